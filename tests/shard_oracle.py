"""A slice store for ShardedState backed by the CPU oracle (test infrastructure).

It has the interface of paper_2602_09020_gb300.shard.LibrarySlices, but each
rank's buffer is a host complex128 array and every rotation and reduction is
the oracle's: the textbook gate decomposition and the gate-wise expectation.
With it the sharded host logic (the library's planner, the exchanges, the
rank sums) runs on CPU ranks -- in one process or as gloo processes -- and is
checked against the oracle's run of the whole state.
"""
import numpy as np
import torch

import oracle


class OracleSlices:
    def __init__(self, local_qubits, ranks):
        self.L = int(local_qubits)
        self.buf = {r: np.zeros(2 << self.L, dtype=np.complex128) for r in ranks}
        # torch views sharing the buffers, for the communicator
        self.tbuf = {r: torch.from_numpy(self.buf[r]) for r in ranks}
        self.rotations = 0
        self.pair_rotations = 0

    def own(self, r):
        return self.tbuf[r][: 1 << self.L]

    def recv(self, r):
        return self.tbuf[r][1 << self.L:]

    def clear(self, r):
        self.buf[r][:] = 0

    def set_one(self, r, k):
        self.buf[r][: 1 << self.L] = 0
        self.buf[r][k] = 1.0

    def rotate(self, r, pair, x, z, theta):
        if pair:
            oracle.apply_rotations(self.buf[r], self.L + 1, x, z, theta)
            self.pair_rotations += len(theta)
        else:
            oracle.apply_rotations(self.buf[r][: 1 << self.L], self.L, x, z, theta)
            self.rotations += len(theta)

    def expval(self, r, pair, x, z, c):
        v = self.buf[r] if pair else self.buf[r][: 1 << self.L]
        nq = self.L + 1 if pair else self.L
        return oracle.expval(v, nq, x, z, c), oracle.norm2(v, nq)

    def slice_to_host(self, r):
        return self.buf[r][: 1 << self.L].copy()
