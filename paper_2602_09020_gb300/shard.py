"""A statevector sharded over ranks by its top qubits.

The paper spreads the amplitudes of its full-state simulator over MPI ranks by
the top g index bits, the global qubits, and a rotation whose x-mask touches a
global qubit makes the two ranks it pairs exchange their slices (Sec.
"Multi-qubit rotations in a fullstate simulator", distributed-memory paragraph).
:class:`ShardedState` does the same for 2^g ranks:

* rank r holds the 2^L amplitudes (L = n - g) whose top bits are r, in the lower
  half of a buffer of 2^(L+1) amplitudes; the upper half receives a partner's
  slice, and the two halves form the rank's pair state of L + 1 qubits;
* the library's host planner (``shard_rotations``, ``shard_terms``) rewrites each
  rotation and each Pauli term for the rank: onto its slice (no global x-bit) or
  onto its pair state with the partner r ^ X (global x-part X), and it cuts the
  rotation list into steps so that consecutive rotations sharing a partner
  share one exchange;
* an exchange is one send and one receive of the whole slice with the partner;
  every rotation and reduction then runs in the library's kernels on the slice
  or the pair state; <H> and the norm are summed over ranks in FP64;
* a Clifford frame (the ``cliff_*`` host object) holds the Clifford gates, as in
  the single-state hybrid simulator: rotations and terms are mapped through it
  by the planner, and :meth:`ShardedState.materialize` applies it as rotations.

Where the slices live and how they travel are separate objects: a slice store
(:class:`LibrarySlices`: device memory and libpaulirot handles) and a
communicator (:class:`ProcessGroupComm`: one rank per process over
``torch.distributed`` point-to-point and all-reduce; :class:`InProcessComm`: every
rank in this process, an exchange being a copy between two slices).  The store
and the communicator only move data and call the library; the planner decides
what is computed.
"""
from __future__ import annotations

from typing import Dict, List, Optional, Sequence

import numpy as np
import torch

from . import capi

_TORCH_DT = {capi.SV_C128: torch.complex128, capi.SV_C64: torch.complex64}


class LibrarySlices:
    """Each driven rank's slice in device memory (lower half of a buffer of
    2^(L+1) amplitudes) with two library handles on the current torch stream:
    the slice (L qubits) and the pair state (the whole buffer, L + 1 qubits).
    Every operation leaves both handles with the identity Pauli frame."""

    def __init__(self, local_qubits: int, dtype, ranks: Sequence[int], device=None):
        if not torch.cuda.is_available():
            raise capi.PauliRotError(capi.SV_ECUDA, "LibrarySlices needs a CUDA device")
        self.L = int(local_qubits)
        self.dtype = capi.dtype_code(dtype)
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        stream = int(torch.cuda.current_stream(self.device).cuda_stream)
        self.buf: Dict[int, torch.Tensor] = {}
        self.h_own: Dict[int, int] = {}
        self.h_pair: Dict[int, int] = {}
        half = 1 << self.L
        for r in ranks:
            b = torch.zeros(2 * half, dtype=_TORCH_DT[self.dtype], device=self.device)
            self.buf[r] = b
            self.h_own[r] = capi.sv_wrap(b.data_ptr(), self.L, self.dtype, stream)
            self.h_pair[r] = capi.sv_wrap(b.data_ptr(), self.L + 1, self.dtype, stream)

    def close(self) -> None:
        for h in list(self.h_own.values()) + list(self.h_pair.values()):
            capi.sv_free(h)
        self.h_own.clear()
        self.h_pair.clear()
        self.buf.clear()

    def own(self, r: int) -> torch.Tensor:
        return self.buf[r][: 1 << self.L]

    def recv(self, r: int) -> torch.Tensor:
        return self.buf[r][1 << self.L:]

    def clear(self, r: int) -> None:
        self.buf[r].zero_()

    def set_one(self, r: int, k: int) -> None:
        capi.sv_set_basis_state(self.h_own[r], k)

    def rotate(self, r: int, pair: bool, x, z, theta) -> None:
        h = self.h_pair[r] if pair else self.h_own[r]
        capi.apply_pauli_rotations(h, x, z, theta)
        capi.sv_materialize(h)

    def expval(self, r: int, pair: bool, x, z, c):
        return capi.expval_pauli_sum(self.h_pair[r] if pair else self.h_own[r], x, z, c)

    def slice_to_host(self, r: int) -> np.ndarray:
        return capi.sv_to_host(self.h_own[r], True)


class InProcessComm:
    """Every rank driven by this process: an exchange copies the partner's slice
    into the upper half of each rank's buffer; sums over ranks are local."""

    def __init__(self, world: int):
        self.world = int(world)
        self.ranks = list(range(self.world))

    def exchange(self, store, partner_of: Dict[int, int]) -> None:
        for r in self.ranks:
            store.recv(r).copy_(store.own(partner_of[r]))

    def allreduce_sum(self, values: np.ndarray, store) -> np.ndarray:
        return np.asarray(values, dtype=np.float64)

    def all_slices(self, store) -> List[np.ndarray]:
        return [store.slice_to_host(r) for r in range(self.world)]


class ProcessGroupComm:
    """One rank per process over torch.distributed (backend of the default or
    given group: gloo for host tensors, nccl for device tensors).  An exchange is
    a paired isend/irecv of the whole slice with the partner."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.world = dist.get_world_size(group)
        self.ranks = [dist.get_rank(group)]

    def exchange(self, store, partner_of: Dict[int, int]) -> None:
        r = self.ranks[0]
        p = partner_of[r]
        ops = [self.dist.P2POp(self.dist.isend, store.own(r).contiguous(), p, self.group),
               self.dist.P2POp(self.dist.irecv, store.recv(r), p, self.group)]
        for q in self.dist.batch_isend_irecv(ops):
            q.wait()

    def allreduce_sum(self, values: np.ndarray, store) -> np.ndarray:
        t = torch.tensor(np.asarray(values, dtype=np.float64), device=store.own(self.ranks[0]).device)
        self.dist.all_reduce(t, group=self.group)
        return t.cpu().numpy()

    def all_slices(self, store) -> List[np.ndarray]:
        mine = store.own(self.ranks[0]).contiguous()
        parts = [torch.empty_like(mine) for _ in range(self.world)]
        self.dist.all_gather(parts, mine, group=self.group)
        return [p.cpu().numpy() for p in parts]


class ShardedState:
    """An n-qubit state over 2^g ranks (g = global_qubits), |0..0> with the
    origin Clifford frame.  ``comm.world`` must be 2^g; ``store`` defaults to
    :class:`LibrarySlices` on the current CUDA device."""

    def __init__(self, n_qubits: int, dtype, global_qubits: int, comm, store=None):
        self.n = int(n_qubits)
        self.g = int(global_qubits)
        if not 0 <= self.g < self.n:
            raise ValueError("global_qubits must be in 0..n-1")
        if comm.world != (1 << self.g):
            raise ValueError(f"the communicator has {comm.world} ranks, the state needs {1 << self.g}")
        self.L = self.n - self.g
        self.dtype = capi.dtype_code(dtype)
        self.comm = comm
        self.store = store if store is not None else LibrarySlices(self.L, self.dtype, comm.ranks)
        self.frame = capi.cliff_create(self.n)
        self.set_basis_state(0)

    def close(self) -> None:
        if getattr(self, "frame", None):
            capi.cliff_free(self.frame)
            self.frame = None
        if getattr(self, "store", None) is not None and hasattr(self.store, "close"):
            self.store.close()

    # -- state set-up
    def set_basis_state(self, k: int) -> None:
        """|k> on the origin frame: rank k >> L holds the one amplitude."""
        owner, local = int(k) >> self.L, int(k) & ((1 << self.L) - 1)
        for r in self.comm.ranks:
            self.store.clear(r)
            if r == owner:
                self.store.set_one(r, local)
        capi.cliff_reset(self.frame)

    # -- evolution
    def apply_pauli_rotations(self, x, z, theta) -> None:
        """exp(-i theta_j/2 P_j) for j in order on the represented state."""
        self._run(x, z, theta, self.frame)

    def apply_gates(self, gates) -> None:
        """A gate stream (see capi.cliff_apply_gates): Clifford gates update the
        host frame, rotation gates run on the slices."""
        x, z, t = capi.cliff_apply_gates(self.frame, gates)
        self._run(x, z, t, None)

    def materialize(self) -> None:
        """Apply the Clifford frame to the slices (<= 4n rotations by pi/2) and
        reset it: the slices then hold the state up to a global phase."""
        x, z, t = capi.cliff_inverse_rotations(self.frame)
        self._run(x, z, t, None)
        capi.cliff_reset(self.frame)

    def _run(self, x, z, theta, frame) -> None:
        plans = {r: capi.shard_rotations(self.n, self.g, r, x, z, theta, frame) for r in self.comm.ranks}
        steps = plans[self.comm.ranks[0]][0]
        for s, (kind, _, first, count) in enumerate(steps):
            if kind == 1:
                self.comm.exchange(self.store, {r: plans[r][0][s][1] for r in self.comm.ranks})
            sl = slice(first, first + count)
            for r in self.comm.ranks:
                _, rx, rz, rt = plans[r]
                self.store.rotate(r, kind == 1, rx[sl], rz[sl], rt[sl])

    # -- reductions
    def expval_pauli_sum(self, x, z, coeff):
        """(<psi|sum_j c_j P_j|psi>, <psi|psi>), FP64, summed over all ranks."""
        plans = {r: capi.shard_terms(self.n, self.g, r, x, z, coeff, self.frame) for r in self.comm.ranks}
        groups = plans[self.comm.ranks[0]][0]
        parts = np.zeros(2, dtype=np.float64)
        for k, (kind, _, first, count) in enumerate(groups):
            if kind == 1:
                self.comm.exchange(self.store, {r: plans[r][0][k][1] for r in self.comm.ranks})
            sl = slice(first, first + count)
            for r in self.comm.ranks:
                _, tx, tz, tc = plans[r]
                e, nrm = self.store.expval(r, kind == 1, tx[sl], tz[sl], tc[sl])
                parts += (e, nrm if k == 0 else 0.0)
        tot = self.comm.allreduce_sum(parts, self.store)
        return float(tot[0]), float(tot[1])

    def gather(self) -> np.ndarray:
        """The whole stored state (every slice, rank order) on the host of every
        process; the Clifford frame is not applied (see materialize)."""
        return np.concatenate(self.comm.all_slices(self.store))
