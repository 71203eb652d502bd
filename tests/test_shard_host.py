"""Global-qubit sharding on CPU: the library's host planner and the sharded
driver, with the oracle doing every slice's arithmetic.

* the planner (shard_rotations / shard_terms through the C ABI, no GPU): steps
  cover the list in order, pair steps name the partner r ^ X, rewritten masks
  fit the slice or pair state, every rank gets the same steps, bad arguments
  fail;
* the whole distributed scheme (paper, Sec. "Multi-qubit rotations in a
  fullstate simulator", distributed-memory paragraph) with 2, 4 and 8 ranks in
  one process and with 2 and 4 gloo processes: a Trotter evolution with
  Clifford gates on global qubits, <H> and the norm summed over ranks, and the
  gathered state, against the oracle's run of the whole state.
"""
import os
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2602_09020_gb300 import capi, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _workload(n, seed=3):
    ham = synth.jw_hamiltonian(n, 4 * n + 8, seed)
    rx, rz, rt = capi.trotter_expand(ham.x, ham.z, ham.c, 0.15, 1, 1, False)
    # Clifford gates on the top qubits (global for every g >= 1) and across the cut
    gates = [("h", n - 1), ("cnot", n - 1, 0), ("s", n - 2), ("cnot", 1, n - 2), ("h", 2), ("sdg", n - 1),
             ("rz", n - 1, 0.37), ("ry", 0, -0.81), ("rx", n - 2, 1.3)]
    return ham, (rx, rz, rt), gates


def _oracle_reference(orc, n, ham, rots, gates, basis):
    rx, rz, rt = rots
    psi = orc.basis_state(n, basis)
    orc.apply_rotations(psi, n, rx, rz, rt)
    for g in gates:
        name = g[0]
        if name in ("rx", "ry"):  # exp(-i theta/2 sigma) as a one-qubit rotation
            q, th = g[1], g[2]
            orc.apply_rotation(psi, n, 1 << q, (1 << q) if name == "ry" else 0, th)
        elif name == "rz":
            orc.gate(psi, n, "rz", g[1], theta=g[2])
        elif name == "cnot":
            orc.gate(psi, n, "cnot", g[1], g[2])
        else:
            orc.gate(psi, n, name, g[1])
    orc.apply_rotations(psi, n, rx, rz, rt)
    return psi, orc.expval(psi, n, ham.x, ham.z, ham.c)


def _sharded_run(st, ham, rots, gates, basis):
    rx, rz, rt = rots
    st.set_basis_state(basis)
    st.apply_pauli_rotations(rx, rz, rt)
    st.apply_gates(gates)
    st.apply_pauli_rotations(rx, rz, rt)
    e, nrm = st.expval_pauli_sum(ham.x, ham.z, ham.c)
    st.materialize()
    return e, nrm, st.gather()


def _phase_aligned(ref, got):
    k = int(np.argmax(np.abs(ref)))
    return got * (ref[k] / got[k]) / abs(ref[k] / got[k])


# ---------------------------------------------------------------- the planner

def test_planner_steps_partition_and_partners():
    n, g = 9, 2
    L = n - g
    ham, (rx, rz, rt), _ = _workload(n)
    ref = None
    for r in range(1 << g):
        steps, ox, oz, ot = capi.shard_rotations(n, g, r, rx, rz, rt)
        pos = 0
        for kind, partner, first, count in steps:
            assert first == pos and count > 0
            pos += count
            sl = slice(first, first + count)
            if kind == 0:
                assert partner == r
                assert all(int(x) >> L == 0 for x in rx[sl])
                assert int(np.max(ox[sl] | oz[sl])) < (1 << L)
            else:
                X = r ^ partner
                assert X != 0 and all(int(x) >> L in (0, X) for x in rx[sl])
                assert int(np.max(ox[sl] | oz[sl])) < (1 << (L + 1))
                # the rotation that opens a pair step crosses the pair
                assert int(rx[first]) >> L == X and (int(ox[first]) >> L) & 1
        assert pos == len(rt)
        assert np.array_equal(np.abs(ot), np.abs(rt))
        cut = [(k, f, c) for k, _, f, c in steps]
        assert ref is None or cut == ref
        ref = cut


def test_planner_without_global_qubits_is_identity():
    ham, (rx, rz, rt), _ = _workload(7)
    steps, ox, oz, ot = capi.shard_rotations(7, 0, 0, rx, rz, rt)
    assert steps == [(0, 0, 0, len(rt))]
    assert np.array_equal(ox, rx) and np.array_equal(oz, rz) and np.array_equal(ot, rt)
    groups, tx, tz, tc = capi.shard_terms(7, 0, 0, ham.x, ham.z, ham.c)
    assert groups == [(0, 0, 0, len(ham.c))]
    assert np.array_equal(tc, ham.c)


def test_planner_terms_groups():
    n, g = 8, 3
    L = n - g
    ham, _, _ = _workload(n, seed=5)
    for r in range(1 << g):
        groups, tx, tz, tc = capi.shard_terms(n, g, r, ham.x, ham.z, ham.c)
        assert groups[0][0] == 0 and sum(c for *_, c in groups) == len(ham.c)
        seen = set()
        for kind, partner, first, count in groups[1:]:
            X = r ^ partner
            assert kind == 1 and X not in seen and X != 0
            seen.add(X)
        # pair terms are halved, local ones keep their size
        assert np.allclose(np.sort(np.abs(tc[: groups[0][3]])),
                           np.sort(np.abs(ham.c[(ham.x >> np.uint64(L)) == 0])))


def test_planner_rejects_bad_arguments():
    x = np.array([1 << 9], dtype=np.uint64)
    z = np.zeros(1, dtype=np.uint64)
    t = np.ones(1)
    with pytest.raises(capi.PauliRotError) as e:
        capi.shard_rotations(9, 2, 4, np.array([1], np.uint64), z, t)
    assert e.value.code == capi.SV_EINVAL
    with pytest.raises(capi.PauliRotError) as e:
        capi.shard_rotations(9, 2, 0, x, z, t)  # bit 9 on 9 qubits
    assert e.value.code == capi.SV_EINVAL
    with pytest.raises(capi.PauliRotError) as e:
        capi.shard_terms(9, 9, 0, z, z, t)  # every qubit global
    assert e.value.code == capi.SV_EINVAL


# ---------------------------------------------------------------- the scheme, all ranks in one process

class _CountingComm:
    def __init__(self, inner):
        self.inner, self.world, self.ranks, self.exchanges = inner, inner.world, inner.ranks, 0

    def exchange(self, store, partner_of):
        self.exchanges += 1
        self.inner.exchange(store, partner_of)

    def allreduce_sum(self, v, store):
        return self.inner.allreduce_sum(v, store)

    def all_slices(self, store):
        return self.inner.all_slices(store)


@pytest.mark.parametrize("g", [1, 2, 3])
def test_sharded_evolution_in_process_matches_oracle(orc, g):
    from paper_2602_09020_gb300.shard import InProcessComm, ShardedState
    from shard_oracle import OracleSlices
    n = 9
    ham, rots, gates = _workload(n)
    basis = synth.hartree_fock_index(4)
    want, e_ref = _oracle_reference(orc, n, ham, rots, gates, basis)
    comm = _CountingComm(InProcessComm(1 << g))
    st = ShardedState(n, "c128", g, comm, store=OracleSlices(n - g, comm.ranks))
    try:
        e, nrm, got = _sharded_run(st, ham, rots, gates, basis)
    finally:
        st.close()
    assert abs(e - e_ref) <= 1e-12 and abs(nrm - 1.0) <= 1e-12
    np.testing.assert_allclose(_phase_aligned(want, got), want, atol=1e-12, rtol=0)
    assert comm.exchanges >= 1


def test_sharded_pauli_only_state_needs_no_phase_alignment(orc):
    """Without Clifford gates the frame stays at the origin: the gathered slices
    are the state itself, amplitude for amplitude."""
    from paper_2602_09020_gb300.shard import InProcessComm, ShardedState
    from shard_oracle import OracleSlices
    n, g = 8, 2
    ham, (rx, rz, rt), _ = _workload(n, seed=9)
    st = ShardedState(n, "c128", g, InProcessComm(4), store=OracleSlices(n - g, range(4)))
    try:
        st.set_basis_state(0b1011)
        st.apply_pauli_rotations(rx, rz, rt)
        got = st.gather()
    finally:
        st.close()
    want = orc.apply_rotations(orc.basis_state(n, 0b1011), n, rx, rz, rt)
    np.testing.assert_allclose(got, want, atol=1e-13, rtol=0)


# ---------------------------------------------------------------- the scheme over gloo processes

def _gloo_worker(rank, world, port, n, q):
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch.distributed as dist
    from paper_2602_09020_gb300.shard import ProcessGroupComm, ShardedState
    from shard_oracle import OracleSlices
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = world.bit_length() - 1
        ham, rots, gates = _workload(n)
        comm = ProcessGroupComm()
        st = ShardedState(n, "c128", g, comm, store=OracleSlices(n - g, comm.ranks))
        try:
            e, nrm, got = _sharded_run(st, ham, rots, gates, synth.hartree_fock_index(4))
        finally:
            st.close()
        q.put((rank, e, nrm, got))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_sharded_evolution_gloo_matches_oracle(orc, world):
    n = 9
    ham, rots, gates = _workload(n)
    want, e_ref = _oracle_reference(orc, n, ham, rots, gates, synth.hartree_fock_index(4))
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29600 + (os.getpid() * 7 + world) % 900
    procs = [ctx.Process(target=_gloo_worker, args=(r, world, port, n, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, e, nrm, got in res:
        assert abs(e - e_ref) <= 1e-12 and abs(nrm - 1.0) <= 1e-12
        np.testing.assert_allclose(_phase_aligned(want, got), want, atol=1e-12, rtol=0)
