"""Global-qubit sharding on one GPU: every rank's slice in this GPU's memory
(LibrarySlices), exchanges as device copies between slices (InProcessComm),
all rotations and reductions in the library's kernels on slices and pair
states.  Checked against the oracle's run of the whole state (complex128 to
1e-12, complex64 by infidelity) and against the unsharded library path.
Kernels of different ranks never wait on one another: the ranks run one after
the other on one stream.
"""
import numpy as np
import pytest

from helpers import assert_close_c128, infidelity
from paper_2602_09020_gb300 import capi, synth
from test_shard_host import _oracle_reference, _phase_aligned, _sharded_run, _workload

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("g", [1, 2, 3])
def test_sharded_state_on_one_gpu_matches_oracle(orc, dtype, g):
    from paper_2602_09020_gb300.shard import InProcessComm, ShardedState
    n = 12
    ham, rots, gates = _workload(n)
    basis = synth.hartree_fock_index(6)
    want, e_ref = _oracle_reference(orc, n, ham, rots, gates, basis)
    st = ShardedState(n, dtype, g, InProcessComm(1 << g))
    try:
        e, nrm, got = _sharded_run(st, ham, rots, gates, basis)
    finally:
        st.close()
    got = _phase_aligned(want, got.astype(np.complex128))
    if dtype == "c128":
        assert abs(e - e_ref) <= 1e-12 and abs(nrm - 1.0) <= 1e-12
        assert_close_c128(want, got, what=f"sharded g={g}")
    else:
        assert abs(e - e_ref) <= 1e-4 and abs(nrm - 1.0) <= 1e-5
        assert infidelity(want, got) <= 1e-6


def test_sharded_matches_unsharded_library_path():
    """The same Trotter run sharded over 4 slices and as one state, complex128:
    energies and amplitudes agree to rounding."""
    from paper_2602_09020_gb300.shard import InProcessComm, ShardedState
    n = 14
    ham = synth.jw_hamiltonian(n, 120, 7)
    rx, rz, rt = capi.trotter_expand(ham.x, ham.z, ham.c, 0.1, 2, 1, False)
    basis = synth.hartree_fock_index(7)
    st = ShardedState(n, "c128", 2, InProcessComm(4))
    try:
        st.set_basis_state(basis)
        st.apply_pauli_rotations(rx, rz, rt)
        e, nrm = st.expval_pauli_sum(ham.x, ham.z, ham.c)
        got = st.gather()
    finally:
        st.close()
    sv = capi.sv_alloc(n, "c128")
    try:
        capi.sv_set_basis_state(sv, basis)
        capi.apply_pauli_rotations(sv, rx, rz, rt)
        e1, n1 = capi.expval_pauli_sum(sv, ham.x, ham.z, ham.c)
        want = capi.sv_to_host(sv, True)
    finally:
        capi.sv_free(sv)
    assert abs(e - e1) <= 1e-12 and abs(nrm - n1) <= 1e-12
    assert_close_c128(want, got, what="sharded vs single state")
