"""Adjoint gradients against the oracle's parameter-shift rule, central finite
differences (h = 1e-4, FP64, on the GPU complex128 path) and the autograd
Function."""
import numpy as np
import pytest

from paper_2602_09020_gb300 import capi, synth

pytestmark = pytest.mark.gpu


def energy(n, dtype, psi0, x, z, th, hx, hz, hc):
    sv = capi.sv_alloc(n, dtype)
    capi.sv_from_host(sv, psi0)
    capi.apply_pauli_rotations(sv, x, z, th)
    e, _ = capi.expval_pauli_sum(sv, hx, hz, hc)
    capi.sv_free(sv)
    return e


@pytest.mark.parametrize("n,n_rot", [(4, 30), (7, 60), (10, 120)])
def test_adjoint_matches_parameter_shift(orc, n, n_rot):
    x, z, th, obs = synth.adjoint_workload(n, n_rot, 40, seed=n)
    psi0 = orc.basis_state(n, synth.hartree_fock_index(n // 2))
    e_ref, g_ref = orc.grad_param_shift(n, psi0, x, z, th, obs.x, obs.z, obs.c)
    sv = capi.sv_alloc(n, "c128")
    capi.sv_from_host(sv, psi0)
    e, g = capi.rotation_grads(sv, x, z, th, obs.x, obs.z, obs.c)
    # psi0 is left unchanged
    np.testing.assert_array_equal(capi.sv_to_host(sv, True), psi0)
    capi.sv_free(sv)
    scale = max(1.0, np.abs(g_ref).max())
    assert abs(e - e_ref) < 1e-11
    assert np.max(np.abs(g - g_ref)) < 1e-10 * scale
    # complex64: compared to the complex128 adjoint at a stated looser tolerance
    sv = capi.sv_alloc(n, "c64")
    capi.sv_from_host(sv, psi0.astype(np.complex64))
    e32, g32 = capi.rotation_grads(sv, x, z, th, obs.x, obs.z, obs.c)
    capi.sv_free(sv)
    assert abs(e32 - e_ref) < 1e-4 * max(1.0, abs(e_ref))
    assert np.max(np.abs(g32 - g_ref)) < 1e-4 * scale


def test_adjoint_matches_central_differences():
    n, n_rot = 9, 50
    x, z, th, obs = synth.adjoint_workload(n, n_rot, 60, seed=3)
    psi0 = synth.random_state(n, 3)
    sv = capi.sv_alloc(n, "c128")
    capi.sv_from_host(sv, psi0)
    _, g = capi.rotation_grads(sv, x, z, th, obs.x, obs.z, obs.c)
    capi.sv_free(sv)
    h = 1e-4
    fd = np.empty(n_rot)
    for j in range(n_rot):
        tp = th.copy(); tp[j] += h
        tm = th.copy(); tm[j] -= h
        fd[j] = (energy(n, "c128", psi0, x, z, tp, obs.x, obs.z, obs.c) -
                 energy(n, "c128", psi0, x, z, tm, obs.x, obs.z, obs.c)) / (2 * h)
    assert np.max(np.abs(g - fd)) <= 1e-6 * max(1.0, np.abs(g).max())


def test_adjoint_with_frame_on_initial_state(orc):
    n, n_rot = 8, 40
    x, z, th, obs = synth.adjoint_workload(n, n_rot, 30, seed=12)
    psi0 = synth.random_state(n, 12)
    # reference: the frame gates applied as gates to the initial state
    ref0 = psi0.copy()
    orc.apply_pauli(ref0, n, 1 << 2, 1 << 2)  # Y on qubit 2
    orc.apply_pauli(ref0, n, 0, 1 << 5)       # Z on qubit 5
    e_ref, g_ref = orc.grad_param_shift(n, ref0, x, z, th, obs.x, obs.z, obs.c)
    sv = capi.sv_alloc(n, "c128")
    capi.sv_from_host(sv, psi0)
    capi.frame_apply_pauli(sv, "Y", 2)
    capi.frame_apply_pauli(sv, "Z", 5)
    e, g = capi.rotation_grads(sv, x, z, th, obs.x, obs.z, obs.c)
    capi.sv_free(sv)
    assert abs(e - e_ref) < 1e-11
    assert np.max(np.abs(g - g_ref)) < 1e-10 * max(1.0, np.abs(g_ref).max())


def test_autograd_function(orc):
    torch = pytest.importorskip("torch")
    from paper_2602_09020_gb300.torch_api import StateVector, pauli_rotation_energy
    n, n_rot = 6, 25
    x, z, th, obs = synth.adjoint_workload(n, n_rot, 20, seed=5)
    psi0 = StateVector(n, "c128").set_basis_state(synth.hartree_fock_index(3))
    theta = torch.tensor(th, dtype=torch.float64, requires_grad=True)
    e = pauli_rotation_energy(theta, psi0, x, z, obs.x, obs.z, obs.c)
    e.backward()
    e_ref, g_ref = orc.grad_param_shift(n, orc.basis_state(n, 7), x, z, th, obs.x, obs.z, obs.c)
    assert abs(e.item() - e_ref) < 1e-11
    assert np.max(np.abs(theta.grad.numpy() - g_ref)) < 1e-10 * max(1.0, np.abs(g_ref).max())


def test_autograd_forward_alone_and_psi0_unchanged(orc):
    """Forward is E only (rotations on a copy, then <H>): under no_grad it gives
    the oracle's energy, leaves psi0 as it was, and a later backward still
    gives the oracle's parameter-shift gradient."""
    torch = pytest.importorskip("torch")
    from paper_2602_09020_gb300.torch_api import StateVector, pauli_rotation_energy
    n, n_rot = 7, 30
    x, z, th, obs = synth.adjoint_workload(n, n_rot, 25, seed=8)
    basis = synth.hartree_fock_index(3)
    psi0 = StateVector(n, "c128").set_basis_state(basis)
    psi0.frame_apply_pauli("X", 4)
    before = psi0.to_host(False)
    theta = torch.tensor(th, dtype=torch.float64, requires_grad=True)
    start = orc.gate(orc.basis_state(n, basis), n, "x", 4)
    e_ref, g_ref = orc.grad_param_shift(n, start, x, z, th, obs.x, obs.z, obs.c)
    with torch.no_grad():
        e0 = pauli_rotation_energy(theta, psi0, x, z, obs.x, obs.z, obs.c)
    assert abs(e0.item() - e_ref) < 1e-11
    np.testing.assert_array_equal(psi0.to_host(False), before)
    e = pauli_rotation_energy(theta, psi0, x, z, obs.x, obs.z, obs.c)
    e.backward()
    assert abs(e.item() - e_ref) < 1e-11
    assert np.max(np.abs(theta.grad.numpy() - g_ref)) < 1e-10 * max(1.0, np.abs(g_ref).max())
