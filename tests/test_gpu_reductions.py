"""GPU parity of the FP64 reductions (norm, <H>, H|psi>) against the oracle."""
import numpy as np
import pytest

from helpers import random_paulis
from paper_2602_09020_gb300 import capi, synth

pytestmark = pytest.mark.gpu


def upload(n, dtype, psi):
    sv = capi.sv_alloc(n, dtype)
    capi.sv_from_host(sv, psi.astype(np.complex64 if dtype == "c64" else np.complex128))
    return sv


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 8, 12])
def test_expval_random_terms(orc, n):
    psi = synth.random_state(n, 50 + n)
    x, z = random_paulis(n, 60, seed=n, diag_frac=0.3)
    c = np.random.default_rng(n).normal(size=60)
    want = orc.expval(psi, n, x, z, c)
    sv = upload(n, "c128", psi)
    e, nrm = capi.expval_pauli_sum(sv, x, z, c)
    capi.sv_free(sv)
    assert abs(e - want) < 1e-12 * max(1.0, np.abs(c).sum()), (e, want)
    assert abs(nrm - 1.0) < 1e-13
    sv = upload(n, "c64", psi)
    e32, nrm32 = capi.expval_pauli_sum(sv, x, z, c)
    ref32 = orc.expval(psi.astype(np.complex64).astype(np.complex128), n, x, z, c)
    capi.sv_free(sv)
    # FP64 accumulation over FP32 amplitudes: agrees with the oracle on the same
    # rounded amplitudes to FP64 accuracy
    assert abs(e32 - ref32) < 1e-12 * max(1.0, np.abs(c).sum())


def test_expval_jw_hamiltonian_and_determinism(orc):
    n = 12
    ham = synth.jw_hamiltonian(n, 300, 8)
    psi = synth.random_state(n, 8)
    want = orc.expval(psi, n, ham.x, ham.z, ham.c)
    sv = upload(n, "c128", psi)
    e1, _ = capi.expval_pauli_sum(sv, ham.x, ham.z, ham.c)
    e2, _ = capi.expval_pauli_sum(sv, ham.x, ham.z, ham.c)
    capi.sv_free(sv)
    assert abs(e1 - want) < 1e-11
    assert e1 == e2  # fixed reduction order: bitwise reproducible


def test_expval_empty_and_identity_terms(orc):
    n = 6
    psi = synth.random_state(n, 2) * 1.5
    sv = upload(n, "c128", psi)
    e, nrm = capi.expval_pauli_sum(sv, [], [], [])
    assert e == 0.0 and abs(nrm - 2.25) < 1e-13
    e, _ = capi.expval_pauli_sum(sv, [0, 0], [0, 0], [0.5, 0.25])
    capi.sv_free(sv)
    assert abs(e - 0.75 * 2.25) < 1e-13


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_apply_pauli_sum(orc, dtype):
    n = 9
    psi = synth.random_state(n, 77)
    ham = synth.jw_hamiltonian(n, 120, 77)
    want = orc.apply_pauli_sum(psi, n, ham.x, ham.z, ham.c)
    src = upload(n, dtype, psi)
    dst = capi.sv_alloc(n, dtype)
    capi.apply_pauli_sum(dst, src, ham.x, ham.z, ham.c)
    got = capi.sv_to_host(dst, True)
    capi.sv_free(src)
    capi.sv_free(dst)
    tol = 1e-12 if dtype == "c128" else 2e-5
    assert np.max(np.abs(got - want)) < tol * max(1.0, np.abs(ham.c).sum() / 10)
