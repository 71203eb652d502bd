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


@pytest.mark.parametrize("dtype,scale", [("c64", 1.0), ("c64", 1.5), ("c64", 1e-3), ("c64", 1e-20),
                                         ("c128", 1.0), ("c128", 1e-3), ("c128", 1e-150), ("c128", 1e120)])
def test_expval_group_structure(orc, dtype, scale):
    """<H> with x-masks that are XOR combinations of one another (so a run
    holds x-masks whose coordinates in the run basis are 3, 5, 6, 7, ...), both
    Re and Im parts, one x-mask with 40 terms (more than one run holds), 70
    diagonal terms and identities spread over several runs, at several state
    norms.  The fixed-point grid 2^-S follows the norm (S = 60 - ceil(log2
    <a|a>), bounded where the norm is too small for the estimate), and each
    sum is exact up to 2^-(S+1) per transform entry (complex64: exact products;
    complex128: 62-bit fixed-point products on one exponent per 16-amplitude
    tile): the result matches the oracle on the same rounded amplitudes to
    FP64 accuracy relative to the norm, and repeated calls agree bitwise."""
    n = 11
    rng = np.random.default_rng(17)
    psi = synth.random_state(n, 31) * scale
    gens = [int(v) for v in rng.integers(1, 1 << n, size=4)]
    xs_unique = []
    for k in range(1, 16):
        v = 0
        for b in range(4):
            if (k >> b) & 1:
                v ^= gens[b]
        if v:
            xs_unique.append(v)
    x, z = [], []
    for v in xs_unique:
        for _ in range(3):
            x.append(v)
            z.append(int(rng.integers(0, 1 << n)))
    for _ in range(40):
        x.append(gens[0])
        z.append(int(rng.integers(0, 1 << n)))
    for _ in range(70):
        x.append(0)
        z.append(int(rng.integers(0, 1 << n)))
    x += [0, 0]
    z += [0, 0]
    x = np.array(x, dtype=np.uint64)
    z = np.array(z, dtype=np.uint64)
    c = rng.normal(size=len(x))
    psi_r = psi.astype(np.complex64).astype(np.complex128) if dtype == "c64" else psi
    ref = orc.expval(psi_r, n, x, z, c)
    sv = upload(n, dtype, psi)
    e1, nrm1 = capi.expval_pauli_sum(sv, x, z, c)
    e2, nrm2 = capi.expval_pauli_sum(sv, x, z, c)
    capi.sv_free(sv)
    norm = float(np.vdot(psi_r, psi_r).real)
    assert abs(e1 - ref) < 1e-12 * np.abs(c).sum() * norm, (e1, ref)
    assert abs(nrm1 - norm) <= 1e-13 * norm
    assert e1 == e2 and nrm1 == nrm2
