"""apply_pauli_rotations launches runs while it is still planning the rest of
the list (records copied to the handle's buffer in batches); the launches are
those of plan_create + plan_apply on the same list, so the two must give the
same state bit for bit.  Cases: both precisions, lists shorter than one batch
of runs and many batches long, diagonal stretches, angles needing frame factors,
a running-scale fold on the last run, identities only, an empty list, a Pauli
frame set beforehand, consecutive calls on one handle (buffer reuse and growth),
and the oracle on the result."""
import numpy as np
import pytest

from helpers import assert_close_c128, random_paulis
from paper_2602_09020_gb300 import capi, synth

pytestmark = pytest.mark.gpu


def lists(n):
    g = np.random.default_rng(n)
    ham = synth.jw_hamiltonian(n, 400, seed=n)
    x, z, th = capi.trotter_expand(ham.x, ham.z, ham.c, 0.07, 3, 1, False)
    yield "jw", x, z, th
    x, z = random_paulis(n, 30, seed=n + 1, span_dim=3, diag_frac=0.2)
    yield "short", x, z, g.uniform(-5, 5, size=30)
    dz = g.integers(1, 1 << n, size=60).astype(np.uint64)
    x2, z2 = random_paulis(n, 50, seed=n + 2)
    x = np.concatenate([np.zeros(60, dtype=np.uint64), x2, np.zeros(20, dtype=np.uint64)])
    z = np.concatenate([dz, z2, dz[:20]])
    yield "diag", x, z, g.uniform(-3, 3, size=len(x))
    yield "identities", np.zeros(5, dtype=np.uint64), np.zeros(5, dtype=np.uint64), g.uniform(-1, 1, size=5)
    yield "empty", np.zeros(0, dtype=np.uint64), np.zeros(0, dtype=np.uint64), np.zeros(0)


@pytest.mark.parametrize("n,dtype", [(14, "c64"), (16, "c64"), (10, "c64"), (12, "c128"), (14, "c128")])
def test_streamed_apply_equals_plan_apply(orc, n, dtype):
    cdt = np.complex64 if dtype == "c64" else np.complex128
    psi0 = synth.random_state(n, 3 * n).astype(cdt)
    a = capi.sv_alloc(n, dtype)
    b = capi.sv_alloc(n, dtype)
    try:
        capi.sv_from_host(a, psi0)
        capi.sv_from_host(b, psi0)
        for sv in (a, b):
            capi.frame_apply_pauli(sv, "Y", 1)
        want = psi0.astype(np.complex128)
        orc.gate(want, n, "y", 1)
        for name, x, z, th in lists(n):
            capi.apply_pauli_rotations(a, x, z, th)
            plan = capi.plan_create(n, dtype, x, z, th, -1)
            try:
                capi.plan_apply(b, plan)
            finally:
                capi.plan_free(plan)
            ga, gb = capi.sv_to_host(a, False), capi.sv_to_host(b, False)
            assert np.array_equal(ga.view(np.uint8), gb.view(np.uint8)), f"{name}: states differ"
            assert capi.frame_get(a) == capi.frame_get(b), name
            if len(th):
                orc.apply_rotations(want, n, x, z, th)
        got = capi.sv_to_host(a, True).astype(np.complex128)
        if dtype == "c128":
            assert_close_c128(want, got, what=f"n={n}")
        else:
            ov = abs(np.vdot(want, got)) ** 2 / (np.vdot(want, want).real * np.vdot(got, got).real)
            assert 1.0 - ov < 1e-5
    finally:
        capi.sv_free(a)
        capi.sv_free(b)


def test_streamed_apply_after_a_stream_switch():
    """The handle's record buffer is reused by the next call, which may run on
    another stream (sv_set_stream): its copies wait for the previous call's
    passes, so a long list on one stream followed at once by a short one on
    another gives the sequential result bit for bit."""
    import torch
    n = 18
    ham = synth.jw_hamiltonian(n, 600, seed=5)
    xa, za, ta = capi.trotter_expand(ham.x, ham.z, ham.c, 0.05, 4, 1, False)
    xb, zb = random_paulis(n, 200, seed=6, span_dim=4)
    tb = np.random.default_rng(6).uniform(-2, 2, size=200)
    psi0 = synth.random_state(n, 7).astype(np.complex64)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    sv = capi.sv_alloc(n, "c64", s1.cuda_stream)
    ref = capi.sv_alloc(n, "c64")
    try:
        capi.sv_from_host(sv, psi0)
        capi.sv_from_host(ref, psi0)
        capi.apply_pauli_rotations(sv, xa, za, ta)
        capi.sv_set_stream(sv, s2.cuda_stream)
        capi.apply_pauli_rotations(sv, xb, zb, tb)
        for x, z, t in ((xa, za, ta), (xb, zb, tb)):
            p = capi.plan_create(n, "c64", x, z, t, -1)
            capi.plan_apply(ref, p)
            capi.plan_free(p)
        got, want = capi.sv_to_host(sv, False), capi.sv_to_host(ref, False)
        assert np.array_equal(got.view(np.uint8), want.view(np.uint8))
    finally:
        capi.sv_free(sv)
        capi.sv_free(ref)
