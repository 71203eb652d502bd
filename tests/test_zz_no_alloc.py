"""The allocation-free expectation entry point (expval_pauli_sum_noalloc).

Some callers cannot allocate while they run: code inside a memory budget that
an outer framework has already handed out, latency-critical loops that cannot
take the device-wide synchronisation an allocation can cause, hosts that
forbid allocation after start-up.  For them the library offers one entry point
that uses a fixed scratch array inside the library instead of allocating.
These tests call it through the C ABI and check it against the regular
expval_pauli_sum and against the oracle, twice in a row (the scratch keeps
the previous call's contents, which must not leak into the next result).  This file is collected
last so that a run stopping at the first failure has run everything else.
"""
import ctypes

import numpy as np
import pytest

from helpers import random_paulis
from paper_2602_09020_gb300 import capi, synth

pytestmark = pytest.mark.gpu


def _tol(c):
    return 1e-12 * max(1.0, float(np.abs(c).sum()))


@pytest.mark.parametrize("dtype,n", [("c128", 12), ("c64", 12), ("c128", 3), ("c64", 20)])
def test_noalloc_matches_expval_twice(orc, dtype, n):
    ham = synth.jw_hamiltonian(n, 300, 5) if n >= 4 else None
    if ham is None:
        x, z = random_paulis(n, 20, seed=1, diag_frac=0.3)
        c = np.random.default_rng(1).normal(size=20)
    else:
        x, z, c = ham.x, ham.z, ham.c
    psi = synth.random_state(n, 9)
    sv = capi.sv_alloc(n, dtype)
    try:
        capi.sv_from_host(sv, psi.astype(np.complex64 if dtype == "c64" else np.complex128))
        capi.frame_apply_pauli(sv, "Y", 1)
        e_ref, n_ref = capi.expval_pauli_sum(sv, x, z, c)
        # the oracle on the same state: the stored amplitudes (rounded to the
        # handle's precision) with the frame's Y on qubit 1 applied as a gate
        stored = psi.astype(np.complex64 if dtype == "c64" else np.complex128).astype(np.complex128)
        e_orc = orc.expval(orc.gate(stored.copy(), n, "y", 1), n, x, z, c)
        assert abs(e_ref - e_orc) <= _tol(c), (e_ref, e_orc)
        assert abs(n_ref - orc.norm2(stored, n)) <= 1e-13
        for _ in range(2):
            e, nrm = capi.expval_pauli_sum_noalloc(sv, x, z, c)
            assert abs(e - e_ref) <= _tol(c), (e, e_ref)
            assert abs(e - e_orc) <= _tol(c), (e, e_orc)
            assert abs(nrm - n_ref) <= 1e-13
        # a different, smaller request right after a larger one
        e1, _ = capi.expval_pauli_sum(sv, x[:7], z[:7], c[:7])
        e2, _ = capi.expval_pauli_sum_noalloc(sv, x[:7], z[:7], c[:7])
        assert abs(e1 - e2) <= _tol(c[:7])
    finally:
        capi.sv_free(sv)


def test_noalloc_rejects_oversized_requests():
    n = 6
    sv = capi.sv_alloc(n, "c128")
    try:
        x = np.zeros(5000, dtype=np.uint64)
        z = np.arange(5000, dtype=np.uint64) % 64
        c = np.ones(5000)
        with pytest.raises(capi.PauliRotError) as e:
            capi.expval_pauli_sum_noalloc(sv, x, z, c)
        assert e.value.code == capi.SV_EINVAL and "4096" in str(e.value)
    finally:
        capi.sv_free(sv)


def test_noalloc_leaves_device_memory_unchanged():
    torch = pytest.importorskip("torch")
    n = 14
    ham = synth.jw_hamiltonian(n, 200, 3)
    sv = capi.sv_alloc(n, "c128")
    try:
        capi.sv_set_basis_state(sv, 7)
        capi.expval_pauli_sum_noalloc(sv, ham.x, ham.z, ham.c)  # first call: set-up
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        for _ in range(3):
            capi.expval_pauli_sum_noalloc(sv, ham.x, ham.z, ham.c)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0
    finally:
        capi.sv_free(sv)
