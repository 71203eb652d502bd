"""Bounds checks by guard words (compute-sanitizer is not available): the state
lives in the middle of a larger device buffer whose two guard regions hold a
canary pattern, and after every kind of launch the regions must be unchanged
bit for bit.  Covers fused passes of every depth (packed and generic kernels),
diagonal phase-sum runs, both <H> reductions, frame materialisation, the
gate-decomposed path, Pauli measurement, the batched launch, the adjoint (which
reads the state) and checkpoint loading, at sizes from 1 qubit up."""
import numpy as np
import pytest
import torch

from paper_2602_09020_gb300 import capi, synth

pytestmark = pytest.mark.gpu

GUARD = 4096  # amplitudes on each side (32 KB / 64 KB: keeps 16-byte alignment)


def rotation_list(n, seed):
    rng = np.random.default_rng(seed)
    m = 120
    x = rng.integers(0, 1 << n, size=m).astype(np.uint64)
    z = rng.integers(0, 1 << n, size=m).astype(np.uint64)
    x[rng.random(m) < 0.2] &= np.uint64(1)          # x with bit 0
    x[rng.random(m) < 0.2] = np.uint64(1 << (n - 1))  # the top bit
    x[40:52] = 0                                     # a diagonal stretch
    th = rng.uniform(-3, 3, size=m)
    return x, z, th


class Guarded:
    def __init__(self, n, dtype):
        self.dt = torch.complex128 if dtype == "c128" else torch.complex64
        self.buf = torch.empty(GUARD + (1 << n) + GUARD, dtype=self.dt, device="cuda")
        self.buf.fill_(complex(12345.678, -98765.4321))
        self.canary = self.buf[:GUARD].clone()
        self.state = self.buf[GUARD:GUARD + (1 << n)]
        self.sv = capi.sv_wrap(self.state.data_ptr(), n, dtype, torch.cuda.current_stream().cuda_stream)
        capi.sv_set_basis_state(self.sv, 0)

    def check(self, what):
        torch.cuda.synchronize()
        lo, hi = self.buf[:GUARD], self.buf[-GUARD:]
        for g in (lo, hi):
            assert torch.equal(torch.view_as_real(g), torch.view_as_real(self.canary)), what

    def close(self):
        capi.sv_free(self.sv)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("n", [1, 2, 5, 9, 12, 17])
def test_no_kernel_writes_outside_the_state(tmp_path, n, dtype):
    g = Guarded(n, dtype)
    try:
        x, z, th = rotation_list(n, n)
        if n >= 5:
            ham = synth.jw_hamiltonian(n, 30, n)
            hx, hz, hc = ham.x, ham.z, ham.c
        else:
            rng = np.random.default_rng(7)
            hx, hz = rng.integers(0, 1 << n, size=6), rng.integers(0, 1 << n, size=6)
            hc = rng.normal(size=6)
        capi.sv_from_host(g.sv, synth.random_state(n, 3).astype(np.complex64 if dtype == "c64" else np.complex128))
        g.check("from_host")
        for depth in range(0, 6):
            p = capi.plan_create(n, dtype, x, z, th, depth)
            try:
                capi.plan_apply(g.sv, p)
            finally:
                capi.plan_free(p)
            g.check(f"plan depth {depth}")
        capi.frame_apply_pauli(g.sv, "Y", n - 1)
        capi.apply_pauli_rotations(g.sv, x[:20], z[:20], th[:20])
        g.check("apply with a frame")
        capi.expval_pauli_sum(g.sv, hx, hz, hc)
        g.check("expval")
        capi.sv_materialize(g.sv)
        g.check("materialize")
        if n >= 2:  # the gate-decomposed path needs two qubits (SV_EUNSUPPORTED below)
            capi.apply_pauli_rotations_gates(g.sv, x[:10], z[:10], th[:10])
            g.check("gate-decomposed")
        else:
            with pytest.raises(capi.PauliRotError) as e:
                capi.apply_pauli_rotations_gates(g.sv, x[:10], z[:10], th[:10])
            assert e.value.code == capi.SV_EUNSUPPORTED
        capi.cfhs_measure_pauli(g.sv, None, int(x[0]) | 1, int(z[0]), 0.3)
        g.check("measure")
        capi.rotation_grads(g.sv, x[:30], z[:30], th[:30], hx, hz, hc)
        g.check("adjoint")
        path = str(tmp_path / "g.ckpt")
        capi.sv_save(g.sv, path, 1)
        capi.sv_load(g.sv, path)
        g.check("checkpoint load")
    finally:
        g.close()


def test_batched_launch_stays_inside_every_state():
    stream = torch.cuda.Stream()
    sh = int(stream.cuda_stream)
    sizes = [3, 9, 12, 16, 17, 18]
    with torch.cuda.stream(stream):
        guarded = [Guarded(n, "c64") for n in sizes]
    for gd in guarded:
        capi.sv_set_stream(gd.sv, sh)
    plans = []
    try:
        for k, (gd, n) in enumerate(zip(guarded, sizes)):
            rx, rz, rt = rotation_list(n, 50 + k)
            capi.sv_from_host(gd.sv, synth.random_state(n, k).astype(np.complex64))
            plans.append(capi.plan_create(n, "c64", rx, rz, rt, 4, sh))
        capi.batch_run([gd.sv for gd in guarded], plans, use_graph=True)
        capi.batch_run([gd.sv for gd in guarded], plans, use_graph=False)
        for gd in guarded:
            gd.check("batched")
    finally:
        for p in plans:
            capi.plan_free(p)
        for gd in guarded:
            gd.close()
