"""Parity at the maximum state sizes (n = 34 complex64, n = 33 complex128: 128 GiB
each), where every kernel runs its 64-bit-index instantiation.

The rotations act on a register of 12 "active" qubits that includes the top
ones; the other qubits hold fixed bits, and some z-masks reach one of them, so
those rotations pick up the sign of its bit.  The state therefore stays
|fixed> (x) |12-qubit state>, whose 4096 amplitudes are gathered on the device
and compared with the oracle at n = 12 (qubit j of the oracle = active[j]),
together with <H> of a Hamiltonian on the same register.  The list holds a
stretch of Z / ZZ strings (a diagonal phase-sum run) between random strings,
and Pauli gates on the register go into the frame first (the oracle applies
them as gates); the launch trace shows the diagonal pass and, for complex64,
the two-run pass ran.
"""
import numpy as np
import pytest
import torch

from helpers import C128_ATOL, C64_INFIDELITY, infidelity
from paper_2602_09020_gb300 import capi

pytestmark = pytest.mark.gpu


def embed(v: int, active) -> int:
    out = 0
    for j, q in enumerate(active):
        if (v >> j) & 1:
            out |= 1 << q
    return out


@pytest.mark.parametrize("n,dtype", [(34, "c64"), (33, "c128")])
def test_maximum_size_register_against_oracle(orc, n, dtype):
    active = [0, 1, 2, 3, 4, 5, 6, 7, n - 4, n - 3, n - 2, n - 1]
    m = len(active)
    outside = 20  # a fixed qubit some z-masks touch; its bit is 1
    fixed = (1 << outside) | (1 << 12) | (1 << 25)
    rng = np.random.default_rng(n)
    count = 80
    xo = rng.integers(0, 1 << m, size=count)
    xo[rng.random(count) < 0.2] = 0  # some diagonal rotations
    zo = rng.integers(0, 1 << m, size=count)
    # a diagonal stretch in the middle: every Z_j and Z_j Z_{j+1} on the register
    zd = [1 << j for j in range(m)] + [(3 << j) for j in range(m - 1)]
    half = count // 2
    xo = np.concatenate([xo[:half], np.zeros(len(zd), dtype=xo.dtype), xo[half:]])
    zo = np.concatenate([zo[:half], np.array(zd, dtype=zo.dtype), zo[half:]])
    count = len(xo)
    th = rng.uniform(-3, 3, size=count)
    touch = rng.random(count) < 0.5
    X = np.array([embed(int(v), active) for v in xo], dtype=np.uint64)
    Z = np.array([embed(int(v), active) | ((1 << outside) if t else 0) for v, t in zip(zo, touch)], dtype=np.uint64)
    th_oracle = np.where(touch, -th, th)  # Z on a qubit holding 1 flips the rotation's sign
    b0 = int(rng.integers(0, 1 << m))
    hx = rng.integers(0, 1 << m, size=40)
    hz = rng.integers(0, 1 << m, size=40)
    hc = rng.normal(size=40)
    HX = np.array([embed(int(v), active) for v in hx], dtype=np.uint64)
    HZ = np.array([embed(int(v), active) for v in hz], dtype=np.uint64)

    gates = [("X", m - 1), ("Z", m - 3), ("Y", 0), ("X", m - 2)]  # (Pauli, register qubit)
    psi = orc.basis_state(m, b0)
    for p, j in gates:
        orc.gate(psi, m, p.lower(), j)
    orc.apply_rotations(psi, m, xo.astype(np.uint64), zo.astype(np.uint64), th_oracle)
    e_ref = orc.expval(psi, m, hx.astype(np.uint64), hz.astype(np.uint64), hc)

    amp_dt = torch.complex64 if dtype == "c64" else torch.complex128
    t = torch.empty(1 << n, dtype=amp_dt, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    sv = capi.sv_wrap(t.data_ptr(), n, dtype, stream)
    try:
        capi.sv_set_basis_state(sv, fixed | embed(b0, active))
        for p, j in gates:
            capi.frame_apply_pauli(sv, p, active[j])
        capi.sv_trace_start(sv)
        capi.apply_pauli_rotations(sv, X, Z, th)
        rows = capi.sv_trace_stop(sv)
        e, nrm = capi.expval_pauli_sum(sv, HX, HZ, hc)
        capi.sv_materialize(sv)
        torch.cuda.synchronize()
        idx = torch.tensor([fixed | embed(j, active) for j in range(1 << m)], device="cuda")
        got = t[idx].cpu().numpy().astype(np.complex128)
    finally:
        capi.sv_free(sv)
        del t
        torch.cuda.empty_cache()
    assert rows.get("k_diag_sum", (0,))[0] >= 1, rows
    if dtype == "c64":
        assert rows.get("k_chain2", (0,))[0] >= 1, rows
    # nothing leaked outside the register: its amplitudes carry the whole norm
    assert abs(nrm - float(np.vdot(got, got).real)) <= (1e-12 if dtype == "c128" else 1e-5)
    if dtype == "c128":
        assert np.max(np.abs(got - psi)) <= C128_ATOL
        assert abs(e - e_ref) <= 1e-12 * max(1.0, np.abs(hc).sum())
        assert abs(nrm - 1.0) <= 1e-12
    else:
        assert infidelity(psi, got) <= C64_INFIDELITY
        assert abs(e - e_ref) <= 1e-4 * max(1.0, np.abs(hc).sum())
