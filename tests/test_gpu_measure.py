"""Pauli measurement and qubit preparation (App. "Complete workflow of the hybrid
Clifford fullstate simulation": Meas and Prep on the frame-rewritten axis).

The reference is the oracle's state with the plain definition of a projective
measurement: p_+ = (1 + <P>/<psi|psi>)/2 from the oracle's <P>, outcome +1 iff
u < p_+, post-state (psi + s P psi)/(2 sqrt(p_s <psi|psi>)) with P psi applied
gate-wise by the oracle; preparation flips a -1 outcome with Z (X or Y axis) or
X (Z axis).
"""
import numpy as np
import pytest
import torch

from helpers import C128_ATOL, C64_INFIDELITY, infidelity
from paper_2602_09020_gb300 import capi, synth

pytestmark = pytest.mark.gpu

CLIFF1 = ["h", "s", "sdg", "x", "y", "z"]


def oracle_measure(orc, n, psi, x, z, u):
    e = orc.expval(psi, n, [x], [z], [1.0])
    nrm = orc.norm2(psi, n)
    p_plus = min(1.0, max(0.0, 0.5 * (1.0 + e / nrm)))
    s = 1 if u < p_plus else -1
    p = p_plus if s > 0 else 1.0 - p_plus
    if p <= 1e-14:
        s, p = -s, 1.0 - p
    ppsi = orc.apply_pauli(psi.copy(), n, x, z)
    psi[:] = (psi + s * ppsi) * (0.5 / np.sqrt(p * nrm))
    return s, p


def oracle_prepare(orc, n, psi, q, axis, u):
    x = (1 << q) if axis in "XY" else 0
    z = (1 << q) if axis in "YZ" else 0
    s, _ = oracle_measure(orc, n, psi, x, z, u)
    if s < 0:
        orc.gate(psi, n, "z" if axis in "XY" else "x", q)
    return s


def clifford_circuit(n, length, rng):
    out = []
    for _ in range(length):
        r = rng.random()
        if r < 0.25:
            out.append(("rz", int(rng.integers(n)), float(rng.uniform(-3, 3))))
        elif r < 0.6:
            out.append((CLIFF1[rng.integers(6)], int(rng.integers(n))))
        else:
            a, b = rng.choice(n, size=2, replace=False)
            out.append(("cnot", int(a), int(b)))
    return out


def oracle_circuit(orc, n, gates, psi):
    for g in gates:
        if g[0] == "rz":
            orc.gate(psi, n, "rz", g[1], theta=g[2])
        elif g[0] == "cnot":
            orc.gate(psi, n, "cnot", g[1], g[2])
        else:
            orc.gate(psi, n, g[0], g[1])
    return psi


def align_phase(ref, got):
    k = int(np.argmax(np.abs(ref)))
    ph = got[k] / ref[k]
    return got / (ph / abs(ph))


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_measurements_on_a_state_with_a_pauli_frame(orc, dtype):
    n = 10
    rng = np.random.default_rng(5)
    psi = synth.random_state(n, 17)
    stream = torch.cuda.current_stream().cuda_stream
    sv = capi.sv_alloc(n, dtype, stream)
    try:
        capi.sv_from_host(sv, psi.astype(np.complex64 if dtype == "c64" else np.complex128))
        for p, q in (("X", 3), ("Y", 5), ("Z", 0)):
            capi.frame_apply_pauli(sv, p, q)
            orc.gate(psi, n, p.lower(), q)
        tol = 1e-12 if dtype == "c128" else 1e-5
        for _ in range(8):
            x, z = int(rng.integers(0, 1 << n)), int(rng.integers(0, 1 << n))
            p_plus = 0.5 * (1.0 + orc.expval(psi, n, [x], [z], [1.0]) / orc.norm2(psi, n))
            u = float(rng.random())
            while abs(u - p_plus) < 1e-3:  # keep the draw away from the outcome boundary
                u = float(rng.random())
            s_ref, p_ref = oracle_measure(orc, n, psi, x, z, u)
            s, p = capi.cfhs_measure_pauli(sv, None, x, z, u)
            assert s == s_ref and abs(p - p_ref) <= tol
        got = capi.sv_to_host(sv, True).astype(np.complex128)
    finally:
        capi.sv_free(sv)
    if dtype == "c128":
        assert np.max(np.abs(got - psi)) <= C128_ATOL
    else:
        assert infidelity(psi, got) <= C64_INFIDELITY


def test_measure_and_prepare_through_a_clifford_frame(orc):
    n = 9
    rng = np.random.default_rng(8)
    stream = torch.cuda.current_stream().cuda_stream
    sv = capi.sv_alloc(n, "c128", stream)
    f = capi.cliff_create(n)
    psi = orc.basis_state(n, 0)
    try:
        capi.sv_set_basis_state(sv, 0)
        for _ in range(5):
            gates = clifford_circuit(n, 60, rng)
            capi.cfhs_apply_gates(sv, f, gates)
            oracle_circuit(orc, n, gates, psi)
            x, z, u = int(rng.integers(1, 1 << n)), int(rng.integers(0, 1 << n)), float(rng.random())
            s_ref, p_ref = oracle_measure(orc, n, psi, x, z, u)
            s, p = capi.cfhs_measure_pauli(sv, f, x, z, u)
            assert s == s_ref and abs(p - p_ref) <= 1e-12
            q, axis, u = int(rng.integers(n)), "XYZ"[rng.integers(3)], float(rng.random())
            s_ref = oracle_prepare(orc, n, psi, q, axis, u)
            assert capi.cfhs_prepare_qubit(sv, f, q, axis, u) == s_ref
            # the prepared qubit is in the +1 eigenstate of its axis
            mx = (1 << q) if axis in "XY" else 0
            mz = (1 << q) if axis in "YZ" else 0
            e, _ = capi.cfhs_expval(sv, f, [mx], [mz], [1.0])
            assert abs(e - 1.0) <= 1e-12
        capi.cfhs_materialize(sv, f)
        got = capi.sv_to_host(sv, True)
    finally:
        capi.cliff_free(f)
        capi.sv_free(sv)
    assert np.max(np.abs(align_phase(psi, got) - psi)) <= C128_ATOL


def test_deterministic_outcomes_and_preparation():
    n = 6
    stream = torch.cuda.current_stream().cuda_stream
    sv = capi.sv_alloc(n, "c128", stream)
    try:
        capi.sv_set_basis_state(sv, 0b000100)
        # an eigenstate: the outcome does not depend on u
        for u in (0.0, 0.5, 0.999999):
            assert capi.cfhs_measure_pauli(sv, None, 0, 0b000100, u) == (-1, 1.0)
            assert capi.cfhs_measure_pauli(sv, None, 0, 0b000001, u) == (1, 1.0)
        s, p = capi.cfhs_measure_pauli(sv, None, 0b000001, 0, 0.25)  # X on |0>: a fair coin
        assert s == 1 and abs(p - 0.5) <= 1e-15
        capi.sv_set_basis_state(sv, 0b000100)
        assert capi.cfhs_prepare_qubit(sv, None, 2, "Z", 0.3) == -1
        want = np.zeros(1 << n, dtype=np.complex128)
        want[0] = 1.0
        assert np.max(np.abs(capi.sv_to_host(sv, True) - want)) <= 1e-15
    finally:
        capi.sv_free(sv)


def test_rejected_arguments_leave_the_state():
    n = 5
    stream = torch.cuda.current_stream().cuda_stream
    sv = capi.sv_alloc(n, "c128", stream)
    try:
        capi.sv_from_host(sv, synth.random_state(n, 3))
        before = capi.sv_to_host(sv, True)
        for args in ((1, 0, 1.0), (1, 0, -0.1), (1, 0, float("nan")), (1 << n, 0, 0.5), (0, 1 << 7, 0.5)):
            with pytest.raises(capi.PauliRotError) as e:
                capi.cfhs_measure_pauli(sv, None, *args)
            assert e.value.code == capi.SV_EINVAL
        for q, axis in ((n, "Z"), (-1, "X"), (0, "W")):
            with pytest.raises(capi.PauliRotError):
                capi.cfhs_prepare_qubit(sv, None, q, axis, 0.5)
        f = capi.cliff_create(n + 1)
        try:
            with pytest.raises(capi.PauliRotError):
                capi.cfhs_measure_pauli(sv, f, 1, 0, 0.5)
        finally:
            capi.cliff_free(f)
        np.testing.assert_array_equal(capi.sv_to_host(sv, True), before)
    finally:
        capi.sv_free(sv)
