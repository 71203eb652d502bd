"""Clifford-fullstate hybrid on the GPU (Sec. "Clifford-Fullstate Hybrid
Simulator"): a general Clifford frame kept on the host, the non-Clifford gates
run on the state through the rotation kernels.

Against the oracle, which applies every gate of the same circuit to a plain
statevector:
* <H> through the frame (Eq. chfsexp) matches the oracle's <H> with no phase
  freedom (complex128 to FP64 accuracy, complex64 to 1e-4);
* after cfhs_materialize (the App. A rotations) the frame is the origin and the
  amplitudes equal the oracle's up to one global phase (a Clifford frame does
  not fix it): complex128 within 1e-12 after aligning that phase, complex64 by
  infidelity;
* multi-qubit rotations through the frame, interleaved with Clifford gates.
"""
import numpy as np
import pytest
import torch

from helpers import C128_ATOL, C64_INFIDELITY, infidelity
from paper_2602_09020_gb300 import capi, synth

pytestmark = pytest.mark.gpu

CLIFF1 = ["h", "s", "sdg", "x", "y", "z"]
CLIFF2 = ["cnot", "cz", "swap"]


def random_circuit(n, length, rng, rot_frac=0.3):
    out = []
    for _ in range(length):
        r = rng.random()
        if r < rot_frac:
            out.append((["rx", "ry", "rz"][rng.integers(3)], int(rng.integers(n)), float(rng.uniform(-3, 3))))
        elif r < 0.65:
            out.append((CLIFF1[rng.integers(6)], int(rng.integers(n))))
        else:
            a, b = rng.choice(n, size=2, replace=False)
            out.append((CLIFF2[rng.integers(3)], int(a), int(b)))
    return out


def oracle_circuit(orc, n, gates, psi):
    """The same circuit as the oracle's own gates (rx = H rz H, ry = S rx S^dag,
    cz = H_b cnot H_b, swap = three cnots)."""
    for g in gates:
        name, q = g[0], g[1]
        if name in ("h", "s", "sdg", "x", "y", "z"):
            orc.gate(psi, n, name, q)
        elif name == "cnot":
            orc.gate(psi, n, "cnot", q, g[2])
        elif name == "cz":
            orc.gate(psi, n, "h", g[2])
            orc.gate(psi, n, "cnot", q, g[2])
            orc.gate(psi, n, "h", g[2])
        elif name == "swap":
            for a, b in ((q, g[2]), (g[2], q), (q, g[2])):
                orc.gate(psi, n, "cnot", a, b)
        elif name == "rz":
            orc.gate(psi, n, "rz", q, theta=g[2])
        elif name == "rx":
            orc.gate(psi, n, "h", q)
            orc.gate(psi, n, "rz", q, theta=g[2])
            orc.gate(psi, n, "h", q)
        elif name == "ry":
            orc.gate(psi, n, "sdg", q)
            orc.gate(psi, n, "h", q)
            orc.gate(psi, n, "rz", q, theta=g[2])
            orc.gate(psi, n, "h", q)
            orc.gate(psi, n, "s", q)
    return psi


def align_phase(ref, got):
    k = int(np.argmax(np.abs(ref)))
    ph = got[k] / ref[k]
    return got / (ph / abs(ph))


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("seed", [1, 2])
def test_cfhs_gate_stream_matches_oracle(orc, dtype, seed):
    n = 10
    rng = np.random.default_rng(seed)
    gates = random_circuit(n, 400, rng)
    basis = synth.hartree_fock_index(n // 2)
    ham = synth.jw_hamiltonian(n, 120, seed)
    psi = oracle_circuit(orc, n, gates, orc.basis_state(n, basis))
    e_ref = orc.expval(psi, n, ham.x, ham.z, ham.c)
    stream = torch.cuda.current_stream().cuda_stream
    sv = capi.sv_alloc(n, dtype, stream)
    f = capi.cliff_create(n)
    try:
        capi.sv_set_basis_state(sv, basis)
        capi.cfhs_apply_gates(sv, f, gates)
        e, nrm = capi.cfhs_expval(sv, f, ham.x, ham.z, ham.c)
        capi.cfhs_materialize(sv, f)
        assert capi.cliff_is_origin(f)
        got = capi.sv_to_host(sv, True).astype(np.complex128)
    finally:
        capi.cliff_free(f)
        capi.sv_free(sv)
    scale = max(1.0, np.abs(ham.c).sum())
    if dtype == "c128":
        assert abs(e - e_ref) <= 1e-12 * scale
        assert abs(nrm - 1.0) <= 1e-12
        assert np.max(np.abs(align_phase(psi, got) - psi)) <= C128_ATOL
    else:
        assert abs(e - e_ref) <= 1e-4 * scale
        assert infidelity(psi, got) <= C64_INFIDELITY


def test_cfhs_multi_qubit_rotations_through_the_frame(orc):
    n = 9
    rng = np.random.default_rng(11)
    stream = torch.cuda.current_stream().cuda_stream
    sv = capi.sv_alloc(n, "c128", stream)
    f = capi.cliff_create(n)
    psi = orc.basis_state(n, 0b101010101)
    try:
        capi.sv_set_basis_state(sv, 0b101010101)
        for _ in range(6):
            gates = random_circuit(n, 30, rng, rot_frac=0.0)
            capi.cfhs_apply_gates(sv, f, gates)
            oracle_circuit(orc, n, gates, psi)
            x = rng.integers(0, 1 << n, size=20).astype(np.uint64)
            z = rng.integers(0, 1 << n, size=20).astype(np.uint64)
            th = rng.uniform(-3, 3, size=20)
            capi.cfhs_apply_rotations(sv, f, x, z, th)
            orc.apply_rotations(psi, n, x, z, th)
        capi.cfhs_materialize(sv, f)
        got = capi.sv_to_host(sv, True)
    finally:
        capi.cliff_free(f)
        capi.sv_free(sv)
    assert np.max(np.abs(align_phase(psi, got) - psi)) <= C128_ATOL
