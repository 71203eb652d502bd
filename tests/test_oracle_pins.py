"""Pins for the CPU oracle: each check ties it to something other than itself.

* gates against the textbook matrices (dense Kronecker products),
* rotations against the closed form cos(theta/2) I - i sin(theta/2) P and
  against scipy's matrix exponential, for every Pauli string on 3 qubits,
* hand-derived values in tests/golden/closed_forms.txt,
* identities the paper states (XYZ = iI, 2(k-1) CNOTs, SWAP from pi/4 XX, YY, ZZ
  rotations, f_P an involution) and invariants (norm, inverse, R(2pi) = -I,
  R(pi) = -iP, commuting rotations commute),
* Trotter products against dense products and against exp(-iHt) with the
  convergence order (1 for the first-order product, 2 for the symmetric one),
* expectation values against dense psi^dag P psi,
* parameter-shift gradients against central finite differences and a closed form.
"""
import os

import numpy as np
import pytest
import scipy.linalg

import dense
from paper_2602_09020_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "closed_forms.txt")
RNG = np.random.default_rng(12345)


def rand_state(n, seed):
    return synth.random_state(n, seed)


# ---------------------------------------------------------------- gates

@pytest.mark.parametrize("name,mat", [("x", dense.X), ("y", dense.Y), ("z", dense.Z), ("h", dense.H),
                                      ("s", dense.S), ("sdg", dense.SDG)])
def test_one_qubit_gates_match_textbook(orc, name, mat):
    n = 3
    for q in range(n):
        psi = rand_state(n, 10 + q)
        want = dense.one_qubit(n, q, mat) @ psi
        got = orc.gate(psi.copy(), n, name, q)
        np.testing.assert_allclose(got, want, atol=1e-14, rtol=0)


def test_rz_and_cnot_match_textbook(orc):
    n = 4
    for q in range(n):
        psi = rand_state(n, 20 + q)
        np.testing.assert_allclose(orc.gate(psi.copy(), n, "rz", q, theta=0.731),
                                   dense.rz(n, q, 0.731) @ psi, atol=1e-14, rtol=0)
    for c in range(n):
        for t in range(n):
            if c == t:
                continue
            psi = rand_state(n, 30 + 4 * c + t)
            np.testing.assert_allclose(orc.gate(psi.copy(), n, "cnot", c, t),
                                       dense.cnot(n, c, t) @ psi, atol=1e-15, rtol=0)


def test_xyz_is_i_identity():
    # paper: XYZ = i I
    np.testing.assert_allclose(dense.X @ dense.Y @ dense.Z, 1j * np.eye(2), atol=0)


# ---------------------------------------------------------------- rotations

def test_every_rotation_on_three_qubits_matches_closed_form_and_expm(orc):
    n = 3
    psi0 = rand_state(n, 1)
    for x, z in dense.all_paulis(n):
        theta = float(RNG.uniform(-4 * np.pi, 4 * np.pi))
        want = dense.rotation(n, x, z, theta) @ psi0
        got = orc.apply_rotation(psi0.copy(), n, x, z, theta)
        np.testing.assert_allclose(got, want, atol=2e-14, rtol=0)
        want2 = scipy.linalg.expm(-0.5j * theta * dense.pauli(n, x, z)) @ psi0
        np.testing.assert_allclose(got, want2, atol=1e-12, rtol=0)


def test_random_rotations_on_six_qubits(orc):
    n = 6
    for s in range(40):
        x, z = int(RNG.integers(0, 64)), int(RNG.integers(0, 64))
        theta = float(RNG.normal())
        psi0 = rand_state(n, 100 + s)
        np.testing.assert_allclose(orc.apply_rotation(psi0.copy(), n, x, z, theta),
                                   dense.rotation(n, x, z, theta) @ psi0, atol=2e-14, rtol=0)


def _parse_amps(spec):
    out = {}
    for item in spec.split(";"):
        k, v = item.strip().split("=")
        re, im = v.split(",")
        out[int(k)] = complex(float(re), float(im))
    return out


def _golden_lines():
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                yield line


def test_golden_closed_forms(orc):
    n_rot = n_exp = 0
    for line in _golden_lines():
        head, tail = line.split(":", 1)
        kind, n, label, theta, k = head.split()
        n, theta, k = int(n), float(theta), int(k)
        x, z = synth.parse_label(label)
        psi = orc.basis_state(n, k)
        orc.apply_rotation(psi, n, x, z, theta)
        if kind == "rot":
            want = np.zeros(1 << n, dtype=complex)
            for kk, v in _parse_amps(tail).items():
                want[kk] = v
            np.testing.assert_allclose(psi, want, atol=1e-15, rtol=0, err_msg=line)
            n_rot += 1
        else:
            for item in tail.split(";"):
                lab, v = item.strip().split("=")
                ox, oz = synth.parse_label(lab)
                e = orc.expval(psi, n, [ox], [oz], [1.0])
                assert abs(e - float(v)) < 1e-15, (line, lab, e)
                n_exp += 1
    assert n_rot >= 10 and n_exp >= 5


def test_cnot_ladder_count(orc):
    # paper: the staircase uses 2(k-1) CNOTs for a k-local string
    n = 8
    for _ in range(50):
        x, z = int(RNG.integers(0, 256)), int(RNG.integers(0, 256))
        k = bin(x | z).count("1")
        ncnot, _, nrz = orc.rotation_gate_count(n, x, z)
        assert ncnot == (2 * (k - 1) if k else 0)
        assert nrz == (1 if k else 0)


def test_swap_from_quarter_pi_rotations(orc):
    # paper (footnote on SWAP): pi/4 rotations about X0X1, Y0Y1, Z0Z1 give SWAP up to phase;
    # exp(-i pi/4 P) is R_P(pi/2)
    n = 2
    psi0 = rand_state(n, 7)
    psi = psi0.copy()
    for lab in ("XX", "YY", "ZZ"):
        x, z = synth.parse_label(lab)
        orc.apply_rotation(psi, n, x, z, np.pi / 2)
    swapped = psi0[[0, 2, 1, 3]]
    ov = np.vdot(swapped, psi)
    assert abs(abs(ov) - 1) < 1e-14
    np.testing.assert_allclose(psi, ov * swapped, atol=1e-14)


def test_pauli_involution_and_pairing(orc):
    # f_P(f_P(k)) = k, and P^2 = I on states
    n = 5
    for _ in range(30):
        x, z = int(RNG.integers(0, 32)), int(RNG.integers(0, 32))
        psi0 = rand_state(n, 3)
        twice = orc.apply_pauli(orc.apply_pauli(psi0.copy(), n, x, z), n, x, z)
        np.testing.assert_allclose(twice, psi0, atol=1e-15)
        np.testing.assert_allclose(orc.apply_pauli(psi0.copy(), n, x, z), dense.pauli(n, x, z) @ psi0,
                                   atol=1e-15)


def test_rotation_invariants(orc):
    n = 7
    psi0 = rand_state(n, 5)
    for _ in range(12):
        x, z = int(RNG.integers(0, 128)), int(RNG.integers(0, 128))
        th = float(RNG.uniform(-3, 3))
        p = orc.apply_rotation(psi0.copy(), n, x, z, th)
        assert abs(orc.norm2(p, n) - 1) < 1e-14
        back = orc.apply_rotation(p, n, x, z, -th)
        np.testing.assert_allclose(back, psi0, atol=1e-14)
        np.testing.assert_allclose(orc.apply_rotation(psi0.copy(), n, x, z, 2 * np.pi), -psi0, atol=1e-14)
        minus_ip = -1j * orc.apply_pauli(psi0.copy(), n, x, z)
        np.testing.assert_allclose(orc.apply_rotation(psi0.copy(), n, x, z, np.pi), minus_ip, atol=1e-14)


def test_commuting_rotations_commute(orc):
    n = 6
    psi0 = rand_state(n, 9)
    found = 0
    while found < 15:
        x1, z1, x2, z2 = (int(v) for v in RNG.integers(0, 64, size=4))
        anti = bin((x1 & z2) ^ (z1 & x2)).count("1") & 1
        if anti:
            continue
        found += 1
        a = orc.apply_rotation(orc.apply_rotation(psi0.copy(), n, x1, z1, 0.4), n, x2, z2, -1.1)
        b = orc.apply_rotation(orc.apply_rotation(psi0.copy(), n, x2, z2, -1.1), n, x1, z1, 0.4)
        np.testing.assert_allclose(a, b, atol=1e-14)


def test_forward_then_reverse_returns_initial(orc):
    n = 10
    ham = synth.jw_hamiltonian(n, 120, 3)
    x, z, t = orc.trotter_rotations(ham.x, ham.z, ham.c, 0.05, 2, 1)
    psi0 = orc.basis_state(n, synth.hartree_fock_index(5))
    psi = orc.apply_rotations(psi0.copy(), n, x, z, t)
    back = orc.apply_rotations(psi, n, x[::-1], z[::-1], -t[::-1])
    np.testing.assert_allclose(back, psi0, atol=1e-13)


# ---------------------------------------------------------------- Trotter products

def _small_ham(n=6, seed=4):
    g = np.random.default_rng(seed)
    terms = set()
    while len(terms) < 10:
        x, z = int(g.integers(0, 1 << n)), int(g.integers(0, 1 << n))
        if x or z:
            terms.add((x, z))
    terms = sorted(terms)
    xs = np.array([t[0] for t in terms], dtype=np.uint64)
    zs = np.array([t[1] for t in terms], dtype=np.uint64)
    return xs, zs, g.uniform(-1, 1, size=len(terms))


def _dense_ham(n, xs, zs, cs):
    return sum(c * dense.pauli(n, int(x), int(z)) for x, z, c in zip(xs, zs, cs))


def test_trotter_product_equals_dense_product(orc):
    n = 6
    xs, zs, cs = _small_ham(n)
    psi0 = rand_state(n, 11)
    for order in (1, 2):
        rx, rz, rt = orc.trotter_rotations(xs, zs, cs, 0.07, 3, order)
        assert len(rt) == 3 * len(cs) * order
        u = np.eye(1 << n, dtype=complex)
        for x, z, t in zip(rx, rz, rt):
            u = dense.rotation(n, int(x), int(z), t) @ u
        np.testing.assert_allclose(orc.apply_rotations(psi0.copy(), n, rx, rz, rt), u @ psi0, atol=1e-13)


@pytest.mark.parametrize("order,expected", [(1, 2.0), (2, 4.0)])
def test_trotter_converges_to_expm_with_its_order(orc, order, expected):
    n = 6
    xs, zs, cs = _small_ham(n)
    psi0 = rand_state(n, 12)
    t_total = 0.4
    exact = scipy.linalg.expm(-1j * t_total * _dense_ham(n, xs, zs, cs)) @ psi0
    errs = []
    for steps in (8, 16, 32):
        rx, rz, rt = orc.trotter_rotations(xs, zs, cs, t_total / steps, steps, order)
        errs.append(np.linalg.norm(orc.apply_rotations(psi0.copy(), n, rx, rz, rt) - exact))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert abs(r1 - expected) < 0.25 * expected and abs(r2 - expected) < 0.15 * expected, errs


def test_small_workload_subcase_against_expm(orc):
    # the n=10 workload restricted to its first 6 qubits: terms supported on 0..5
    circ = synth.small_workload(0)
    keep = [(int(x) | int(z)) < 64 for x, z in zip(circ.ham.x, circ.ham.z)]
    xs, zs, cs = circ.ham.x[keep], circ.ham.z[keep], circ.ham.c[keep]
    assert len(cs) >= 8
    n = 6
    psi0 = orc.basis_state(n, 0b011111)
    hd = _dense_ham(n, xs, zs, cs)
    for steps in (1, 4):
        rx, rz, rt = orc.trotter_rotations(xs, zs, cs, 0.1 / steps, steps, 1)
        got = orc.apply_rotations(psi0.copy(), n, rx, rz, rt)
        exact = scipy.linalg.expm(-1j * 0.1 * hd) @ psi0
        # first-order bound: ||U - prod|| <= t^2/(2M) sum_{j<k} ||[h_j, h_k]||
        bound = 0.0
        mats = [c * dense.pauli(n, int(x), int(z)) for x, z, c in zip(xs, zs, cs)]
        for a in range(len(mats)):
            for b in range(a + 1, len(mats)):
                bound += np.linalg.norm(mats[a] @ mats[b] - mats[b] @ mats[a], 2)
        bound *= 0.1 ** 2 / (2 * steps)
        assert np.linalg.norm(got - exact) <= bound + 1e-14


# ---------------------------------------------------------------- expectations and gradients

def test_expval_matches_dense(orc):
    n = 6
    psi = rand_state(n, 13)
    xs, zs, cs = _small_ham(n, 8)
    e, ei = orc.expval(psi, n, xs, zs, cs, return_imag=True)
    want = np.vdot(psi, _dense_ham(n, xs, zs, cs) @ psi)
    assert abs(e - want.real) < 1e-13 and abs(ei) < 1e-13
    np.testing.assert_allclose(orc.apply_pauli_sum(psi, n, xs, zs, cs), _dense_ham(n, xs, zs, cs) @ psi,
                               atol=1e-14)


def test_gradient_closed_form_single_qubit(orc):
    # E(theta) = <0| R_X(theta)^dag Z R_X(theta) |0> = cos(theta), dE/dtheta = -sin(theta)
    for th in (0.3, -1.2, 2.9):
        e, g = orc.grad_param_shift(1, orc.basis_state(1, 0), [1], [0], [th], [0], [1], [1.0])
        assert abs(e - np.cos(th)) < 1e-15 and abs(g[0] + np.sin(th)) < 1e-15


def test_param_shift_matches_finite_differences(orc):
    n = 5
    g = np.random.default_rng(2)
    m = 12
    x = g.integers(0, 32, size=m).astype(np.uint64)
    z = g.integers(0, 32, size=m).astype(np.uint64)
    th = g.uniform(-np.pi, np.pi, size=m)
    ox, oz, oc = _small_ham(n, 3)
    psi0 = rand_state(n, 17)
    e0, grads = orc.grad_param_shift(n, psi0, x, z, th, ox, oz, oc)
    h = 1e-4
    for j in range(m):
        tp = th.copy(); tp[j] += h
        tm = th.copy(); tm[j] -= h
        ep = orc.expval(orc.apply_rotations(psi0.copy(), n, x, z, tp), n, ox, oz, oc)
        em = orc.expval(orc.apply_rotations(psi0.copy(), n, x, z, tm), n, ox, oz, oc)
        assert abs((ep - em) / (2 * h) - grads[j]) < 1e-7 * max(1.0, abs(grads[j]))


# ---------------------------------------------------------------- circuits with interleaved Pauli gates

def _dense_circuit(circ):
    """The circuit as a dense product: the Trotter rotations (Eq. trotter, theta
    = 2 c dt) in list order, and a gate (position p, Pauli, qubit) applied once
    the first p rotations have acted (the Circuit convention).  Gates at one
    position act in the order they are listed."""
    n = circ.n
    hx, hz, hc = circ.ham.x, circ.ham.z, circ.ham.c
    if circ.order != 1:
        raise ValueError("first-order circuits only")
    rots = [(int(a), int(b), 2.0 * float(c) * circ.dt) for a, b, c in zip(hx, hz, hc)] * circ.steps
    masks = {"X": (1, 0), "Y": (1, 1), "Z": (0, 1)}
    psi = np.zeros(1 << n, dtype=complex)
    psi[circ.basis_state] = 1.0
    for p in range(len(rots) + 1):
        for pos, kind, q in circ.gates:
            if pos == p:
                xb, zb = masks[kind]
                psi = dense.pauli(n, xb << q, zb << q) @ psi
        if p < len(rots):
            psi = dense.rotation(n, *rots[p]) @ psi
    return psi


def test_run_circuit_matches_dense_gate_placement(orc):
    """Pauli gates interleaved with rotations (the CFHS gate-flow workflow: gates
    and rotations act in stream order) against a dense product, with gates at the
    first and last insertion points and two at one position.  A gate moved one
    rotation later, a wrong Pauli or a swapped pair at one position fails."""
    n = 5
    g = np.random.default_rng(77)
    T = 9
    x = g.integers(0, 1 << n, size=T).astype(np.uint64)
    z = g.integers(0, 1 << n, size=T).astype(np.uint64)
    x[0] |= 1  # no pure identity, and a non-diagonal first rotation
    x[3] |= 2  # the Z gate on qubit 1 at position 3 anticommutes with rotation 3
    ham = synth.PauliSum(n, x, z, g.uniform(-1.0, 1.0, size=T))
    L = 2 * T  # two first-order steps
    gates = [(0, "Y", 2), (0, "X", 0), (3, "Z", 1), (T, "Y", 4), (T + 1, "X", 3), (L, "Z", 0), (L, "Y", 1)]
    circ = synth.Circuit(n=n, ham=ham, dt=0.37, steps=2, order=1, gates=gates, basis_state=0b00101)
    want = _dense_circuit(circ)
    got = orc.run_circuit(circ)
    np.testing.assert_allclose(got, want, atol=1e-13, rtol=0)
    kind, sx, sz, st = orc.circuit_sequence(circ)
    assert len(kind) == L + len(gates) and int(kind.sum()) == len(gates)
    assert list(kind[:3]) == [1, 1, 0] and list(kind[-3:]) == [0, 1, 1]
    # moving one gate one rotation later changes the state (the check is sensitive)
    moved = synth.Circuit(n=n, ham=ham, dt=0.37, steps=2, order=1,
                          gates=[(4 if p == 3 else p, k, q) for p, k, q in gates], basis_state=0b00101)
    assert np.max(np.abs(_dense_circuit(moved) - want)) > 1e-3


def test_run_circuit_small_workload_recipe_against_dense(orc):
    """The small workload's recipe (JW-shaped terms, one first-order step at
    dt = 0.1, 5 seeded Pauli gates at uniform gaps, Hartree-Fock state) at
    n = 6, where the dense product is cheap."""
    ham = synth.small_jw_hamiltonian(6, 6, 4, 3)
    sub = synth.Circuit(n=6, ham=ham, dt=0.1, steps=1, order=1,
                        gates=synth.random_pauli_gates(6, 5, len(ham) + 1, 4),
                        basis_state=synth.hartree_fock_index(3))
    np.testing.assert_allclose(orc.run_circuit(sub), _dense_circuit(sub), atol=1e-13, rtol=0)


# ---------------------------------------------------------------- the generators (inputs, not arithmetic)

def test_generators_are_seeded_and_well_formed():
    h1 = synth.jw_hamiltonian(24, 2000, 1)
    h2 = synth.jw_hamiltonian(24, 2000, 1)
    assert np.array_equal(h1.x, h2.x) and np.array_equal(h1.c, h2.c)
    assert len(h1) == 2000 and len(set(zip(h1.x.tolist(), h1.z.tolist()))) == 2000
    assert int(np.max(h1.x | h1.z)) < (1 << 24)
    L = synth.locality(h1.x, h1.z)
    assert 10.5 < L.mean() < 12.5 and 4.0 < L.std() < 6.0
    circ = synth.small_workload(0)
    assert len(circ.ham) == 60 and len(circ.gates) == 5 and circ.basis_state == 0b11111


def test_random_klocal_generator():
    """Sec. "Evaluation on Random Hamiltonians": distinct strings of weight exactly
    k, coefficients of L1 norm 1, seeded."""
    for k in (2, 4, 12, 24):
        h = synth.random_klocal_hamiltonian(24, 100, k, seed=5)
        assert len(h) == 100 and len(set(zip(h.x.tolist(), h.z.tolist()))) == 100
        assert set(synth.locality(h.x, h.z).tolist()) == {k}
        assert abs(np.abs(h.c).sum() - 1.0) < 1e-12
        assert int(np.max(h.x | h.z)) < (1 << 24)
        g = synth.random_klocal_hamiltonian(24, 100, k, seed=5)
        assert np.array_equal(h.x, g.x) and np.array_equal(h.z, g.z) and np.array_equal(h.c, g.c)
    assert len(synth.random_klocal_hamiltonian(24, 72, 1, seed=5)) == 72  # every weight-1 string
    for args in ((8, 10, 9), (24, 73, 1)):  # k > n; more strings than exist
        with pytest.raises(ValueError):
            synth.random_klocal_hamiltonian(*args, seed=0)
