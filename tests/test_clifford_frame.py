"""General Clifford frames (host only, no GPU): the cliff_* calls of the library
against dense matrices.

* every frame entry and every mapped Pauli equals U^dag P U of the dense Clifford
  U (the product of the gate matrices), signs included;
* a gate stream with rotation gates emits rotations R_k such that the dense
  circuit equals U_Clifford R_m ... R_1 exactly (Eq. single_to_multirot);
* a rotation fed in its textbook gate decomposition (basis change, CNOT ladder,
  Rz, undo) emits exactly that rotation and leaves the frame at the origin;
* the inverse rotations (App. A) multiply to U up to a global phase, with at
  most 4n of them;
* malformed streams are rejected without changing the frame.
"""
import numpy as np
import pytest

import dense
from paper_2602_09020_gb300 import capi

CLIFF1 = ["h", "s", "sdg", "x", "y", "z"]
CLIFF2 = ["cnot", "cz", "swap"]
MAT1 = {"h": dense.H, "s": dense.S, "sdg": dense.SDG, "x": dense.X, "y": dense.Y, "z": dense.Z}


def gate_matrix(n, g):
    name = g[0]
    if name in MAT1:
        return dense.one_qubit(n, g[1], MAT1[name])
    if name == "cnot":
        return dense.cnot(n, g[1], g[2])
    if name == "cz":
        return dense.one_qubit(n, g[2], dense.H) @ dense.cnot(n, g[1], g[2]) @ dense.one_qubit(n, g[2], dense.H)
    if name == "swap":
        a, b = g[1], g[2]
        return dense.cnot(n, a, b) @ dense.cnot(n, b, a) @ dense.cnot(n, a, b)
    sig = {"rx": (1, 0), "ry": (1, 1), "rz": (0, 1)}[name]
    return dense.rotation(n, sig[0] << g[1], sig[1] << g[1], g[2])


def random_circuit(n, length, rng, rotations=False):
    out = []
    for _ in range(length):
        r = rng.random()
        if rotations and r < 0.25:
            out.append((["rx", "ry", "rz"][rng.integers(3)], int(rng.integers(n)), float(rng.uniform(-3, 3))))
        elif r < 0.6 or n == 1:
            out.append((CLIFF1[rng.integers(6)], int(rng.integers(n))))
        else:
            a, b = rng.choice(n, size=2, replace=False)
            out.append((CLIFF2[rng.integers(3)], int(a), int(b)))
    return out


def dense_product(n, gates):
    U = np.eye(1 << n, dtype=complex)
    for g in gates:
        U = gate_matrix(n, g) @ U
    return U


@pytest.mark.parametrize("seed", range(6))
def test_frame_matches_dense_conjugation(seed):
    n = 3
    rng = np.random.default_rng(seed)
    gates = random_circuit(n, 40, rng)
    f = capi.cliff_create(n)
    try:
        capi.cliff_apply_gates(f, gates)
        U = dense_product(n, gates)
        xs, zs = zip(*[(x, z) for x in range(1 << n) for z in range(1 << n)])
        ox, oz, sg = capi.cliff_map_paulis(f, xs, zs)
        for x, z, mx, mz, s in zip(xs, zs, ox, oz, sg):
            want = U.conj().T @ dense.pauli(n, x, z) @ U
            np.testing.assert_allclose(s * dense.pauli(n, int(mx), int(mz)), want, atol=1e-12)
        for q in range(n):
            (zx, zz, zsg), (xx, xz, xsg) = capi.cliff_entry(f, q)
            np.testing.assert_allclose(zsg * dense.pauli(n, zx, zz), U.conj().T @ dense.pauli(n, 0, 1 << q) @ U,
                                       atol=1e-12)
            np.testing.assert_allclose(xsg * dense.pauli(n, xx, xz), U.conj().T @ dense.pauli(n, 1 << q, 0) @ U,
                                       atol=1e-12)
    finally:
        capi.cliff_free(f)


@pytest.mark.parametrize("seed", range(4))
def test_rotation_gates_become_frame_rotations(seed):
    n = 4
    rng = np.random.default_rng(100 + seed)
    gates = random_circuit(n, 50, rng, rotations=True)
    f = capi.cliff_create(n)
    try:
        rx, rz, rt = capi.cliff_apply_gates(f, gates)
    finally:
        capi.cliff_free(f)
    assert len(rt) == sum(g[0] in ("rx", "ry", "rz") for g in gates)
    C = dense_product(n, gates)
    U = dense_product(n, [g for g in gates if g[0] not in ("rx", "ry", "rz")])
    V = np.eye(1 << n, dtype=complex)
    for x, z, t in zip(rx, rz, rt):
        V = dense.rotation(n, int(x), int(z), float(t)) @ V
    np.testing.assert_allclose(C, U @ V, atol=1e-12)


def staircase(x, z, theta):
    """Textbook gate decomposition of exp(-i theta/2 P) (time order)."""
    sup = [q for q in range(64) if ((x | z) >> q) & 1]
    basis = []
    for q in sup:
        if (x >> q) & 1 and (z >> q) & 1:
            basis += [("sdg", q), ("h", q)]
        elif (x >> q) & 1:
            basis += [("h", q)]
    ladder = [("cnot", a, b) for a, b in zip(sup, sup[1:])]
    undo = [("s" if g[0] == "sdg" else g[0], g[1]) for g in reversed(basis)]
    return basis + ladder + [("rz", sup[-1], theta)] + list(reversed(ladder)) + undo


@pytest.mark.parametrize("seed", range(8))
def test_gate_decomposed_rotation_returns_itself(seed):
    n = 7
    rng = np.random.default_rng(200 + seed)
    f = capi.cliff_create(n)
    try:
        for _ in range(10):
            x, z = int(rng.integers(0, 1 << n)), int(rng.integers(0, 1 << n))
            if x | z == 0:
                continue
            theta = float(rng.uniform(-3, 3))
            ox, oz, ot = capi.cliff_apply_gates(f, staircase(x, z, theta))
            assert list(ox) == [x] and list(oz) == [z] and list(ot) == [theta]
            assert capi.cliff_is_origin(f)
    finally:
        capi.cliff_free(f)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_inverse_rotations_implement_the_frame(n):
    rng = np.random.default_rng(300 + n)
    for trial in range(4):
        gates = random_circuit(n, 12 * n, rng)
        f = capi.cliff_create(n)
        try:
            capi.cliff_apply_gates(f, gates)
            x, z, t = capi.cliff_inverse_rotations(f)
            origin = capi.cliff_is_origin(f)
        finally:
            capi.cliff_free(f)
        assert len(t) <= 4 * n and (len(t) == 0) == origin
        assert np.allclose(np.abs(t), np.pi / 2)
        V = np.eye(1 << n, dtype=complex)
        for xx, zz, tt in zip(x, z, t):
            V = dense.rotation(n, int(xx), int(zz), float(tt)) @ V
        U = dense_product(n, gates)
        # equal up to a global phase
        assert abs(abs(np.trace(U.conj().T @ V)) - (1 << n)) < 1e-9


def test_circuit_then_inverse_is_origin():
    n = 6
    rng = np.random.default_rng(7)
    gates = random_circuit(n, 200, rng)
    inv = {"s": "sdg", "sdg": "s"}
    back = [(inv.get(g[0], g[0]),) + tuple(g[1:]) for g in reversed(gates)]
    f = capi.cliff_create(n)
    try:
        capi.cliff_apply_gates(f, gates)
        assert not capi.cliff_is_origin(f)
        capi.cliff_apply_gates(f, back)
        assert capi.cliff_is_origin(f)
    finally:
        capi.cliff_free(f)


def test_rejected_streams_leave_the_frame():
    f = capi.cliff_create(3)
    try:
        capi.cliff_apply_gates(f, [("h", 0), ("cnot", 0, 2)])
        before = [capi.cliff_entry(f, q) for q in range(3)]
        bad = [
            [("h", 1), ("cnot", 1, 1)],          # equal qubits
            [("s", 0), ("x", 3)],                # qubit out of range
            [("h", 2), ("rz", 0, float("nan"))],  # angle not finite
        ]
        for stream in bad:
            with pytest.raises(capi.PauliRotError) as e:
                capi.cliff_apply_gates(f, stream)
            assert e.value.code == capi.SV_EINVAL
            assert [capi.cliff_entry(f, q) for q in range(3)] == before
        with pytest.raises(capi.PauliRotError):
            capi.cliff_map_paulis(f, [8], [0])  # bit at n
    finally:
        capi.cliff_free(f)


def test_bench_gate_stream_reproduces_the_rotations():
    """The gate-level circuit bench.py feeds to the hybrid path (every rotation as
    basis changes, CNOT ladder, Rz, undo) emits exactly the original rotations
    and leaves the frame at the origin."""
    import bench
    from paper_2602_09020_gb300 import synth

    ham = synth.jw_hamiltonian(12, 60, 3)
    stream = []
    for x, z, c in zip(ham.x, ham.z, ham.c):
        bench.staircase_stream(int(x), int(z), 2 * float(c), stream)
    names = {0: "h", 1: "s", 2: "sdg", 6: "cnot", 11: "rz"}
    gates = [(names[g], q0, q1) if g == 6 else (names[g], q0, t) if g == 11 else (names[g], q0)
             for g, q0, q1, t in stream]
    f = capi.cliff_create(12)
    try:
        ox, oz, ot = capi.cliff_apply_gates(f, gates)
        assert capi.cliff_is_origin(f)
    finally:
        capi.cliff_free(f)
    keep = (ham.x | ham.z) != 0
    assert np.array_equal(ox, ham.x[keep]) and np.array_equal(oz, ham.z[keep])
    np.testing.assert_array_equal(ot, 2 * ham.c[keep])


def _anti(a, b):
    return bin((a[0] & b[1]) ^ (a[1] & b[0])).count("1") & 1


@pytest.mark.parametrize("seed", range(4))
def test_frame_stays_a_symplectic_basis_after_every_gate(seed):
    """The entries F(Z_q), F(X_q) keep the Pauli commutation relations of the
    Z_q, X_q they stand for after every gate: F(Z_i), F(Z_j) commute, F(X_i),
    F(X_j) commute, and F(Z_i), F(X_j) anticommute exactly when i = j."""
    n = 6
    rng = np.random.default_rng(400 + seed)
    f = capi.cliff_create(n)
    try:
        for g in random_circuit(n, 150, rng):
            capi.cliff_apply_gates(f, [g])
            ent = [capi.cliff_entry(f, q) for q in range(n)]
            zs = [(e[0][0], e[0][1]) for e in ent]
            xs = [(e[1][0], e[1][1]) for e in ent]
            assert all(e[0][2] in (1, -1) and e[1][2] in (1, -1) for e in ent)
            for i in range(n):
                for j in range(n):
                    assert _anti(zs[i], zs[j]) == 0 and _anti(xs[i], xs[j]) == 0
                    assert _anti(zs[i], xs[j]) == (1 if i == j else 0)
    finally:
        capi.cliff_free(f)
