"""Seeded synthetic workloads shared by the CUDA path, the tests and the oracle.

This module only draws inputs: Pauli strings as symplectic bit masks, real
coefficients, angles, Pauli-gate insertions and basis states.  It holds none of
the simulation arithmetic (no Trotter expansion, no rotation, no frame), so both
sides of every parity test can read it without sharing any of the method.

Conventions (paper, Sec. "Multi-qubit rotations in a fullstate simulator"):
qubit j is bit j of the amplitude index (qubit 0 is the least significant bit).
A Pauli string is a pair of n-bit masks (x, z) with X on bits x & ~z, Z on bits
z & ~x and Y on bits x & z.  Strings are printed most-significant qubit first.

The chemistry workloads of the paper (Jordan-Wigner Hamiltonians from a public
dataset, Sec. "Evaluation on Chemistry Hamiltonians") are not available; the
generators below build Jordan-Wigner-*shaped* Hamiltonians of the same kinds of
strings (number terms Z_p, Coulomb terms Z_p Z_q, hopping strings
X_p Z..Z X_q / Y_p Z..Z Y_q and the 8-string double-excitation blocks
s_p Z..Z s_q s_r Z..Z s_s) with seeded coefficients.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Tuple

import numpy as np

__all__ = [
    "PauliSum",
    "Circuit",
    "pauli_label",
    "parse_label",
    "locality",
    "jw_hamiltonian",
    "small_jw_hamiltonian",
    "small_workload",
    "random_pauli_gates",
    "adjoint_workload",
    "batch_workload",
    "random_state",
    "hartree_fock_index",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


@dataclass
class PauliSum:
    """H = sum_j c_j P_j with P_j given by symplectic masks (x_j, z_j)."""

    n: int
    x: np.ndarray  # uint64[T]
    z: np.ndarray  # uint64[T]
    c: np.ndarray  # float64[T]
    kinds: List[str] = field(default_factory=list)

    def __len__(self) -> int:
        return int(self.x.shape[0])

    def labels(self) -> List[str]:
        return [pauli_label(self.n, int(a), int(b)) for a, b in zip(self.x, self.z)]


@dataclass
class Circuit:
    """A term list plus Pauli gates interleaved at given positions.

    ``gates`` holds (position, pauli, qubit): the gate acts after the first
    ``position`` rotations of the expanded rotation list have been applied.
    """

    n: int
    ham: PauliSum
    dt: float
    steps: int
    order: int
    gates: List[Tuple[int, str, int]]
    basis_state: int


def pauli_label(n: int, x: int, z: int) -> str:
    """Most-significant-qubit-first label, e.g. 'IXZY' for n=4."""
    out = []
    for q in reversed(range(n)):
        xb, zb = (x >> q) & 1, (z >> q) & 1
        out.append("IXZY"[xb | (zb << 1)])
    return "".join(out)


def parse_label(label: str) -> Tuple[int, int]:
    """Inverse of :func:`pauli_label` (leftmost character is qubit n-1)."""
    n = len(label)
    x = z = 0
    for pos, ch in enumerate(label):
        q = n - 1 - pos
        if ch in "XY":
            x |= 1 << q
        if ch in "ZY":
            z |= 1 << q
        if ch not in "IXYZ":
            raise ValueError(f"bad Pauli character {ch!r}")
    return x, z


def locality(x: np.ndarray, z: np.ndarray) -> np.ndarray:
    """Pauli weight |P| (number of non-identity factors), Def. of locality."""
    s = np.asarray(x, dtype=np.uint64) | np.asarray(z, dtype=np.uint64)
    return np.array([bin(int(v)).count("1") for v in s], dtype=np.int64)


def _chain(lo: int, hi: int) -> int:
    """Bits lo+1 .. hi-1 (the Jordan-Wigner Z chain strictly between lo and hi)."""
    if hi - lo <= 1:
        return 0
    return ((1 << hi) - 1) & ~((1 << (lo + 1)) - 1)


def _hopping_strings(p: int, q: int) -> List[Tuple[int, int]]:
    """X_p Z..Z X_q and Y_p Z..Z Y_q (p < q)."""
    x = (1 << p) | (1 << q)
    ch = _chain(p, q)
    return [(x, ch), (x, ch | x)]


# even-Y patterns of a double excitation, sigma in {X, Y} on (p, q, r, s)
_DOUBLE_PATTERNS = [
    (0, 0, 0, 0), (0, 0, 1, 1), (0, 1, 0, 1), (0, 1, 1, 0),
    (1, 0, 0, 1), (1, 0, 1, 0), (1, 1, 0, 0), (1, 1, 1, 1),
]


def _double_strings(p: int, q: int, r: int, s: int) -> List[Tuple[int, int]]:
    """The 8 strings s_p Z..Z s_q s_r Z..Z s_s with an even number of Y's."""
    x = (1 << p) | (1 << q) | (1 << r) | (1 << s)
    ch = _chain(p, q) | _chain(r, s)
    out = []
    for pat in _DOUBLE_PATTERNS:
        y = 0
        for bit, qb in zip(pat, (p, q, r, s)):
            if bit:
                y |= 1 << qb
        out.append((x, ch | y))
    return out


def _finish(n, xs, zs, cs, kinds) -> PauliSum:
    return PauliSum(
        n=n,
        x=np.array(xs, dtype=np.uint64),
        z=np.array(zs, dtype=np.uint64),
        c=np.array(cs, dtype=np.float64),
        kinds=kinds,
    )


def small_jw_hamiltonian(n: int = 10, n_hop: int = 20, n_zz: int = 10, seed: int = 0) -> PauliSum:
    """Small JW-shaped Hamiltonian: n single Z, ``n_zz`` distinct Z_pZ_q and
    ``n_hop`` distinct hopping pairs (2 strings each), coefficients U[-1, 1].

    Emission order: all Z_p (p ascending), then the Z_pZ_q, then the hopping
    pairs with X..X immediately followed by Y..Y of the same pair.
    """
    g = _rng(seed)
    xs, zs, cs, kinds = [], [], [], []
    for p in range(n):
        xs.append(0); zs.append(1 << p); cs.append(g.uniform(-1, 1)); kinds.append("Z")
    pairs = [(p, q) for p in range(n) for q in range(p + 1, n)]
    zz = g.choice(len(pairs), size=n_zz, replace=False)
    for k in zz:
        p, q = pairs[k]
        xs.append(0); zs.append((1 << p) | (1 << q)); cs.append(g.uniform(-1, 1)); kinds.append("ZZ")
    hop = g.choice(len(pairs), size=n_hop, replace=False)
    for k in hop:
        p, q = pairs[k]
        c = g.uniform(-1, 1)
        for (x, z) in _hopping_strings(p, q):
            xs.append(x); zs.append(z); cs.append(c); kinds.append("hop")
    return _finish(n, xs, zs, cs, kinds)


def jw_hamiltonian(n: int, n_terms: int, seed: int, *, sigma: float = 0.5,
                   zz_frac: float = 0.04, hop_frac: float = 0.08) -> PauliSum:
    """JW-shaped Hamiltonian with exactly ``n_terms`` distinct strings.

    Kinds: all n single Z_p; ``zz_frac`` of the terms Z_pZ_q; ``hop_frac`` of
    the terms hopping strings (pairs X..X / Y..Y sharing one coefficient); the
    rest double-excitation blocks of 8 strings sharing one x-mask, each string
    with its own coefficient.  Coefficients are N(0, sigma^2).

    Emission order: the Z_p, then the Z_pZ_q, then the hopping pairs and
    double blocks in a seeded shuffle (each pair or block stays contiguous).
    """
    if n < 4:
        raise ValueError("need n >= 4 for double excitations")
    g = _rng(seed)
    seen = set()
    xs, zs, cs, kinds = [], [], [], []

    def emit(x, z, c, kind):
        seen.add((x, z))
        xs.append(x); zs.append(z); cs.append(c); kinds.append(kind)

    for p in range(n):
        emit(0, 1 << p, g.normal(0.0, sigma), "Z")
    pairs = [(p, q) for p in range(n) for q in range(p + 1, n)]
    n_zz = min(len(pairs), max(0, int(round(zz_frac * n_terms))))
    for k in g.choice(len(pairs), size=n_zz, replace=False):
        p, q = pairs[k]
        emit(0, (1 << p) | (1 << q), g.normal(0.0, sigma), "ZZ")
    remaining = n_terms - len(xs)
    if remaining < 0:
        raise ValueError("n_terms too small for the diagonal part")
    n_hop = min(len(pairs), (int(round(hop_frac * n_terms)) // 2))
    n_hop = min(n_hop, remaining // 2)
    groups = []
    for k in g.choice(len(pairs), size=n_hop, replace=False):
        p, q = pairs[k]
        groups.append(("hop", (p, q)))
    left = remaining - 2 * n_hop
    n_quads = n * (n - 1) * (n - 2) * (n - 3) // 24
    n_dbl = min(left // 8, n_quads // 2)
    tail = left - 8 * n_dbl
    quads = set()
    while len(quads) < n_dbl:
        quad = tuple(sorted(g.choice(n, size=4, replace=False).tolist()))
        quads.add(quad)
    for quad in sorted(quads):
        groups.append(("dbl", quad))
    order = g.permutation(len(groups))
    body = []
    for k in order:
        kind, idx = groups[k]
        if kind == "hop":
            c = g.normal(0.0, sigma)
            body.extend((x, z, c, "hop") for (x, z) in _hopping_strings(*idx))
        else:
            body.extend((x, z, g.normal(0.0, sigma), "dbl") for (x, z) in _double_strings(*idx))
    for (x, z, c, kind) in body:
        emit(x, z, c, kind)
    # pad to exactly n_terms with fresh hopping-type strings carrying one extra Z
    # (the shape of JW one-body terms dressed by a number operator)
    # (small n: any unused string once those run out)
    attempts = 0
    while tail > 0:
        attempts += 1
        if attempts > 64 * n_terms + 4096:
            raise ValueError(f"cannot draw {n_terms} distinct strings on {n} qubits")
        if attempts <= 16 * n_terms:
            p, q = sorted(g.choice(n, size=2, replace=False).tolist())
            r = int(g.integers(0, n))
            x = (1 << p) | (1 << q)
            z = _chain(p, q) ^ ((1 << r) if r not in (p, q) else 0)
            kind = "hopz"
        else:
            x, z = int(g.integers(0, 1 << n)), int(g.integers(0, 1 << n))
            kind = "any"
        if (x, z) in seen or (x == 0 and z == 0):
            continue
        emit(x, z, g.normal(0.0, sigma), kind)
        tail -= 1
    return _finish(n, xs, zs, cs, kinds)


def random_klocal_hamiltonian(n: int, n_terms: int, k: int, seed: int) -> PauliSum:
    """Random k-local Hamiltonian of the paper's locality study (Sec. "Evaluation
    on Random Hamiltonians"): n_terms distinct strings of Pauli weight exactly k,
    each drawn uniformly from the C(n, k) 3^k such strings, coefficients
    U[-1, 1] divided by their L1 norm."""
    if not 1 <= k <= n:
        raise ValueError(f"locality {k} out of range 1..{n}")
    if n_terms > math.comb(n, k) * 3 ** k:
        raise ValueError(f"only {math.comb(n, k) * 3 ** k} distinct strings of weight {k} on {n} qubits")
    g = _rng(seed)
    seen, xs, zs = set(), [], []
    while len(xs) < n_terms:
        x = z = 0
        for q in g.choice(n, size=k, replace=False):
            p = int(g.integers(3))  # 0 = X, 1 = Y, 2 = Z
            if p < 2:
                x |= 1 << int(q)
            if p > 0:
                z |= 1 << int(q)
        if (x, z) in seen:
            continue
        seen.add((x, z))
        xs.append(x)
        zs.append(z)
    c = g.uniform(-1.0, 1.0, size=n_terms)
    c = c / np.abs(c).sum()
    return PauliSum(n, np.array(xs, dtype=np.uint64), np.array(zs, dtype=np.uint64), c, [f"w{k}"] * n_terms)


def hartree_fock_index(n_electrons: int) -> int:
    """Basis index with qubits 0..n_electrons-1 occupied."""
    return (1 << n_electrons) - 1


def random_pauli_gates(n: int, count: int, n_positions: int, seed: int) -> List[Tuple[int, str, int]]:
    """``count`` Pauli gates of seeded type and qubit at uniform gaps of the
    ``n_positions`` insertion points 0..n_positions-1."""
    g = _rng(seed)
    gaps = n_positions // (count + 1)
    out = []
    for k in range(count):
        pos = gaps * (k + 1)
        out.append((pos, "XYZ"[int(g.integers(0, 3))], int(g.integers(0, n))))
    return out


def small_workload(seed: int = 0) -> Circuit:
    """n=10, complex128, HF state |0b0000011111>, 60 JW-shaped terms with
    coefficients U[-1,1], one first-order step at dt=0.1 and 5 Pauli gates
    interleaved among the 61 positions of the 60-rotation list."""
    ham = small_jw_hamiltonian(10, 20, 10, seed)
    gates = random_pauli_gates(10, 5, len(ham) + 1, seed + 1)
    return Circuit(n=10, ham=ham, dt=0.1, steps=1, order=1, gates=gates,
                   basis_state=hartree_fock_index(5))


def adjoint_workload(n: int, n_rot: int, n_obs: int, seed: int):
    """Parameterised circuit for gradients: ``n_rot`` axes taken in order from a
    JW-shaped Hamiltonian, independent angles U[-pi, pi]; observable a separate
    ``n_obs``-term JW-shaped Hamiltonian.  Returns (axes_x, axes_z, theta, obs)."""
    axes = jw_hamiltonian(n, max(n_rot, 4 * n + 8), seed)
    g = _rng(seed + 7919)
    theta = g.uniform(-np.pi, np.pi, size=n_rot)
    obs = jw_hamiltonian(n, n_obs, seed + 104729)
    return axes.x[:n_rot].copy(), axes.z[:n_rot].copy(), theta, obs


def batch_workload(n_states: int = 64, seed: int = 0, n_min: int = 12, n_max: int = 22,
                   t_min: int = 100, t_max: int = 800):
    """Independent uneven problems: n ~ U{n_min..n_max}, T ~ U{t_min..t_max},
    dt ~ U[0.01, 0.2], steps ~ U{1..8}, each with its own seeded Hamiltonian.
    Returns a list of Circuit (first-order, no interleaved gates)."""
    g = _rng(seed)
    out = []
    for k in range(n_states):
        n = int(g.integers(n_min, n_max + 1))
        T = int(g.integers(t_min, t_max + 1))
        dt = float(g.uniform(0.01, 0.2))
        steps = int(g.integers(1, 9))
        ham = jw_hamiltonian(n, T, seed * 1000 + k + 1)
        out.append(Circuit(n=n, ham=ham, dt=dt, steps=steps, order=1, gates=[],
                           basis_state=hartree_fock_index(n // 2)))
    return out


def random_state(n: int, seed: int) -> np.ndarray:
    """Normalised complex128 vector with N(0,1) real and imaginary parts."""
    g = _rng(seed)
    v = g.normal(size=1 << n) + 1j * g.normal(size=1 << n)
    return (v / np.linalg.norm(v)).astype(np.complex128)
