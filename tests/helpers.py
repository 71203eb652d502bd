"""Shared helpers for the parity tests (inputs and comparisons only)."""
import numpy as np

from paper_2602_09020_gb300 import synth

C128_ATOL = 1e-12        # complex128 amplitudes, absolute (spec tolerance)
C64_INFIDELITY = 1e-5    # complex64 states
C64_ATOL = 1e-4          # complex64 amplitudes, absolute, short sequences


def infidelity(ref: np.ndarray, got: np.ndarray) -> float:
    """1 - |<ref|got>|^2 / (<ref|ref><got|got>) in FP64."""
    r = ref.astype(np.complex128)
    g = got.astype(np.complex128)
    ov = np.vdot(r, g)
    return float(1.0 - abs(ov) ** 2 / (np.vdot(r, r).real * np.vdot(g, g).real))


def random_paulis(n: int, count: int, seed: int, span_dim=None, diag_frac: float = 0.0):
    """Random strings; with span_dim the x-masks are drawn from a random
    subspace of that dimension (so runs fuse), diag_frac of them have x = 0."""
    g = np.random.default_rng(seed)
    full = (1 << n) - 1
    if span_dim is not None:
        basis = [int(g.integers(1, full + 1)) for _ in range(span_dim)]
    xs, zs = [], []
    for _ in range(count):
        if g.random() < diag_frac:
            x = 0
        elif span_dim is not None:
            x = 0
            for b in basis:
                if g.random() < 0.5:
                    x ^= b
        else:
            x = int(g.integers(0, full + 1))
        z = int(g.integers(0, full + 1))
        if x == 0 and z == 0:
            z = 1
        xs.append(x)
        zs.append(z)
    return np.array(xs, dtype=np.uint64), np.array(zs, dtype=np.uint64)


def covering_paulis(n: int, seed: int = 0):
    """Strings that cover the layouts the kernels special-case: x with the
    lowest and highest bit, single-bit x, nY = 0..3 (mod 4), diagonal strings,
    and the identity."""
    g = np.random.default_rng(seed)
    full = (1 << n) - 1
    out = {(0, 0), (0, 1), (1, 0), (1, 1)}
    top = 1 << (n - 1)
    out |= {(top, 0), (top, top), (0, top), (top | 1, 0), (full, 0), (full, full), (0, full)}
    for q in range(n):
        out.add((1 << q, 0))
        out.add((1 << q, 1 << q))
    for target in range(4):
        for _ in range(50):
            x = int(g.integers(1, full + 1))
            z = int(g.integers(0, full + 1))
            if bin(x & z).count("1") % 4 == target:
                out.add((x, z))
                break
    for _ in range(8):
        out.add((int(g.integers(0, full + 1)), int(g.integers(0, full + 1))))
    xs = np.array([p[0] for p in sorted(out)], dtype=np.uint64)
    zs = np.array([p[1] for p in sorted(out)], dtype=np.uint64)
    return xs, zs


def assert_close_c128(ref, got, atol=C128_ATOL, what=""):
    err = float(np.max(np.abs(ref - got))) if len(ref) else 0.0
    assert err <= atol, f"{what}: max |diff| = {err:.3e} > {atol:.1e}"
    return err


def assert_close_c64(ref, got, what="", atol=C64_ATOL, infid=C64_INFIDELITY):
    err = float(np.max(np.abs(ref - got.astype(np.complex128))))
    inf = infidelity(ref, got)
    assert err <= atol and inf <= infid, f"{what}: max |diff| = {err:.3e}, infidelity = {inf:.3e}"
    return err, inf


def hf_state(n: int) -> int:
    return synth.hartree_fock_index(n // 2)
