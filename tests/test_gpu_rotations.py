"""GPU parity of the rotation path against the FP64 oracle, through the C ABI.

Covers: every mask layout the kernels special-case at n = 1..12, fused runs of
every span dimension 0..5 with ragged lengths, long diagonal phase-sum runs,
angles outside [-pi/2, pi/2] (reduction into the frame) and beyond 2 pi, the
Pauli frame with interleaved gates, and the n = 10 workload with its 6-qubit
expm sub-case.  complex128 to 1e-12 absolute, complex64 by infidelity.
"""
import numpy as np
import pytest
import scipy.linalg

from helpers import (C128_ATOL, assert_close_c128, assert_close_c64, covering_paulis, infidelity,
                     random_paulis)
from paper_2602_09020_gb300 import capi, synth

pytestmark = pytest.mark.gpu


def run_gpu(n, dtype, psi0, x, z, theta, depth=-1):
    sv = capi.sv_alloc(n, dtype)
    try:
        capi.sv_from_host(sv, psi0)
        plan = capi.plan_create(n, dtype, x, z, theta, depth)
        try:
            capi.plan_apply(sv, plan)
            stats = capi.plan_stats(plan)
        finally:
            capi.plan_free(plan)
        return capi.sv_to_host(sv, True), stats
    finally:
        capi.sv_free(sv)


def run_oracle(orc, n, psi0, x, z, theta):
    return orc.apply_rotations(psi0.astype(np.complex128).copy(), n, x, z, theta)


@pytest.mark.parametrize("n", list(range(1, 13)))
def test_single_rotations_every_layout(orc, n):
    xs, zs = covering_paulis(n, seed=n)
    g = np.random.default_rng(100 + n)
    psi0 = synth.random_state(n, 7 + n)
    for x, z in zip(xs, zs):
        th = np.array([g.uniform(-7.0, 7.0)])
        want = run_oracle(orc, n, psi0, [x], [z], th)
        got, _ = run_gpu(n, "c128", psi0, [x], [z], th)
        assert_close_c128(want, got, what=f"n={n} x={int(x):#x} z={int(z):#x} theta={th[0]:.3f}")
        got64, _ = run_gpu(n, "c64", psi0.astype(np.complex64), [x], [z], th)
        assert_close_c64(want, got64, what=f"c64 n={n} x={int(x):#x} z={int(z):#x}")


@pytest.mark.parametrize("depth", [0, 1, 2, 3, 4, 5])
@pytest.mark.parametrize("n", [5, 9, 12])
def test_fused_runs_match_oracle(orc, n, depth):
    psi0 = synth.random_state(n, 40 + n)
    for count, span, diag in [(1, 1, 0.0), (7, 2, 0.2), (33, 3, 0.1), (130, 5, 0.05), (300, None, 0.3)]:
        x, z = random_paulis(n, count, seed=count * 31 + n, span_dim=span, diag_frac=diag)
        th = np.random.default_rng(count).uniform(-np.pi, np.pi, size=count)
        want = run_oracle(orc, n, psi0, x, z, th)
        got, stats = run_gpu(n, "c128", psi0, x, z, th, depth)
        assert_close_c128(want, got, what=f"n={n} depth={depth} count={count} span={span}")
        got64, _ = run_gpu(n, "c64", psi0.astype(np.complex64), x, z, th, depth)
        # longer sequences accumulate FP32 rounding: scale the amplitude bound
        assert_close_c64(want, got64, what=f"c64 n={n} depth={depth} count={count}",
                         atol=1e-4 * max(1.0, count / 50))


def test_fusion_reduces_passes():
    n = 12
    x, z = random_paulis(n, 200, seed=5, span_dim=3)
    th = np.full(200, 0.1)
    for depth, bound in [(0, 200), (3, 1)]:
        p = capi.plan_create(n, "c128", x, z, th, depth)
        nrot, nruns, _ = capi.plan_stats(p)
        capi.plan_free(p)
        assert nrot == 200 and nruns <= bound


@pytest.mark.parametrize("n", [9, 11, 14])
def test_diagonal_phase_sum_runs(orc, n):
    g = np.random.default_rng(n)
    count = 700
    x = np.zeros(count, dtype=np.uint64)
    z = g.integers(1, 1 << n, size=count).astype(np.uint64)
    th = g.uniform(-9, 9, size=count)
    # interleave a non-diagonal rotation so the run is split in two stretches
    x[350] = 3
    psi0 = synth.random_state(n, 3)
    p = capi.plan_create(n, "c128", x, z, th, -1)
    _, nruns, ndiag = capi.plan_stats(p)
    capi.plan_free(p)
    assert ndiag >= 2
    want = run_oracle(orc, n, psi0, x, z, th)
    got, _ = run_gpu(n, "c128", psi0, x, z, th)
    assert_close_c128(want, got, what=f"diag n={n}")
    got64, _ = run_gpu(n, "c64", psi0.astype(np.complex64), x, z, th)
    assert_close_c64(want, got64, what=f"c64 diag n={n}", atol=2e-4)


@pytest.mark.parametrize("kind", ["distinct", "zz"])
def test_diagonal_runs_cut_at_the_pattern_cap(orc, kind):
    # a diagonal run holds at most 128 distinct z patterns on index bits 0..8
    # (its rotations are grouped by pattern); longer stretches become several runs
    n = 12
    g = np.random.default_rng(21)
    if kind == "distinct":
        count = 400
        z = np.array([(j % 511) + 1 + (int(g.integers(0, 8)) << 9) for j in range(count)], dtype=np.uint64)
        want_runs = 4
    else:  # every Z_p and Z_p Z_q, as in a Jordan-Wigner Hamiltonian's number terms
        z = [1 << p for p in range(n)] + [(1 << p) | (1 << q) for p in range(n) for q in range(p + 1, n)]
        z = np.array(z, dtype=np.uint64)
        count = len(z)
        want_runs = 1
    x = np.zeros(count, dtype=np.uint64)
    th = g.uniform(-5, 5, size=count)
    psi0 = synth.random_state(n, 4)
    p = capi.plan_create(n, "c128", x, z, th, -1)
    _, nruns, ndiag = capi.plan_stats(p)
    capi.plan_free(p)
    assert ndiag == nruns == want_runs
    want = run_oracle(orc, n, psi0, x, z, th)
    got, _ = run_gpu(n, "c128", psi0, x, z, th)
    assert_close_c128(want, got, what=f"diag {kind}")
    got64, _ = run_gpu(n, "c64", psi0.astype(np.complex64), x, z, th)
    assert_close_c64(want, got64, what=f"c64 diag {kind}", atol=2e-4)


def test_identity_strings_are_global_phase(orc):
    n = 6
    psi0 = synth.random_state(n, 1)
    x = np.array([0, 5, 0, 0], dtype=np.uint64)
    z = np.array([0, 3, 0, 6], dtype=np.uint64)
    th = np.array([0.7, -0.4, 11.0, 1.9])
    want = run_oracle(orc, n, psi0, x, z, th)
    got, _ = run_gpu(n, "c128", psi0, x, z, th)
    assert_close_c128(want, got, what="identity")


def test_empty_rotation_list_is_noop():
    n = 7
    psi0 = synth.random_state(n, 2)
    got, stats = run_gpu(n, "c128", psi0, [], [], [])
    assert stats[1] == 0
    np.testing.assert_array_equal(got, psi0)


def _frame_sequence(orc, n, seed, n_rot=120, n_gates=25):
    g = np.random.default_rng(seed)
    x, z = random_paulis(n, n_rot, seed=seed, span_dim=4, diag_frac=0.2)
    th = g.uniform(-4, 4, size=n_rot)
    gate_pos = sorted(g.integers(0, n_rot + 1, size=n_gates).tolist())
    gates = [(p, "XYZ"[int(g.integers(0, 3))], int(g.integers(0, n))) for p in gate_pos]
    return x, z, th, gates


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_pauli_frame_with_interleaved_gates(orc, dtype):
    n = 10
    x, z, th, gates = _frame_sequence(orc, n, 11)
    psi0 = synth.random_state(n, 12)
    # oracle: gates as gates
    want = psi0.copy()
    gi = 0
    pm = {"X": (1, 0), "Y": (1, 1), "Z": (0, 1)}
    for j in range(len(th) + 1):
        while gi < len(gates) and gates[gi][0] == j:
            _, p, q = gates[gi]
            orc.apply_pauli(want, n, pm[p][0] << q, pm[p][1] << q)
            gi += 1
        if j < len(th):
            orc.apply_rotation(want, n, int(x[j]), int(z[j]), th[j])
    # GPU: gates into the frame, rotations in chunks between them
    sv = capi.sv_alloc(n, dtype)
    capi.sv_from_host(sv, psi0.astype(np.complex64 if dtype == "c64" else np.complex128))
    start = 0
    gi = 0
    for j in range(len(th) + 1):
        while gi < len(gates) and gates[gi][0] == j:
            if j > start:
                capi.apply_pauli_rotations(sv, x[start:j], z[start:j], th[start:j])
                start = j
            capi.frame_apply_pauli(sv, gates[gi][1], gates[gi][2])
            gi += 1
    capi.apply_pauli_rotations(sv, x[start:], z[start:], th[start:])
    # expectation through the frame equals the oracle's on the materialised state
    hx, hz = random_paulis(n, 30, seed=3)
    hc = np.random.default_rng(4).normal(size=30)
    e_gpu, norm = capi.expval_pauli_sum(sv, hx, hz, hc)
    e_ref = orc.expval(want, n, hx, hz, hc)
    got = capi.sv_to_host(sv, True)
    assert capi.frame_get(sv) == (0, 0, 0)
    capi.sv_free(sv)
    if dtype == "c128":
        assert_close_c128(want, got, what="frame")
        assert abs(e_gpu - e_ref) < 1e-11 and abs(norm - 1) < 1e-12
    else:
        assert_close_c64(want, got, what="frame c64", atol=2e-4)
        assert abs(e_gpu - e_ref) < 1e-4


def test_small_workload_against_oracle_and_expm(orc):
    circ = synth.small_workload(0)
    n = circ.n
    want = orc.run_circuit(circ)
    rx, rz, rt = capi.trotter_expand(circ.ham.x, circ.ham.z, circ.ham.c, circ.dt, circ.steps, 1, False)
    for dtype in ("c128", "c64"):
        sv = capi.sv_alloc(n, dtype)
        capi.sv_set_basis_state(sv, circ.basis_state)
        start = 0
        for pos, p, q in sorted(circ.gates):
            capi.apply_pauli_rotations(sv, rx[start:pos], rz[start:pos], rt[start:pos])
            capi.frame_apply_pauli(sv, p, q)
            start = pos
        capi.apply_pauli_rotations(sv, rx[start:], rz[start:], rt[start:])
        e_gpu, norm = capi.expval_pauli_sum(sv, circ.ham.x, circ.ham.z, circ.ham.c)
        got = capi.sv_to_host(sv, True)
        capi.sv_free(sv)
        e_ref = orc.expval(want, n, circ.ham.x, circ.ham.z, circ.ham.c)
        if dtype == "c128":
            assert_close_c128(want, got, what="small workload")
            assert abs(e_gpu - e_ref) < 1e-12
        else:
            assert_close_c64(want, got, what="small workload c64")
            assert abs(e_gpu - e_ref) < 1e-5
    # 6-qubit sub-case: the terms on qubits 0..5, against exp(-i H dt)
    keep = [(int(a) | int(b)) < 64 for a, b in zip(circ.ham.x, circ.ham.z)]
    xs, zs, cs = circ.ham.x[keep], circ.ham.z[keep], circ.ham.c[keep]
    m = 6
    import dense
    hd = sum(c * dense.pauli(m, int(a), int(b)) for a, b, c in zip(xs, zs, cs))
    psi0 = orc.basis_state(m, 0b011111)
    steps = 64
    rx, rz, rt = capi.trotter_expand(xs, zs, cs, circ.dt / steps, steps, 2, True)
    got, _ = run_gpu(m, "c128", psi0, rx, rz, rt)
    exact = scipy.linalg.expm(-1j * circ.dt * hd) @ psi0
    assert np.linalg.norm(got - exact) < 1e-6


def test_large_angles_and_inverse_sequence(orc):
    n = 13
    x, z = random_paulis(n, 400, seed=9, span_dim=4, diag_frac=0.25)
    th = np.random.default_rng(9).uniform(-20, 20, size=400)
    psi0 = synth.random_state(n, 9)
    sv = capi.sv_alloc(n, "c128")
    capi.sv_from_host(sv, psi0)
    capi.apply_pauli_rotations(sv, x, z, th)
    mid = capi.sv_to_host(sv, True)
    want = run_oracle(orc, n, psi0, x, z, th)
    assert_close_c128(want, mid, what="large angles")
    capi.apply_pauli_rotations(sv, x[::-1], z[::-1], -th[::-1])
    back = capi.sv_to_host(sv, True)
    capi.sv_free(sv)
    assert_close_c128(psi0, back, what="inverse")


def test_second_order_trotter_merge_is_exact(orc):
    n = 8
    ham = synth.jw_hamiltonian(n, 40, 2)
    rx, rz, rt = orc.trotter_rotations(ham.x, ham.z, ham.c, 0.05, 3, 2)
    mx, mz, mt = capi.trotter_expand(ham.x, ham.z, ham.c, 0.05, 3, 2, True)
    assert len(mt) == 3 * (2 * 40 - 1) - 2
    psi0 = orc.basis_state(n, 15)
    want = run_oracle(orc, n, psi0, rx, rz, rt)
    got, _ = run_gpu(n, "c128", psi0, mx, mz, mt)
    assert_close_c128(want, got, what="strang merged")


def test_gate_decomposed_path_matches_oracle(orc):
    n = 9
    x, z = random_paulis(n, 40, seed=21, diag_frac=0.2)
    th = np.random.default_rng(21).uniform(-3, 3, size=40)
    psi0 = synth.random_state(n, 21)
    want = run_oracle(orc, n, psi0, x, z, th)
    for dtype in ("c128", "c64"):
        sv = capi.sv_alloc(n, dtype)
        capi.sv_from_host(sv, psi0.astype(np.complex64 if dtype == "c64" else np.complex128))
        capi.frame_apply_pauli(sv, "Y", 3)   # frame signs apply to this path too
        capi.frame_apply_pauli(sv, "Y", 3)
        ngates = capi.apply_pauli_rotations_gates(sv, x, z, th)
        got = capi.sv_to_host(sv, True)
        capi.sv_free(sv)
        # Y Y = I, so the frame is the identity with phase i^2 * ... = +1
        if dtype == "c128":
            assert_close_c128(want, got, what="gates")
        else:
            assert_close_c64(want, got, what="gates c64")
    expect = 0
    for a, b in zip(x, z):
        k = bin(int(a) | int(b)).count("1")
        nxy = bin(int(a)).count("1")
        ny = bin(int(a) & int(b)).count("1")
        expect += (2 * (k - 1) + 1 + 2 * nxy + 2 * ny) if k else 1
    assert ngates == expect


def test_invalid_inputs_fail_without_side_effects():
    n = 6
    sv = capi.sv_alloc(n, "c128")
    with pytest.raises(capi.PauliRotError) as e:
        capi.apply_pauli_rotations(sv, [1 << n], [0], [0.1])
    assert e.value.code == capi.SV_EINVAL
    with pytest.raises(capi.PauliRotError) as e:
        capi.apply_pauli_rotations(sv, [1], [0], [float("nan")])
    assert e.value.code == capi.SV_EINVAL
    with pytest.raises(capi.PauliRotError) as e:
        capi.frame_apply_pauli(sv, "Q", 0)
    assert e.value.code == capi.SV_EINVAL
    got = capi.sv_to_host(sv, True)
    capi.sv_free(sv)
    assert got[0] == 1 and np.count_nonzero(got) == 1
    with pytest.raises(capi.PauliRotError) as e:
        capi.sv_alloc(40, "c128")
    assert e.value.code == capi.SV_ENOMEM


@pytest.mark.parametrize("scale_exp", [-700, -300, 0, 300, 700])
def test_c128_block_exponent_follows_the_state_scale(orc, scale_exp):
    """The complex128 pass computes in fixed point with one exponent per coset
    chosen from the coset's largest component: a state scaled by 2^k (k up to
    +-700, far outside any fixed grid) must give the scaled result with the
    same relative accuracy, for fused runs of every depth."""
    n = 10
    psi0 = synth.random_state(n, 77)
    s = 2.0 ** scale_exp
    for depth in (1, 3, 5):
        x, z = random_paulis(n, 90, seed=5 + depth, span_dim=depth, diag_frac=0.1)
        th = np.random.default_rng(depth).uniform(-np.pi, np.pi, size=90)
        want = run_oracle(orc, n, psi0, x, z, th)
        got, _ = run_gpu(n, "c128", psi0 * s, x, z, th, depth)
        assert_close_c128(want, got / s, what=f"scale 2^{scale_exp} depth {depth}")


def test_c128_long_runs_of_large_angles(orc):
    """Runs of up to 256 rotations at angles near +-pi/2 grow the tan-form norm
    by up to half a bit per rotation (about 128 bits per run): the fixed-point
    pass halves its components as the growth passes each whole bit, and the
    running scale folds the cos factors back in."""
    n = 9
    psi0 = synth.random_state(n, 3)
    g = np.random.default_rng(11)
    for span in (1, 2, 3):
        x, z = random_paulis(n, 256, seed=20 + span, span_dim=span)
        th = np.where(g.random(256) < 0.5, -1.0, 1.0) * g.uniform(1.45, np.pi / 2, size=256)
        want = run_oracle(orc, n, psi0, x, z, th)
        got, (nrot, nruns, _) = run_gpu(n, "c128", psi0, x, z, th, span)
        assert nruns <= 4, nruns  # long runs really are fused
        assert_close_c128(want, got, what=f"large angles, span {span}")


def test_c128_tiny_components_beside_large_ones(orc):
    """A coset holding components of very different size: the fixed point is
    set by the largest, so values below 2^-57 of it may be dropped, within the
    complex128 tolerance of 1e-12 absolute (the state is normalised)."""
    n = 8
    psi0 = synth.random_state(n, 5)
    psi0[::2] *= 1e-30  # every even amplitude tiny, odd ones of normal size
    psi0 /= np.linalg.norm(psi0)
    x, z = random_paulis(n, 60, seed=9, span_dim=3)
    th = np.random.default_rng(9).uniform(-np.pi, np.pi, size=60)
    want = run_oracle(orc, n, psi0, x, z, th)
    got, _ = run_gpu(n, "c128", psi0, x, z, th, 3)
    assert_close_c128(want, got, what="tiny beside large")
