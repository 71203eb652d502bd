"""The fusion planner on the host (plan_inspect, no GPU): the runs partition the
rotation list in order, each fused run's x-masks lie in the span of its reduced
basis of dimension <= the fusion depth, diagonal runs hold only x = 0 stretches,
identity strings are dropped, and fusion_depth = -1 follows the tune table."""
import numpy as np
import pytest

from paper_2602_09020_gb300 import capi, synth


def reduce(v, basis):
    for b in sorted(basis, key=lambda u: -u):  # highest pivot first
        if (v >> (b.bit_length() - 1)) & 1:
            v ^= b
    return v


def rank(vs):
    basis = []
    for v in vs:
        r = reduce(int(v), basis)
        if r:
            basis.append(r)
    return len(basis)


def check_runs(runs, x, z, depth, n):
    keep = [(int(a), int(b)) for a, b in zip(x, z) if (a | b) != 0]
    assert sum(c for _, _, c, _ in runs) == len(keep)
    pos = 0
    for kind, d, count, basis in runs:
        members = keep[pos:pos + count]
        pos += count
        if kind == 1:
            assert all(mx == 0 for mx, _ in members)
            assert count >= 8 and n >= 9
            continue
        assert d <= depth and len(basis) == d
        pivots = [b.bit_length() - 1 for b in basis]
        assert len(set(pivots)) == d and all(b > 0 for b in basis)
        # reduced: no basis vector has another vector's pivot bit set
        for b in basis:
            for p in pivots:
                if p != b.bit_length() - 1:
                    assert not (b >> p) & 1
        for mx, _ in members:
            assert reduce(mx, basis) == 0
        assert rank([mx for mx, _ in members if mx]) <= d
        assert count <= 256


@pytest.mark.parametrize("depth", [1, 2, 3, 4, 5])
def test_runs_partition_a_jw_trotter_list(depth):
    n = 14
    ham = synth.jw_hamiltonian(n, 300, 2)
    x, z, t = capi.trotter_expand(ham.x, ham.z, ham.c, 0.05, 3, 1, False)
    runs, nrot = capi.plan_inspect(n, "c64", x, z, t, depth)
    assert nrot == len(t)
    check_runs(runs, x, z, depth, n)


def test_random_lists_with_identities_and_every_depth():
    rng = np.random.default_rng(5)
    for n in (1, 3, 8, 12):
        m = 200
        x = rng.integers(0, 1 << n, size=m).astype(np.uint64)
        z = rng.integers(0, 1 << n, size=m).astype(np.uint64)
        x[rng.random(m) < 0.3] = 0
        ident = rng.random(m) < 0.1
        x[ident] = 0
        z[ident] = 0
        t = rng.uniform(-7, 7, size=m)  # large angles are reduced into the frame
        for depth in range(0, 6):
            runs, nrot = capi.plan_inspect(n, "c128", x, z, t, depth)
            assert nrot == m - int(np.sum((x | z) == 0))  # drawn identities included
            check_runs(runs, x, z, max(depth, 1), n)


def test_long_diagonal_stretches_get_their_own_runs():
    n = 10
    x = np.array([3] * 4 + [0] * 20 + [5] * 3, dtype=np.uint64)
    z = np.arange(1, 28, dtype=np.uint64) % (1 << n)
    t = np.full(27, 0.2)
    runs, _ = capi.plan_inspect(n, "c64", x, z, t, 4)
    assert [(k, c) for k, _, c, _ in runs] == [(0, 4), (1, 20), (0, 3)]
    # below the diagonal kernel's size the stretch stays inside a fused run
    runs, _ = capi.plan_inspect(8, "c64", x, z % (1 << 8), t, 4)
    assert all(k == 0 for k, *_ in runs)


def test_diagonal_runs_hold_at_most_128_low_bit_patterns():
    # the diagonal kernel groups a run's rotations by their z pattern on index
    # bits 0..8; a stretch with more distinct patterns is cut into several runs
    n = 12
    g = np.random.default_rng(4)
    z = np.array([(j % 511) + 1 + (int(g.integers(0, 8)) << 9) for j in range(400)], dtype=np.uint64)
    x = np.zeros(400, dtype=np.uint64)
    runs, _ = capi.plan_inspect(n, "c64", x, z, np.full(400, 0.3), 4)
    assert [(k, c) for k, _, c, _ in runs] == [(1, 128), (1, 128), (1, 128), (1, 16)]
    # the same count of rotations on few patterns stays one run, up to 1024 rotations
    z2 = np.array([1 << (j % 12) for j in range(1100)], dtype=np.uint64)
    runs, _ = capi.plan_inspect(n, "c64", np.zeros(1100, dtype=np.uint64), z2, np.full(1100, 0.3), 4)
    assert [(k, c) for k, _, c, _ in runs] == [(1, 1024), (1, 76)]


def test_run_length_is_capped():
    n = 10
    x = np.full(1000, 6, dtype=np.uint64)
    z = np.full(1000, 1, dtype=np.uint64)
    runs, _ = capi.plan_inspect(n, "c64", x, z, np.full(1000, 0.01), 4)
    assert all(c <= 256 for _, _, c, _ in runs) and sum(c for _, _, c, _ in runs) == 1000


def test_default_depth_follows_the_tune_table():
    n = 13
    ham = synth.jw_hamiltonian(n, 200, 4)
    x, z, t = capi.trotter_expand(ham.x, ham.z, ham.c, 0.05, 1, 1, False)
    assert capi.plan_inspect(n, "c64", x, z, t, -1) == capi.plan_inspect(n, "c64", x, z, t, 4)
    assert capi.plan_inspect(n, "c128", x, z, t, -1) == capi.plan_inspect(n, "c128", x, z, t, 3)
    try:
        capi.plan_set_tuned_depth(n, "c64", 2)
        assert capi.plan_inspect(n, "c64", x, z, t, -1) == capi.plan_inspect(n, "c64", x, z, t, 2)
    finally:
        capi.plan_set_tuned_depth(n, "c64", -1)


def test_bad_lists_are_rejected():
    for args in ((4, "c64", [1 << 4], [0], [0.1], 2), (4, "c64", [1], [0], [np.nan], 2),
                 (4, "c64", [1], [0], [0.1], 6), (0, "c64", [], [], [], 2)):
        with pytest.raises(capi.PauliRotError) as e:
            capi.plan_inspect(*args)
        assert e.value.code == capi.SV_EINVAL
