"""Fusion-depth autotuner on the GPU.

* plan_autotune times every depth, records the fastest for (n, dtype) and
  leaves the state evolved by exactly the applications it timed (one warm-up
  and 2 x reps per depth), which the oracle reproduces;
* plan_create(-1) follows the recorded depth (same runs as an explicit depth).
"""
import numpy as np
import pytest
import torch

from helpers import C128_ATOL
from paper_2602_09020_gb300 import capi, synth

pytestmark = pytest.mark.gpu


def rotation_list(n, count, seed):
    rng = np.random.default_rng(seed)
    x = rng.integers(0, 1 << n, size=count).astype(np.uint64)
    x[rng.random(count) < 0.3] = 0
    x[rng.random(count) < 0.3] &= np.uint64(0b111)  # low, overlapping spans
    z = rng.integers(0, 1 << n, size=count).astype(np.uint64)
    th = rng.uniform(-3, 3, size=count)
    return x, z, th


def test_autotune_times_every_depth_and_evolves_the_state(orc):
    n, max_depth, reps = 10, 4, 2
    x, z, th = rotation_list(n, 60, 1)
    psi = synth.random_state(n, 5)
    stream = torch.cuda.current_stream().cuda_stream
    sv = capi.sv_alloc(n, "c128", stream)
    try:
        capi.sv_from_host(sv, psi)
        capi.frame_apply_pauli(sv, "Y", 4)  # the tuner's applications go through the frame
        orc.gate(psi, n, "y", 4)
        depth, ms = capi.plan_autotune(sv, x, z, th, max_depth=max_depth, reps=reps)
        got = capi.sv_to_host(sv, True)
        assert capi.plan_tuned_depth(n, "c128") == (depth, True)
    finally:
        capi.plan_set_tuned_depth(n, "c128", -1)
        capi.sv_free(sv)
    assert 1 <= depth <= max_depth
    assert np.all(ms[:max_depth] > 0) and ms[max_depth] == -1
    assert depth == int(np.argmin(ms[:max_depth])) + 1
    for _ in range(max_depth * (1 + 2 * reps)):
        orc.apply_rotations(psi, n, x, z, th)
    assert np.max(np.abs(got - psi)) <= C128_ATOL


def test_plan_create_default_follows_the_recorded_depth():
    n = 12
    x, z, th = rotation_list(n, 200, 2)
    stream = torch.cuda.current_stream().cuda_stream

    def runs(depth):
        p = capi.plan_create(n, "c64", x, z, th, depth, stream)
        try:
            return capi.plan_stats(p)
        finally:
            capi.plan_free(p)

    explicit = {d: runs(d) for d in (1, 2, 4)}
    assert explicit[1][1] > explicit[4][1]  # the depths give different plans
    try:
        for d in (1, 2, 4):
            capi.plan_set_tuned_depth(n, "c64", d)
            assert runs(-1) == explicit[d]
        capi.plan_set_tuned_depth(n, "c64", -1)
        assert runs(-1) == explicit[4]  # the complex64 default
    finally:
        capi.plan_set_tuned_depth(n, "c64", -1)


def test_autotune_on_a_full_size_state_records_a_depth():
    n = 24
    ham = synth.jw_hamiltonian(n, 2000, 2)
    rx, rz, rt = capi.trotter_expand(ham.x, ham.z, ham.c, 0.05, 1, 1, False)
    stream = torch.cuda.current_stream().cuda_stream
    sv = capi.sv_alloc(n, "c64", stream)
    try:
        depth, ms = capi.plan_autotune(sv, rx, rz, rt, reps=1)
        assert capi.plan_tuned_depth(n, "c64") == (depth, True)
        # 15 applications of 2000 rotations in complex64 keep the norm
        _, nrm = capi.expval_pauli_sum(sv, [0], [0], [1.0])
        assert abs(nrm - 1.0) <= 1e-3
    finally:
        capi.plan_set_tuned_depth(n, "c64", -1)
        capi.sv_free(sv)
    assert np.all(ms > 0) and depth == int(np.argmin(ms)) + 1


def test_tuning_writes_the_cache_named_by_the_environment(tmp_path):
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cache = tmp_path / "tune.txt"
    code = (
        "import numpy as np, torch\n"
        "from paper_2602_09020_gb300 import capi\n"
        "rng = np.random.default_rng(3)\n"
        "x = rng.integers(0, 1 << 12, size=40).astype(np.uint64)\n"
        "z = rng.integers(0, 1 << 12, size=40).astype(np.uint64)\n"
        "sv = capi.sv_alloc(12, 'c64', torch.cuda.current_stream().cuda_stream)\n"
        "d, _ = capi.plan_autotune(sv, x, z, rng.uniform(-1, 1, 40), max_depth=3, reps=1)\n"
        "capi.sv_free(sv)\n"
        "print(d)\n")
    env = dict(os.environ, PAULIROT_TUNE_CACHE=str(cache))
    out = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True, text=True,
                         timeout=300)
    assert out.returncode == 0, out.stderr
    depth = int(out.stdout.strip())
    lines = [l.split() for l in cache.read_text().splitlines() if not l.startswith("#")]
    assert lines == [["c64", "12", str(depth)]]
    # a second process finds the depth without tuning
    code2 = "from paper_2602_09020_gb300 import capi\nprint(capi.plan_tuned_depth(12, 'c64'))\n"
    out = subprocess.run([sys.executable, "-c", code2], cwd=root, env=env, capture_output=True, text=True,
                         timeout=300)
    assert out.stdout.strip() == f"({depth}, True)"


def test_autotune_on_states_smaller_than_the_depths(orc):
    # n = 2: only depths 1 and 2 exist; the tuner's applications still match the oracle
    n = 2
    x = np.array([1, 2, 3, 0, 1], dtype=np.uint64)
    z = np.array([0, 1, 3, 2, 1], dtype=np.uint64)
    th = np.array([0.3, -1.1, 2.0, 0.7, -2.9])
    psi = synth.random_state(n, 1)
    stream = torch.cuda.current_stream().cuda_stream
    sv = capi.sv_alloc(n, "c128", stream)
    try:
        capi.sv_from_host(sv, psi)
        depth, ms = capi.plan_autotune(sv, x, z, th, reps=1)
        got = capi.sv_to_host(sv, True)
        assert capi.plan_tuned_depth(n, "c128") == (depth, True)
    finally:
        capi.plan_set_tuned_depth(n, "c128", -1)
        capi.sv_free(sv)
    assert depth in (1, 2) and np.all(ms[:2] > 0) and np.all(ms[2:] == -1)
    for _ in range(2 * (1 + 2 * 1)):
        orc.apply_rotations(psi, n, x, z, th)
    assert np.max(np.abs(got - psi)) <= C128_ATOL


def test_autotune_rejects_bad_lists_before_device_work():
    stream = torch.cuda.current_stream().cuda_stream
    sv = capi.sv_alloc(6, "c64", stream)
    try:
        capi.sv_set_basis_state(sv, 5)
        before = capi.sv_to_host(sv, True)
        for x, z, th in (([1 << 6], [0], [0.1]), ([1], [0], [np.inf]), ([], [], [])):
            with pytest.raises(capi.PauliRotError) as e:
                capi.plan_autotune(sv, x, z, th)
            assert e.value.code == capi.SV_EINVAL
        assert capi.sv_to_host(sv, True).tobytes() == before.tobytes()
        assert capi.plan_tuned_depth(6, "c64") == (4, False)
    finally:
        capi.sv_free(sv)
