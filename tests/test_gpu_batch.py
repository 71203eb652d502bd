"""Batched independent states in one persistent launch (batch_run).

Checks: every state of an uneven batch equals the same plan applied on its own
(bitwise: each coset's arithmetic does not depend on which CTA runs it) and
every one matches the oracle; CUDA-graph replay gives the same result as a direct launch;
states large enough to span several CTAs are exercised (their CTAs meet at
bounded barriers); and the failure path: when one CTA skips a barrier arrival,
its peers' waits run out, the call returns SV_ETIMEOUT and the context stays
usable (no fault, no hang).
"""
import numpy as np
import pytest
import torch

from helpers import assert_close_c128, assert_close_c64
from paper_2602_09020_gb300 import capi, synth

pytestmark = pytest.mark.gpu


def _problems(ns, seed, dtype):
    out = []
    for k, n in enumerate(ns):
        ham = synth.jw_hamiltonian(n, 60 + 20 * (k % 5), seed + k)
        rx, rz, rt = capi.trotter_expand(ham.x, ham.z, ham.c, 0.07, 1 + k % 3, 1, False)
        psi0 = synth.random_state(n, seed + 100 + k)
        out.append((n, rx, rz, rt, psi0.astype(np.complex64 if dtype == "c64" else np.complex128)))
    return out


LAST_INFO = {}


def _run(problems, dtype, stream, mode):
    states, plans = [], []
    for (n, rx, rz, rt, psi0) in problems:
        sv = capi.sv_alloc(n, dtype, stream)
        capi.sv_from_host(sv, psi0)
        states.append(sv)
        plans.append(capi.plan_create(n, dtype, rx, rz, rt, -1, stream))
    try:
        if mode == "single":
            for sv, p in zip(states, plans):
                capi.plan_apply(sv, p)
        else:
            capi.batch_run(states, plans, use_graph=(mode == "graph"))
            if mode == "graph":  # second replay from fresh inputs through the cached graph
                for sv, (n, rx, rz, rt, psi0) in zip(states, problems):
                    capi.sv_from_host(sv, psi0)
                capi.batch_run(states, plans, use_graph=True)
            # read before the states and plans are freed (freeing one drops the graph)
            LAST_INFO[mode] = capi.batch_info()
        return [capi.sv_to_host(sv, True) for sv in states]
    finally:
        for p in plans:
            capi.plan_free(p)
        for sv in states:
            capi.sv_free(sv)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_batch_matches_single_launches_and_oracle(orc, dtype):
    stream = torch.cuda.Stream()
    ns = [10, 12, 17, 11, 18, 13, 14, 10, 16, 12, 19, 15]
    probs = _problems(ns, 7, dtype)
    single = _run(probs, dtype, stream.cuda_stream, "single")
    direct = _run(probs, dtype, stream.cuda_stream, "direct")
    graph = _run(probs, dtype, stream.cuda_stream, "graph")
    grid, multi, used_graph = LAST_INFO["graph"]
    assert multi >= 1, "no state spanned several CTAs"
    # the barriers need every CTA resident: only the cooperative launch is
    # captured (1), or the capture failed (negative) and it ran without a graph
    assert used_graph == 1 or used_graph < 0, used_graph
    for a, b, c in zip(single, direct, graph):
        np.testing.assert_array_equal(a, b)
        np.testing.assert_array_equal(a, c)
    for k in range(len(probs)):  # every state of the batch against the oracle
        n, rx, rz, rt, psi0 = probs[k]
        want = orc.apply_rotations(psi0.astype(np.complex128).copy(), n, rx, rz, rt)
        if dtype == "c128":
            assert_close_c128(want, direct[k], what=f"batch state {k}")
        else:
            assert_close_c64(want, direct[k], what=f"batch state {k}", atol=3e-4)


def test_batch_barrier_timeout_reports_and_recovers():
    stream = torch.cuda.Stream()
    ns = [18, 12, 17, 11]
    probs = _problems(ns, 3, "c64")
    states, plans = [], []
    for (n, rx, rz, rt, psi0) in probs:
        sv = capi.sv_alloc(n, "c64", stream.cuda_stream)
        capi.sv_from_host(sv, psi0)
        states.append(sv)
        plans.append(capi.plan_create(n, "c64", rx, rz, rt, -1, stream.cuda_stream))
    try:
        with pytest.raises(capi.PauliRotError) as e:
            capi.batch_run_ex(states, plans, use_graph=False, wait_timeout_s=0.05, test_skip_arrival=True)
        assert e.value.code == capi.SV_ETIMEOUT
        _, multi, _ = capi.batch_info()
        assert multi >= 1
        # the context is intact: the same batch runs normally afterwards
        for sv, (n, rx, rz, rt, psi0) in zip(states, probs):
            capi.sv_from_host(sv, psi0)
        capi.batch_run(states, plans, use_graph=False)
        got = [capi.sv_to_host(sv, True) for sv in states]
    finally:
        for p in plans:
            capi.plan_free(p)
        for sv in states:
            capi.sv_free(sv)
    ref = _run(probs, "c64", stream.cuda_stream, "single")
    for a, b in zip(got, ref):
        np.testing.assert_array_equal(a, b)


def test_batch_autotune_records_the_fastest_depth_for_every_size():
    problems = _problems([10, 11, 12, 12, 16, 18], 40, "c64")
    stream = torch.cuda.Stream()
    sh = int(stream.cuda_stream)
    states = [capi.sv_alloc(n, "c64", sh) for (n, *_rest) in problems]
    sizes = sorted({p[0] for p in problems})
    try:
        depth, ms = capi.batch_autotune(states, [(rx, rz, rt) for (_, rx, rz, rt, _) in problems],
                                        max_depth=4, reps=2)
        assert 1 <= depth <= 4 and np.all(ms > 0)
        assert depth == int(np.argmin(ms)) + 1
        for n in sizes:
            assert capi.plan_tuned_depth(n, "c64") == (min(depth, n), True)
        # the tuned plans run in the batched launch and equal single launches
        for sv, (n, rx, rz, rt, psi0) in zip(states, problems):
            capi.sv_from_host(sv, psi0)
        plans = [capi.plan_create(n, "c64", rx, rz, rt, -1, sh) for (n, rx, rz, rt, _) in problems]
        try:
            capi.batch_run(states, plans, use_graph=True)
            got = [capi.sv_to_host(sv, True) for sv in states]
            for sv, p, (n, rx, rz, rt, psi0) in zip(states, plans, problems):
                capi.sv_from_host(sv, psi0)
                capi.plan_apply(sv, p)
            want = [capi.sv_to_host(sv, True) for sv in states]
        finally:
            for p in plans:
                capi.plan_free(p)
        for g, w in zip(got, want):
            assert g.tobytes() == w.tobytes()
        with pytest.raises(capi.PauliRotError) as e:
            capi.batch_autotune(states[:2], [(problems[0][1], problems[0][2], problems[0][3]),
                                             (problems[1][1][:3], problems[1][2][:3],
                                              np.array([0.1, np.nan, 0.2]))])
        assert e.value.code == capi.SV_EINVAL
    finally:
        for n in sizes:
            capi.plan_set_tuned_depth(n, "c64", -1)
        for sv in states:
            capi.sv_free(sv)
