"""The batched launch's work assignment on the host (batch_inspect, no GPU):
large states are split over CTAs so that no CTA carries much more than the
mean load, small states are packed, and every CTA range fits the grid."""
import numpy as np
import pytest

from paper_2602_09020_gb300 import capi, synth


def workload_shape(n_states, seed):
    n, rot, passes = [], [], []
    for c in synth.batch_workload(n_states, seed=seed):
        x, z, t = capi.trotter_expand(c.ham.x, c.ham.z, c.ham.c, c.dt, c.steps, 1, False)
        runs, nrot = capi.plan_inspect(c.n, "c64", x, z, t, 4)
        n.append(c.n)
        rot.append(nrot)
        passes.append(len(runs))
    return n, rot, passes


@pytest.mark.parametrize("seed", [4, 7, 11])
def test_uneven_batch_is_balanced(seed):
    n, rot, passes = workload_shape(64, seed)
    ctas, ratio = capi.batch_inspect(n, rot, passes, 304)
    # the busiest CTA carries at most a fifth more than the mean (it was 2.9x
    # when split states were scaled down to fit three quarters of the grid)
    assert ratio <= 1.2
    cost = np.array([(1 << a) * (r + 4 * (p + 1)) for a, r, p in zip(n, rot, passes)], dtype=float)
    share = cost.sum() / 304
    split = ctas > 1
    assert ctas[split].sum() <= 304
    assert np.all(np.array(n)[split] >= 16)
    # a split state's load per CTA stays near the share
    assert np.all(cost[split] / ctas[split] <= 1.2 * share)


def test_single_large_state_takes_the_grid():
    ctas, ratio = capi.batch_inspect([22], [1000], [40], 304)
    assert ctas[0] == 304 and ratio == pytest.approx(1.0)


def test_small_states_are_packed():
    n = [12] * 400
    ctas, ratio = capi.batch_inspect(n, [100] * 400, [5] * 400, 304)
    assert np.all(ctas == 1)
    # 400 equal items over 304 CTAs: two on some CTAs
    assert ratio == pytest.approx(2 * 304 / 400)


def test_bad_arguments():
    with pytest.raises(capi.PauliRotError):
        capi.batch_inspect([40], [1], [1], 304)
    with pytest.raises(capi.PauliRotError):
        capi.batch_inspect([10], [1], [1], 0)
