"""Launch tracing: per-launch event pairs and per-block events (one event where
the kernel changes) count the same launches and algorithmic bytes, and block
times add up to the traced region."""
import numpy as np
import pytest
import torch

from paper_2602_09020_gb300 import capi, synth

pytestmark = pytest.mark.gpu


def traced_apply(sv, plan, ham, blocks):
    capi.sv_set_basis_state(sv, synth.hartree_fock_index(6))
    torch.cuda.synchronize()
    capi.sv_trace_start(sv, blocks=blocks)
    capi.plan_apply(sv, plan)
    capi.expval_pauli_sum(sv, ham.x, ham.z, ham.c)
    return capi.sv_trace_stop(sv)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_block_trace_counts_match_launch_trace(dtype):
    n = 14
    ham = synth.jw_hamiltonian(n, 300, 3)
    rx, rz, rt = capi.trotter_expand(ham.x, ham.z, ham.c, 0.05, 2, 1, False)
    stream = torch.cuda.current_stream().cuda_stream
    sv = capi.sv_alloc(n, dtype, stream)
    plan = capi.plan_create(n, dtype, rx, rz, rt, -1, stream)
    try:
        n_runs = capi.plan_sweeps(plan)  # passes over the state: a chained pass applies several runs
        per_launch = traced_apply(sv, plan, ham, False)
        per_block = traced_apply(sv, plan, ham, True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        capi.sv_set_basis_state(sv, synth.hartree_fock_index(6))
        capi.sv_trace_start(sv, blocks=True)
        e0.record()
        capi.plan_apply(sv, plan)
        e1.record()
        rows = capi.sv_trace_stop(sv)
        wall = e0.elapsed_time(e1)
        with pytest.raises(capi.PauliRotError) as err:
            capi._check(capi.lib().sv_trace_start_ex(sv, 7))
        assert err.value.code == capi.SV_EINVAL
    finally:
        capi.plan_free(plan)
        capi.sv_free(sv)
    assert set(per_launch) == set(per_block)
    for k in per_launch:
        assert per_launch[k][0] == per_block[k][0], k           # launches
        assert per_launch[k][2] == pytest.approx(per_block[k][2])  # bytes
        assert per_block[k][1] > 0
    rot_launches = sum(v[0] for k, v in per_block.items() if k.startswith(("k_coset", "k_diag_sum", "k_chain")))
    assert rot_launches == n_runs
    # the blocks of one plan application tile the region between the two events
    total = sum(v[1] for v in rows.values())
    assert total <= wall * 1.05 + 0.05 and total >= wall * 0.5
    assert np.isfinite(total)
