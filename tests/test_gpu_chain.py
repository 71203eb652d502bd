"""GPU parity of the chained complex64 pass (two fused runs in one HBM pass).

A chained pass applies, per element, the same arithmetic in the same order as
the two runs it replaces, so the state must be bitwise equal to the unchained
application (PAULIROT_CHAIN=0 when the plan is created); the oracle fixes the
values.  Cases: the Jordan-Wigner workload's shape, random strings whose
x-masks touch bit 0 and bits 0..3 (which the block layout treats specially),
runs of dimension below 4 (padded to 4 inside the chain), plans of depth 1 to
4, diagonal rotations
inside runs, angles beyond pi/2 (frame factors), a running-scale fold, a Pauli
frame set before the plan is applied, and n = 13 (two blocks of 2^12) to 17.
"""
import os

import numpy as np
import pytest

from helpers import assert_close_c64, random_paulis
from paper_2602_09020_gb300 import capi, synth

pytestmark = pytest.mark.gpu


def apply(n, psi0, x, z, th, depth, chain, frame=()):
    old = os.environ.get("PAULIROT_CHAIN")
    os.environ["PAULIROT_CHAIN"] = "1" if chain else "0"
    try:
        plan = capi.plan_create(n, "c64", x, z, th, depth)
    finally:
        if old is None:
            os.environ.pop("PAULIROT_CHAIN", None)
        else:
            os.environ["PAULIROT_CHAIN"] = old
    sv = capi.sv_alloc(n, "c64")
    try:
        capi.sv_from_host(sv, psi0)
        for p, q in frame:
            capi.frame_apply_pauli(sv, p, q)
        capi.sv_trace_start(sv)
        capi.plan_apply(sv, plan)
        rows = capi.sv_trace_stop(sv)
        rows["_sweeps"] = capi.plan_sweeps(plan)
        rows["_runs"] = capi.plan_stats(plan)[1]
        return capi.sv_to_host(sv, True), rows
    finally:
        capi.sv_free(sv)
        capi.plan_free(plan)


def low_bit_paulis(n, count, seed):
    """x-masks mixing bits 0..3 with a few higher bits (and some bit-0-only
    strings, which keep a run out of the packed kernels)."""
    g = np.random.default_rng(seed)
    xs, zs = [], []
    for _ in range(count):
        r = g.random()
        if r < 0.3:
            x = int(g.integers(1, 16))
        elif r < 0.35:
            x = 1
        elif r < 0.45:
            x = 0
        else:
            x = int(g.integers(1, 16)) ^ (1 << int(g.integers(4, n))) ^ (1 << int(g.integers(4, n)))
        z = int(g.integers(0, 1 << n))
        if x == 0 and z == 0:
            z = 2
        xs.append(x)
        zs.append(z)
    return np.array(xs, dtype=np.uint64), np.array(zs, dtype=np.uint64)


CASES = [
    # (name, n, depth)
    ("jw", 13, 4), ("jw", 14, 4), ("jw", 15, 4), ("jw", 17, 4), ("jw", 15, 3), ("jw", 15, 2),
    ("span6", 14, 4), ("span6", 16, 3), ("lowbits", 14, 4), ("lowbits", 16, 4), ("random", 15, 1),
]


def workload(name, n):
    if name == "jw":
        ham = synth.jw_hamiltonian(n, 300, seed=n)
        x, z, th = capi.trotter_expand(ham.x, ham.z, ham.c, 0.3, 2, 1, False)
        return x, z, th
    g = np.random.default_rng(7 * n + len(name))
    if name == "span6":
        x, z = random_paulis(n, 400, seed=n, span_dim=6, diag_frac=0.1)
    elif name == "lowbits":
        x, z = low_bit_paulis(n, 400, seed=n)
    else:
        x, z = random_paulis(n, 120, seed=n, diag_frac=0.2)
    th = g.uniform(-4.0, 4.0, size=len(x))
    return x, z, th


@pytest.mark.parametrize("name,n,depth", CASES)
def test_chained_equals_unchained_and_oracle(orc, name, n, depth):
    x, z, th = workload(name, n)
    psi0 = synth.random_state(n, 100 + n).astype(np.complex64)
    frame = [("X", 3), ("Y", 0), ("Z", n - 1)]
    got_c, rows_c = apply(n, psi0, x, z, th, depth, True, frame)
    got_u, rows_u = apply(n, psi0, x, z, th, depth, False, frame)
    assert "k_chain2" not in rows_u
    chained = rows_c.get("k_chain2", (0,))[0]
    assert rows_u["_sweeps"] == rows_u["_runs"] == rows_c["_runs"]
    # a chained pass takes two runs
    singles = sum(v[0] for k, v in rows_c.items() if k.startswith(("k_coset", "k_diag_sum")))
    assert rows_c["_sweeps"] == singles + chained == rows_c["_runs"] - chained
    if name in ("jw", "span6"):
        assert chained > 0, rows_c
    assert np.array_equal(got_c.view(np.uint32), got_u.view(np.uint32)), \
        f"{name} n={n} depth={depth}: chained state differs from the unchained one"
    # values: the oracle applies the frame's Pauli gates, then the rotations
    want = psi0.astype(np.complex128)
    for p, q in frame:
        orc.gate(want, n, p.lower(), q)
    orc.apply_rotations(want, n, x, z, th)
    assert_close_c64(want, got_c, what=f"{name} n={n} depth={depth}", atol=1e-4 * max(1.0, len(th) / 50))
