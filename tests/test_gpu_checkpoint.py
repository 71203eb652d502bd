"""Checkpoint and resume of a state handle (sv_save / sv_load).

* a saved and reloaded state equals the original bit for bit, frame and tag
  included;
* a Trotter sequence compiled as two plans and interrupted between them by a
  save, a fresh handle and a load ends bit for bit where the uninterrupted run
  ends;
* damaged or mismatched files are rejected with the documented codes, and
  header problems leave the handle unchanged.
"""
import os

import numpy as np
import pytest
import torch

from paper_2602_09020_gb300 import capi, synth

pytestmark = pytest.mark.gpu


def stream():
    return torch.cuda.current_stream().cuda_stream


@pytest.mark.parametrize("n,dtype", [(11, "c128"), (11, "c64"), (24, "c128")])
def test_round_trip_is_bitwise(tmp_path, n, dtype):
    psi = synth.random_state(n, 4)
    a = capi.sv_alloc(n, dtype, stream())
    b = capi.sv_alloc(n, dtype, stream())
    path = str(tmp_path / "state.ckpt")
    try:
        capi.sv_from_host(a, psi.astype(np.complex64 if dtype == "c64" else np.complex128))
        for p, q in (("X", 1), ("Y", n - 1), ("Z", 3)):
            capi.frame_apply_pauli(a, p, q)
        capi.sv_save(a, path, 2 ** 40 + 7)
        assert os.path.getsize(path) == 72 + ((16 if dtype == "c128" else 8) << n)
        assert not os.path.exists(path + ".tmp")
        assert capi.sv_load(b, path) == 2 ** 40 + 7
        assert capi.frame_get(b) == capi.frame_get(a)
        ra, rb = capi.sv_to_host(a, False), capi.sv_to_host(b, False)
        assert ra.tobytes() == rb.tobytes()
        assert capi.sv_to_host(a, True).tobytes() == capi.sv_to_host(b, True).tobytes()
    finally:
        capi.sv_free(a)
        capi.sv_free(b)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_resumed_trotter_run_matches_the_uninterrupted_one(tmp_path, dtype):
    n = 16
    ham = synth.jw_hamiltonian(n, 400, 6)
    x1, z1, t1 = capi.trotter_expand(ham.x, ham.z, ham.c, 0.05, 5, 1, False)
    hf = synth.hartree_fock_index(n // 2)
    path = str(tmp_path / "mid.ckpt")
    pa = capi.plan_create(n, dtype, x1, z1, t1, -1, stream())
    pb = capi.plan_create(n, dtype, x1, z1, t1, -1, stream())  # the second 5 steps are the same list
    try:
        ref = capi.sv_alloc(n, dtype, stream())
        capi.sv_set_basis_state(ref, hf)
        capi.plan_apply(ref, pa)
        capi.frame_apply_pauli(ref, "Y", 5)
        capi.plan_apply(ref, pb)
        want = capi.sv_to_host(ref, False)
        want_frame = capi.frame_get(ref)
        capi.sv_free(ref)

        s = capi.sv_alloc(n, dtype, stream())
        capi.sv_set_basis_state(s, hf)
        capi.plan_apply(s, pa)
        capi.frame_apply_pauli(s, "Y", 5)
        capi.sv_save(s, path, 1)
        capi.sv_free(s)

        t = capi.sv_alloc(n, dtype, stream())
        try:
            assert capi.sv_load(t, path) == 1
            capi.plan_apply(t, pb)
            got = capi.sv_to_host(t, False)
            assert capi.frame_get(t) == want_frame
        finally:
            capi.sv_free(t)
    finally:
        capi.plan_free(pa)
        capi.plan_free(pb)
    assert got.tobytes() == want.tobytes()


def test_damaged_and_mismatched_files(tmp_path):
    n = 10
    a = capi.sv_alloc(n, "c128", stream())
    path = str(tmp_path / "good.ckpt")
    try:
        capi.sv_from_host(a, synth.random_state(n, 9))
        capi.frame_apply_pauli(a, "X", 2)
        capi.sv_save(a, path, 3)
        good = open(path, "rb").read()
        before, frame = capi.sv_to_host(a, False), capi.frame_get(a)

        def load_bytes(data, name):
            p = str(tmp_path / name)
            with open(p, "wb") as f:
                f.write(data)
            with pytest.raises(capi.PauliRotError) as e:
                capi.sv_load(a, p)
            return e.value.code

        # header problems: nothing changes
        assert load_bytes(b"not a checkpoint" * 8, "junk") == capi.SV_EINVAL
        assert load_bytes(good[:40], "short_header") == capi.SV_EIO
        hdr = bytearray(good)
        hdr[41] ^= 0x01  # the tag, under the header checksum
        assert load_bytes(bytes(hdr), "bad_header") == capi.SV_EIO
        assert load_bytes(good[:-8], "truncated") == capi.SV_EIO
        with pytest.raises(capi.PauliRotError) as e:
            capi.sv_load(a, str(tmp_path / "absent"))
        assert e.value.code == capi.SV_EIO
        assert capi.sv_to_host(a, False).tobytes() == before.tobytes() and capi.frame_get(a) == frame
        for nn, dt in ((n + 1, "c128"), (n, "c64")):
            b = capi.sv_alloc(nn, dt, stream())
            try:
                with pytest.raises(capi.PauliRotError) as e:
                    capi.sv_load(b, path)
                assert e.value.code == capi.SV_EINVAL
            finally:
                capi.sv_free(b)
        # a flipped amplitude bit is caught by the amplitude checksum
        amp = bytearray(good)
        amp[72 + 1000] ^= 0x10
        assert load_bytes(bytes(amp), "bad_amps") == capi.SV_EIO
        assert capi.frame_get(a) == frame
        # the good file still loads
        assert capi.sv_load(a, path) == 3
        assert capi.sv_to_host(a, False).tobytes() == before.tobytes()
    finally:
        capi.sv_free(a)


def test_single_qubit_checkpoint(tmp_path):
    stream_ = stream()
    a = capi.sv_alloc(1, "c64", stream_)
    b = capi.sv_alloc(1, "c64", stream_)
    path = str(tmp_path / "one.ckpt")
    try:
        capi.sv_from_host(a, np.array([0.6, 0.8j], dtype=np.complex64))
        capi.frame_apply_pauli(a, "Y", 0)
        capi.sv_save(a, path, 0)
        assert os.path.getsize(path) == 72 + 16
        assert capi.sv_load(b, path) == 0
        assert capi.sv_to_host(b, True).tobytes() == capi.sv_to_host(a, True).tobytes()
    finally:
        capi.sv_free(a)
        capi.sv_free(b)


def test_torch_state_vector_checkpoint_and_tuning(tmp_path):
    from paper_2602_09020_gb300.torch_api import Plan, StateVector
    n = 12
    ham = synth.jw_hamiltonian(n, 120, 8)
    x, z, t = capi.trotter_expand(ham.x, ham.z, ham.c, 0.05, 2, 1, False)
    a = StateVector(n, "c64")
    try:
        depth, ms = a.autotune(x, z, t, max_depth=4, reps=1)
        assert capi.plan_tuned_depth(n, "c64") == (depth, True)
        a.set_basis_state(synth.hartree_fock_index(n // 2))
        plan = Plan(n, "c64", x, z, t)
        a.apply_plan(plan)
        a.frame_apply_pauli("X", 2)
        path = str(tmp_path / "sv.ckpt")
        a.save(path, tag=5)
        b = StateVector(n, "c64")
        assert b.load(path) == 5
        assert b.frame() == a.frame()
        assert b.to_host().tobytes() == a.to_host().tobytes()
        plan.close()
        b.close()
    finally:
        capi.plan_set_tuned_depth(n, "c64", -1)
        a.close()
