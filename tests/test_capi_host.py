"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every function include/paulirot.h declares, and its host-only logic (Trotter
expansion, argument validation, error reporting) behaves."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2602_09020_gb300 import capi, synth

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "paulirot.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_]+\s*\**\s*([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    L = capi.lib()
    names = declared_functions()
    assert len(names) >= 25
    for name in names:
        assert hasattr(L, name), name
    assert set(names) == set(capi.exported_symbols())
    assert L.sv_version() >> 16 == 1


def test_trotter_expand_matches_oracle_expansion(orc):
    ham = synth.jw_hamiltonian(12, 150, 4)
    for order in (1, 2):
        ox, oz, ot = orc.trotter_rotations(ham.x, ham.z, ham.c, 0.03, 3, order)
        lx, lz, lt = capi.trotter_expand(ham.x, ham.z, ham.c, 0.03, 3, order, False)
        np.testing.assert_array_equal(ox, lx)
        np.testing.assert_array_equal(oz, lz)
        np.testing.assert_allclose(ot, lt, rtol=0, atol=0)
        mx, mz, mt = capi.trotter_expand(ham.x, ham.z, ham.c, 0.03, 3, order, True)
        # merging keeps the total angle per string
        for s in set(zip(ox.tolist(), oz.tolist())):
            a = ot[(ox == s[0]) & (oz == s[1])].sum()
            b = mt[(mx == s[0]) & (mz == s[1])].sum()
            assert abs(a - b) < 1e-13
    # 5000 terms, 4 second-order steps, merged: 4 (2T - 1) - 3
    big = synth.jw_hamiltonian(30, 5000, 1)
    mx, _, _ = capi.trotter_expand(big.x, big.z, big.c, 0.05, 4, 2, True)
    assert len(mx) == 4 * (2 * 5000 - 1) - 3 == 39993


def test_plan_create_rejects_bad_input_before_touching_a_device():
    with pytest.raises(capi.PauliRotError) as e:
        capi.plan_create(5, "c128", [1 << 5], [0], [0.1])
    assert e.value.code == capi.SV_EINVAL and "mask bit" in str(e.value)
    with pytest.raises(capi.PauliRotError) as e:
        capi.plan_create(5, "c64", [1], [0], [np.inf])
    assert e.value.code == capi.SV_EINVAL
    with pytest.raises(capi.PauliRotError) as e:
        capi.plan_create(5, "c64", [1], [0], [0.1], fusion_depth=9)
    assert e.value.code == capi.SV_EINVAL
    with pytest.raises(ValueError):
        capi.plan_create(5, "c32", [1], [0], [0.1])


def test_trotter_expand_validation():
    with pytest.raises(capi.PauliRotError):
        capi.trotter_expand([1], [0], [1.0], 0.1, 1, 3)
    assert len(capi.trotter_expand([], [], [], 0.1, 4, 2, True)[0]) == 0


def test_null_handles_are_rejected_not_crashed():
    L = capi.lib()
    assert L.sv_free(None) == capi.SV_OK
    assert L.frame_apply_pauli(None, b"X", 0) == capi.SV_EINVAL
    assert L.expval_pauli_sum(None, None, None, None, 0, None, None) == capi.SV_EINVAL
    assert L.plan_apply(None, None) == capi.SV_EINVAL
    assert b"NULL" in L.sv_last_error()
