"""FP64 CPU oracle for the Pauli-rotation path.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA library and never imports it.

The heavy lifting is ``oracle.c`` (plain C99 complex double, OpenMP over
amplitudes, textbook gate decomposition of every rotation); this module loads
it with ctypes and adds the small pieces written directly from the paper:

* ``trotter_rotations`` -- the first-order product of Eq. (trotter) and the
  symmetric second-order product (the paper gives only the first order; the
  second order used here is the standard Strang splitting, one half step per
  term forward then backward, no merging of neighbours).
* ``run_circuit`` -- rotations with interleaved Pauli gates applied as gates
  (the oracle has no Pauli frame).
* ``expval`` -- sum_j c_j <psi|P_j|psi> by applying P_j gate-wise to a copy
  (Sec. "Extraction of Expectation Values", Eq. (chfsexp) with the origin frame).
* ``grad_param_shift`` -- dE/dtheta_j by the parameter-shift rule
  [E(theta_j + pi/2) - E(theta_j - pi/2)] / 2, exact for exp(-i theta P / 2)
  because P^2 = I (Sec. "Pauli and Clifford Group").
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Iterable, List, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

__all__ = [
    "build", "lib", "num_threads", "set_num_threads", "basis_state", "apply_rotations", "apply_rotation",
    "apply_pauli", "apply_sequence", "norm2", "inner", "expval", "apply_pauli_sum",
    "trotter_rotations", "circuit_sequence", "run_circuit", "grad_param_shift",
    "rotation_gate_count", "gate",
]


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, -O2, OpenMP, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared", "-Wall",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        cx = ctypes.c_void_p
        i64, u64, d = ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        vp = ctypes.c_void_p
        for name in ["orc_gate_x", "orc_gate_y", "orc_gate_z", "orc_gate_h", "orc_gate_s", "orc_gate_sdg"]:
            getattr(L, name).argtypes = [cx, ctypes.c_int, ctypes.c_int]
            getattr(L, name).restype = None
        L.orc_gate_rz.argtypes = [cx, ctypes.c_int, ctypes.c_int, d]
        L.orc_gate_cnot.argtypes = [cx, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.orc_apply_pauli.argtypes = [cx, ctypes.c_int, u64, u64]
        L.orc_rotation.argtypes = [cx, ctypes.c_int, u64, u64, d]
        L.orc_apply_rotations.argtypes = [cx, ctypes.c_int, vp, vp, vp, i64]
        L.orc_apply_sequence.argtypes = [cx, ctypes.c_int, vp, vp, vp, vp, i64]
        L.orc_norm2.argtypes = [cx, ctypes.c_int]
        L.orc_norm2.restype = d
        L.orc_inner.argtypes = [cx, cx, ctypes.c_int, ctypes.POINTER(d), ctypes.POINTER(d)]
        L.orc_expval.argtypes = [cx, ctypes.c_int, vp, vp, vp, i64, cx, ctypes.POINTER(d)]
        L.orc_expval.restype = d
        L.orc_apply_pauli_sum.argtypes = [cx, ctypes.c_int, vp, vp, vp, i64, cx, cx]
        L.orc_rotation_gate_count.argtypes = [u64, u64, ctypes.c_int] + [ctypes.POINTER(ctypes.c_int)] * 3
        L.orc_num_threads.restype = ctypes.c_int
        L.orc_set_num_threads.argtypes = [ctypes.c_int]
        _lib = L
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _state(psi: np.ndarray, n: int) -> np.ndarray:
    if psi.dtype != np.complex128 or not psi.flags.c_contiguous or psi.shape != (1 << n,):
        raise ValueError("oracle state must be a contiguous complex128 vector of length 2^n")
    return psi


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_num_threads(k: int) -> None:
    """Threads for later calls; k <= 0 = one per processor (timing only)."""
    lib().orc_set_num_threads(int(k))


def basis_state(n: int, k: int) -> np.ndarray:
    v = np.zeros(1 << n, dtype=np.complex128)
    v[k] = 1.0
    return v


def gate(psi: np.ndarray, n: int, name: str, *qubits, theta: float = 0.0) -> np.ndarray:
    """Apply one named gate in place ('x','y','z','h','s','sdg','rz','cnot')."""
    _state(psi, n)
    L = lib()
    if name == "rz":
        L.orc_gate_rz(_ptr(psi), n, qubits[0], theta)
    elif name == "cnot":
        L.orc_gate_cnot(_ptr(psi), n, qubits[0], qubits[1])
    else:
        getattr(L, "orc_gate_" + name)(_ptr(psi), n, qubits[0])
    return psi


def apply_rotation(psi: np.ndarray, n: int, x: int, z: int, theta: float) -> np.ndarray:
    lib().orc_rotation(_ptr(_state(psi, n)), n, int(x), int(z), float(theta))
    return psi


def apply_rotations(psi: np.ndarray, n: int, x, z, theta) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.uint64)
    z = np.ascontiguousarray(z, dtype=np.uint64)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    lib().orc_apply_rotations(_ptr(_state(psi, n)), n, _ptr(x), _ptr(z), _ptr(th), len(th))
    return psi


def apply_pauli(psi: np.ndarray, n: int, x: int, z: int) -> np.ndarray:
    lib().orc_apply_pauli(_ptr(_state(psi, n)), n, int(x), int(z))
    return psi


def apply_sequence(psi: np.ndarray, n: int, kind, x, z, theta) -> np.ndarray:
    k = np.ascontiguousarray(kind, dtype=np.int32)
    x = np.ascontiguousarray(x, dtype=np.uint64)
    z = np.ascontiguousarray(z, dtype=np.uint64)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    lib().orc_apply_sequence(_ptr(_state(psi, n)), n, _ptr(k), _ptr(x), _ptr(z), _ptr(th), len(k))
    return psi


def norm2(psi: np.ndarray, n: int) -> float:
    return float(lib().orc_norm2(_ptr(_state(psi, n)), n))


def inner(a: np.ndarray, b: np.ndarray, n: int) -> complex:
    re, im = ctypes.c_double(), ctypes.c_double()
    lib().orc_inner(_ptr(_state(a, n)), _ptr(_state(b, n)), n, ctypes.byref(re), ctypes.byref(im))
    return complex(re.value, im.value)


def expval(psi: np.ndarray, n: int, x, z, c, return_imag: bool = False):
    x = np.ascontiguousarray(x, dtype=np.uint64)
    z = np.ascontiguousarray(z, dtype=np.uint64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    work = np.empty(1 << n, dtype=np.complex128)
    im = ctypes.c_double()
    e = lib().orc_expval(_ptr(_state(psi, n)), n, _ptr(x), _ptr(z), _ptr(c), len(c), _ptr(work),
                         ctypes.byref(im))
    return (float(e), float(im.value)) if return_imag else float(e)


def apply_pauli_sum(psi: np.ndarray, n: int, x, z, c) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.uint64)
    z = np.ascontiguousarray(z, dtype=np.uint64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    out = np.empty(1 << n, dtype=np.complex128)
    work = np.empty(1 << n, dtype=np.complex128)
    lib().orc_apply_pauli_sum(_ptr(_state(psi, n)), n, _ptr(x), _ptr(z), _ptr(c), len(c),
                              _ptr(out), _ptr(work))
    return out


def rotation_gate_count(n: int, x: int, z: int) -> Tuple[int, int, int]:
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    lib().orc_rotation_gate_count(int(x), int(z), n, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
    return a.value, b.value, c.value


# ---- Trotter products ------------------------------------------------------------

def trotter_rotations(x, z, c, dt: float, steps: int, order: int = 1):
    """Rotation list (x, z, theta) in application order, theta of exp(-i theta/2 P).

    First order, Eq. (trotter): each step applies exp(-i c_j P_j dt) for
    j = 1..T in term order, i.e. theta_j = 2 c_j dt.
    Second order (symmetric): each step applies exp(-i c_j P_j dt/2) for
    j = 1..T, then again for j = T..1, i.e. theta = c_j dt per half step.
    No neighbouring rotations are merged.
    """
    x = np.asarray(x, dtype=np.uint64)
    z = np.asarray(z, dtype=np.uint64)
    c = np.asarray(c, dtype=np.float64)
    if order == 1:
        one_x, one_z, one_t = x, z, 2.0 * c * dt
    elif order == 2:
        one_x = np.concatenate([x, x[::-1]])
        one_z = np.concatenate([z, z[::-1]])
        one_t = np.concatenate([c * dt, (c * dt)[::-1]])
    else:
        raise ValueError("order must be 1 or 2")
    return (np.tile(one_x, steps), np.tile(one_z, steps), np.tile(one_t, steps))


_PAULI_MASK = {"X": (1, 0), "Y": (1, 1), "Z": (0, 1)}


def circuit_sequence(circ):
    """Expand a synth.Circuit into (kind, x, z, theta) with gates as kind 1."""
    rx, rz, rt = trotter_rotations(circ.ham.x, circ.ham.z, circ.ham.c, circ.dt, circ.steps, circ.order)
    gates = sorted(circ.gates, key=lambda g: g[0])
    kind: List[int] = []
    xs: List[int] = []
    zs: List[int] = []
    ts: List[float] = []
    gi = 0
    for j in range(len(rt) + 1):
        while gi < len(gates) and gates[gi][0] == j:
            _, p, q = gates[gi]
            xb, zb = _PAULI_MASK[p]
            kind.append(1); xs.append(xb << q); zs.append(zb << q); ts.append(0.0)
            gi += 1
        if j < len(rt):
            kind.append(0); xs.append(int(rx[j])); zs.append(int(rz[j])); ts.append(float(rt[j]))
    return (np.array(kind, dtype=np.int32), np.array(xs, dtype=np.uint64),
            np.array(zs, dtype=np.uint64), np.array(ts, dtype=np.float64))


def run_circuit(circ) -> np.ndarray:
    psi = basis_state(circ.n, circ.basis_state)
    k, x, z, t = circuit_sequence(circ)
    apply_sequence(psi, circ.n, k, x, z, t)
    return psi


def grad_param_shift(n: int, psi0: np.ndarray, x, z, theta, ox, oz, oc):
    """Energy E = <psi|H|psi>, psi = prod_j R_j(theta_j) psi0, and all dE/dtheta_j
    by the parameter-shift rule (2 extra full evaluations per angle)."""
    x = np.asarray(x, dtype=np.uint64)
    z = np.asarray(z, dtype=np.uint64)
    theta = np.asarray(theta, dtype=np.float64)

    def energy(th):
        psi = psi0.astype(np.complex128).copy()
        apply_rotations(psi, n, x, z, th)
        return expval(psi, n, ox, oz, oc)

    e0 = energy(theta)
    g = np.empty(len(theta))
    for j in range(len(theta)):
        tp = theta.copy(); tp[j] += np.pi / 2
        tm = theta.copy(); tm[j] -= np.pi / 2
        g[j] = 0.5 * (energy(tp) - energy(tm))
    return e0, g
