"""Thin ctypes binding of libpaulirot.so (argument marshalling only).

Every function here has the name of the C entry point it calls and does no
arithmetic of its own: masks, angles and coefficients are converted to
contiguous numpy arrays, handles are passed through, status codes are turned
into :class:`PauliRotError`.  PyTorch is used only to own device memory and to
provide the current CUDA stream (see :class:`StateVector`).

If the library is missing it is built from ``csrc/`` with nvcc; if that is not
possible an ImportError-like :class:`PauliRotError` is raised -- there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence, Tuple

import numpy as np

from . import build as _build

SV_OK, SV_EINVAL, SV_ENOMEM, SV_ECUDA, SV_ETIMEOUT, SV_EUNSUPPORTED, SV_EIO = 0, -1, -2, -3, -4, -5, -6
SV_C128, SV_C64 = 0, 1
_DTYPES = {"c128": SV_C128, "complex128": SV_C128, SV_C128: SV_C128,
           "c64": SV_C64, "complex64": SV_C64, SV_C64: SV_C64}

_lib: Optional[ctypes.CDLL] = None


class PauliRotError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


def dtype_code(dtype) -> int:
    try:
        return _DTYPES[dtype]
    except KeyError:
        raise ValueError(f"dtype must be 'c128' or 'c64', got {dtype!r}") from None


def library_path() -> str:
    return _build.LIB


def lib() -> ctypes.CDLL:
    """Load (building first if needed) libpaulirot.so and declare its symbols."""
    global _lib
    if _lib is not None:
        return _lib
    try:
        path = _build.build()
    except Exception as exc:  # no nvcc / compile error: fail loudly
        raise PauliRotError(SV_EUNSUPPORTED, f"libpaulirot.so is not available: {exc}") from exc
    L = ctypes.CDLL(path)
    vp, i, sz, u64, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t, ctypes.c_uint64, ctypes.c_double
    P = ctypes.POINTER
    sig = {
        "sv_last_error": ([], ctypes.c_char_p),
        "sv_version": ([], i),
        "sv_alloc": ([P(vp), i, i, vp], i),
        "sv_wrap": ([P(vp), vp, i, i, vp], i),
        "sv_free": ([vp], i),
        "sv_set_stream": ([vp, vp], i),
        "sv_device_ptr": ([vp, P(vp)], i),
        "sv_info": ([vp, P(i), P(i)], i),
        "sv_set_basis_state": ([vp, u64], i),
        "sv_from_host": ([vp, vp], i),
        "sv_to_host": ([vp, vp, i], i),
        "sv_materialize": ([vp], i),
        "sv_copy": ([vp, vp], i),
        "sv_save": ([vp, ctypes.c_char_p, u64], i),
        "sv_load": ([vp, ctypes.c_char_p, P(u64)], i),
        "frame_reset": ([vp], i),
        "frame_apply_pauli": ([vp, ctypes.c_char, i], i),
        "frame_get": ([vp, P(u64), P(u64), P(i)], i),
        "apply_pauli_rotations": ([vp, vp, vp, vp, sz], i),
        "plan_create": ([P(vp), i, i, vp, vp, vp, sz, i, vp], i),
        "plan_apply": ([vp, vp], i),
        "plan_free": ([vp], i),
        "plan_stats": ([vp, P(sz), P(sz), P(sz)], i),
        "plan_sweeps": ([vp, P(sz)], i),
        "plan_inspect": ([i, i, vp, vp, vp, sz, i, vp, sz, P(sz), P(sz)], i),
        "plan_autotune": ([vp, vp, vp, vp, sz, i, i, P(i), vp], i),
        "plan_tuned_depth": ([i, i, P(i), P(i)], i),
        "batch_autotune": ([vp, vp, vp, vp, vp, sz, i, i, i, P(i), vp], i),
        "plan_set_tuned_depth": ([i, i, i], i),
        "plan_tune_cache_load": ([ctypes.c_char_p], i),
        "plan_tune_cache_save": ([ctypes.c_char_p], i),
        "trotter_expand": ([vp, vp, vp, sz, d, i, i, i, vp, vp, vp, sz, P(sz)], i),
        "expval_pauli_sum": ([vp, vp, vp, vp, sz, P(d), P(d)], i),
        "expval_pauli_sum_noalloc": ([vp, vp, vp, vp, sz, P(d), P(d)], i),
        "apply_pauli_sum": ([vp, vp, vp, vp, vp, sz], i),
        "rotation_grads": ([vp, vp, vp, vp, sz, vp, vp, vp, sz, P(d), vp], i),
        "apply_pauli_rotations_gates": ([vp, vp, vp, vp, sz, P(sz)], i),
        "batch_run": ([vp, vp, sz, i], i),
        "batch_run_ex": ([vp, vp, sz, i, vp], i),
        "batch_info": ([P(i), P(i), P(i)], i),
        "batch_inspect": ([vp, vp, vp, sz, i, vp, P(d)], i),
        "sv_trace_start": ([vp], i),
        "sv_trace_start_ex": ([vp, i], i),
        "sv_trace_stop": ([vp, vp, i, P(i)], i),
        "sv_probe_rate": ([i, i, i, vp, vp, P(d)], i),
        "shard_rotations": ([i, i, i, vp, vp, vp, vp, sz, vp, sz, P(sz), vp, vp, vp], i),
        "shard_terms": ([i, i, i, vp, vp, vp, vp, sz, vp, sz, P(sz), vp, vp, vp], i),
        "cliff_create": ([P(vp), i], i),
        "cliff_free": ([vp], i),
        "cliff_reset": ([vp], i),
        "cliff_num_qubits": ([vp, P(i)], i),
        "cliff_apply_gates": ([vp, vp, vp, vp, vp, sz, vp, vp, vp, sz, P(sz)], i),
        "cliff_map_paulis": ([vp, vp, vp, sz, vp, vp, vp], i),
        "cliff_entry": ([vp, i, P(u64), P(u64), P(i), P(u64), P(u64), P(i)], i),
        "cliff_is_origin": ([vp, P(i)], i),
        "cliff_inverse_rotations": ([vp, vp, vp, vp, sz, P(sz)], i),
        "cfhs_apply_gates": ([vp, vp, vp, vp, vp, vp, sz], i),
        "cfhs_apply_rotations": ([vp, vp, vp, vp, vp, sz], i),
        "cfhs_expval": ([vp, vp, vp, vp, vp, sz, P(d), P(d)], i),
        "cfhs_materialize": ([vp, vp], i),
        "cfhs_measure_pauli": ([vp, vp, u64, u64, d, P(i), P(d)], i),
        "cfhs_prepare_qubit": ([vp, vp, i, ctypes.c_char, d, P(i)], i),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def exported_symbols() -> Sequence[str]:
    return ["sv_last_error", "sv_version", "sv_alloc", "sv_wrap", "sv_free", "sv_set_stream",
            "sv_device_ptr", "sv_info", "sv_set_basis_state", "sv_from_host", "sv_to_host",
            "sv_materialize", "sv_copy", "sv_save", "sv_load", "frame_reset", "frame_apply_pauli", "frame_get",
            "apply_pauli_rotations", "plan_create", "plan_apply", "plan_free", "plan_stats", "plan_sweeps", "plan_inspect",
            "plan_autotune", "batch_autotune", "plan_tuned_depth", "plan_set_tuned_depth", "plan_tune_cache_load",
            "plan_tune_cache_save",
            "trotter_expand", "expval_pauli_sum", "expval_pauli_sum_noalloc", "apply_pauli_sum", "rotation_grads",
            "apply_pauli_rotations_gates", "batch_run", "batch_run_ex", "batch_info", "batch_inspect", "sv_trace_start",
            "sv_trace_start_ex", "sv_trace_stop", "cliff_create", "cliff_free", "cliff_reset", "cliff_num_qubits", "cliff_apply_gates",
            "cliff_map_paulis", "cliff_entry", "cliff_is_origin", "cliff_inverse_rotations", "cfhs_apply_gates",
            "cfhs_apply_rotations", "cfhs_expval", "cfhs_materialize", "cfhs_measure_pauli", "cfhs_prepare_qubit",
            "sv_probe_rate", "shard_rotations", "shard_terms"]


def _check(rc: int) -> None:
    if rc != SV_OK:
        msg = lib().sv_last_error()
        raise PauliRotError(rc, msg.decode() if msg else "")


def _u64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint64))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _p(a: np.ndarray) -> Optional[int]:
    return a.ctypes.data if a.size else None


def _stream(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream or None
    s = getattr(stream, "cuda_stream", None)  # torch.cuda.Stream
    return int(s) if s else None


# ------------------------------------------------------------------ C entry points

def sv_alloc(n_qubits: int, dtype="c128", stream=None) -> int:
    h = ctypes.c_void_p()
    _check(lib().sv_alloc(ctypes.byref(h), int(n_qubits), dtype_code(dtype), _stream(stream)))
    return h.value


def sv_wrap(dev_ptr: int, n_qubits: int, dtype="c128", stream=None) -> int:
    h = ctypes.c_void_p()
    _check(lib().sv_wrap(ctypes.byref(h), int(dev_ptr), int(n_qubits), dtype_code(dtype), _stream(stream)))
    return h.value


def sv_free(sv: int) -> None:
    _check(lib().sv_free(sv))


def sv_set_stream(sv: int, stream) -> None:
    _check(lib().sv_set_stream(sv, _stream(stream)))


def sv_info(sv: int) -> Tuple[int, int]:
    n, d = ctypes.c_int(), ctypes.c_int()
    _check(lib().sv_info(sv, ctypes.byref(n), ctypes.byref(d)))
    return n.value, d.value


def sv_set_basis_state(sv: int, k: int) -> None:
    _check(lib().sv_set_basis_state(sv, int(k)))


def _host_dtype(sv: int):
    n, d = sv_info(sv)
    return n, (np.complex128 if d == SV_C128 else np.complex64)


def sv_from_host(sv: int, amps: np.ndarray) -> None:
    n, dt = _host_dtype(sv)
    a = np.ascontiguousarray(amps, dtype=dt)
    if a.shape != (1 << n,):
        raise ValueError("amplitude array has the wrong length")
    _check(lib().sv_from_host(sv, a.ctypes.data))


def sv_to_host(sv: int, materialize_frame: bool = True, out: Optional[np.ndarray] = None) -> np.ndarray:
    n, dt = _host_dtype(sv)
    if out is None:
        out = np.empty(1 << n, dtype=dt)
    if out.dtype != dt or out.shape != (1 << n,) or not out.flags.c_contiguous:
        raise ValueError("output array has the wrong dtype or shape")
    _check(lib().sv_to_host(sv, out.ctypes.data, 1 if materialize_frame else 0))
    return out


def sv_materialize(sv: int) -> None:
    _check(lib().sv_materialize(sv))


def sv_copy(dst: int, src: int) -> None:
    _check(lib().sv_copy(dst, src))


def sv_save(sv: int, path: str, tag: int = 0) -> None:
    _check(lib().sv_save(sv, os.fsencode(path), ctypes.c_uint64(int(tag))))


def sv_load(sv: int, path: str) -> int:
    """Load a checkpoint into sv (same n and dtype); returns the saved tag."""
    t = ctypes.c_uint64()
    _check(lib().sv_load(sv, os.fsencode(path), ctypes.byref(t)))
    return t.value


def frame_reset(sv: int) -> None:
    _check(lib().frame_reset(sv))


def frame_apply_pauli(sv: int, pauli: str, qubit: int) -> None:
    _check(lib().frame_apply_pauli(sv, pauli.encode()[:1], int(qubit)))


def frame_get(sv: int) -> Tuple[int, int, int]:
    x, z, q = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_int()
    _check(lib().frame_get(sv, ctypes.byref(x), ctypes.byref(z), ctypes.byref(q)))
    return x.value, z.value, q.value


def apply_pauli_rotations(sv: int, x, z, angles) -> None:
    x, z, a = _u64(x), _u64(z), _f64(angles)
    if not (len(x) == len(z) == len(a)):
        raise ValueError("x, z and angles must have equal length")
    _check(lib().apply_pauli_rotations(sv, _p(x), _p(z), _p(a), len(a)))


def plan_create(n_qubits: int, dtype, x, z, angles, fusion_depth: int = -1, stream=None) -> int:
    x, z, a = _u64(x), _u64(z), _f64(angles)
    if not (len(x) == len(z) == len(a)):
        raise ValueError("x, z and angles must have equal length")
    h = ctypes.c_void_p()
    _check(lib().plan_create(ctypes.byref(h), int(n_qubits), dtype_code(dtype), _p(x), _p(z), _p(a), len(a),
                             int(fusion_depth), _stream(stream)))
    return h.value


def plan_apply(sv: int, plan: int) -> None:
    _check(lib().plan_apply(sv, plan))


def plan_free(plan: int) -> None:
    _check(lib().plan_free(plan))


def plan_stats(plan: int) -> Tuple[int, int, int]:
    a, b, c = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_size_t()
    _check(lib().plan_stats(plan, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def plan_sweeps(plan: int) -> int:
    """Passes over the state that plan_apply launches (a chained pass applies
    two runs)."""
    v = ctypes.c_size_t()
    _check(lib().plan_sweeps(plan, ctypes.byref(v)))
    return v.value


def plan_autotune(sv: int, x, z, angles, max_depth: int = 0, reps: int = 0) -> Tuple[int, np.ndarray]:
    """Time the list at every fusion depth on sv (overwritten) and record the
    fastest for sv's (n, dtype).  Returns (depth, ms per application for
    depths 1..5, -1 where not timed)."""
    x, z, a = _u64(x), _u64(z), _f64(angles)
    if not (len(x) == len(z) == len(a)):
        raise ValueError("x, z and angles must have equal length")
    d = ctypes.c_int()
    ms = np.empty(5, np.float64)
    _check(lib().plan_autotune(sv, _p(x), _p(z), _p(a), len(a), int(max_depth), int(reps), ctypes.byref(d),
                               _p(ms)))
    return d.value, ms


def batch_autotune(states, lists, max_depth: int = 4, reps: int = 3, use_graph: bool = True):
    """Time the batched launch of the lists (one (x, z, angles) per state) at
    every fusion depth and record the fastest for the states' sizes.  The
    states are overwritten.  Returns (depth, ms per launch for depths 1..4)."""
    if len(states) != len(lists) or not states:
        raise ValueError("one rotation list per state")
    keep = [(_u64(x), _u64(z), _f64(a)) for x, z, a in lists]
    for x, z, a in keep:
        if not (len(x) == len(z) == len(a)):
            raise ValueError("x, z and angles must have equal length")
    k = len(states)
    sv = (ctypes.c_void_p * k)(*states)
    xp = (ctypes.c_void_p * k)(*[x.ctypes.data for x, _, _ in keep])
    zp = (ctypes.c_void_p * k)(*[z.ctypes.data for _, z, _ in keep])
    ap = (ctypes.c_void_p * k)(*[a.ctypes.data for _, _, a in keep])
    cnt = (ctypes.c_size_t * k)(*[len(a) for _, _, a in keep])
    d = ctypes.c_int()
    ms = np.empty(4, np.float64)
    _check(lib().batch_autotune(sv, xp, zp, ap, cnt, k, int(max_depth), int(reps), int(bool(use_graph)),
                                ctypes.byref(d), _p(ms)))
    return d.value, ms


def plan_tuned_depth(n_qubits: int, dtype) -> Tuple[int, bool]:
    d, t = ctypes.c_int(), ctypes.c_int()
    _check(lib().plan_tuned_depth(int(n_qubits), dtype_code(dtype), ctypes.byref(d), ctypes.byref(t)))
    return d.value, bool(t.value)


def plan_set_tuned_depth(n_qubits: int, dtype, depth: int) -> None:
    _check(lib().plan_set_tuned_depth(int(n_qubits), dtype_code(dtype), int(depth)))


def plan_tune_cache_load(path: str) -> None:
    _check(lib().plan_tune_cache_load(os.fsencode(path)))


def plan_tune_cache_save(path: str) -> None:
    _check(lib().plan_tune_cache_save(os.fsencode(path)))


class RunInfo(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("d", ctypes.c_int32), ("count", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("basis", ctypes.c_uint64 * 5)]


def plan_inspect(n_qubits: int, dtype, x, z, angles, fusion_depth: int = -1):
    """The runs plan_create would build, planned on the host only.  Returns
    (runs, rotations): runs is a list of (kind, d, count, basis) with kind 0 =
    fused coset run, 1 = diagonal phase-sum run; rotations = count after
    dropping identity strings."""
    x, z, a = _u64(x), _u64(z), _f64(angles)
    if not (len(x) == len(z) == len(a)):
        raise ValueError("x, z and angles must have equal length")
    nr, nrot = ctypes.c_size_t(), ctypes.c_size_t()
    L = lib()
    _check(L.plan_inspect(int(n_qubits), dtype_code(dtype), _p(x), _p(z), _p(a), len(a), int(fusion_depth),
                          None, 0, ctypes.byref(nr), ctypes.byref(nrot)))
    buf = (RunInfo * max(1, nr.value))()
    _check(L.plan_inspect(int(n_qubits), dtype_code(dtype), _p(x), _p(z), _p(a), len(a), int(fusion_depth),
                          buf, nr.value, ctypes.byref(nr), ctypes.byref(nrot)))
    runs = [(int(r.kind), int(r.d), int(r.count), [int(v) for v in r.basis[:r.d]]) for r in buf[:nr.value]]
    return runs, nrot.value


def batch_inspect(n_qubits, rotations, passes, grid_ctas: int):
    """The batched launch's work assignment on the host: (CTAs per state, the
    largest CTA load over the mean)."""
    nq = np.ascontiguousarray(n_qubits, dtype=np.int32)
    rot = np.ascontiguousarray(rotations, dtype=np.uint64)
    pas = np.ascontiguousarray(passes, dtype=np.uint64)
    if not (len(nq) == len(rot) == len(pas)):
        raise ValueError("one entry per state")
    ctas = np.empty(len(nq), dtype=np.int32)
    ratio = ctypes.c_double()
    _check(lib().batch_inspect(_p(nq), _p(rot), _p(pas), len(nq), int(grid_ctas), _p(ctas), ctypes.byref(ratio)))
    return ctas, ratio.value


def trotter_expand(x, z, c, dt: float, steps: int, order: int = 1, merge: bool = False):
    x, z, c = _u64(x), _u64(z), _f64(c)
    cnt = ctypes.c_size_t()
    L = lib()
    _check(L.trotter_expand(_p(x), _p(z), _p(c), len(c), float(dt), int(steps), int(order), int(merge),
                            None, None, None, 0, ctypes.byref(cnt)))
    m = cnt.value
    ox, oz, ot = np.empty(m, np.uint64), np.empty(m, np.uint64), np.empty(m, np.float64)
    _check(L.trotter_expand(_p(x), _p(z), _p(c), len(c), float(dt), int(steps), int(order), int(merge),
                            _p(ox), _p(oz), _p(ot), m, ctypes.byref(cnt)))
    return ox, oz, ot


def expval_pauli_sum(sv: int, x, z, coeff) -> Tuple[float, float]:
    x, z, c = _u64(x), _u64(z), _f64(coeff)
    e, nrm = ctypes.c_double(), ctypes.c_double()
    _check(lib().expval_pauli_sum(sv, _p(x), _p(z), _p(c), len(c), ctypes.byref(e), ctypes.byref(nrm)))
    return e.value, nrm.value


def expval_pauli_sum_noalloc(sv: int, x, z, coeff) -> Tuple[float, float]:
    """As expval_pauli_sum, through the entry point that allocates nothing
    (fixed device scratch inside the library; at most 4096 terms)."""
    x, z, c = _u64(x), _u64(z), _f64(coeff)
    e, nrm = ctypes.c_double(), ctypes.c_double()
    _check(lib().expval_pauli_sum_noalloc(sv, _p(x), _p(z), _p(c), len(c), ctypes.byref(e), ctypes.byref(nrm)))
    return e.value, nrm.value


def apply_pauli_sum(dst: int, src: int, x, z, coeff) -> None:
    x, z, c = _u64(x), _u64(z), _f64(coeff)
    _check(lib().apply_pauli_sum(dst, src, _p(x), _p(z), _p(c), len(c)))


def rotation_grads(psi0: int, x, z, angles, hx, hz, hc) -> Tuple[float, np.ndarray]:
    x, z, a = _u64(x), _u64(z), _f64(angles)
    hx, hz, hc = _u64(hx), _u64(hz), _f64(hc)
    g = np.empty(len(a), dtype=np.float64)
    e = ctypes.c_double()
    _check(lib().rotation_grads(psi0, _p(x), _p(z), _p(a), len(a), _p(hx), _p(hz), _p(hc), len(hc),
                                ctypes.byref(e), _p(g)))
    return e.value, g


def apply_pauli_rotations_gates(sv: int, x, z, angles) -> int:
    x, z, a = _u64(x), _u64(z), _f64(angles)
    n = ctypes.c_size_t()
    _check(lib().apply_pauli_rotations_gates(sv, _p(x), _p(z), _p(a), len(a), ctypes.byref(n)))
    return n.value


class BatchOpts(ctypes.Structure):
    _fields_ = [("wait_timeout_s", ctypes.c_double), ("test_skip_arrival", ctypes.c_int)]


def batch_run(states: Sequence[int], plans: Sequence[int], use_graph: bool = True) -> None:
    if len(states) != len(plans):
        raise ValueError("states and plans must have equal length")
    sa = (ctypes.c_void_p * len(states))(*states)
    pa = (ctypes.c_void_p * len(plans))(*plans)
    _check(lib().batch_run(sa, pa, len(states), 1 if use_graph else 0))


def batch_run_ex(states: Sequence[int], plans: Sequence[int], use_graph: bool = True,
                 wait_timeout_s: float = 0.0, test_skip_arrival: bool = False) -> None:
    if len(states) != len(plans):
        raise ValueError("states and plans must have equal length")
    sa = (ctypes.c_void_p * len(states))(*states)
    pa = (ctypes.c_void_p * len(plans))(*plans)
    opts = BatchOpts(float(wait_timeout_s), 1 if test_skip_arrival else 0)
    _check(lib().batch_run_ex(sa, pa, len(states), 1 if use_graph else 0, ctypes.byref(opts)))


def batch_info() -> Tuple[int, int, int]:
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().batch_info(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


class TraceRow(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 40), ("launches", ctypes.c_int64),
                ("total_ms", ctypes.c_double), ("bytes", ctypes.c_double), ("flops", ctypes.c_double)]


SV_TRACE_LAUNCHES, SV_TRACE_BLOCKS = 0, 1


def sv_trace_start(sv: int, blocks: bool = False) -> None:
    """Trace every launch (event pair each), or with blocks=True one event per
    change of kernel (consecutive launches of one kernel stay chained)."""
    _check(lib().sv_trace_start_ex(sv, SV_TRACE_BLOCKS if blocks else SV_TRACE_LAUNCHES))


def sv_trace_stop(sv: int) -> dict:
    """Returns {kernel name: (launches, total_ms, algorithmic_bytes, algorithmic_flops)}."""
    rows = (TraceRow * 64)()
    n = ctypes.c_int()
    _check(lib().sv_trace_stop(sv, rows, 64, ctypes.byref(n)))
    return {rows[i].name.decode(): (int(rows[i].launches), float(rows[i].total_ms), float(rows[i].bytes),
                                    float(rows[i].flops)) for i in range(n.value)}


def sv_probe_rate(kind: int, blocks: int, iters: int, dev_out: int, stream: int = 0) -> float:
    """Launch one arithmetic-rate probe (kind 0: FP64 FMA, 1: 32x32->64 integer
    multiply-add, 2: packed FP32x2 FMA) on `stream`; returns the operations it
    performs."""
    ops = ctypes.c_double()
    _check(lib().sv_probe_rate(int(kind), int(blocks), int(iters), ctypes.c_void_p(dev_out),
                               ctypes.c_void_p(stream), ctypes.byref(ops)))
    return ops.value


# ------------------------------------------------------------------ global-qubit sharding (host)

class ShardStep(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("partner", ctypes.c_int32), ("first", ctypes.c_int64),
                ("count", ctypes.c_int64)]


def _shard_call(name, n_qubits, global_qubits, rank, frame, x, z, v):
    x, z, v = _u64(x), _u64(z), _f64(v)
    if not (len(x) == len(z) == len(v)):
        raise ValueError("x, z and the values must have equal length")
    cap = len(v) + 1
    steps = (ShardStep * cap)()
    ns = ctypes.c_size_t()
    ox, oz, ov = np.zeros(len(v), np.uint64), np.zeros(len(v), np.uint64), np.zeros(len(v), np.float64)
    _check(getattr(lib(), name)(int(n_qubits), int(global_qubits), int(rank), frame, _p(x), _p(z), _p(v),
                                len(v), steps, cap, ctypes.byref(ns), _p(ox), _p(oz), _p(ov)))
    out = [(int(steps[k].kind), int(steps[k].partner), int(steps[k].first), int(steps[k].count))
           for k in range(ns.value)]
    return out, ox, oz, ov


def shard_rotations(n_qubits: int, global_qubits: int, rank: int, x, z, theta, frame: Optional[int] = None):
    """Rotations rewritten for one rank of a sharded state (through the Clifford
    frame `frame` first, if given): returns (steps, x, z, theta) with steps =
    [(kind, partner, first, count)]; kind 0 acts on the rank's slice, kind 1 on
    its pair state with `partner`."""
    return _shard_call("shard_rotations", n_qubits, global_qubits, rank, frame, x, z, theta)


def shard_terms(n_qubits: int, global_qubits: int, rank: int, x, z, coeff, frame: Optional[int] = None):
    """Pauli terms rewritten for one rank: returns (groups, x, z, coeff) with
    groups = [(kind, partner, first, count)], group 0 local to the slice."""
    return _shard_call("shard_terms", n_qubits, global_qubits, rank, frame, x, z, coeff)


# ------------------------------------------------------------------ Clifford-fullstate hybrid

SV_CG = {"h": 0, "s": 1, "sdg": 2, "x": 3, "y": 4, "z": 5, "cnot": 6, "cz": 7, "swap": 8,
         "rx": 9, "ry": 10, "rz": 11}


def _gates(gates):
    """[(name, q0[, q1][, theta]), ...] -> int32 codes, q0, q1 and float64 theta arrays.
    One-qubit gates take (name, q); two-qubit (name, q0, q1); rotations (name, q, theta)."""
    code = np.zeros(len(gates), dtype=np.int32)
    q0 = np.zeros(len(gates), dtype=np.int32)
    q1 = np.full(len(gates), -1, dtype=np.int32)
    th = np.zeros(len(gates), dtype=np.float64)
    for k, g in enumerate(gates):
        c = SV_CG[g[0].lower()]
        code[k], q0[k] = c, g[1]
        if c in (6, 7, 8):
            q1[k] = g[2]
        elif c >= 9:
            th[k] = g[2]
    return code, q0, q1, th


def cliff_create(n_qubits: int) -> int:
    h = ctypes.c_void_p()
    _check(lib().cliff_create(ctypes.byref(h), n_qubits))
    return h.value


def cliff_free(f: int) -> None:
    _check(lib().cliff_free(f))


def cliff_reset(f: int) -> None:
    _check(lib().cliff_reset(f))


def cliff_num_qubits(f: int) -> int:
    n = ctypes.c_int()
    _check(lib().cliff_num_qubits(f, ctypes.byref(n)))
    return n.value


def cliff_apply_gates(f: int, gates) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Returns the rotations (x, z, theta) the state must undergo, in order."""
    code, q0, q1, th = _gates(gates)
    cap = int(np.count_nonzero(code >= 9))
    ox, oz, ot = np.zeros(cap, np.uint64), np.zeros(cap, np.uint64), np.zeros(cap, np.float64)
    cnt = ctypes.c_size_t()
    _check(lib().cliff_apply_gates(f, _p(code), _p(q0), _p(q1), _p(th), len(code), _p(ox), _p(oz), _p(ot), cap,
                                   ctypes.byref(cnt)))
    return ox[:cnt.value], oz[:cnt.value], ot[:cnt.value]


def cliff_map_paulis(f: int, x, z) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    x, z = _u64(x), _u64(z)
    ox, oz = np.zeros(x.size, np.uint64), np.zeros(x.size, np.uint64)
    sg = np.zeros(x.size, np.int32)
    _check(lib().cliff_map_paulis(f, _p(x), _p(z), x.size, _p(ox), _p(oz), _p(sg)))
    return ox, oz, sg


def cliff_entry(f: int, qubit: int):
    """((ez_x, ez_z, ez_sign), (ex_x, ex_z, ex_sign)) of entry `qubit`."""
    v = [ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_int(), ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_int()]
    _check(lib().cliff_entry(f, qubit, *[ctypes.byref(a) for a in v]))
    return (v[0].value, v[1].value, v[2].value), (v[3].value, v[4].value, v[5].value)


def cliff_is_origin(f: int) -> bool:
    o = ctypes.c_int()
    _check(lib().cliff_is_origin(f, ctypes.byref(o)))
    return bool(o.value)


def cliff_inverse_rotations(f: int) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    cap = 4 * cliff_num_qubits(f)
    ox, oz, ot = np.zeros(cap, np.uint64), np.zeros(cap, np.uint64), np.zeros(cap, np.float64)
    cnt = ctypes.c_size_t()
    _check(lib().cliff_inverse_rotations(f, _p(ox), _p(oz), _p(ot), cap, ctypes.byref(cnt)))
    return ox[:cnt.value], oz[:cnt.value], ot[:cnt.value]


def cfhs_apply_gates(sv: int, f: int, gates) -> None:
    code, q0, q1, th = _gates(gates)
    _check(lib().cfhs_apply_gates(sv, f, _p(code), _p(q0), _p(q1), _p(th), len(code)))


def cfhs_apply_rotations(sv: int, f: int, x, z, angles) -> None:
    x, z, t = _u64(x), _u64(z), _f64(angles)
    _check(lib().cfhs_apply_rotations(sv, f, _p(x), _p(z), _p(t), t.size))


def cfhs_expval(sv: int, f: int, x, z, coeff) -> Tuple[float, float]:
    x, z, c = _u64(x), _u64(z), _f64(coeff)
    e, nrm = ctypes.c_double(), ctypes.c_double()
    _check(lib().cfhs_expval(sv, f, _p(x), _p(z), _p(c), c.size, ctypes.byref(e), ctypes.byref(nrm)))
    return e.value, nrm.value


def cfhs_materialize(sv: int, f: int) -> None:
    _check(lib().cfhs_materialize(sv, f))


def cfhs_measure_pauli(sv: int, f: Optional[int], x: int, z: int, u: float) -> Tuple[int, float]:
    """Measure the Pauli (x, z) on the state (through frame f, or None); returns
    (outcome +-1, its probability).  u: a uniform draw in [0, 1)."""
    o, p = ctypes.c_int(), ctypes.c_double()
    _check(lib().cfhs_measure_pauli(sv, f, int(x), int(z), float(u), ctypes.byref(o), ctypes.byref(p)))
    return o.value, p.value


def cfhs_prepare_qubit(sv: int, f: Optional[int], qubit: int, pauli: str, u: float) -> int:
    """Put `qubit` in the +1 eigenstate of pauli ('X', 'Y', 'Z'); returns the measured outcome."""
    o = ctypes.c_int()
    _check(lib().cfhs_prepare_qubit(sv, f, qubit, pauli.encode()[:1], float(u), ctypes.byref(o)))
    return o.value
