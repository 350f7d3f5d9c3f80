"""Thin ctypes binding of ``include/sptrsv.h``.

The functions here carry the C entry points' names and only marshal
arguments: integers, raw device pointers (``tensor.data_ptr()``) and CUDA
stream handles (``torch.cuda.Stream.cuda_stream``).  Every step of the solver
runs in the CUDA library; if the library cannot be loaded this module raises
instead of falling back to anything else.

``Plan`` is a convenience wrapper that takes torch tensors.
"""
from __future__ import annotations

import ctypes
import os
import threading
from ctypes import (byref, c_char_p, c_double, c_int32, c_int64, c_size_t, c_void_p,
                    create_string_buffer, POINTER, Structure)

from . import _build

SPTRSV_OK = 0
STATUS_NAMES = {
    0: "OK", 1: "INVALID_ARG", 2: "NOT_LOWER", 3: "UNSORTED", 4: "ZERO_DIAG",
    5: "MISSING_DIAG", 6: "OOM", 7: "CUDA", 8: "TIMEOUT", 9: "BAD_STATE",
    10: "UNSUPPORTED", 11: "BREAKDOWN", 12: "CODEGEN",
}
SELECT_NONE, SELECT_HEURISTIC, SELECT_COSTMODEL, SELECT_FIXED, SELECT_AUTO, SELECT_CRITPATH = \
    0, 1, 2, 3, 4, 5
SELECT_SEGMODEL = 6
SEG_FEATURES = 8
SOLVE_AUTO, SOLVE_BARRIER, SOLVE_SYNCFREE = 0, 1, 2
F64, F32_IR = 0, 1
OP_LOWER, OP_UPPER, OP_LOWER_TRANS, OP_UPPER_TRANS = 0, 1, 2, 3
PRECOND_SGS, PRECOND_IC0 = 0, 1


class SptrsvError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        self.name = STATUS_NAMES.get(code, str(code))
        super().__init__(f"{what}: SPTRSV_ERR_{self.name} ({_status_string(code)})")


class TransformParams(Structure):
    _fields_ = [
        ("select_mode", c_int32), ("depth", c_int32), ("thin_rows", c_int32),
        ("max_depth", c_int32), ("flop_budget", c_double),
        ("max_row_fill", c_int32), ("solve_mode", c_int32),
        ("precision", c_int32), ("ir_tol", c_double), ("ir_max_iter", c_int32),
        ("lanes_per_row", c_int32), ("block_threads", c_int32),
        ("cta_run_rows", c_int32), ("wait_timeout_ms", c_int32),
        ("grid_blocks", c_int32), ("poll_backoff_ns", c_int32), ("nrhs_hint", c_int32),
        ("tail_rows", c_int32), ("stage_z", c_int32), ("hop_weight", c_int32),
        ("codegen_rows", c_int32),
    ]


class Info(Structure):
    _fields_ = [
        ("n", c_int32), ("nnz", c_int64), ("nlev", c_int32), ("nlev_new", c_int32),
        ("rows_rewritten", c_int32), ("nnz_x", c_int64), ("nnz_b", c_int64),
        ("flops_plain", c_int64), ("flops_new", c_int64),
        ("select_mode", c_int32), ("solve_mode", c_int32), ("precision", c_int32),
        ("lanes_per_row", c_int32), ("block_threads", c_int32),
        ("grid_blocks", c_int32), ("cta_run_rows", c_int32),
        ("thin_rows", c_int32), ("max_depth", c_int32), ("flop_budget", c_double),
        ("ir_iters_last", c_int32), ("num_sms", c_int32), ("poll_backoff_ns", c_int32),
        ("chosen_depth", c_int32),
        ("analyze_ms", c_double), ("transform_ms", c_double), ("op", c_int32),
        ("tuned_from_cache", c_int32), ("tail_rows", c_int32), ("tail_levels", c_int32),
        ("stage_z", c_int32), ("codegen_segments", c_int32), ("codegen_ms", c_double),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_lock = threading.Lock()
_lib = None

# name -> (restype, argtypes)
_SIGS = {
    "sptrsv_status_string": (c_char_p, [c_int32]),
    "sptrsv_default_params": (None, [POINTER(TransformParams)]),
    "sptrsv_analyze": (c_int32, [c_int32, c_int64, c_void_p, c_void_p, c_void_p,
                                 c_void_p, POINTER(c_void_p)]),
    "sptrsv_analyze_ex": (c_int32, [c_int32, c_int64, c_void_p, c_void_p, c_void_p,
                                    c_int32, c_void_p, POINTER(c_void_p)]),
    "sptrsv_autotune_cache_clear": (None, []),
    "sptrsv_transform": (c_int32, [c_void_p, POINTER(TransformParams), c_void_p]),
    "sptrsv_solve": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_void_p]),
    "sptrsv_check": (c_int32, [c_void_p, c_void_p]),
    "sptrsv_get_info": (c_int32, [c_void_p, POINTER(Info)]),
    "sptrsv_plan_destroy": (None, [c_void_p]),
    "sptrsv_get_levels": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "sptrsv_get_segments": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "sptrsv_get_transformed": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p,
                                         c_void_p, c_void_p, c_void_p, c_void_p,
                                         c_void_p]),
    "sptrsv_debug_inject_wait": (c_int32, [c_void_p, c_int32]),
    "sptrsv_critical_path": (c_int32, [c_void_p, c_int32, POINTER(c_int64), c_void_p]),
    "sptrsv_codegen_source": (c_int32, [c_void_p, c_int32, c_char_p, c_size_t,
                                        POINTER(c_size_t)]),
    "sptrsv_codegen_source_from_records": (c_int32, [c_int32, c_int32, c_int32, c_void_p,
                                                     c_void_p, c_void_p, c_void_p, c_char_p,
                                                     c_size_t, POINTER(c_size_t)]),
    "sptrsv_level_features": (c_int32, [c_void_p, c_int32, c_void_p, c_void_p]),
    "sptrsv_costmodel_features": (c_int32, [c_void_p, c_void_p, c_int32, c_void_p, c_void_p]),
    "sptrsv_set_costmodel": (c_int32, [c_void_p, c_void_p]),
    "sptrsv_mlp_num_params": (c_int64, [c_int32, c_int32]),
    "sptrsv_mlp_create": (c_int32, [c_int32, c_int32, c_void_p, POINTER(c_void_p)]),
    "sptrsv_mlp_get_params": (c_int32, [c_void_p, c_void_p]),
    "sptrsv_mlp_set_normalization": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "sptrsv_mlp_forward": (c_int32, [c_void_p, c_void_p, c_int32, c_void_p, c_void_p]),
    "sptrsv_mlp_grads": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_void_p, c_void_p,
                                   c_void_p]),
    "sptrsv_mlp_train_step": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, ctypes.c_float,
                                        c_void_p, c_void_p]),
    "sptrsv_mlp_destroy": (None, [c_void_p]),
    "sptrsv_mlp_fit_normalization": (c_int32, [c_void_p, c_void_p, c_int32, c_void_p]),
    "sptrsv_mlp_normalize": (c_int32, [c_void_p, c_void_p, c_int32, c_void_p, c_void_p]),
    "sptrsv_mlp_get_normalization": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "sptrsv_mlp_save": (c_int32, [c_void_p, ctypes.c_char_p]),
    "sptrsv_mlp_load": (c_int32, [ctypes.c_char_p, POINTER(c_void_p)]),
    "sptrsv_costmodel_load": (c_int32, [ctypes.c_char_p]),
    "sptrsv_costmodel_save": (c_int32, [ctypes.c_char_p]),
    "sptrsv_costmodel_set_default": (c_int32, [c_void_p]),
    "sptrsv_segmodel_load": (c_int32, [c_char_p]),
    "sptrsv_segmodel_set_default": (c_int32, [c_void_p]),
    "sptrsv_segment_features": (c_int32, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p]),
    "sptrsv_level_times": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_void_p, c_void_p]),
    "sptrsv_batch_create": (c_int32, [c_void_p, c_int32, POINTER(c_void_p)]),
    "sptrsv_batch_solve": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "sptrsv_batch_check": (c_int32, [c_void_p, c_void_p]),
    "sptrsv_batch_get_info": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "sptrsv_batch_destroy": (None, [c_void_p]),
    "sptrsv_batch_get_times": (c_int32, [c_void_p, c_void_p]),
    "sptrsv_set_profiling": (c_int32, [c_void_p, c_int32]),
    "sptrsv_solve_ir_noalloc": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_void_p]),
    "sptrsv_last_kernel_ms": (c_int32, [c_void_p, POINTER(ctypes.c_float)]),
    "sptrsv_pcg_create": (c_int32, [c_int32, c_int64, c_void_p, c_void_p, c_void_p, c_int32,
                                    c_void_p, c_void_p, c_void_p, POINTER(c_void_p)]),
    "sptrsv_pcg_get_factor": (c_int32, [c_void_p, POINTER(c_int64), c_void_p, c_void_p]),
    "sptrsv_pcg_get_plans": (c_int32, [c_void_p, POINTER(c_void_p), POINTER(c_void_p)]),
    "sptrsv_pcg_solve": (c_int32, [c_void_p, c_void_p, c_void_p, c_double, c_int32,
                                   POINTER(c_int32), POINTER(c_double), c_void_p]),
    "sptrsv_pcg_destroy": (None, [c_void_p]),
}


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libsptrsv.so (building it from source if needed)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing:
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"the sptrsv CUDA library is missing ({path}); "
                               "build it with paper_2103_11445_gb300._build.build()")
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            if hasattr(lib, name):
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
        _lib = lib
        return lib


def _status_string(code: int) -> str:
    try:
        return load().sptrsv_status_string(code).decode()
    except Exception:  # pragma: no cover - only while the library is absent
        return STATUS_NAMES.get(code, "?")


def _check(code: int, what: str) -> None:
    if code != SPTRSV_OK:
        raise SptrsvError(code, what)


# --- C entry points, same names -------------------------------------------

def sptrsv_autotune_cache_clear() -> None:
    load().sptrsv_autotune_cache_clear()


def sptrsv_default_params() -> TransformParams:
    prm = TransformParams()
    load().sptrsv_default_params(byref(prm))
    return prm


def sptrsv_analyze(n: int, nnz: int, d_row_ptr: int, d_col: int, d_val: int,
                   stream: int = 0) -> int:
    out = c_void_p()
    _check(load().sptrsv_analyze(n, nnz, d_row_ptr, d_col, d_val, stream, byref(out)),
           "sptrsv_analyze")
    return out.value


def sptrsv_analyze_ex(n: int, nnz: int, d_row_ptr: int, d_col: int, d_val: int, op: int,
                      stream: int = 0) -> int:
    out = c_void_p()
    _check(load().sptrsv_analyze_ex(n, nnz, d_row_ptr, d_col, d_val, op, stream, byref(out)),
           "sptrsv_analyze_ex")
    return out.value


def sptrsv_transform(plan: int, prm: TransformParams, stream: int = 0) -> None:
    _check(load().sptrsv_transform(plan, byref(prm), stream), "sptrsv_transform")


def sptrsv_solve(plan: int, d_b: int, d_x: int, nrhs: int, stream: int = 0) -> None:
    _check(load().sptrsv_solve(plan, d_b, d_x, nrhs, stream), "sptrsv_solve")


def sptrsv_check(plan: int, stream: int = 0) -> int:
    return int(load().sptrsv_check(plan, stream))


def sptrsv_get_info(plan: int) -> Info:
    info = Info()
    _check(load().sptrsv_get_info(plan, byref(info)), "sptrsv_get_info")
    return info


def sptrsv_plan_destroy(plan: int) -> None:
    if plan:
        load().sptrsv_plan_destroy(plan)


def sptrsv_get_levels(plan: int, d_level: int, d_level_ptr: int, d_perm: int,
                      stream: int = 0) -> None:
    _check(load().sptrsv_get_levels(plan, d_level, d_level_ptr, d_perm, stream),
           "sptrsv_get_levels")


def sptrsv_get_segments(plan: int, nseg: int):
    first = (c_int32 * max(nseg, 1))()
    depth = (c_int32 * max(nseg, 1))()
    _check(load().sptrsv_get_segments(plan, first, depth), "sptrsv_get_segments")
    return list(first)[:nseg], list(depth)[:nseg]


def sptrsv_get_transformed(plan: int, d_new_level: int, d_xptr: int, d_xcol: int,
                           d_xval: int, d_bptr: int, d_bcol: int, d_bw: int,
                           stream: int = 0) -> None:
    _check(load().sptrsv_get_transformed(plan, d_new_level, d_xptr, d_xcol, d_xval,
                                         d_bptr, d_bcol, d_bw, stream),
           "sptrsv_get_transformed")


def sptrsv_debug_inject_wait(plan: int, row: int) -> None:
    _check(load().sptrsv_debug_inject_wait(plan, row), "sptrsv_debug_inject_wait")


def sptrsv_level_features(plan: int, nlev: int, lifts: int = 2, stream: int = 0):
    import numpy as np
    out = np.zeros((max(nlev, 0), 11 + lifts), dtype=np.float32)
    _check(load().sptrsv_level_features(plan, lifts, out.ctypes.data, stream),
           "sptrsv_level_features")
    return out


def sptrsv_critical_path(plan: int, hop_weight: int = 0, stream: int = 0) -> int:
    cp = c_int64()
    _check(load().sptrsv_critical_path(plan, hop_weight, byref(cp), stream),
           "sptrsv_critical_path")
    return cp.value


def sptrsv_codegen_source(plan: int, seg: int) -> str:
    n = c_size_t()
    _check(load().sptrsv_codegen_source(plan, seg, None, 0, byref(n)), "sptrsv_codegen_source")
    buf = create_string_buffer(n.value + 1)
    _check(load().sptrsv_codegen_source(plan, seg, buf, n.value + 1, byref(n)),
           "sptrsv_codegen_source")
    return buf.value.decode()


def sptrsv_codegen_source_from_records(nlev: int, row, nn, term, diag) -> str:
    """The generator on host records: row, nn int32 [nrows], term int32
    [K, nrows, 4], diag float64 [nrows, 2] (see the header)."""
    import numpy as np
    row = np.ascontiguousarray(row, np.int32)
    nn = np.ascontiguousarray(nn, np.int32)
    term = np.ascontiguousarray(term, np.int32)
    diag = np.ascontiguousarray(diag, np.float64)
    K, nrows = term.shape[0], term.shape[1]
    args = (nrows, K, nlev, row.ctypes.data, nn.ctypes.data, term.ctypes.data, diag.ctypes.data)
    n = c_size_t()
    _check(load().sptrsv_codegen_source_from_records(*args, None, 0, byref(n)),
           "sptrsv_codegen_source_from_records")
    buf = create_string_buffer(n.value + 1)
    _check(load().sptrsv_codegen_source_from_records(*args, buf, n.value + 1, byref(n)),
           "sptrsv_codegen_source_from_records")
    return buf.value.decode()


def sptrsv_solve_ir_noalloc(plan: int, d_b: int, d_x: int, nrhs: int,
                            stream: int = 0) -> None:
    _check(load().sptrsv_solve_ir_noalloc(plan, d_b, d_x, nrhs, stream),
           "sptrsv_solve_ir_noalloc")


def sptrsv_set_profiling(plan: int, on: bool) -> None:
    _check(load().sptrsv_set_profiling(plan, 1 if on else 0), "sptrsv_set_profiling")


def sptrsv_last_kernel_ms(plan: int) -> float:
    ms = ctypes.c_float()
    _check(load().sptrsv_last_kernel_ms(plan, byref(ms)), "sptrsv_last_kernel_ms")
    return float(ms.value)


COSTMODEL_FEATURES = 17


def sptrsv_costmodel_features(plan: int, codes, stream: int = 0):
    import numpy as np
    d = np.ascontiguousarray(codes, dtype=np.int32)
    out = np.zeros((d.size, COSTMODEL_FEATURES), dtype=np.float32)
    _check(load().sptrsv_costmodel_features(plan, d.ctypes.data, d.size, out.ctypes.data,
                                            stream), "sptrsv_costmodel_features")
    return out


def sptrsv_set_costmodel(plan: int, mlp: int) -> None:
    _check(load().sptrsv_set_costmodel(plan, mlp), "sptrsv_set_costmodel")


def sptrsv_mlp_num_params(n_in: int, hidden: int) -> int:
    return int(load().sptrsv_mlp_num_params(n_in, hidden))


def sptrsv_mlp_create(n_in: int, hidden: int, params) -> int:
    import numpy as np
    p = np.ascontiguousarray(params, dtype=np.float32)
    if p.size != sptrsv_mlp_num_params(n_in, hidden):
        raise ValueError("wrong number of network weights")
    out = c_void_p()
    _check(load().sptrsv_mlp_create(n_in, hidden, p.ctypes.data, byref(out)),
           "sptrsv_mlp_create")
    return out.value


def sptrsv_mlp_get_params(mlp: int, n_in: int, hidden: int):
    import numpy as np
    out = np.zeros(sptrsv_mlp_num_params(n_in, hidden), dtype=np.float32)
    _check(load().sptrsv_mlp_get_params(mlp, out.ctypes.data), "sptrsv_mlp_get_params")
    return out


def sptrsv_mlp_set_normalization(mlp: int, mean, std) -> None:
    import numpy as np
    m = np.ascontiguousarray(mean, dtype=np.float32)
    s = np.ascontiguousarray(std, dtype=np.float32)
    _check(load().sptrsv_mlp_set_normalization(mlp, m.ctypes.data, s.ctypes.data),
           "sptrsv_mlp_set_normalization")


def sptrsv_mlp_forward(mlp: int, d_X: int, N: int, d_y: int, stream: int = 0) -> None:
    _check(load().sptrsv_mlp_forward(mlp, d_X, N, d_y, stream), "sptrsv_mlp_forward")


def sptrsv_mlp_grads(mlp: int, d_X: int, d_t: int, N: int, d_grads: int, d_loss: int,
                     stream: int = 0) -> None:
    _check(load().sptrsv_mlp_grads(mlp, d_X, d_t, N, d_grads, d_loss, stream),
           "sptrsv_mlp_grads")


def sptrsv_mlp_train_step(mlp: int, d_X: int, d_t: int, N: int, lr: float, d_loss: int,
                          stream: int = 0) -> None:
    _check(load().sptrsv_mlp_train_step(mlp, d_X, d_t, N, lr, d_loss, stream),
           "sptrsv_mlp_train_step")


def sptrsv_mlp_destroy(mlp: int) -> None:
    if mlp:
        load().sptrsv_mlp_destroy(mlp)


def sptrsv_mlp_fit_normalization(mlp: int, d_X: int, N: int, stream: int = 0) -> None:
    _check(load().sptrsv_mlp_fit_normalization(mlp, d_X, N, stream),
           "sptrsv_mlp_fit_normalization")


def sptrsv_mlp_normalize(mlp: int, d_X: int, N: int, d_Xn: int, stream: int = 0) -> None:
    _check(load().sptrsv_mlp_normalize(mlp, d_X, N, d_Xn, stream), "sptrsv_mlp_normalize")


def sptrsv_mlp_get_normalization(mlp: int, n_in: int):
    import numpy as np
    mean = np.zeros(n_in, dtype=np.float32)
    std = np.zeros(n_in, dtype=np.float32)
    _check(load().sptrsv_mlp_get_normalization(mlp, mean.ctypes.data, std.ctypes.data),
           "sptrsv_mlp_get_normalization")
    return mean, std


def sptrsv_mlp_save(mlp: int, path: str) -> None:
    _check(load().sptrsv_mlp_save(mlp, os.fsencode(path)), "sptrsv_mlp_save")


def sptrsv_mlp_load(path: str) -> int:
    out = c_void_p()
    _check(load().sptrsv_mlp_load(os.fsencode(path), byref(out)), "sptrsv_mlp_load")
    return out.value


def sptrsv_costmodel_load(path: str) -> None:
    _check(load().sptrsv_costmodel_load(os.fsencode(path)), "sptrsv_costmodel_load")


def sptrsv_costmodel_save(path: str) -> None:
    _check(load().sptrsv_costmodel_save(os.fsencode(path)), "sptrsv_costmodel_save")


def sptrsv_costmodel_set_default(mlp: int) -> None:
    _check(load().sptrsv_costmodel_set_default(mlp), "sptrsv_costmodel_set_default")


def sptrsv_segmodel_load(path: str) -> None:
    _check(load().sptrsv_segmodel_load(os.fsencode(path)), "sptrsv_segmodel_load")


def sptrsv_segmodel_set_default(mlp: int) -> None:
    _check(load().sptrsv_segmodel_set_default(mlp), "sptrsv_segmodel_set_default")


def sptrsv_segment_features(plan: int, nlev: int, d_max: int, stream: int = 0):
    """(features [nlev, d_max + 1, SEG_FEATURES] float32, ok [nlev, d_max + 1] bool)."""
    import numpy as np
    f = np.zeros((nlev, d_max + 1, SEG_FEATURES), np.float32)
    ok = np.zeros((nlev, d_max + 1), np.uint8)
    _check(load().sptrsv_segment_features(plan, d_max, f.ctypes.data, ok.ctypes.data, stream),
           "sptrsv_segment_features")
    return f, ok.astype(bool)


def sptrsv_level_times(plan: int, d_b: int, d_x: int, nlev_new: int, reps: int = 3,
                       stream: int = 0):
    """Microseconds each new level adds to a solve (median over reps)."""
    import numpy as np
    us = np.zeros(nlev_new, np.float64)
    _check(load().sptrsv_level_times(plan, d_b, d_x, reps, us.ctypes.data, stream),
           "sptrsv_level_times")
    return us


def sptrsv_batch_create(plans) -> int:
    arr = (c_void_p * len(plans))(*plans)
    out = c_void_p()
    _check(load().sptrsv_batch_create(arr, len(plans), byref(out)), "sptrsv_batch_create")
    return out.value


def sptrsv_batch_solve(batch: int, b_ptrs, x_ptrs, nrhs, stream: int = 0) -> None:
    m = len(b_ptrs)
    bp = (c_void_p * m)(*b_ptrs)
    xp = (c_void_p * m)(*x_ptrs)
    nr = (c_int32 * m)(*nrhs)
    _check(load().sptrsv_batch_solve(batch, bp, xp, nr, stream), "sptrsv_batch_solve")


def sptrsv_batch_check(batch: int, stream: int = 0) -> int:
    return int(load().sptrsv_batch_check(batch, stream))


def sptrsv_batch_get_info(batch: int, count: int):
    it = (c_int32 * count)()
    cv = (c_int32 * count)()
    ct = (c_int32 * count)()
    g = c_int32()
    _check(load().sptrsv_batch_get_info(batch, it, cv, ct, byref(g)), "sptrsv_batch_get_info")
    return dict(iters=list(it), converged=list(cv), cta_count=list(ct), graph=g.value)


def sptrsv_batch_get_times(batch: int, count: int):
    ms = (ctypes.c_float * count)()
    _check(load().sptrsv_batch_get_times(batch, ms), "sptrsv_batch_get_times")
    return list(ms)


def sptrsv_batch_destroy(batch: int) -> None:
    if batch:
        load().sptrsv_batch_destroy(batch)


def sptrsv_pcg_create(n: int, nnz: int, d_row_ptr: int, d_col: int, d_val: int,
                      precond: int = PRECOND_SGS, prm_lower: TransformParams | None = None,
                      prm_upper: TransformParams | None = None, stream: int = 0) -> int:
    out = c_void_p()
    _check(load().sptrsv_pcg_create(n, nnz, d_row_ptr, d_col, d_val, precond,
                                    byref(prm_lower) if prm_lower is not None else None,
                                    byref(prm_upper) if prm_upper is not None else None,
                                    stream, byref(out)), "sptrsv_pcg_create")
    return out.value


def sptrsv_pcg_get_plans(pcg: int):
    lo, up = c_void_p(), c_void_p()
    _check(load().sptrsv_pcg_get_plans(pcg, byref(lo), byref(up)), "sptrsv_pcg_get_plans")
    return lo.value, up.value


def sptrsv_pcg_get_factor(pcg: int, d_val: int = 0, stream: int = 0) -> int:
    """Entries of the preconditioner's triangle; copies its values to d_val
    when given."""
    nnz = c_int64()
    _check(load().sptrsv_pcg_get_factor(pcg, byref(nnz), d_val or None, stream),
           "sptrsv_pcg_get_factor")
    return nnz.value


def sptrsv_pcg_solve(pcg: int, d_b: int, d_x: int, rtol: float, max_iter: int,
                     stream: int = 0):
    """(iterations, final relative residual norm)."""
    it, rel = c_int32(), c_double()
    _check(load().sptrsv_pcg_solve(pcg, d_b, d_x, rtol, max_iter, byref(it), byref(rel),
                                   stream), "sptrsv_pcg_solve")
    return it.value, rel.value


def sptrsv_pcg_destroy(pcg: int) -> None:
    if pcg:
        load().sptrsv_pcg_destroy(pcg)


# --- torch convenience wrapper ---------------------------------------------

def _stream_handle(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


class Plan:
    """Owns an sptrsv plan built from a CSR matrix held in torch tensors.

    ``row_ptr``/``col`` int32 and ``val`` float64 CUDA tensors (or numpy
    arrays, copied to the current device).  ``op`` (OP_*) names the system:
    A x = b for a lower (default) or upper A, or A^T x = b."""

    def __init__(self, n: int, row_ptr, col, val, stream=None, op: int = OP_LOWER):
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())

        def t(a, dt):
            if isinstance(a, torch.Tensor):
                return a.to(device=dev, dtype=dt).contiguous()
            return torch.as_tensor(a, dtype=dt, device=dev).contiguous()

        self.n = int(n)
        rp, c, v = t(row_ptr, torch.int32), t(col, torch.int32), t(val, torch.float64)
        self.nnz = int(c.numel())
        self._handle = 0
        self.op = int(op)
        self._handle = sptrsv_analyze_ex(self.n, self.nnz, rp.data_ptr(), c.data_ptr(),
                                         v.data_ptr(), self.op, _stream_handle(stream))

    @property
    def handle(self) -> int:
        return self._handle

    def transform(self, stream=None, **kw) -> "Plan":
        prm = sptrsv_default_params()
        for k, val in kw.items():
            if not hasattr(prm, k):
                raise TypeError(f"unknown transform parameter {k}")
            setattr(prm, k, val)
        sptrsv_transform(self._handle, prm, _stream_handle(stream))
        return self

    def solve(self, b, x=None, stream=None):
        """x = L^{-1} b for b of shape (n,) or (n, nrhs), float64 on the GPU."""
        import torch
        if b.dtype != torch.float64 or not b.is_cuda or not b.is_contiguous():
            raise TypeError("b must be a contiguous float64 CUDA tensor")
        nrhs = 1 if b.dim() == 1 else int(b.shape[1])
        if x is None:
            x = torch.empty_like(b)
        sptrsv_solve(self._handle, b.data_ptr(), x.data_ptr(), nrhs,
                     _stream_handle(stream))
        return x

    def check(self, stream=None) -> None:
        _check(sptrsv_check(self._handle, _stream_handle(stream)), "sptrsv_check")

    def info(self) -> dict:
        return sptrsv_get_info(self._handle).as_dict()

    def levels(self):
        import torch
        inf = self.info()
        dev = torch.device("cuda", torch.cuda.current_device())
        lv = torch.empty(self.n, dtype=torch.int32, device=dev)
        lp = torch.empty(inf["nlev"] + 1, dtype=torch.int32, device=dev)
        pm = torch.empty(self.n, dtype=torch.int32, device=dev)
        sptrsv_get_levels(self._handle, lv.data_ptr(), lp.data_ptr(), pm.data_ptr(),
                          _stream_handle(None))
        return lv, lp, pm

    def segments(self):
        return sptrsv_get_segments(self._handle, self.info()["nlev_new"])

    def segment_features(self, d_max: int = 4):
        """Features of every candidate segment (see sptrsv_segment_features)."""
        return sptrsv_segment_features(self._handle, self.info()["nlev"], d_max)

    def level_times(self, b, reps: int = 3):
        """Microseconds each new level adds to a solve of b (one column)."""
        import torch
        x = torch.empty_like(b)
        return sptrsv_level_times(self._handle, b.data_ptr(), x.data_ptr(),
                                  self.info()["nlev_new"], reps)

    def codegen_source(self, seg: int = 0) -> str:
        """Source of the kernel generated for tail segment seg."""
        return sptrsv_codegen_source(self._handle, seg)

    def transformed(self):
        """The transformed rows in original order (see sptrsv_get_transformed)."""
        import torch
        inf = self.info()
        dev = torch.device("cuda", torch.cuda.current_device())
        nl = torch.empty(self.n, dtype=torch.int32, device=dev)
        xp = torch.empty(self.n + 1, dtype=torch.int64, device=dev)
        bp = torch.empty(self.n + 1, dtype=torch.int64, device=dev)
        xc = torch.empty(max(inf["nnz_x"], 1), dtype=torch.int32, device=dev)
        xv = torch.empty(max(inf["nnz_x"], 1), dtype=torch.float64, device=dev)
        bc = torch.empty(max(inf["nnz_b"], 1), dtype=torch.int32, device=dev)
        bw = torch.empty(max(inf["nnz_b"], 1), dtype=torch.float64, device=dev)
        sptrsv_get_transformed(self._handle, nl.data_ptr(), xp.data_ptr(), xc.data_ptr(),
                               xv.data_ptr(), bp.data_ptr(), bc.data_ptr(), bw.data_ptr(),
                               _stream_handle(None))
        return dict(new_level=nl, xptr=xp, xcol=xc[:inf["nnz_x"]], xval=xv[:inf["nnz_x"]],
                    bptr=bp, bcol=bc[:inf["nnz_b"]], bw=bw[:inf["nnz_b"]])

    def close(self) -> None:
        if self._handle:
            sptrsv_plan_destroy(self._handle)
            self._handle = 0

    def __del__(self):  # pragma: no cover - interpreter shutdown order
        try:
            self.close()
        except Exception:
            pass


class PCG:
    """Owns a preconditioned-CG object built from a full symmetric CSR matrix
    in torch tensors or numpy arrays; ``precond`` is PRECOND_SGS or
    PRECOND_IC0; ``lower`` and ``upper`` are dicts of transform parameters
    for its two triangular plans (None: the library defaults)."""

    def __init__(self, n: int, row_ptr, col, val, lower=None, upper=None, stream=None,
                 precond: int = PRECOND_SGS):
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())

        def t(a, dt):
            return torch.as_tensor(a, dtype=dt, device=dev).contiguous()

        def prm(kw):
            if kw is None:
                return None
            p = sptrsv_default_params()
            for k, v in kw.items():
                if not hasattr(p, k):
                    raise TypeError(f"unknown transform parameter {k}")
                setattr(p, k, v)
            return p

        self.n = int(n)
        rp, c, v = t(row_ptr, torch.int32), t(col, torch.int32), t(val, torch.float64)
        self._handle = 0
        self._handle = sptrsv_pcg_create(self.n, int(c.numel()), rp.data_ptr(), c.data_ptr(),
                                         v.data_ptr(), int(precond), prm(lower), prm(upper),
                                         _stream_handle(stream))

    @property
    def handle(self) -> int:
        return self._handle

    def plan_info(self):
        """(info of the D + L plan, info of the (D + L)^T plan)."""
        lo, up = sptrsv_pcg_get_plans(self._handle)
        return sptrsv_get_info(lo).as_dict(), sptrsv_get_info(up).as_dict()

    def factor(self):
        """The triangle's values (D + L, or the IC(0) factor) in the order of
        A's lower-triangle entries."""
        import torch
        nnz = sptrsv_pcg_get_factor(self._handle)
        out = torch.empty(nnz, dtype=torch.float64,
                          device=torch.device("cuda", torch.cuda.current_device()))
        sptrsv_pcg_get_factor(self._handle, out.data_ptr(), _stream_handle(None))
        return out

    def solve(self, b, x=None, rtol: float = 1e-8, max_iter: int = 1000, stream=None):
        """(x, iterations, relative residual); x (if given) is the initial
        guess and is overwritten, else the iteration starts from zero."""
        import torch
        if b.dtype != torch.float64 or not b.is_cuda or not b.is_contiguous() or b.dim() != 1:
            raise TypeError("b must be a contiguous 1-D float64 CUDA tensor")
        if x is None:
            x = torch.zeros_like(b)
        it, rel = sptrsv_pcg_solve(self._handle, b.data_ptr(), x.data_ptr(), rtol, max_iter,
                                   _stream_handle(stream))
        return x, it, rel

    def close(self) -> None:
        if self._handle:
            sptrsv_pcg_destroy(self._handle)
            self._handle = 0

    def __del__(self):  # pragma: no cover - interpreter shutdown order
        try:
            self.close()
        except Exception:
            pass
