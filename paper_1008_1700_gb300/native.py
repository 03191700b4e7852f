"""ctypes binding of ``include/ddps.h`` (argument marshalling only).

Every function here has the name of the C entry point it calls.  Tensors are
passed as raw device pointers on the caller's current CUDA stream; NumPy
arrays as host pointers.  Nothing is computed in Python: if the library is not
built, loading fails with an error instead of falling back to anything.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libddps.so")

DDPS_FP64, DDPS_FP32, DDPS_BF16, DDPS_BF16X3, DDPS_FP16 = 0, 1, 2, 3, 4
DDPS_DROP_NONE, DDPS_DROP_COLUMN, DDPS_DROP_ABS = 0, 1, 2
DDPS_GHAT_EXPLICIT, DDPS_GHAT_IMPLICIT = 0, 1
DDPS_REDUCED_ITERATIVE, DDPS_REDUCED_DIRECT = 0, 1
DDPS_FACTOR_LU, DDPS_FACTOR_ILU0 = 0, 1
STATUS = {0: "DDPS_OK", 1: "DDPS_ERR_INVALID_ARG", 2: "DDPS_ERR_SINGULAR_BLOCK",
          3: "DDPS_ERR_NOT_CONVERGED", 4: "DDPS_ERR_OUT_OF_MEMORY", 5: "DDPS_ERR_CUDA",
          6: "DDPS_ERR_TIMEOUT", 7: "DDPS_ERR_STATE"}


class ddps_options(C.Structure):
    _fields_ = [("drop_mode", C.c_int32), ("drop_tol", C.c_double),
                ("factor_prec", C.c_int32), ("spike_prec", C.c_int32),
                ("ghat_prec", C.c_int32), ("inner_prec", C.c_int32),
                ("tol_out", C.c_double), ("maxit_out", C.c_int32),
                ("tol_in", C.c_double), ("maxit_in", C.c_int32),
                ("pivot_tol", C.c_double), ("leaf_size", C.c_int32),
                ("rhs_chunk", C.c_int32), ("verbose", C.c_int32),
                ("debug_wait_timeout", C.c_int32), ("fused_rows", C.c_int32),
                ("ghat_mode", C.c_int32), ("update_prec", C.c_int32),
                ("reduced_solver", C.c_int32), ("use_graphs", C.c_int32),
                ("persistent_solve", C.c_int32), ("factor_kind", C.c_int32),
                ("autotune", C.c_int32), ("csr_kernel", C.c_int32)]


class ddps_solve_info(C.Structure):
    _fields_ = [("outer_iterations", C.c_double), ("inner_iterations", C.c_int32),
                ("precond_applies", C.c_int32), ("converged", C.c_int32),
                ("guess_used", C.c_int32), ("relres_inf", C.c_double),
                ("first_inner_iters", C.c_double), ("ms_solve", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ddps_sizes(C.Structure):
    _fields_ = [(k, C.c_int64) for k in ("n", "nnz", "nsys", "nblocks", "m", "nnz_rt", "nfronts",
                                          "nlevels", "factor_entries", "factor_lu_entries",
                                          "ghat_entries", "max_front", "max_rhs", "device_bytes")] + \
               [("factor_flops", C.c_double), ("spike_flops", C.c_double),
                ("direct_flops", C.c_double), ("direct_bytes", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class DDPSError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


_lib = None
_p = C.c_void_p
_i32, _i64, _f64 = C.c_int32, C.c_int64, C.c_double


def load():
    """Load ``_build/libddps.so``; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"DDPS CUDA library not built: {LIB_PATH} is missing "
                          "(run __graft_entry__.build() or paper_1008_1700_gb300/build.py)")
    lib = C.CDLL(LIB_PATH)
    sig = {
        "ddps_default_options": (None, [C.POINTER(ddps_options)]),
        "ddps_analyze": (_i32, [_i64, _i64, _p, _p, _i32, _p, _i32, _p, _p,
                                C.POINTER(ddps_options), C.POINTER(_p)]),
        "ddps_factor": (_i32, [_p, _p, _p]),
        "ddps_factor_host": (_i32, [_p, _p, _p]),
        "ddps_solve": (_i32, [_p, _p, _p, _i32, _p, _p, C.POINTER(ddps_solve_info)]),
        "ddps_solve_host": (_i32, [_p, _p, _p, _i32, _p, _p, C.POINTER(ddps_solve_info)]),
        "ddps_set_reduced_guess": (_i32, [_p, _p, _p]),
        "ddps_get_reduced_solution": (_i32, [_p, _p, _p, _p]),
        "ddps_block_solve": (_i32, [_p, _p, _p, _p]),
        "ddps_block_solve_noalloc": (_i32, [_p, _p, _p, _p]),
        "ddps_reduced_matvec": (_i32, [_p, _p, _p, _p]),
        "ddps_reduced_rhs": (_i32, [_p, _p, _p, _p]),
        "ddps_reduced_solve": (_i32, [_p, _p, _p, _p]),
        "ddps_precond_apply": (_i32, [_p, _p, _p, _p]),
        "ddps_spmv": (_i32, [_p, _p, _p, _p]),
        "ddps_get_sizes": (_i32, [_p, C.POINTER(ddps_sizes)]),
        "ddps_get_interface": (_i32, [_p, _p]),
        "ddps_get_tuning": (_i32, [_p, C.c_char_p, _i64, C.POINTER(_i64)]),
        "ddps_get_ghat_layout": (_i32, [_p, _i32, C.POINTER(_i64), C.POINTER(_i64),
                                        C.POINTER(_i64), _p]),
        "ddps_get_ghat_block": (_i32, [_p, _i32, _p, _p]),
        "ddps_destroy": (_i32, [_p]),
        "ddps_last_error": (C.c_char_p, [_p]),
        "ddps_status_string": (C.c_char_p, [_i32]),
        "ddps_launch_count": (_i64, [_p]),
        "ddps_set_profiling": (_i32, [_p, _i32]),
        "ddps_get_profile": (_i32, [_p, _p, _p, _i32]),
        "ddps_symbolic": (_i32, [_i64, _i64, _p, _p, _i32, _p, _i32, _p, _p,
                                 C.POINTER(ddps_options), C.POINTER(ddps_sizes), _p, _p]),
        "ddps_mlp_param_count": (_i64, [_i32, _i32, _i32, _i32]),
        "ddps_mlp_workspace_bytes": (_i64, [_i32, _i32, _i32, _i32, _i32]),
        "ddps_mlp_forward": (_i32, [_p, _i32, _i32, _i32, _i32, _p, _i32, _p, _p, _p]),
        "ddps_mlp_backward": (_i32, [_p, _i32, _i32, _i32, _i32, _p, _p, _i32, _p, _p, _p, _p]),
        "ddps_mlp_adam": (_i32, [_p, _p, _p, _p, _i64, C.c_float, C.c_float, C.c_float,
                                 C.c_float, _i32, _p]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    """Names of the ``ddps_*`` entry points the library exports."""
    lib = load()
    return {n for n in _declared_names() if hasattr(lib, n)}


def _declared_names():
    import re
    hdr = os.path.join(os.path.dirname(_HERE), "include", "ddps.h")
    with open(hdr) as fh:
        text = fh.read()
    return set(re.findall(r"\b(ddps_[a-z0-9_]+)\s*\(", text))


def _ptr(a):
    """Device or host pointer of a torch tensor / numpy array (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays passed to the DDPS library must be contiguous")
        return a.ctypes.data
    if not a.is_contiguous():
        raise ValueError("tensors passed to the DDPS library must be contiguous")
    return a.data_ptr()


def _stream(stream):
    if stream is not None:
        return stream
    import torch
    return torch.cuda.current_stream().cuda_stream


def _check(st, h=None):
    if st != 0:
        msg = load().ddps_last_error(h)
        raise DDPSError(st, msg.decode() if msg else "")


def default_options(**kw) -> ddps_options:
    o = ddps_options()
    load().ddps_default_options(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(f"unknown option {k}")
        setattr(o, k, v)
    return o


def _host_pattern(rowptr, colind, block_ptr, sys_block_ptr, values):
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
    colind = np.ascontiguousarray(colind, dtype=np.int32)
    block_ptr = np.ascontiguousarray(block_ptr, dtype=np.int64)
    sbp = None if sys_block_ptr is None else np.ascontiguousarray(sys_block_ptr, dtype=np.int32)
    vals = None if values is None else np.ascontiguousarray(values, dtype=np.float64)
    return rowptr, colind, block_ptr, sbp, vals


def ddps_analyze(rowptr, colind, block_ptr, sys_block_ptr=None, values=None, options=None):
    """Symbolic phase; returns the handle (c_void_p)."""
    lib = load()
    rowptr, colind, block_ptr, sbp, vals = _host_pattern(rowptr, colind, block_ptr, sys_block_ptr,
                                                         values)
    n = len(rowptr) - 1
    nsys = 1 if sbp is None else len(sbp) - 1
    opt = options if options is not None else default_options()
    h = _p()
    st = lib.ddps_analyze(n, int(rowptr[-1]), _ptr(rowptr), _ptr(colind), len(block_ptr) - 1,
                          _ptr(block_ptr), nsys, _ptr(sbp), _ptr(vals), C.byref(opt), C.byref(h))
    _check(st, None)
    return h


def ddps_symbolic(rowptr, colind, block_ptr, sys_block_ptr=None, values=None, options=None):
    """Host-only analysis: returns (sizes dict, perm, c)."""
    lib = load()
    rowptr, colind, block_ptr, sbp, vals = _host_pattern(rowptr, colind, block_ptr, sys_block_ptr,
                                                         values)
    n = len(rowptr) - 1
    nsys = 1 if sbp is None else len(sbp) - 1
    opt = options if options is not None else default_options()
    sz = ddps_sizes()
    perm = np.zeros(n, dtype=np.int32)
    c = np.zeros(n, dtype=np.int64)
    st = lib.ddps_symbolic(n, int(rowptr[-1]), _ptr(rowptr), _ptr(colind), len(block_ptr) - 1,
                           _ptr(block_ptr), nsys, _ptr(sbp), _ptr(vals), C.byref(opt),
                           C.byref(sz), _ptr(perm), _ptr(c))
    _check(st, None)
    d = sz.as_dict()
    return d, perm, c[: d["m"]].copy()


def ddps_factor(h, values, stream=None):
    _check(load().ddps_factor(h, _ptr(values), _stream(stream)), h)


def ddps_factor_host(h, values, stream=None):
    """ddps_factor with the values in host memory (a NumPy array or a CPU tensor)."""
    _check(load().ddps_factor_host(h, _ptr(values), _stream(stream)), h)


def _nrhs(f):
    shape = tuple(f.shape)
    return 1 if len(shape) == 1 else int(shape[0])


def ddps_solve(h, f, x, x0=None, stream=None, check=True):
    """f, x (and x0): device tensors of shape (n,) or (nrhs, n)."""
    info = ddps_solve_info()
    st = load().ddps_solve(h, _ptr(f), _ptr(x), _nrhs(f), _ptr(x0), _stream(stream),
                           C.byref(info))
    if check and st not in (0, 3):
        _check(st, h)
    return st, info.as_dict()


def ddps_solve_host(h, f, x, x0=None, stream=None):
    """f, x (and x0): host arrays of shape (n,) or (nrhs, n)."""
    info = ddps_solve_info()
    st = load().ddps_solve_host(h, _ptr(f), _ptr(x), _nrhs(f), _ptr(x0), _stream(stream),
                                C.byref(info))
    if st not in (0, 3):
        _check(st, h)
    return st, info.as_dict()


def ddps_set_reduced_guess(h, zhat0, stream=None):
    _check(load().ddps_set_reduced_guess(h, _ptr(zhat0), _stream(stream)), h)


def ddps_get_reduced_solution(h, zhat, ghat, stream=None):
    _check(load().ddps_get_reduced_solution(h, _ptr(zhat), _ptr(ghat), _stream(stream)), h)


def ddps_block_solve(h, y, g, stream=None):
    _check(load().ddps_block_solve(h, _ptr(y), _ptr(g), _stream(stream)), h)


def ddps_block_solve_noalloc(h, y, g, stream=None):
    """ddps_block_solve with scratch from the library's fixed array (no allocation)."""
    _check(load().ddps_block_solve_noalloc(h, _ptr(y), _ptr(g), _stream(stream)), h)


def ddps_reduced_rhs(h, y, ghat, stream=None):
    _check(load().ddps_reduced_rhs(h, _ptr(y), _ptr(ghat), _stream(stream)), h)


def ddps_reduced_matvec(h, v, w, stream=None):
    _check(load().ddps_reduced_matvec(h, _ptr(v), _ptr(w), _stream(stream)), h)


def ddps_reduced_solve(h, ghat, zhat, stream=None):
    _check(load().ddps_reduced_solve(h, _ptr(ghat), _ptr(zhat), _stream(stream)), h)


def ddps_precond_apply(h, y, z, stream=None):
    _check(load().ddps_precond_apply(h, _ptr(y), _ptr(z), _stream(stream)), h)


def ddps_spmv(h, x, y, stream=None):
    _check(load().ddps_spmv(h, _ptr(x), _ptr(y), _stream(stream)), h)


def ddps_get_sizes(h):
    s = ddps_sizes()
    _check(load().ddps_get_sizes(h, C.byref(s)), h)
    return s.as_dict()


def ddps_get_tuning(h):
    """The autotuner's choices (parsed JSON)."""
    import json
    n = _i64()
    _check(load().ddps_get_tuning(h, None, 0, C.byref(n)), h)
    buf = C.create_string_buffer(n.value + 1)
    _check(load().ddps_get_tuning(h, buf, n.value + 1, None), h)
    return json.loads(buf.value.decode())


def ddps_get_interface(h):
    m = ddps_get_sizes(h)["m"]
    c = np.zeros(max(m, 1), dtype=np.int64)
    _check(load().ddps_get_interface(h, _ptr(c)), h)
    return c[:m]


def ddps_get_ghat_layout(h, b):
    q0, q1, nc = _i64(), _i64(), _i64()
    _check(load().ddps_get_ghat_layout(h, b, C.byref(q0), C.byref(q1), C.byref(nc), None), h)
    cols = np.zeros(max(nc.value, 1), dtype=np.int64)
    _check(load().ddps_get_ghat_layout(h, b, C.byref(q0), C.byref(q1), C.byref(nc), _ptr(cols)), h)
    return q0.value, q1.value, cols[: nc.value]


def ddps_get_ghat_block(h, b, stream=None):
    q0, q1, cols = ddps_get_ghat_layout(h, b)
    out = np.zeros(max((q1 - q0) * len(cols), 1))
    _check(load().ddps_get_ghat_block(h, b, _ptr(out), _stream(stream)), h)
    return out[: (q1 - q0) * len(cols)].reshape(q1 - q0, len(cols))


def ddps_launch_count(h):
    return int(load().ddps_launch_count(h))


PROF_CLASSES = ["assemble", "extend_add", "front_lu", "spike_fwd", "spike_bwd", "ghat_extract",
                "block_solve", "ghat_matvec", "spmv", "direct_factor", "direct_solve"]


def ddps_set_profiling(h, mask):
    _check(load().ddps_set_profiling(h, int(mask)), h)


def ddps_get_profile(h, reset=True):
    """{class: (milliseconds, launch groups)} since the last reset."""
    ms = np.zeros(len(PROF_CLASSES))
    cnt = np.zeros(len(PROF_CLASSES), dtype=np.int64)
    _check(load().ddps_get_profile(h, _ptr(ms), _ptr(cnt), 1 if reset else 0), h)
    return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(PROF_CLASSES)}


def ddps_destroy(h):
    if h:
        load().ddps_destroy(h)


def ddps_mlp_param_count(d_in, hidden, layers, d_out):
    return int(load().ddps_mlp_param_count(d_in, hidden, layers, d_out))


def ddps_mlp_workspace_bytes(d_in, hidden, layers, d_out, B):
    return int(load().ddps_mlp_workspace_bytes(d_in, hidden, layers, d_out, B))


def ddps_mlp_forward(params, d_in, hidden, layers, d_out, X, B, Y, workspace, stream=None):
    _check(load().ddps_mlp_forward(_ptr(params), d_in, hidden, layers, d_out, _ptr(X), B, _ptr(Y),
                                   _ptr(workspace), _stream(stream)))


def ddps_mlp_backward(params, d_in, hidden, layers, d_out, X, T, B, grads, loss, workspace,
                      stream=None):
    _check(load().ddps_mlp_backward(_ptr(params), d_in, hidden, layers, d_out, _ptr(X), _ptr(T), B,
                                    _ptr(grads), _ptr(loss), _ptr(workspace), _stream(stream)))


def ddps_mlp_adam(params, grads, m, v, count, lr, beta1, beta2, eps, step, stream=None):
    _check(load().ddps_mlp_adam(_ptr(params), _ptr(grads), _ptr(m), _ptr(v), count, lr, beta1,
                                beta2, eps, step, _stream(stream)))
