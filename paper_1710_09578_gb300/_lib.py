"""ctypes binding of ``include/fm.h`` (argument marshalling only).

Every function here has the name of the C entry point it wraps; it converts Python
arguments to C types, calls the library and raises ``FmError`` on a non-OK status.
There is no fallback: if the shared library is missing, importing this module fails.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libfastmat_gb300.so")

FM_OK = 0
STATUS = {0: "FM_OK", 1: "FM_ERR_INVALID_ARG", 2: "FM_ERR_SHAPE", 3: "FM_ERR_DTYPE",
          4: "FM_ERR_UNSUPPORTED", 5: "FM_ERR_ALIAS", 6: "FM_ERR_OOM", 7: "FM_ERR_CUDA",
          8: "FM_ERR_TIMEOUT", 9: "FM_ERR_NUMERIC"}
FM_I8, FM_I32, FM_F32, FM_F64, FM_C64, FM_C128 = range(6)
FM_HAD_FP32, FM_HAD_BF16, FM_HAD_BF16X2, FM_HAD_INT8 = range(4)


class FmError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")


class fm_fista_params(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("power_iters", ctypes.c_int32),
                ("lambda_rel", ctypes.c_double), ("safety", ctypes.c_double),
                ("accel", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("warm", ctypes.c_int32), ("k0", ctypes.c_int32)]


class fm_fista_report(ctypes.Structure):
    _fields_ = [("L", ctypes.c_void_p), ("lambda_", ctypes.c_void_p),
                ("objective", ctypes.c_void_p), ("status", ctypes.c_void_p)]


class fm_trace_entry(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_char * 64), ("ms", ctypes.c_float)]


class fm_tune_entry(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int64), ("n1", ctypes.c_int64), ("ncand", ctypes.c_int32),
                ("cand_n1", ctypes.c_int64 * 8), ("ms", ctypes.c_float * 8), ("kind", ctypes.c_int32)]


if not os.path.exists(LIB_PATH):
    raise ImportError(f"CUDA library not built: {LIB_PATH} is missing (run __graft_entry__.build())")
lib = ctypes.CDLL(LIB_PATH)

_p = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int
_op = ctypes.c_void_p
_opp = ctypes.POINTER(ctypes.c_void_p)

_SIGS = {
    "fm_fourier": [_i64, _i32, _opp],
    "fm_circulant": [_p, _i64, _i32, _p, _opp],
    "fm_toeplitz": [_p, _i64, _i64, _i32, _p, _opp],
    "fm_hadamard": [_i32, _i32, _opp],
    "fm_diag": [_p, _i64, _i32, _p, _opp],
    "fm_partial": [_p, _i64, _i64, _p, _opp],
    "fm_product": [_opp, _i32, _opp],
    "fm_sum": [_opp, _i32, _opp],
    "fm_blkdiag": [_opp, _i32, _opp],
    "fm_kron": [_opp, _i32, _opp],
    "fm_hermitian": [_op, _opp],
    "fm_blocks": [_opp, _i32, _i32, _opp],
    "fm_toeplitz2": [_p, _i64, _i64, _i64, _i64, _i32, _p, _opp],
    "fm_shape": [_op, ctypes.POINTER(_i64), ctypes.POINTER(_i64)],
    "fm_is_real": [_op, ctypes.POINTER(_i32)],
    "fm_out_dtype": [_op, _i32, ctypes.POINTER(_i32)],
    "fm_forward": [_op, _p, _i64, _i32, _p, _i64, _i32, _i64, _p],
    "fm_backward": [_op, _p, _i64, _i32, _p, _i64, _i32, _i64, _p],
    "fm_reserve": [_op, _i64, _i32, _p],
    "fm_circulant_apply_noalloc": [_op, _i32, _p, _i64, _p, _i64, _i64, _p],
    "fm_batch_create": [_opp, _i64, _p, _opp],
    "fm_batch_sizes": [_p, ctypes.POINTER(_i64), ctypes.POINTER(_i64)],
    "fm_fista": [_opp, _i64, ctypes.POINTER(_p), ctypes.POINTER(_p), ctypes.POINTER(fm_fista_params),
                 ctypes.POINTER(fm_fista_report), _p],
    "fm_fista_batch": [_p, _p, _p, _p, ctypes.POINTER(fm_fista_params), ctypes.POINTER(fm_fista_report), _p],
    "fm_batch_set_order": [_p, _i32],
    "fm_batch_tune": [_p, _p, _p, ctypes.POINTER(fm_fista_params), _p, ctypes.POINTER(ctypes.c_float),
                      ctypes.POINTER(_i32)],
    "fm_calibrate": [_op, _i64, _i32, _p, ctypes.POINTER(fm_tune_entry), _i32, ctypes.POINTER(_i32)],
    "fm_set_split": [_op, _i64, _i64, _p],
    "fm_set_plan": [_op, _i64, _i32, _i64, _p],
    "fm_signature": [_op, ctypes.c_char_p, _i32],
    "fm_param_grad": [_op, _op, _p, _i64, _i32, _p, _i64, _i32, _i64, _p, _i32, _p],
    "fm_omp": [_op, _p, _i32, _i32, _p, _p, _p],
    "fm_lfsr_circulant": [_i32, ctypes.c_uint64, ctypes.c_uint64, _i64, _p, _opp],
    "fm_set_dense": [_op, _i32, _p],
    "fm_calibrate_dense": [_op, _i64, _i32, _p, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float),
                           ctypes.POINTER(_i32)],
    "fm_trace_begin": [_i32],
    "fm_trace_end": [ctypes.POINTER(fm_trace_entry), _i32, ctypes.POINTER(_i32)],
}
for _name, _args in _SIGS.items():
    getattr(lib, _name).argtypes = _args
    getattr(lib, _name).restype = ctypes.c_int
lib.fm_release.argtypes = [_op]
lib.fm_release.restype = None
lib.fm_batch_release.argtypes = [_p]
lib.fm_batch_release.restype = None
lib.fm_status_string.argtypes = [ctypes.c_int]
lib.fm_status_string.restype = ctypes.c_char_p
lib.fm_last_error.argtypes = []
lib.fm_last_error.restype = ctypes.c_char_p
lib.fm_launch_count.argtypes = []
lib.fm_launch_count.restype = ctypes.c_uint64
lib.fm_version.argtypes = []
lib.fm_version.restype = ctypes.c_char_p

EXPORTED = sorted(list(_SIGS) + ["fm_release", "fm_batch_release", "fm_status_string",
                                 "fm_last_error", "fm_launch_count", "fm_version"])


def check(status: int, where: str) -> None:
    if status != FM_OK:
        raise FmError(status, where, lib.fm_last_error().decode(errors="replace"))


def _new(fn, *args):
    h = ctypes.c_void_p()
    check(getattr(lib, fn)(*args, ctypes.byref(h)), fn)
    return h.value


def _arr(handles):
    return (ctypes.c_void_p * len(handles))(*handles)


# ---------------------------------------------------------------- same-name wrappers
def fm_fourier(n: int, ortho: int = 0):
    return _new("fm_fourier", n, ortho)


def fm_circulant(c_ptr: int, n: int, dt: int, stream: int = 0):
    return _new("fm_circulant", c_ptr, n, dt, stream)


def fm_toeplitz(t_ptr: int, rows: int, cols: int, dt: int, stream: int = 0):
    return _new("fm_toeplitz", t_ptr, rows, cols, dt, stream)


def fm_hadamard(log2n: int, mode: int = FM_HAD_FP32):
    return _new("fm_hadamard", log2n, mode)


def fm_diag(d_ptr: int, n: int, dt: int, stream: int = 0):
    return _new("fm_diag", d_ptr, n, dt, stream)


def fm_partial(idx_ptr: int, m: int, n: int, stream: int = 0):
    return _new("fm_partial", idx_ptr, m, n, stream)


def fm_product(handles):
    return _new("fm_product", _arr(handles), len(handles))


def fm_sum(handles):
    return _new("fm_sum", _arr(handles), len(handles))


def fm_blkdiag(handles):
    return _new("fm_blkdiag", _arr(handles), len(handles))


def fm_kron(handles):
    return _new("fm_kron", _arr(handles), len(handles))


def fm_blocks(handles, nrows: int, ncols: int):
    return _new("fm_blocks", _arr(handles), nrows, ncols)


def fm_toeplitz2(t_ptr: int, r1: int, c1: int, r2: int, c2: int, dt: int, stream: int = 0):
    return _new("fm_toeplitz2", t_ptr, r1, c1, r2, c2, dt, stream)


def fm_hermitian(h):
    return _new("fm_hermitian", h)


def fm_shape(h):
    r, c = _i64(), _i64()
    check(lib.fm_shape(h, ctypes.byref(r), ctypes.byref(c)), "fm_shape")
    return r.value, c.value


def fm_is_real(h):
    r = _i32()
    check(lib.fm_is_real(h, ctypes.byref(r)), "fm_is_real")
    return bool(r.value)


def fm_out_dtype(h, in_dt: int) -> int:
    r = _i32()
    check(lib.fm_out_dtype(h, in_dt, ctypes.byref(r)), "fm_out_dtype")
    return r.value


def fm_forward(h, X: int, ldx: int, xdt: int, Y: int, ldy: int, ydt: int, ncols: int, stream: int = 0):
    check(lib.fm_forward(h, X, ldx, xdt, Y, ldy, ydt, ncols, stream), "fm_forward")


def fm_backward(h, Y: int, ldy: int, ydt: int, X: int, ldx: int, xdt: int, ncols: int, stream: int = 0):
    check(lib.fm_backward(h, Y, ldy, ydt, X, ldx, xdt, ncols, stream), "fm_backward")


def fm_reserve(h, ncols: int, xdt: int, stream: int = 0):
    check(lib.fm_reserve(h, ncols, xdt, stream), "fm_reserve")


def fm_calibrate(h, ncols: int, dt: int, stream: int = 0):
    """Time the candidates of every plan setting of h; returns one dict per tuned setting:
    L, kind (0 split, 1 tile shape, 2 radix schedule), the chosen value and {value: ms}."""
    rep = (fm_tune_entry * 64)()
    n = _i32(0)
    check(lib.fm_calibrate(h, ncols, dt, stream, rep, 64, ctypes.byref(n)), "fm_calibrate")
    out = []
    for e in rep[:min(n.value, 64)]:
        out.append({"L": int(e.L), "kind": int(e.kind), "value": int(e.n1),
                    "ms": {int(e.cand_n1[i]): float(e.ms[i]) for i in range(e.ncand)}})
    return out


def fm_set_plan(h, L: int, kind: int, value: int, stream: int = 0):
    check(lib.fm_set_plan(h, L, kind, value, stream), "fm_set_plan")


def fm_signature(h) -> str:
    buf = ctypes.create_string_buffer(1 << 16)
    check(lib.fm_signature(h, buf, len(buf)), "fm_signature")
    return buf.value.decode()


def fm_set_split(h, L: int, n1: int, stream: int = 0):
    check(lib.fm_set_split(h, L, n1, stream), "fm_set_split")


def fm_circulant_apply_noalloc(h, adjoint: int, X: int, ldx: int, Y: int, ldy: int, ncols: int,
                               stream: int = 0):
    check(lib.fm_circulant_apply_noalloc(h, adjoint, X, ldx, Y, ldy, ncols, stream),
          "fm_circulant_apply_noalloc")


def fm_batch_create(handles, stream: int = 0):
    return _new("fm_batch_create", _arr(handles), len(handles), stream)


def fm_batch_sizes(b):
    r, c = _i64(), _i64()
    check(lib.fm_batch_sizes(b, ctypes.byref(r), ctypes.byref(c)), "fm_batch_sizes")
    return r.value, c.value


def fm_fista(handles, b_ptrs, x_ptrs, params: fm_fista_params, report: fm_fista_report | None,
             stream: int = 0):
    """Solve len(handles) instances; b_ptrs / x_ptrs: device pointers, one per instance."""
    n = len(handles)
    if len(b_ptrs) != n or len(x_ptrs) != n:
        raise ValueError("one b and one x pointer per instance")
    bp = (ctypes.c_void_p * n)(*b_ptrs)
    xp = (ctypes.c_void_p * n)(*x_ptrs)
    rep = ctypes.byref(report) if report is not None else None
    check(lib.fm_fista(_arr(handles), n, bp, xp, ctypes.byref(params), rep, stream), "fm_fista")


def fm_batch_set_order(b, order: int):
    check(lib.fm_batch_set_order(b, order), "fm_batch_set_order")


def fm_batch_tune(b, b_ptr: int, x_ptr: int, params: fm_fista_params, stream: int = 0):
    """Time the two work-list orders; returns ([ms largest first, ms smallest first], chosen)."""
    ms = (ctypes.c_float * 2)()
    c = _i32()
    check(lib.fm_batch_tune(b, b_ptr, x_ptr, ctypes.byref(params), stream, ms, ctypes.byref(c)), "fm_batch_tune")
    return [float(ms[0]), float(ms[1])], int(c.value)


def fm_fista_batch(b, b_ptr: int, x_ptr: int, y_ptr: int | None, params: fm_fista_params,
                   report: fm_fista_report | None, stream: int = 0):
    rep = ctypes.byref(report) if report is not None else None
    check(lib.fm_fista_batch(b, b_ptr, x_ptr, y_ptr, ctypes.byref(params), rep, stream), "fm_fista_batch")


def fm_param_grad(h, leaf, X: int, ldx: int, xdt: int, G: int, ldg: int, gdt: int, ncols: int, grad: int,
                  grad_dt: int, stream: int = 0):
    check(lib.fm_param_grad(h, leaf, X, ldx, xdt, G, ldg, gdt, ncols, grad, grad_dt, stream), "fm_param_grad")


def fm_lfsr_circulant(nbits: int, taps: int, state: int, n: int, stream: int = 0):
    return _new("fm_lfsr_circulant", nbits, taps, state, n, stream)


def fm_set_dense(h, dense: int, stream: int = 0):
    check(lib.fm_set_dense(h, dense, stream), "fm_set_dense")


def fm_calibrate_dense(h, ncols: int, dt: int, stream: int = 0):
    """Time forward + adjoint fast and dense; returns (ms_fast, ms_dense, chosen)."""
    a, b, c = ctypes.c_float(), ctypes.c_float(), _i32()
    check(lib.fm_calibrate_dense(h, ncols, dt, stream, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
          "fm_calibrate_dense")
    return a.value, b.value, c.value


def fm_omp(h, b: int, dt: int, K: int, x: int, support: int | None, stream: int = 0):
    check(lib.fm_omp(h, b, dt, K, x, support, stream), "fm_omp")


def fm_trace_begin(max_launches: int):
    check(lib.fm_trace_begin(max_launches), "fm_trace_begin")


def fm_trace_end(max_entries: int = 1 << 16):
    """Stop tracing; returns [(kernel label, ms), ...] in launch order."""
    buf = (fm_trace_entry * max_entries)()
    n = _i32(0)
    check(lib.fm_trace_end(buf, max_entries, ctypes.byref(n)), "fm_trace_end")
    return [(e.kernel.decode(errors="replace"), float(e.ms)) for e in buf[:min(n.value, max_entries)]]


def fm_release(h):
    lib.fm_release(h)


def fm_batch_release(b):
    lib.fm_batch_release(b)


def fm_status_string(s: int) -> str:
    return lib.fm_status_string(s).decode()


def fm_last_error() -> str:
    return lib.fm_last_error().decode(errors="replace")


def fm_launch_count() -> int:
    return int(lib.fm_launch_count())


def fm_version() -> str:
    return lib.fm_version().decode()
