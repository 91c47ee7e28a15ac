"""Structured linear operators on one GB300 GPU (the fastmat method, arXiv 1710.09578).

Thin Python layer over the C ABI in ``include/fm.h``: operators are immutable handles
built from parameter vectors (Sec. 2.1.1), composed with ``product`` / ``sum`` /
``blkdiag`` / ``kron`` / ``.H``, and applied to blocks of columns with ``forward``
(phi, Eq. (3)) and ``backward`` (beta, Eq. (4)).  PyTorch supplies device memory and
the current stream only; every step of a transform runs in the library's CUDA kernels.

Column blocks are torch tensors of shape ``[K, n]`` (K columns of length n, each
contiguous) or 1-D tensors of length n.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import (FM_HAD_BF16, FM_HAD_BF16X2, FM_HAD_FP32, FM_HAD_INT8, FmError,  # noqa: F401
                   fm_fista_params, fm_fista_report)

__all__ = ["Op", "fourier", "circulant", "lfsr_circulant", "toeplitz", "toeplitz2", "hadamard", "diag", "partial",
           "product",
           "blocks",
           "sum_", "blkdiag", "kron", "FmApply", "apply", "param_grad", "FmParamApply", "apply_params",
           "FistaBatch", "fista", "omp", "FmError",
           "FM_HAD_FP32", "FM_HAD_BF16", "FM_HAD_BF16X2", "FM_HAD_INT8", "launch_count"]

_TORCH2FM = {torch.int8: _lib.FM_I8, torch.int32: _lib.FM_I32, torch.float32: _lib.FM_F32,
             torch.float64: _lib.FM_F64, torch.complex64: _lib.FM_C64, torch.complex128: _lib.FM_C128}
_FM2TORCH = {v: k for k, v in _TORCH2FM.items()}
_NP2FM = {np.dtype(np.float32): _lib.FM_F32, np.dtype(np.float64): _lib.FM_F64,
          np.dtype(np.complex64): _lib.FM_C64, np.dtype(np.complex128): _lib.FM_C128}


def launch_count() -> int:
    """Kernels launched by the library in this process."""
    return _lib.fm_launch_count()


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0


def _param(x, allow_int=False):
    """(pointer, fm dtype, keep-alive) for a parameter vector in host or device memory."""
    if isinstance(x, torch.Tensor):
        t = x.contiguous()
        if allow_int:
            return t.data_ptr(), None, t
        return t.data_ptr(), _TORCH2FM[t.dtype], t
    a = np.ascontiguousarray(x)
    if allow_int:
        a = np.ascontiguousarray(a, dtype=np.int32)
        return a.ctypes.data, None, a
    if a.dtype.kind in "iu":
        a = a.astype(np.float64)
    return a.ctypes.data, _NP2FM[a.dtype], a


class Op:
    """An immutable structured operator (handle to the C library)."""

    def __init__(self, handle: int, kids=(), kind: str = ""):
        self._h = handle
        self._kids = tuple(kids)  # composites also hold C references; kept for clarity
        self.kind = kind
        self.rows, self.cols = _lib.fm_shape(handle)
        self.real = _lib.fm_is_real(handle)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _lib.fm_release(h)
            self._h = None

    @property
    def handle(self) -> int:
        return self._h

    @property
    def shape(self):
        return (self.rows, self.cols)

    @property
    def H(self) -> "Op":
        return Op(_lib.fm_hermitian(self._h), (self,))

    def out_dtype(self, dtype: torch.dtype) -> torch.dtype:
        return _FM2TORCH[_lib.fm_out_dtype(self._h, _TORCH2FM[dtype])]

    def _apply(self, X: torch.Tensor, adjoint: bool, out: torch.Tensor | None = None,
               real_out: bool = False) -> torch.Tensor:
        if not isinstance(X, torch.Tensor) or not X.is_cuda:
            raise TypeError("X must be a CUDA tensor")
        one = X.dim() == 1
        X2 = X.unsqueeze(0) if one else X
        if X2.dim() != 2:
            raise ValueError("X must be [K, n] or [n]")
        if X2.stride(-1) != 1:
            X2 = X2.contiguous()
        nin, nout = (self.rows, self.cols) if adjoint else (self.cols, self.rows)
        if X2.shape[1] != nin:
            raise ValueError(f"expected columns of length {nin}, got {X2.shape[1]}")
        k = X2.shape[0]
        odt = self.out_dtype(X2.dtype)
        if real_out and odt.is_complex:
            odt = torch.float32 if odt == torch.complex64 else torch.float64
        if out is None:
            Y = torch.empty((k, nout), dtype=odt, device=X2.device)
        else:
            Y = out.view(k, nout) if out.dim() == 1 else out
            if Y.dtype != odt or Y.stride(-1) != 1 or tuple(Y.shape) != (k, nout):
                raise ValueError("bad output tensor")
        ldx = X2.stride(0) if k > 1 else nin
        ldy = Y.stride(0) if k > 1 else nout
        fn = _lib.fm_backward if adjoint else _lib.fm_forward
        fn(self._h, X2.data_ptr(), ldx, _TORCH2FM[X2.dtype], Y.data_ptr(), ldy, _TORCH2FM[odt], k, _stream())
        return Y[0] if one and out is None else Y

    def forward(self, X, out=None, real_out: bool = False):
        """phi_A(X) = A X (Eq. (3)); real_out: Re(A X) when A X would be complex."""
        return self._apply(X, False, out, real_out)

    def backward(self, Y, out=None, real_out: bool = False):
        """beta_A(Y) = A^H Y (Eq. (4)); real_out: Re(A^H Y), the adjoint of A on real inputs."""
        return self._apply(Y, True, out, real_out)

    def reserve(self, ncols: int, dtype: torch.dtype):
        """Grow the workspace so that later calls on up to ncols columns allocate nothing."""
        _lib.fm_reserve(self._h, ncols, _TORCH2FM[dtype], _stream())

    def signature(self) -> str:
        """Text description of the operator tree (``fm_signature``)."""
        return _lib.fm_signature(self._h)

    def calibrate(self, ncols: int, dtype: torch.dtype = torch.complex64, cache: str | None = None,
                  key: str | None = None):
        """Choose the execution plan of every transform in this operator by timing forward +
        adjoint on ncols probe columns (the GPU form of the paper's calibration): the split of
        long transforms, the tile shape of strided views and the radix schedule.

        With `cache` (a JSON file path) the choices are stored under `key` (default: the
        operator's signature, ncols, dtype and the GPU's SM count) and a later call with the
        same key restores them without timing.  Returns the list of {"L", "kind", "value", "ms"}
        entries that were applied (kind 0 split, 1 tile shape, 2 radix schedule, 3 fused Kron
        pass)."""
        import json
        import os
        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        key = key or f"{self.signature()}|n={self.cols}|ncols={ncols}|{str(dtype).replace('torch.', '')}|sm={sms}"
        table = {}
        if cache and os.path.exists(cache):
            with open(cache) as f:
                table = json.load(f)
        if key in table:
            for e in table[key]:
                _lib.fm_set_plan(self._h, int(e["L"]), int(e["kind"]), int(e["value"]), _stream())
            return table[key]
        res = _lib.fm_calibrate(self._h, ncols, _TORCH2FM[dtype], _stream())
        if cache:
            table[key] = [{"L": e["L"], "kind": e["kind"], "value": e["value"],
                           "ms": {str(k): v for k, v in e["ms"].items()}} for e in res]
            tmp = cache + ".tmp"
            with open(tmp, "w") as f:
                json.dump(table, f, indent=1, sort_keys=True)
            os.replace(tmp, cache)
        return res

    def set_plan(self, L: int, kind: int, value: int):
        """Set one execution-plan choice of every transform of length L (``fm_set_plan``)."""
        _lib.fm_set_plan(self._h, L, kind, value, _stream())

    def set_dense(self, dense: bool = True):
        """Apply this small leaf as a dense matrix product (True) or as the fast transform."""
        _lib.fm_set_dense(self._h, 1 if dense else 0, _stream())

    def calibrate_dense(self, ncols: int, dtype: torch.dtype = torch.complex64):
        """Time the fast transform against the dense product and keep the faster (the
        paper's calibration); returns {"ms_fast", "ms_dense", "dense"}."""
        a, b, c = _lib.fm_calibrate_dense(self._h, ncols, _TORCH2FM[dtype], _stream())
        return {"ms_fast": a, "ms_dense": b, "dense": bool(c)}

    def set_split(self, L: int, n1: int):
        """Use the split N1 x (L / N1) for every two-pass transform of length L (0: default)."""
        _lib.fm_set_split(self._h, L, n1, _stream())

    def __matmul__(self, other):
        if isinstance(other, Op):
            return product(self, other)
        return self.forward(other)

    def __add__(self, other):
        return sum_(self, other)


# ---------------------------------------------------------------- constructors
def fourier(n: int, ortho: bool = False) -> Op:
    return Op(_lib.fm_fourier(n, 1 if ortho else 0))


def circulant(c) -> Op:
    p, dt, keep = _param(c)
    return Op(_lib.fm_circulant(p, len(keep), dt, _stream()), kind="circulant")


def toeplitz(t, rows: int, cols: int | None = None) -> Op:
    cols = rows if cols is None else cols
    p, dt, keep = _param(t)
    if len(keep) != rows + cols - 1:
        raise ValueError("t must hold rows + cols - 1 entries")
    return Op(_lib.fm_toeplitz(p, rows, cols, dt, _stream()), kind="toeplitz")


def lfsr_circulant(nbits: int, taps: int, state: int, n: int) -> Op:
    """Circulant on the +-1 output of a Fibonacci LFSR (``fm_lfsr_circulant``)."""
    return Op(_lib.fm_lfsr_circulant(nbits, taps, state, n, _stream()), kind="circulant")


def toeplitz2(t, r1: int, c1: int, r2: int, c2: int) -> Op:
    """Two-level Toeplitz matrix (r1 r2) x (c1 c2) from the row-major (r1 + c1 - 1) x (r2 + c2 - 1)
    generator t (``fm_toeplitz2``)."""
    if isinstance(t, torch.Tensor):
        t = t.reshape(-1)
    else:
        t = np.asarray(t).reshape(-1)
    p, dt, keep = _param(t)
    if len(keep) != (r1 + c1 - 1) * (r2 + c2 - 1):
        raise ValueError("t must hold (r1 + c1 - 1) (r2 + c2 - 1) entries")
    return Op(_lib.fm_toeplitz2(p, r1, c1, r2, c2, dt, _stream()), kind="toeplitz2")


def blocks(grid) -> Op:
    """Block matrix of operators from a list of block rows (``fm_blocks``)."""
    nr, nc = len(grid), len(grid[0])
    if any(len(r) != nc for r in grid):
        raise ValueError("every block row needs the same number of blocks")
    flat = [b for r in grid for b in r]
    return Op(_lib.fm_blocks([b.handle for b in flat], nr, nc), flat)


def hadamard(log2n: int, mode: int = FM_HAD_FP32) -> Op:
    return Op(_lib.fm_hadamard(log2n, mode))


def diag(d) -> Op:
    p, dt, keep = _param(d)
    return Op(_lib.fm_diag(p, len(keep), dt, _stream()), kind="diag")


def partial(idx, n: int) -> Op:
    if isinstance(idx, torch.Tensor):
        idx = idx.to(torch.int32)
    p, _, keep = _param(idx, allow_int=True)
    return Op(_lib.fm_partial(p, len(keep), n, _stream()))


def product(*ops: Op) -> Op:
    return Op(_lib.fm_product([o.handle for o in ops]), ops)


def sum_(*ops: Op) -> Op:
    return Op(_lib.fm_sum([o.handle for o in ops]), ops)


def blkdiag(*ops: Op) -> Op:
    return Op(_lib.fm_blkdiag([o.handle for o in ops]), ops)


def kron(*ops: Op) -> Op:
    return Op(_lib.fm_kron([o.handle for o in ops]), ops)


# ---------------------------------------------------------------- autograd
class FmApply(torch.autograd.Function):
    """y = A x with the hand-written adjoint as its backward: dL/dx = A^H dL/dy.

    The map is linear in x, so nothing but the operator is saved; composite operators
    (Kron, Product) recompute their intermediates inside the adjoint kernels.
    """

    @staticmethod
    def forward(ctx, X, op: Op):
        ctx.op = op
        ctx.real_in = not X.is_complex()
        return op.forward(X)

    @staticmethod
    def backward(ctx, g):
        # real x: the library returns Re(A^H g), the adjoint of x -> A x on real inputs
        return ctx.op.backward(g.contiguous(), real_out=ctx.real_in), None


def apply(op: Op, X: torch.Tensor) -> torch.Tensor:
    """Differentiable A X."""
    return FmApply.apply(X, op)


def param_grad(A: Op, leaf: Op, X: torch.Tensor, G: torch.Tensor) -> torch.Tensor:
    """Gradient with respect to the parameter vector of `leaf` (a Diag, Circulant or Toeplitz
    term of A) for Y = A X and upstream gradient G = dloss/dconj(Y) (``fm_param_grad``).
    X: [K, cols(A)], G: [K, rows(A)]; returns a vector of the parameter length, complex for a
    complex leaf and real for a real one."""
    X2 = (X.unsqueeze(0) if X.dim() == 1 else X).contiguous()
    G2 = (G.unsqueeze(0) if G.dim() == 1 else G).contiguous()
    if X2.shape[0] != G2.shape[0] or X2.shape[1] != A.cols or G2.shape[1] != A.rows:
        raise ValueError("X must be [K, cols(A)] and G [K, rows(A)]")
    dbl = X2.dtype in (torch.float64, torch.complex128)
    if leaf.real:
        gdt = torch.float64 if dbl else torch.float32
    else:
        gdt = torch.complex128 if dbl else torch.complex64
    plen = leaf.rows + leaf.cols - 1 if leaf.kind == "toeplitz" else leaf.rows
    out = torch.empty(plen, dtype=gdt, device=X2.device)
    _lib.fm_param_grad(A.handle, leaf.handle, X2.data_ptr(), X2.shape[1], _TORCH2FM[X2.dtype], G2.data_ptr(),
                       G2.shape[1], _TORCH2FM[G2.dtype], X2.shape[0], out.data_ptr(), _TORCH2FM[gdt], _stream())
    return out


class FmParamApply(torch.autograd.Function):
    """y = A(params) x, differentiable in x and in the parameter vectors.

    ``build(*params)`` returns (A, leaves) with leaves[i] the Diag / Circulant / Toeplitz
    operator made from params[i].  Only x is saved: the backward recomputes the intermediates
    the parameter gradients need inside the library (``fm_param_grad``).
    """

    @staticmethod
    def forward(ctx, X, build, *params):
        A, leaves = build(*[p.detach() for p in params])
        ctx.A, ctx.leaves = A, list(leaves)
        ctx.real_in = not X.is_complex()
        ctx.pdtypes = [p.dtype for p in params]
        ctx.save_for_backward(X)
        return A.forward(X)

    @staticmethod
    def backward(ctx, g):
        (X,) = ctx.saved_tensors
        g = g.contiguous()
        gx = ctx.A.backward(g, real_out=ctx.real_in) if ctx.needs_input_grad[0] else None
        gps = []
        for i, leaf in enumerate(ctx.leaves):
            if not ctx.needs_input_grad[2 + i]:
                gps.append(None)
                continue
            gp = param_grad(ctx.A, leaf, X, g)
            if not ctx.pdtypes[i].is_complex and gp.is_complex():
                gp = gp.real
            gps.append(gp.to(ctx.pdtypes[i]))
        return (gx, None, *gps)


def apply_params(build, X: torch.Tensor, *params: torch.Tensor) -> torch.Tensor:
    """Differentiable A(params) X: see FmParamApply."""
    return FmParamApply.apply(X, build, *params)


# ---------------------------------------------------------------- OMP
def omp(A: Op, b: torch.Tensor, K: int):
    """Orthogonal matching pursuit with K steps (``fm_omp``): returns (x, support)."""
    if not b.is_cuda or b.dim() != 1 or b.numel() != A.rows:
        raise ValueError("b must be a CUDA vector of rows(A) entries")
    b = b.contiguous()
    x = torch.empty(A.cols, dtype=b.dtype, device=b.device)
    S = torch.empty(K, dtype=torch.int32, device=b.device)
    _lib.fm_omp(A.handle, b.data_ptr(), _TORCH2FM[b.dtype], K, x.data_ptr(), S.data_ptr(), _stream())
    return x, S


# ---------------------------------------------------------------- FISTA
class FistaBatch:
    """Many independent instances A_i = P_i T_i solved together (``fm_fista``)."""

    def __init__(self, ops):
        self.ops = list(ops)
        self._b = _lib.fm_batch_create([o.handle for o in self.ops], _stream())
        self.total_rows, self.total_cols = _lib.fm_batch_sizes(self._b)
        self.count = len(self.ops)

    def __del__(self):
        b = getattr(self, "_b", None)
        if b:
            _lib.fm_batch_release(b)
            self._b = None

    def tune(self, b: torch.Tensor, x: torch.Tensor | None = None, iters: int = 200, power_iters: int = 20,
             lambda_rel: float = 0.01, safety: float = 1.05, accel: bool = True):
        """Choose the work-list order of the persistent solve by timing both (``fm_batch_tune``);
        returns {"ms": [largest first, smallest first], "order": 0 or 1}."""
        if x is None:
            x = torch.empty(self.total_cols, dtype=torch.float32, device=b.device)
        params = fm_fista_params(iters, power_iters, lambda_rel, safety, 1 if accel else 0, 0, 0, 0)
        ms, c = _lib.fm_batch_tune(self._b, b.data_ptr(), x.data_ptr(), params, _stream())
        return {"ms": ms, "order": c}

    def set_order(self, order: int):
        """Work-list order of the persistent solve: 0 largest instances first, 1 smallest first."""
        _lib.fm_batch_set_order(self._b, order)

    def solve(self, b: torch.Tensor, x: torch.Tensor | None = None, iters: int = 200, power_iters: int = 20,
              lambda_rel: float = 0.01, safety: float = 1.05, accel: bool = True, mode: int = 0,
              report: bool | dict = False, y: torch.Tensor | None = None, resume_from: int | None = None):
        """Solve every instance (``fm_fista_batch``).

        y (packed like x) receives the momentum state y_{K+1}.  ``resume_from=k0`` continues a
        run that has taken k0 steps: x and y hold its x_k0 and y_{k0+1}, and ``report`` must be
        the dict that run returned (its L and lambda are reused)."""
        if b.dtype != torch.float32 or not b.is_cuda or b.numel() != self.total_rows:
            raise ValueError("b must be a packed float32 CUDA tensor of the batch's total rows")
        if x is None:
            if resume_from is not None:
                raise ValueError("a resumed run needs its x")
            x = torch.empty(self.total_cols, dtype=torch.float32, device=b.device)
        warm = resume_from is not None
        if warm and (y is None or not isinstance(report, dict)):
            raise ValueError("a resumed run needs its y and the report of the run it continues")
        params = fm_fista_params(iters, power_iters, lambda_rel, safety, 1 if accel else 0, mode,
                                 1 if warm else 0, int(resume_from or 0))
        rep = None
        out = None
        if report:
            out = report if isinstance(report, dict) else {
                "L": torch.empty(self.count, dtype=torch.float64, device=b.device),
                "lambda": torch.empty(self.count, dtype=torch.float64, device=b.device),
                "objective": torch.empty(self.count, dtype=torch.float64, device=b.device),
                "status": torch.empty(self.count, dtype=torch.int32, device=b.device)}
            rep = fm_fista_report(out["L"].data_ptr(), out["lambda"].data_ptr(),
                                  out["objective"].data_ptr(), out["status"].data_ptr())
        _lib.fm_fista_batch(self._b, b.data_ptr(), x.data_ptr(), None if y is None else y.data_ptr(),
                            params, rep, _stream())
        return (x, out) if report else x


def fista(ops, bs, xs=None, iters: int = 200, power_iters: int = 20, lambda_rel: float = 0.01,
          safety: float = 1.05, accel: bool = True, mode: int = 0, report: bool = False):
    """Solve independent instances given as separate tensors (``fm_fista``): ops[i] =
    P_i T_i, bs[i] its float32 measurements, xs[i] (created if None) its solution."""
    ops = list(ops)
    if xs is None:
        xs = [torch.empty(o.cols, dtype=torch.float32, device=b.device) for o, b in zip(ops, bs)]
    for b, x, o in zip(bs, xs, ops):
        if b.dtype != torch.float32 or x.dtype != torch.float32 or not b.is_cuda or not x.is_cuda:
            raise ValueError("b and x must be float32 CUDA tensors")
        if b.numel() != o.rows or x.numel() != o.cols or not b.is_contiguous() or not x.is_contiguous():
            raise ValueError("b[i] must hold rows(A_i) and x[i] cols(A_i) contiguous floats")
    params = fm_fista_params(iters, power_iters, lambda_rel, safety, 1 if accel else 0, mode, 0, 0)
    rep, out = None, None
    if report:
        dev = bs[0].device
        out = {"L": torch.empty(len(ops), dtype=torch.float64, device=dev),
               "lambda": torch.empty(len(ops), dtype=torch.float64, device=dev),
               "objective": torch.empty(len(ops), dtype=torch.float64, device=dev),
               "status": torch.empty(len(ops), dtype=torch.int32, device=dev)}
        rep = fm_fista_report(out["L"].data_ptr(), out["lambda"].data_ptr(),
                              out["objective"].data_ptr(), out["status"].data_ptr())
    _lib.fm_fista([o.handle for o in ops], [b.data_ptr() for b in bs], [x.data_ptr() for x in xs],
                  params, rep, _stream())
    return (xs, out) if report else xs
