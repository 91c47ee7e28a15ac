"""Structured operators of the fastmat method, written out in FP64 (oracle).

TEST INFRASTRUCTURE: imported only by tests, the smoke check and the CPU
baseline of the benchmark.  Vectors are the columns of an array of shape
``[cols, K]``; results are complex128 unless every factor is real (float64) or
the input is integer and the operator is Hadamard (int64, exact).

Paper passages followed (fastmat, arXiv 1710.09578):
* Eq. (1)  DFT matrix, read 0-based: F[k, j] = exp(-2 pi i j k / n).
* Eq. (2)  dense matrix-vector product (``dense`` / ``row``).
* Eq. (3), Eq. (4)  forward phi(x) = M x and backward beta(x) = M^H x.
* Eq. (5)  circulant product as ifft(fft(c) * fft(x)), and Sec. 2.1.1: the
  circulant is the product F^H . Diag . F with the spectrum precomputed once.
* Sec. 2.1.1  Toeplitz = non-circular convolution evaluated in the frequency
  domain (here by circulant embedding of length 2^ceil(log2(rows+cols-1))).
* Eq. (7)  Kron, Diag, Fourier and the row selector P (``Partial``).
* Sec. 3 (compressed model)  BlkDiag of blocks; Product / Sum of terms.
The Sylvester-Hadamard matrix is not in the paper; it is the textbook
H[i, j] = (-1)^popcount(i & j) in natural order, unnormalised.
"""
from __future__ import annotations

import numpy as np


def _as2d(X):
    X = np.asarray(X)
    return (X[:, None], True) if X.ndim == 1 else (X, False)


def _out(Y, was1d):
    return Y[:, 0] if was1d else Y


def _popcount(a: np.ndarray) -> np.ndarray:
    a = a.astype(np.uint64)
    c = np.zeros(a.shape, dtype=np.int64)
    while np.any(a):
        c += (a & np.uint64(1)).astype(np.int64)
        a >>= np.uint64(1)
    return c


class Op:
    """A linear map of shape (rows, cols); ``real`` when all its entries are real."""

    rows: int
    cols: int
    real: bool

    def dense(self) -> np.ndarray:
        raise NotImplementedError

    def row(self, i: int) -> np.ndarray:
        return self.dense()[i]

    def _apply(self, X: np.ndarray, adjoint: bool) -> np.ndarray:
        raise NotImplementedError

    def apply(self, X, adjoint: bool = False) -> np.ndarray:
        """phi(X) = A X (Eq. (3)) or beta(X) = A^H X (Eq. (4)), column by column."""
        X, was1d = _as2d(X)
        need = self.rows if adjoint else self.cols
        if X.shape[0] != need:
            raise ValueError(f"expected {need} rows, got {X.shape[0]}")
        if X.dtype.kind in "iu" and not isinstance(self, Hadamard):
            X = X.astype(np.float64)
        if X.dtype.kind == "f":
            X = X.astype(np.float64)
        elif X.dtype.kind == "c":
            X = X.astype(np.complex128)
        return _out(self._apply(X, adjoint), was1d)

    def forward(self, X):
        return self.apply(X, False)

    def backward(self, Y):
        return self.apply(Y, True)

    def rows_of(self, idx) -> np.ndarray:
        """Stack of rows ``idx`` of the matrix (definition), shape [len(idx), cols]."""
        return np.stack([self.row(int(i)) for i in idx])

    @property
    def shape(self):
        return (self.rows, self.cols)


def _cplx(X):
    return X.astype(np.complex128)


# --------------------------------------------------------------------------- leaves
class Fourier(Op):
    """DFT matrix of Eq. (1), 0-based; ``ortho`` scales it by 1/sqrt(n)."""

    def __init__(self, n: int, ortho: bool = False):
        self.n = self.rows = self.cols = int(n)
        self.ortho = bool(ortho)
        self.real = False

    def _scale(self):
        return 1.0 / np.sqrt(self.n) if self.ortho else 1.0

    def dense(self):
        j = np.arange(self.n, dtype=np.int64)
        jk = np.outer(j, j) % self.n            # exact integer phase index
        return np.exp(-2j * np.pi * jk / self.n) * self._scale()

    def row(self, i):
        jk = (int(i) * np.arange(self.n, dtype=np.int64)) % self.n
        return np.exp(-2j * np.pi * jk / self.n) * self._scale()

    def _apply(self, X, adjoint):
        # The FFT evaluates Eq. (2) for the matrix of Eq. (1); F^H has the opposite sign
        # and no 1/n, so F^H y = n * ifft(y).
        if adjoint:
            Y = np.fft.ifft(_cplx(X), axis=0) * self.n
        else:
            Y = np.fft.fft(_cplx(X), axis=0)
        return Y * self._scale()


class Circulant(Op):
    """C[i, j] = c[(i - j) mod n] (c is the first column); C x = ifft(fft(c) * fft(x)), Eq. (5)."""

    def __init__(self, c):
        c = np.asarray(c)
        self.c = c.astype(np.float64 if c.dtype.kind in "fiu" else np.complex128)
        self.n = self.rows = self.cols = len(c)
        self.real = self.c.dtype.kind == "f"
        self.spectrum = np.fft.fft(self.c)        # precomputed once (Sec. 2.1.1)

    def dense(self):
        i = np.arange(self.n)
        return self.c[(i[:, None] - i[None, :]) % self.n]

    def row(self, i):
        return self.c[(int(i) - np.arange(self.n)) % self.n]

    def _apply(self, X, adjoint):
        s = np.conj(self.spectrum) if adjoint else self.spectrum
        Y = np.fft.ifft(s[:, None] * np.fft.fft(_cplx(X), axis=0), axis=0)
        return Y.real if (self.real and X.dtype.kind == "f") else Y


def embedding_spectrum(t, rows: int, cols: int):
    """First column and FFT of the circulant of length L >= rows+cols-1 that embeds T.

    L is the smallest power of two >= rows + cols - 1.  The embedding column is
    [t_col(0..rows-1), 0, ..., 0, t_row(cols-1..1)] so that C_L[i, j] = T[i, j] for
    i < rows, j < cols.
    """
    t = np.asarray(t)
    L = 1
    while L < rows + cols - 1:
        L *= 2
    dt = np.float64 if t.dtype.kind in "fiu" else np.complex128
    c = np.zeros(L, dtype=dt)
    c[:rows] = t[:rows]
    if cols > 1:
        c[L - (cols - 1):] = t[rows:][::-1]
    return L, c, np.fft.fft(c)


class Toeplitz(Op):
    """T[i, j] = t[i - j] for i >= j, t[rows - 1 + (j - i)] for i < j.

    t = [first column (rows entries); first row without t0 (cols - 1 entries)].
    Applied as a non-circular convolution in the frequency domain (Sec. 2.1.1).
    """

    def __init__(self, t, rows: int, cols: int | None = None):
        cols = rows if cols is None else cols
        t = np.asarray(t)
        if len(t) != rows + cols - 1:
            raise ValueError("t must have rows + cols - 1 entries")
        self.t = t.astype(np.float64 if t.dtype.kind in "fiu" else np.complex128)
        self.rows, self.cols = int(rows), int(cols)
        self.real = self.t.dtype.kind == "f"
        self.L, self.embed, self.spectrum = embedding_spectrum(self.t, self.rows, self.cols)

    def _entry(self, i, j):
        d = i - j
        return np.where(d >= 0, self.t[np.clip(d, 0, None)],
                        self.t[np.clip(self.rows - 1 - d, 0, len(self.t) - 1)])

    def dense(self):
        i = np.arange(self.rows)[:, None]
        j = np.arange(self.cols)[None, :]
        return self._entry(i, j)

    def row(self, i):
        return self._entry(int(i), np.arange(self.cols))

    def _apply(self, X, adjoint):
        nin, nout = (self.rows, self.cols) if adjoint else (self.cols, self.rows)
        Z = np.zeros((self.L, X.shape[1]), dtype=np.complex128)
        Z[:nin] = X
        s = np.conj(self.spectrum) if adjoint else self.spectrum
        Y = np.fft.ifft(s[:, None] * np.fft.fft(Z, axis=0), axis=0)[:nout]
        return Y.real if (self.real and X.dtype.kind == "f") else Y


class Hadamard(Op):
    """Sylvester Hadamard matrix, natural order, unnormalised: H[i, j] = (-1)^popcount(i & j)."""

    def __init__(self, n: int):
        if n < 1 or (n & (n - 1)):
            raise ValueError("n must be a power of two")
        self.n = self.rows = self.cols = int(n)
        self.real = True

    def dense(self):
        i = np.arange(self.n)
        return np.where(_popcount(np.bitwise_and.outer(i, i)) % 2 == 0, 1, -1).astype(np.int64)

    def row(self, i):
        return np.where(_popcount(np.bitwise_and(int(i), np.arange(self.n))) % 2 == 0, 1, -1)

    def _apply(self, X, adjoint):
        # Radix-2 butterflies H_{2h} = [[H_h, H_h], [H_h, -H_h]] on the index bit of weight h
        # (symmetric matrix, so the adjoint is the same map).
        Y = X.astype(np.int64) if X.dtype.kind in "iu" else X.copy()
        n, k = Y.shape
        h = 1
        while h < n:
            V = Y.reshape(n // (2 * h), 2, h, k)
            a, b = V[:, 0].copy(), V[:, 1].copy()
            V[:, 0], V[:, 1] = a + b, a - b
            Y = V.reshape(n, k)
            h *= 2
        return Y


class Diag(Op):
    """Diag(d): y_i = d_i x_i; adjoint conj(d_i) y_i (Eq. (7))."""

    def __init__(self, d):
        d = np.asarray(d)
        self.d = d.astype(np.float64 if d.dtype.kind in "fiu" else np.complex128)
        self.n = self.rows = self.cols = len(d)
        self.real = self.d.dtype.kind == "f"

    def dense(self):
        return np.diag(self.d)

    def row(self, i):
        r = np.zeros(self.n, dtype=self.d.dtype)
        r[int(i)] = self.d[int(i)]
        return r

    def _apply(self, X, adjoint):
        d = np.conj(self.d) if adjoint else self.d
        return d[:, None] * X


class Partial(Op):
    """Row selection P (Eq. (7), Sec. 3): y_r = x_{idx[r]}; adjoint scatters (sums repeats)."""

    def __init__(self, idx, n: int):
        self.idx = np.asarray(idx, dtype=np.int64)
        if np.any(self.idx < 0) or np.any(self.idx >= n):
            raise ValueError("index out of range")
        self.rows, self.cols = len(self.idx), int(n)
        self.real = True

    def dense(self):
        P = np.zeros((self.rows, self.cols))
        P[np.arange(self.rows), self.idx] = 1.0
        return P

    def row(self, i):
        r = np.zeros(self.cols)
        r[self.idx[int(i)]] = 1.0
        return r

    def _apply(self, X, adjoint):
        if not adjoint:
            return X[self.idx].copy()
        Y = np.zeros((self.cols, X.shape[1]), dtype=X.dtype)
        np.add.at(Y, self.idx, X)
        return Y


# --------------------------------------------------------------------------- composites
class Product(Op):
    """A_1 A_2 ... A_k: forward applies A_k first; adjoint applies A_1^H first."""

    def __init__(self, *terms):
        self.terms = list(terms)
        for a, b in zip(self.terms[:-1], self.terms[1:]):
            if a.cols != b.rows:
                raise ValueError("inner dimensions differ")
        self.rows, self.cols = self.terms[0].rows, self.terms[-1].cols
        self.real = all(t.real for t in self.terms)

    def dense(self):
        M = self.terms[0].dense()
        for t in self.terms[1:]:
            M = M @ t.dense()
        return M

    def row(self, i):
        # row_i(A B) = row_i(A) B = conj(B^H conj(row_i(A)))
        r = np.asarray(self.terms[0].row(i))
        for t in self.terms[1:]:
            r = np.conj(t.apply(np.conj(r).astype(np.complex128), adjoint=True))
        return r

    def _apply(self, X, adjoint):
        if adjoint:
            for t in self.terms:
                X = t.apply(X, adjoint=True)
        else:
            for t in reversed(self.terms):
                X = t.apply(X, adjoint=False)
        return X


class Sum(Op):
    """A_1 + ... + A_k (all the same shape)."""

    def __init__(self, *terms):
        self.terms = list(terms)
        if len({t.shape for t in self.terms}) != 1:
            raise ValueError("terms must share a shape")
        self.rows, self.cols = self.terms[0].shape
        self.real = all(t.real for t in self.terms)

    def dense(self):
        return sum(t.dense().astype(np.complex128) for t in self.terms)

    def row(self, i):
        return sum(np.asarray(t.row(i), dtype=np.complex128) for t in self.terms)

    def _apply(self, X, adjoint):
        return sum(t.apply(X, adjoint) for t in self.terms)


class BlkDiag(Op):
    """Block-diagonal arrangement: x splits into segments of sizes cols(A_i); outputs stack."""

    def __init__(self, *blocks):
        self.blocks = list(blocks)
        self.rows = sum(b.rows for b in self.blocks)
        self.cols = sum(b.cols for b in self.blocks)
        self.real = all(b.real for b in self.blocks)

    def dense(self):
        M = np.zeros((self.rows, self.cols), dtype=np.complex128)
        r = c = 0
        for b in self.blocks:
            M[r:r + b.rows, c:c + b.cols] = b.dense()
            r += b.rows
            c += b.cols
        return M

    def row(self, i):
        out = np.zeros(self.cols, dtype=np.complex128)
        r = c = 0
        for b in self.blocks:
            if i < r + b.rows:
                out[c:c + b.cols] = b.row(i - r)
                return out
            r += b.rows
            c += b.cols
        raise IndexError(i)

    def _apply(self, X, adjoint):
        outs, off = [], 0
        for b in self.blocks:
            n = b.rows if adjoint else b.cols
            outs.append(b.apply(X[off:off + n], adjoint))
            off += n
        kind = np.result_type(*[o.dtype for o in outs])
        return np.concatenate([o.astype(kind) for o in outs], axis=0)


class Kron(Op):
    """A_1 (x) A_2 (x) ... (x) A_k, with vectors read as row-major tensors (n_1, ..., n_k).

    Kronecker entry rule: (A (x) B)[(i1, i2), (j1, j2)] = A[i1, j1] B[i2, j2], the first
    factor on the most significant index digit.  Applied as mode products: A_i acts
    along axis i; the adjoint is the Kron of the adjoints (Eq. (7)).
    """

    def __init__(self, *factors):
        self.factors = list(factors)
        self.rows = int(np.prod([f.rows for f in self.factors]))
        self.cols = int(np.prod([f.cols for f in self.factors]))
        self.real = all(f.real for f in self.factors)

    def dense(self):
        M = np.ones((1, 1))
        for f in self.factors:
            D = f.dense()
            M = (M[:, None, :, None] * D[None, :, None, :]).reshape(
                M.shape[0] * D.shape[0], M.shape[1] * D.shape[1])
        return M

    def row(self, i):
        digits = []
        for f in reversed(self.factors):
            digits.append(i % f.rows)
            i //= f.rows
        digits.reverse()
        r = np.ones(1)
        for f, d in zip(self.factors, digits):
            r = (r[:, None] * np.asarray(f.row(d))[None, :]).reshape(-1)
        return r

    def _apply(self, X, adjoint):
        k = X.shape[1]
        dims = [f.cols if not adjoint else f.rows for f in self.factors]
        T = X.reshape(*dims, k)
        for ax, f in enumerate(self.factors):
            T = np.moveaxis(T, ax, 0)
            sh = T.shape
            Y = f.apply(T.reshape(sh[0], -1), adjoint)
            nout = f.cols if adjoint else f.rows
            T = np.moveaxis(Y.reshape(nout, *sh[1:]), 0, ax)
        return T.reshape(-1, k)
