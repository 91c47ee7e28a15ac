"""Block matrices of operators and two-level Toeplitz matrices, FP64 (oracle).

TEST INFRASTRUCTURE: imported only by tests, the smoke check and the CPU baseline of
the benchmark.

The ultrasound model of Sec. 3 is a block matrix H = [H_ij] whose blocks H_ij are 2-level
Toeplitz matrices (2-D non-cyclic convolutions); Eq. (7) writes each as a zero-padded
2-level circulant.  Definitions used here:

* ``Blocks([[B_00, B_01, ...], ...])``: output segment i = sum_j B_ij (input segment j);
  the adjoint maps segment j to sum_i B_ij^H (segment i).
* ``Toeplitz2(t, r1, c1, r2, c2)``: vectors are row-major grids (r1 x r2 out, c1 x c2 in) and
  T2[(i1, i2), (j1, j2)] = t[k(i1, j1; r1), k(i2, j2; r2)] with the 1-D Toeplitz rule
  k(i, j; r) = i - j for i >= j, r - 1 + j - i for i < j on each level; t is an
  (r1 + c1 - 1) x (r2 + c2 - 1) array.  The fast route embeds t in an L1 x L2 two-level
  circulant (each level by the 1-D embedding rule) and convolves with numpy's 2-D FFT.

Pinned by tests/test_oracle_pins.py: a separable generator gives kron(T(a), T(b)) with
scipy's Toeplitz constructor, a hand-worked example, np.block for Blocks, the fast route
against the definition and the adjoint identity.
"""
from __future__ import annotations

import numpy as np

from .operators import Op


def _level_index(i, j, r):
    d = i - j
    return np.where(d >= 0, d, r - 1 - d)


class Toeplitz2(Op):
    def __init__(self, t, r1: int, c1: int, r2: int, c2: int):
        t = np.asarray(t)
        if t.shape != (r1 + c1 - 1, r2 + c2 - 1):
            raise ValueError("t must be (r1 + c1 - 1) x (r2 + c2 - 1)")
        self.t = t.astype(np.float64 if t.dtype.kind in "fiu" else np.complex128)
        self.r1, self.c1, self.r2, self.c2 = int(r1), int(c1), int(r2), int(c2)
        self.rows, self.cols = self.r1 * self.r2, self.c1 * self.c2
        self.real = self.t.dtype.kind == "f"
        L1 = 1
        while L1 < r1 + c1 - 1:
            L1 *= 2
        L2 = 1
        while L2 < r2 + c2 - 1:
            L2 *= 2
        self.L1, self.L2 = L1, L2
        e = np.zeros((L1, L2), dtype=np.complex128)
        m1 = np.array([k for k in range(r1)] + [L1 - d for d in range(1, c1)])
        m2 = np.array([k for k in range(r2)] + [L2 - d for d in range(1, c2)])
        e[np.ix_(m1, m2)] = self.t
        self.spectrum = np.fft.fft2(e)

    def dense(self):
        i1, i2 = np.divmod(np.arange(self.rows), self.r2)
        j1, j2 = np.divmod(np.arange(self.cols), self.c2)
        k1 = _level_index(i1[:, None], j1[None, :], self.r1)
        k2 = _level_index(i2[:, None], j2[None, :], self.r2)
        return self.t[k1, k2]

    def row(self, i):
        return self.dense()[int(i)]

    def _apply(self, X, adjoint):
        k = X.shape[1]
        (a1, a2), (b1, b2) = ((self.r1, self.r2), (self.c1, self.c2)) if adjoint else \
            ((self.c1, self.c2), (self.r1, self.r2))
        Z = np.zeros((self.L1, self.L2, k), dtype=np.complex128)
        Z[:a1, :a2] = X.reshape(a1, a2, k)
        s = np.conj(self.spectrum) if adjoint else self.spectrum
        Y = np.fft.ifft2(s[:, :, None] * np.fft.fft2(Z, axes=(0, 1)), axes=(0, 1))[:b1, :b2]
        Y = Y.reshape(b1 * b2, k)
        return Y.real if (self.real and X.dtype.kind == "f") else Y


class Blocks(Op):
    def __init__(self, grid):
        self.grid = [list(r) for r in grid]
        nc = len(self.grid[0])
        if any(len(r) != nc for r in self.grid):
            raise ValueError("ragged block grid")
        for r in self.grid:
            if len({b.rows for b in r}) != 1:
                raise ValueError("blocks of a block row differ in rows")
        for j in range(nc):
            if len({r[j].cols for r in self.grid}) != 1:
                raise ValueError("blocks of a block column differ in columns")
        self.rows = sum(r[0].rows for r in self.grid)
        self.cols = sum(b.cols for b in self.grid[0])
        self.real = all(b.real for r in self.grid for b in r)

    def dense(self):
        return np.block([[b.dense().astype(np.complex128) for b in r] for r in self.grid])

    def _apply(self, X, adjoint):
        if not adjoint:
            offs = np.cumsum([0] + [b.cols for b in self.grid[0]])
            outs = [sum(b.apply(X[offs[j]:offs[j + 1]]).astype(np.complex128) for j, b in enumerate(r))
                    for r in self.grid]
        else:
            offs = np.cumsum([0] + [r[0].rows for r in self.grid])
            outs = [sum(self.grid[i][j].apply(X[offs[i]:offs[i + 1]], adjoint=True).astype(np.complex128)
                        for i in range(len(self.grid))) for j in range(len(self.grid[0]))]
        Y = np.concatenate(outs, axis=0)
        return Y.real if (self.real and X.dtype.kind == "f") else Y
