"""Orthogonal matching pursuit, FP64 (oracle).

TEST INFRASTRUCTURE: imported only by tests, the smoke check and the CPU baseline of
the benchmark.

OMP is the greedy sparse-recovery loop Sec. 3 cites beside (F)ISTA and Sec. 4 names for its
rank-1 update implementation; like them it touches the operator only through phi (A x) and
beta (A^H y).  Steps for b and K (0-based, written out plainly):

1. r_0 = b, S = [];
2. for k = 1..K: c = A^H r_{k-1}; j = argmax_i |c_i| (the lowest index among equal
   magnitudes); append j to S; x_S = argmin_z ||A_S z - b||_2 (least squares over the
   selected columns A_S, each obtained as A e_j); r_k = b - A_S x_S;
3. x = 0 except x[S] = x_S.

The least-squares solve is done afresh with numpy's lstsq at every step; the rank-1 QR
update of a fast implementation reaches the same solution.  Pinned by
tests/test_oracle_pins.py: a hand-worked example with a tie, exact recovery and pick order
for orthonormal A, and the orthogonality of the residual to the selected columns.
"""
from __future__ import annotations

import numpy as np


def column(A, j: int) -> np.ndarray:
    e = np.zeros(A.cols)
    e[j] = 1.0
    return A.apply(e)


def omp(A, b, K: int, return_residuals: bool = False):
    b = np.asarray(b)
    b = b.astype(np.complex128 if b.dtype.kind == "c" or not A.real else np.float64)
    r = b.copy()
    S, cols, res = [], [], [float(np.linalg.norm(b))]
    xs = np.zeros(0)
    for _ in range(K):
        c = A.apply(r, adjoint=True)
        j = int(np.argmax(np.abs(c)))
        S.append(j)
        cols.append(column(A, j).astype(b.dtype if np.iscomplexobj(b) else np.complex128))
        AS = np.stack(cols, axis=1)
        xs = np.linalg.lstsq(AS, b.astype(AS.dtype), rcond=None)[0]
        r = b - AS @ xs
        res.append(float(np.linalg.norm(r)))
    x = np.zeros(A.cols, dtype=np.complex128)
    x[S] = xs
    if A.real and not np.iscomplexobj(b):
        x = x.real
    return (x, S, res) if return_residuals else (x, S)
