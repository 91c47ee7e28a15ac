"""Gradients with respect to the parameter vectors of Diag, Circulant and Toeplitz, FP64 (oracle).

TEST INFRASTRUCTURE: imported only by tests, the smoke check and the CPU baseline of
the benchmark.

The operators of Sec. 2.1.1 are built from parameter vectors (the diagonal d, the first
column c of a circulant, the generator t of a Toeplitz matrix), and Y = A(theta) X is
bilinear in (theta, X).  For a real loss with upstream gradient G = dloss/dY (PyTorch's
convention for complex tensors: the derivative with respect to conj(Y), so that the
gradient of X is A^H G), the gradient of a parameter entry theta_k is

    grad_k = sum over columns and over the entries (i, j) with A[i, j] = theta_k of
             G[i] * conj(X[j]),

and, for a real parameter, the real part of that sum.  Per operator:

* Diag:      grad_d[i] = sum_cols G[i] conj(X[i]);
* Circulant: C[i, j] = c[(i - j) mod n], so grad_c[k] = sum_cols sum_i G[i] conj(X[(i - k) mod n])
             -- the circular cross-correlation of G with X;
* Toeplitz:  T[i, j] = t[i - j] (i >= j) and t[rows - 1 + j - i] (i < j), so grad_t[k] sums
             G[i] conj(X[j]) over the k-th diagonal: i - j = k for k < rows, and
             j - i = k - rows + 1 for k >= rows.

Each is given twice: ``*_definition`` loops over the entries exactly as above (small
sizes), and the fast routes use the Fourier diagonalisation of the circulant (Eq. (5):
the correlation is ifft(fft(G) conj(fft(X)))) and, for Toeplitz, the circulant embedding
of the products (the same rule as the operator, read backwards).  ``product_param_grad``
evaluates a Product by recomputing the input of the leaf (the product of the terms
applied before it) and the upstream gradient at its output (the adjoints of the terms
applied after it).

Pinned by tests/test_oracle_pins.py: hand-worked examples (tests/golden), central
differences of the bilinear map, and the definitions against the fast routes.
"""
from __future__ import annotations

import numpy as np

from .operators import Circulant, Diag, Product, Toeplitz


def _cols(a):
    a = np.asarray(a)
    return a[:, None] if a.ndim == 1 else a


def _real_if(v, real):
    return v.real.copy() if real else v


def grad_diag(X, G, real=False):
    """sum over columns of G * conj(X) (X, G: [n, K])."""
    X, G = _cols(X), _cols(G)
    return _real_if(np.sum(G * np.conj(X), axis=1), real)


def grad_circulant_definition(X, G, real=False):
    X, G = _cols(X), _cols(G)
    n = X.shape[0]
    out = np.zeros(n, dtype=np.complex128)
    for k in range(n):
        for i in range(n):
            out[k] += np.sum(G[i] * np.conj(X[(i - k) % n]))
    return _real_if(out, real)


def grad_circulant(X, G, real=False):
    """Circular cross-correlation of G with X, summed over columns, through the DFT."""
    X, G = _cols(X).astype(np.complex128), _cols(G).astype(np.complex128)
    r = np.fft.ifft(np.sum(np.fft.fft(G, axis=0) * np.conj(np.fft.fft(X, axis=0)), axis=1))
    return _real_if(r, real)


def grad_toeplitz_definition(X, G, rows, cols, real=False):
    X, G = _cols(X), _cols(G)
    out = np.zeros(rows + cols - 1, dtype=np.complex128)
    for i in range(rows):
        for j in range(cols):
            k = i - j if i >= j else rows - 1 + j - i
            out[k] += np.sum(G[i] * np.conj(X[j]))
    return _real_if(out, real)


def grad_toeplitz(X, G, rows, cols, real=False):
    """Toeplitz generator gradient through the circulant embedding: the correlation of the
    zero-padded G (length L) with the zero-padded X, read back at the embedding's positions
    (entry m < rows at m, entry rows - 1 + d at L - d)."""
    X, G = _cols(X).astype(np.complex128), _cols(G).astype(np.complex128)
    L = 1
    while L < rows + cols - 1:
        L *= 2
    Xp = np.zeros((L, X.shape[1]), dtype=np.complex128)
    Gp = np.zeros((L, G.shape[1]), dtype=np.complex128)
    Xp[:cols] = X
    Gp[:rows] = G
    r = grad_circulant(Xp, Gp)
    out = np.concatenate([r[:rows], r[L - np.arange(1, cols)]])
    return _real_if(out, real)


def leaf_param_grad(op, X, G):
    """Gradient of the parameter vector of a Diag, Circulant or Toeplitz leaf `op` given its
    input X and the upstream gradient G at its output."""
    real = bool(op.real)
    if isinstance(op, Diag):
        return grad_diag(X, G, real)
    if isinstance(op, Circulant):
        return grad_circulant(X, G, real)
    if isinstance(op, Toeplitz):
        return grad_toeplitz(X, G, op.rows, op.cols, real)
    raise TypeError("parameter gradients exist for Diag, Circulant and Toeplitz leaves")


def product_param_grad(A, index, X, G):
    """Gradient of the parameters of term `index` of A = terms[0] ... terms[k-1] (or of A
    itself when it is not a Product): the term's input Z = terms[index+1] ... terms[k-1] X is
    recomputed, and the gradient at its output is terms[index-1]^H ... terms[0]^H G."""
    if not isinstance(A, Product):
        return leaf_param_grad(A, X, G)
    Z = _cols(X).astype(np.complex128)
    for t in reversed(A.terms[index + 1:]):
        Z = t.apply(Z)
    Gt = _cols(G).astype(np.complex128)
    for t in A.terms[:index]:
        Gt = t.apply(Gt, adjoint=True)
    return leaf_param_grad(A.terms[index], Z, Gt)
