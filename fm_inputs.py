"""Seeded synthetic inputs for the structured-operator workloads.

This module only draws random numbers (numpy ``default_rng``, PCG64) and
arranges them in the block-of-columns layout used everywhere in this
repository: a block of K columns of length n is a C-contiguous array of shape
``[K, n]`` (column k is row k of the array, so each column is contiguous and
the leading dimension is n).  It holds none of the operator arithmetic; the
oracle (``oracle/``) and the CUDA library both receive the arrays made here.

The one exception is ``fista_measurements``: the sparse-recovery workload needs
synthetic measurements b = P·T·x0 + n (the measurement model of Eq. (6)), which
are an *input* of the recovery method.  They are synthesised by summing the few
columns of T that the sparse x0 selects, straight from the Toeplitz entry rule,
with noise scaled to an exact 30 dB SNR.

Complex standard normal ("CN(0,1)") means real and imaginary parts i.i.d.
N(0, 1/2), so E|z|^2 = 1.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "cn",
    "circulant_tiny",
    "hadamard_block",
    "cs_operator",
    "fista_instance",
    "fista_measurements",
    "ndt_model",
    "compressed_rows",
    "kron_generator",
    "kron_large",
    "kron_small",
    "column_block",
]


def cn(rng: np.random.Generator, shape, dtype=np.complex128) -> np.ndarray:
    """Complex standard normal CN(0,1): re, im ~ N(0, 1/2), drawn re-block then im-block."""
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    z = (re + 1j * im) * np.sqrt(0.5)
    return z.astype(dtype)


def column_block(rng: np.random.Generator, k: int, n: int, dtype) -> np.ndarray:
    """A [k, n] block of i.i.d. columns: CN(0,1) for complex dtypes, N(0,1) for real."""
    dt = np.dtype(dtype)
    if dt.kind == "c":
        return cn(rng, (k, n), dt)
    return rng.standard_normal((k, n)).astype(dt)


def circulant_tiny(n: int = 4096, k: int = 16, seed: int = 0):
    """Circulant workload: generator c ~ CN(0,1)^n, then X, then Y (both [k, n]), complex128.

    Draw order from one stream: c, X, Y.
    """
    rng = np.random.default_rng(seed)
    c = cn(rng, (n,))
    X = cn(rng, (k, n))
    Y = cn(rng, (k, n))
    return c, X, Y


def hadamard_block(log2n: int = 16, k: int = 256, seed: int = 1):
    """Hadamard workload: X_f32 ~ N(0,1) [k, 2^log2n] float32, then X_i8 ~ U{-128..127} int8."""
    rng = np.random.default_rng(seed)
    n = 1 << log2n
    xf = rng.standard_normal((k, n), dtype=np.float32)
    xi = rng.integers(-128, 128, size=(k, n), dtype=np.int8)
    return xf, xi


def cs_operator(log2n: int = 18, k: int = 64, seed: int = 2, m_div: int = 4):
    """Compressed-sensing operator inputs for Phi = P·Diag(d)·C.

    Draw order: c in {+1,-1}^n (Rademacher), theta ~ U[0, 2pi) (d = exp(i theta)),
    the row selection idx = sorted(choice(n, n/m_div, replace=False)), X ~ CN(0,1) [k, n],
    Y ~ CN(0,1) [k, m], G ~ CN(0,1) [k, m] (an upstream gradient).
    Returns c (float64 +-1), d (complex64), idx (int32), X, Y, G (complex64).
    """
    rng = np.random.default_rng(seed)
    n = 1 << log2n
    m = n // m_div
    c = np.where(rng.integers(0, 2, size=n) == 1, 1.0, -1.0)
    theta = rng.uniform(0.0, 2.0 * np.pi, size=n)
    d = np.exp(1j * theta).astype(np.complex64)
    idx = np.sort(rng.choice(n, size=m, replace=False)).astype(np.int32)
    X = cn(rng, (k, n), np.complex64)
    Y = cn(rng, (k, m), np.complex64)
    G = cn(rng, (k, m), np.complex64)
    return c, d, idx, X, Y, G


def fista_instance(j: int, seed: int = 3, log2n_range=(10, 14)):
    """Random draws of sparse-recovery instance j (its own stream ``default_rng([seed, j])``).

    Draw order: log2 N ~ U{lo..hi}; t ~ N(0, 1/N)^(2N-1) float32 (Toeplitz parameter
    vector [first column; first row without t0]); idx = sorted(choice(N, N/2)) int32;
    support = choice(N, N/64); amplitudes ~ N(0,1); noise direction g ~ N(0,1)^M.
    """
    rng = np.random.default_rng([seed, j])
    lo, hi = log2n_range
    n = 1 << int(rng.integers(lo, hi + 1))
    t = (rng.standard_normal(2 * n - 1) / np.sqrt(n)).astype(np.float32)
    m = n // 2
    idx = np.sort(rng.choice(n, size=m, replace=False)).astype(np.int32)
    kk = max(1, n // 64)
    support = rng.choice(n, size=kk, replace=False)
    amps = rng.standard_normal(kk)
    g = rng.standard_normal(m)
    x0 = np.zeros(n)
    x0[support] = amps
    return {"n": n, "t": t, "idx": idx, "x0": x0, "g": g}


def fista_measurements(inst: dict, snr_db: float = 30.0) -> np.ndarray:
    """Measurements b = P·T·x0 + noise with exact SNR (Eq. (6)), rounded to float32.

    T x0 on the selected rows is the sum of the columns of T picked by the support of
    x0, with T[i, j] = t[i-j] for i >= j and t[N-1+j-i] for i < j.  The noise is the
    drawn direction g scaled so that ||noise|| = ||P T x0|| * 10^(-snr/20).
    """
    n, t, idx, x0, g = inst["n"], inst["t"].astype(np.float64), inst["idx"], inst["x0"], inst["g"]
    supp = np.flatnonzero(x0)
    diff = idx[:, None].astype(np.int64) - supp[None, :].astype(np.int64)
    ent = np.where(diff >= 0, t[np.clip(diff, 0, None)], t[n - 1 - np.clip(diff, None, 0)])
    clean = ent @ x0[supp]
    noise = g * (np.linalg.norm(clean) / np.linalg.norm(g)) * 10.0 ** (-snr_db / 20.0)
    return (clean + noise).astype(np.float32)


def ndt_model(n1: int = 4, n2: int = 8, n3: int = 8, k: int = 3, seed: int = 5, dtype=np.complex64):
    """Block model of Sec. 3: an n1 x n1 grid of two-level Toeplitz blocks with levels of
    2 n2 - 1 and 2 n3 - 1 points (square blocks).  Draw order: the generators h[i][j]
    ~ CN(0,1) of shape (2(2 n2 - 1) - 1) x (2(2 n3 - 1) - 1), row-major over (i, j); then
    X ~ CN(0,1) [k, n1 (2 n2 - 1)(2 n3 - 1)] and Y the same."""
    rng = np.random.default_rng(seed)
    a, b = 2 * n2 - 1, 2 * n3 - 1
    h = cn(rng, (n1, n1, 2 * a - 1, 2 * b - 1), dtype)
    X = cn(rng, (k, n1 * a * b), dtype)
    Y = cn(rng, (k, n1 * a * b), dtype)
    return h, X, Y


def compressed_rows(n_meas: int, n_t: int, n_f: int, seed: int = 6):
    """Row selections of the compressed model (Eq. (9)): for each of n_meas pulse-echo signals
    of n_t samples, n_f distinct Fourier rows, sorted (choice(n_t, n_f) per signal)."""
    rng = np.random.default_rng(seed)
    return [np.sort(rng.choice(n_t, size=n_f, replace=False)).astype(np.int32) for _ in range(n_meas)]


def kron_generator(seed: int = 4, n_c: int = 1024) -> np.ndarray:
    """The circulant generator of the Kron workload alone (the first draw of its stream)."""
    return cn(np.random.default_rng(seed), (n_c,))


def kron_large(k: int = 4, seed: int = 4, n_c: int = 1024, n_total: int = 1 << 24,
               dtype=np.complex64):
    """Large Kron workload: circulant generator c ~ CN(0,1)^n_c, X ~ CN(0,1) [k, n_total], Y the same."""
    rng = np.random.default_rng(seed)
    c = cn(rng, (n_c,))
    X = cn(rng, (k, n_total), dtype)
    Y = cn(rng, (k, n_total), dtype)
    return c, X, Y


def kron_small(k: int = 4, seed: int = 4):
    """Analogue of the large Kron workload at n = 2^12 (factors 16 x 16 x 16)."""
    return kron_large(k=k, seed=seed, n_c=16, n_total=1 << 12, dtype=np.complex128)
