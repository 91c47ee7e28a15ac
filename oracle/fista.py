"""FISTA for the l1-regularised least-squares problem, FP64 (oracle).

TEST INFRASTRUCTURE: imported only by tests, the smoke check and the CPU
baseline of the benchmark.

Problem (Eq. (8), written with a 1/2 on the data term so that the paper's tau
equals 2*lambda):  min_x  1/2 ||A x - b||_2^2 + lambda ||x||_1.

The paper states the ISTA step in Sec. 3 without the gradient step x_k - g/L and
cites the accelerated variant (FISTA, Beck & Teboulle) for its reconstructions.
The steps below are that accelerated proximal-gradient method with a constant
step 1/L, in the order the method defines them:

1. lambda = 0.01 * ||A^T b||_inf;
2. L = min(1.05 * lam_hat, max_k |c_hat_k|^2), lam_hat = ||A v_20||^2 after 20
   power iterations v <- A^T A v / ||A^T A v|| from v_0 = 1/sqrt(N) * ones, and
   c_hat the spectrum of the circulant embedding of T (a guaranteed bound,
   since ||P T|| <= ||T|| <= ||C_L|| = max |c_hat|);
3. x_0 = 0, y_1 = x_0, t_1 = 1;
4. for k = 1..K:  g = A^T (A y_k - b);  x_k = soft(y_k - g/L, lambda/L);
   t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2;  y_{k+1} = x_k + ((t_k - 1)/t_{k+1}) (x_k - x_{k-1});
5. return x_K (no early stop, no restart).  ``accel=False`` keeps t = 1 (plain ISTA).
"""
from __future__ import annotations

import numpy as np

from .operators import Partial, Product, Toeplitz


def soft(z: np.ndarray, s: float) -> np.ndarray:
    """Soft threshold to level s: real sign(z) max(|z|-s, 0); complex z max(1 - s/|z|, 0)."""
    z = np.asarray(z)
    if z.dtype.kind == "c":
        mag = np.abs(z)
        scale = np.where(mag > s, 1.0 - s / np.where(mag > 0, mag, 1.0), 0.0)
        return z * scale
    return np.sign(z) * np.maximum(np.abs(z) - s, 0.0)


def lambda_from_b(A, b, rel: float = 0.01) -> float:
    """lambda = rel * ||A^T b||_inf."""
    return rel * float(np.max(np.abs(A.apply(b, adjoint=True))))


def lipschitz(A, spectrum_cap: float | None = None, iters: int = 20, safety: float = 1.05) -> float:
    """Step-size constant L by the fixed power-iteration protocol of step 2."""
    n = A.cols
    v = np.full(n, 1.0 / np.sqrt(n))
    for _ in range(iters):
        w = A.apply(A.apply(v), adjoint=True)
        v = w / np.linalg.norm(w)
    lam_hat = float(np.linalg.norm(A.apply(v)) ** 2)
    L = safety * lam_hat
    if spectrum_cap is not None:
        L = min(L, float(spectrum_cap))
    return L


def objective(A, b, x, lam) -> float:
    r = A.apply(x) - b
    return 0.5 * float(np.vdot(r, r).real) + lam * float(np.sum(np.abs(x)))


def fista(A, b, lam: float, L: float, iters: int = 200, accel: bool = True,
          state=None, return_state: bool = False):
    """Run K = ``iters`` accelerated proximal-gradient steps.

    ``state`` = (x_k, y_{k+1}, t_{k+1}) resumes a run exactly; the default is the
    start x_0 = 0, y_1 = 0, t_1 = 1.  With ``return_state`` the final
    (x_K, y_{K+1}, t_{K+1}) is returned as well, so K1 + K2 steps equal K1 steps
    followed by K2 resumed steps.
    """
    b = np.asarray(b)
    b = b.astype(np.complex128 if b.dtype.kind == "c" else np.float64)
    n = A.cols
    if state is None:
        x, y, t = np.zeros(n), np.zeros(n), 1.0
    else:
        x, y, t = np.array(state[0], dtype=np.float64), np.array(state[1], dtype=np.float64), float(state[2])
    for _ in range(iters):
        g = A.apply(A.apply(y) - b, adjoint=True)
        x_new = soft(y - g / L, lam / L)
        if accel:
            t_next = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t * t))
            y = x_new + ((t - 1.0) / t_next) * (x_new - x)
            t = t_next
        else:
            y = x_new
        x = x_new
    if return_state:
        return x, (x, y, t)
    return x


def fista_problem(inst: dict, b: np.ndarray):
    """Operator A = P T(t), lambda and L for one sparse-recovery instance."""
    n = inst["n"]
    T = Toeplitz(inst["t"].astype(np.float64), n, n)
    A = Product(Partial(inst["idx"], n), T)
    lam = lambda_from_b(A, b)
    cap = float(np.max(np.abs(T.spectrum)) ** 2)
    L = lipschitz(A, spectrum_cap=cap)
    return A, lam, L
