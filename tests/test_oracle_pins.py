"""Pins of the FP64 oracle against facts fixed outside it (CPU only).

Each test checks the oracle against something other than itself: hand-typed
closed forms (tests/golden), independent library routines (numpy.fft for the
*dense* definitions, scipy.linalg constructors, numpy.kron), mathematical
invariants (adjoint identity, unitarity, diagonalisation, H H^T = n I, the
mixed-product rule) and brute force on tiny inputs.  ``test_planted_*`` plant
a plausible mistake in a copy of the oracle and check that a pin catches it.
"""
import os

import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
import oracle.gradients as OG
import oracle.omp as OMP
import oracle.lfsr as OL

GOLD = os.path.join(os.path.dirname(__file__), "golden")
RNG = np.random.default_rng(1234)


def crand(*shape):
    return RNG.standard_normal(shape) + 1j * RNG.standard_normal(shape)


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


def _golden(name):
    rows = []
    for line in open(os.path.join(GOLD, name)):
        if line.strip() and not line.startswith("#"):
            rows.append(line.split())
    return rows


def _kv(name):
    return {r[0]: np.array([float(v) for v in r[1:]]) for r in _golden(name)}


# ----------------------------------------------------------------- golden, hand-typed
def test_golden_dft4():
    want = np.array([[complex(*map(float, e.split(","))) for e in r] for r in _golden("dft4.txt")])
    assert np.allclose(O.Fourier(4).dense(), want, atol=1e-15)


def test_golden_hadamard8():
    want = np.array([[int(v) for v in r] for r in _golden("hadamard8.txt")])
    assert np.array_equal(O.Hadamard(8).dense(), want)


def test_golden_circulant3():
    g = _kv("circulant3.txt")
    C = O.Circulant(g["c"])
    assert np.allclose(C.dense() @ g["x"], g["y"])
    assert np.allclose(C.apply(g["x"]), g["y"])
    assert np.allclose(C.apply(g["x"], adjoint=True), g["yadj"])


def test_golden_toeplitz3():
    g = _kv("toeplitz3.txt")
    T = O.Toeplitz(g["t"], 3, 3)
    assert np.allclose(T.dense() @ g["x"], g["y"])
    assert np.allclose(T.apply(g["x"]), g["y"])
    assert np.allclose(T.apply(g["x"], adjoint=True), g["yadj"])


def _lasso_cases():
    g = _kv("lasso_toeplitz2.txt")
    return [(O.Toeplitz(g["sq_t"], 2, 2), g["sq_b"], g["sq_x"], float(g["sq_lam"][0]), float(g["sq_objective"][0]),
             float(g["sq_lambda"][0])),
            (O.Toeplitz(g["re_t"], 2, 3), g["re_b"], g["re_x"], float(g["re_lam"][0]), float(g["re_objective"][0]),
             float(g["re_lambda"][0]))]


def test_golden_lasso_objective_and_lambda():
    # objective = 1/2 ||A x - b||^2 + lam ||x||_1 and lambda = 0.01 ||A^T b||_inf, worked by hand
    for A, b, x, lam, obj, lam_b in _lasso_cases():
        assert abs(O.objective(A, b, x, lam) - obj) <= 1e-12 * obj
        assert abs(O.lambda_from_b(A, b) - lam_b) <= 1e-12 * lam_b


# ----------------------------------------------------------------- Fourier, Eq. (1)
@pytest.mark.parametrize("n", [1, 2, 3, 8, 12, 64, 256])
def test_fourier_dense_matches_library_dft(n):
    # numpy's FFT of the identity columns is an independent evaluation of Eq. (1)
    assert rel(O.Fourier(n).dense(), np.fft.fft(np.eye(n), axis=0)) < 1e-13


@pytest.mark.parametrize("n", [8, 64, 1024])
def test_fourier_closed_forms(n):
    F = O.Fourier(n)
    e0 = np.zeros(n)
    e0[0] = 1
    assert np.allclose(F.apply(e0), np.ones(n))               # DFT of an impulse
    m = 3 % n
    j = np.arange(n)
    tone = np.exp(2j * np.pi * m * j / n)                      # DFT of a tone is n * e_m
    want = np.zeros(n, complex)
    want[m] = n
    assert np.allclose(F.apply(tone), want, atol=1e-9)
    x = crand(n)
    assert np.isclose(np.linalg.norm(F.apply(x)) ** 2, n * np.linalg.norm(x) ** 2)  # Parseval
    D = F.dense()
    assert rel(D.conj().T @ D, n * np.eye(n)) < 1e-12          # F^H F = n I
    U = O.Fourier(n, ortho=True).dense()
    assert rel(U.conj().T @ U, np.eye(n)) < 1e-12              # F / sqrt(n) is unitary


@pytest.mark.parametrize("n,ortho", [(16, False), (12, True), (512, False)])
def test_fourier_fast_route_matches_definition(n, ortho):
    F = O.Fourier(n, ortho)
    X = crand(n, 3)
    D = F.dense()
    assert rel(F.apply(X), D @ X) < 1e-12
    assert rel(F.apply(X, adjoint=True), D.conj().T @ X) < 1e-12
    for i in [0, 1, n - 1]:
        assert rel(F.row(i), D[i]) < 1e-13


# ----------------------------------------------------------------- Circulant, Eq. (5)
@pytest.mark.parametrize("n", [1, 5, 16, 128])
def test_circulant_dense_matches_scipy(n):
    c = crand(n)
    assert np.array_equal(O.Circulant(c).dense(), sla.circulant(c))


@pytest.mark.parametrize("n", [8, 64, 100])
def test_circulant_diagonalised_by_dft(n):
    c = crand(n)
    C = O.Circulant(c).dense()
    F = O.Fourier(n).dense()
    # F C F^H = n Diag(F c)
    assert rel(F @ C @ F.conj().T, n * np.diag(F @ c)) < 1e-11
    # commutes with the cyclic shift
    S = np.roll(np.eye(n), 1, axis=0)
    assert rel(S @ C, C @ S) < 1e-14


@pytest.mark.parametrize("n", [8, 64, 100, 4096])
def test_circulant_fast_route_matches_definition(n):
    C = O.Circulant(crand(n))
    X = crand(n, 2)
    D = C.dense()
    assert rel(C.apply(X), D @ X) < 1e-12
    assert rel(C.apply(X, adjoint=True), D.conj().T @ X) < 1e-12
    Cr = O.Circulant(RNG.standard_normal(n))
    xr = RNG.standard_normal((n, 2))
    yr = Cr.apply(xr)
    assert yr.dtype == np.float64 and rel(yr, Cr.dense() @ xr) < 1e-12


# ----------------------------------------------------------------- Toeplitz (Sec. 2.1.1)
@pytest.mark.parametrize("rows,cols", [(1, 1), (3, 3), (7, 7), (5, 9), (9, 5), (64, 64), (100, 37)])
def test_toeplitz_dense_matches_scipy(rows, cols):
    t = crand(rows + cols - 1)
    col, row = t[:rows], np.concatenate([t[:1], t[rows:]])
    assert np.array_equal(O.Toeplitz(t, rows, cols).dense(), sla.toeplitz(col, row))


@pytest.mark.parametrize("rows,cols", [(3, 3), (64, 64), (5, 9), (9, 5), (1024, 1024), (100, 37)])
def test_toeplitz_embedding_matches_definition(rows, cols):
    T = O.Toeplitz(crand(rows + cols - 1), rows, cols)
    assert T.L >= rows + cols - 1 and (T.L & (T.L - 1)) == 0
    D = T.dense()
    X = crand(cols, 2)
    Y = crand(rows, 2)
    assert rel(T.apply(X), D @ X) < 1e-12
    assert rel(T.apply(Y, adjoint=True), D.conj().T @ Y) < 1e-12
    # embedding identity: T = [I 0] C_L [I; 0]
    C = O.Circulant(T.embed).dense()
    assert rel(C[:rows, :cols], D) < 1e-15


def test_toeplitz_embedding_any_length():
    # the identity holds for any embedding length >= rows + cols - 1, not only 2^k
    rows, cols = 6, 4
    t = crand(rows + cols - 1)
    D = O.Toeplitz(t, rows, cols).dense()
    for L in [9, 10, 13]:
        c = np.zeros(L, complex)
        c[:rows] = t[:rows]
        c[L - (cols - 1):] = t[rows:][::-1]
        assert rel(O.Circulant(c).dense()[:rows, :cols], D) < 1e-15


# ----------------------------------------------------------------- Hadamard (textbook)
@pytest.mark.parametrize("n", [1, 2, 4, 16, 256])
def test_hadamard_dense_matches_scipy(n):
    assert np.array_equal(O.Hadamard(n).dense(), sla.hadamard(n))


@pytest.mark.parametrize("n", [2, 64, 1024])
def test_hadamard_invariants(n):
    H = O.Hadamard(n)
    D = H.dense()
    assert np.array_equal(D @ D.T, n * np.eye(n, dtype=np.int64))    # H H^T = n I
    x = RNG.integers(-128, 128, size=(n, 3))
    assert np.array_equal(H.apply(H.apply(x)), n * x)                # H H x = n x, exact int64
    e0 = np.zeros((n, 1), dtype=np.int64)
    e0[0] = 1
    assert np.array_equal(H.apply(e0)[:, 0], np.ones(n, dtype=np.int64))
    assert np.array_equal(H.apply(x), D @ x)                         # butterflies = definition
    xf = crand(n, 2)
    assert rel(H.apply(xf), D @ xf) < 1e-13


def test_hadamard_int8_extremes_exact():
    n = 1 << 16
    x = np.full((n, 1), -128, dtype=np.int8)
    y = O.Hadamard(n).apply(x)
    assert y.dtype == np.int64 and y[0, 0] == -128 * n and np.all(y[1:, 0] == 0)
    assert abs(int(y[0, 0])) <= 2 ** 23


# ----------------------------------------------------------------- Diag, Partial
def test_diag_and_partial():
    n = 50
    d = crand(n)
    Dg = O.Diag(d)
    x = crand(n, 2)
    assert np.allclose(Dg.apply(x), np.diag(d) @ x)
    assert np.allclose(Dg.apply(x, adjoint=True), np.diag(d.conj()) @ x)
    idx = np.sort(RNG.choice(n, 17, replace=False))
    P = O.Partial(idx, n)
    ramp = np.arange(n, dtype=np.float64)
    assert np.array_equal(P.apply(ramp), idx.astype(np.float64))     # forward on x_j = j gives idx
    for r in [0, 5, 16]:
        e = np.zeros(17)
        e[r] = 1
        z = P.apply(e, adjoint=True)
        assert z[idx[r]] == 1 and np.count_nonzero(z) == 1           # adjoint of e_r is e_idx[r]
    with pytest.raises(ValueError):
        O.Partial([n], n)


# ----------------------------------------------------------------- composites
def _zoo(n=16):
    c = crand(n)
    d = np.exp(2j * np.pi * RNG.random(n))
    idx = np.sort(RNG.choice(n, n // 4, replace=False))
    t = crand(2 * n - 1)
    return {
        "fourier": O.Fourier(n),
        "fourier_ortho": O.Fourier(n, True),
        "circulant": O.Circulant(c),
        "toeplitz": O.Toeplitz(t, n, n),
        "toeplitz_rect": O.Toeplitz(crand(n + 5 - 1), n, 5),
        "hadamard": O.Hadamard(n),
        "diag": O.Diag(d),
        "partial": O.Partial(idx, n),
        "product_PDC": O.Product(O.Partial(idx, n), O.Diag(d), O.Circulant(c)),
        "sum": O.Sum(O.Circulant(c), O.Hadamard(n), O.Fourier(n)),
        "blkdiag": O.BlkDiag(O.Fourier(4), O.Partial([1, 3], 5), O.Hadamard(8)),
        "kron": O.Kron(O.Hadamard(4), O.Circulant(crand(4)), O.Fourier(2)),
        "kron_rect": O.Kron(O.Partial([0, 2], 3), O.Fourier(4)),
        "nested": O.Product(O.Kron(O.Fourier(4), O.Fourier(4)), O.Diag(d),
                            O.Kron(O.Fourier(4), O.Fourier(4))),
    }


@pytest.mark.parametrize("name", list(_zoo().keys()))
def test_adjoint_identity(name):
    A = _zoo()[name]
    x = crand(A.cols)
    y = crand(A.rows)
    lhs = np.vdot(y, A.apply(x))                 # <A x, y>
    rhs = np.vdot(A.apply(y, adjoint=True), x)   # <x, A^H y>
    assert abs(lhs - rhs) <= 1e-10 * max(1.0, abs(lhs))


@pytest.mark.parametrize("name", list(_zoo().keys()))
def test_rows_and_apply_match_dense(name):
    A = _zoo()[name]
    D = A.dense()
    X = crand(A.cols, 2)
    assert rel(A.apply(X), D @ X) < 1e-12
    Y = crand(A.rows, 2)
    assert rel(A.apply(Y, adjoint=True), D.conj().T @ Y) < 1e-12
    for i in sorted({0, A.rows // 2, A.rows - 1}):
        assert rel(A.row(i), D[i]) < 1e-12


def test_product_order():
    A, B = O.Diag(crand(6)), O.Fourier(6)
    P = O.Product(A, B)
    assert rel(P.dense(), A.dense() @ B.dense()) < 1e-14
    assert rel(P.dense(), B.dense() @ A.dense()) > 1e-3       # order matters


def test_kron_definition_matches_numpy_kron():
    fs = [O.Hadamard(4), O.Circulant(crand(4)), O.Fourier(4)]
    K = O.Kron(*fs)
    want = np.kron(fs[0].dense(), np.kron(fs[1].dense(), fs[2].dense()))
    assert rel(K.dense(), want) < 1e-14


def test_kron_mixed_product():
    A, B = O.Circulant(crand(4)), O.Fourier(8)
    C, D = O.Diag(crand(4)), O.Hadamard(8)
    lhs = O.Kron(A, B).dense() @ O.Kron(C, D).dense()
    rhs = O.Kron(O.Product(A, C), O.Product(B, D)).dense()
    assert rel(lhs, rhs) < 1e-13


def test_kron_analogue_4096_by_adjoint_and_rows():
    # the 2^12 analogue of Kron(H_256, C_1024, F_64) keeps the three-factor structure
    K = O.Kron(O.Hadamard(16), O.Circulant(crand(16)), O.Fourier(16))
    x = crand(K.cols)
    y = K.apply(x)
    for i in [0, 17, 4095]:
        assert abs(np.dot(K.row(i), x) - y[i]) < 1e-9 * np.linalg.norm(y)
    z = crand(K.rows)
    assert abs(np.vdot(z, y) - np.vdot(K.apply(z, adjoint=True), x)) < 1e-9 * abs(np.vdot(z, y))


# ----------------------------------------------------------------- FISTA
def test_soft_threshold_closed_forms():
    z = np.array([-3.0, -1.0, -0.5, 0.0, 0.5, 1.0, 3.0])
    assert np.array_equal(O.soft(z, 1.0), np.array([-2.0, 0.0, 0.0, 0.0, 0.0, 0.0, 2.0]))
    zc = np.array([3 + 4j, 0.3 + 0.4j, 0j])
    out = O.soft(zc, 1.0)
    assert np.allclose(out, [(3 + 4j) * 0.8, 0, 0])


def test_fista_orthonormal_closed_form():
    # A = H / sqrt(n) is orthonormal: with L = 1 the lasso solution soft(A^T b, lambda) is
    # reached at k = 1 and kept.
    n = 64
    A = O.Product(O.Diag(np.full(n, 1 / np.sqrt(n))), O.Hadamard(n))
    b = RNG.standard_normal(n)
    lam = 0.3
    x_star = O.soft(A.apply(b, adjoint=True), lam)
    for k in [1, 2, 7]:
        assert np.allclose(O.fista(A, b, lam, 1.0, iters=k), x_star, atol=1e-12)


def _small_problem(n=64, seed=7):
    rng = np.random.default_rng(seed)
    t = rng.standard_normal(2 * n - 1) / np.sqrt(n)
    idx = np.sort(rng.choice(n, n // 2, replace=False))
    A = O.Product(O.Partial(idx, n), O.Toeplitz(t, n, n))
    x0 = np.zeros(n)
    x0[rng.choice(n, 3, replace=False)] = rng.standard_normal(3)
    b = A.apply(x0) + 0.01 * rng.standard_normal(n // 2)
    return A, b


def test_lipschitz_bounds_against_svd():
    for seed in range(3):
        A, _ = _small_problem(seed=seed)
        smax2 = np.linalg.svd(A.dense(), compute_uv=False)[0] ** 2
        T = A.terms[1]
        cap = np.max(np.abs(T.spectrum)) ** 2
        L = O.lipschitz(A, spectrum_cap=cap)
        assert cap >= smax2 * (1 - 1e-12)            # the spectral cap is an upper bound
        assert L >= smax2 * (1 - 1e-9) or L == cap   # safe step
        assert L <= 1.05 * smax2 * (1 + 1e-9)


def test_fista_rate_bound_and_kkt():
    A, b = _small_problem()
    lam = O.lambda_from_b(A, b)
    smax2 = np.linalg.svd(A.dense(), compute_uv=False)[0] ** 2
    L = 1.01 * smax2
    x_star = O.fista(A, b, lam, L, iters=10000)
    # KKT: |A^T (A x* - b)|_j <= lambda, with equality and the sign of -x_j on the support
    g = A.apply(A.apply(x_star) - b, adjoint=True)
    assert np.all(np.abs(g) <= lam * (1 + 1e-6))
    on = np.abs(x_star) > 1e-9
    assert np.any(on)
    assert np.allclose(g[on], -lam * np.sign(x_star[on]), rtol=1e-5, atol=1e-9)
    # Beck-Teboulle: F(x_k) - F* <= 2 L ||x_0 - x*||^2 / (k + 1)^2
    F_star = O.objective(A, b, x_star, lam)
    for k in [1, 5, 20, 100]:
        xk = O.fista(A, b, lam, L, iters=k)
        bound = 2 * L * np.linalg.norm(x_star) ** 2 / (k + 1) ** 2
        assert O.objective(A, b, xk, lam) - F_star <= bound * (1 + 1e-9) + 1e-12


def test_ista_monotone_and_resume():
    A, b = _small_problem(seed=3)
    lam = O.lambda_from_b(A, b)
    L = 1.01 * np.linalg.svd(A.dense(), compute_uv=False)[0] ** 2
    prev = np.inf
    for k in range(1, 30):
        f = O.objective(A, b, O.fista(A, b, lam, L, iters=k, accel=False), lam)
        assert f <= prev + 1e-12                       # ISTA with step 1/L never increases F
        prev = f
    x1, st = O.fista(A, b, lam, L, iters=13, return_state=True)
    x2 = O.fista(A, b, lam, L, iters=17, state=st)
    assert np.array_equal(x2, O.fista(A, b, lam, L, iters=30))


# ----------------------------------------------------------------- parameter gradients
def test_golden_param_grads():
    g = _kv("param_grads2.txt")
    x, gg = g["x"], g["g"]
    assert np.allclose(OG.grad_diag(x, gg, real=True), g["grad_d"])
    for f in (OG.grad_circulant, OG.grad_circulant_definition):
        assert np.allclose(f(x, gg, real=True), g["grad_c"])
    for f in (OG.grad_toeplitz, OG.grad_toeplitz_definition):
        assert np.allclose(f(x, gg, 2, 2, real=True), g["grad_t"])


@pytest.mark.parametrize("rows,cols", [(5, 5), (4, 7), (9, 3), (1, 4)])
def test_param_grad_fast_routes_match_definitions(rows, cols):
    X, G = crand(cols, 3), crand(rows, 3)
    assert rel(OG.grad_toeplitz(X, G, rows, cols), OG.grad_toeplitz_definition(X, G, rows, cols)) < 1e-12
    Xc, Gc = crand(8, 3), crand(8, 3)
    assert rel(OG.grad_circulant(Xc, Gc), OG.grad_circulant_definition(Xc, Gc)) < 1e-12


def _loss(A, X, G):
    return float(np.real(np.vdot(G, A.apply(X))))


@pytest.mark.parametrize("kind", ["diag", "circulant", "toeplitz"])
@pytest.mark.parametrize("cplx", [False, True])
def test_param_grads_match_central_differences(kind, cplx):
    # loss(theta) = Re <G, A(theta) X> is linear in theta: central differences are exact up to
    # rounding; for a complex parameter the real and imaginary directions give Re and Im of
    # the gradient (d loss = Re <grad, d theta>)
    rng = np.random.default_rng(3)
    n, m = 8, 6
    mk = {"diag": lambda p: O.Diag(p), "circulant": lambda p: O.Circulant(p),
          "toeplitz": lambda p: O.Toeplitz(p, m, n)}[kind]
    plen = {"diag": n, "circulant": n, "toeplitz": m + n - 1}[kind]
    rows = m if kind == "toeplitz" else n
    p0 = rng.standard_normal(plen) + (1j * rng.standard_normal(plen) if cplx else 0)
    X, G = crand(n, 2), crand(rows, 2)
    grad = OG.leaf_param_grad(mk(p0), X, G)
    eps = 0.5
    for k in range(plen):
        for unit in ([1.0, 1j] if cplx else [1.0]):
            e = np.zeros(plen, dtype=complex if cplx else float)
            e[k] = unit
            fd = (_loss(mk(p0 + eps * e), X, G) - _loss(mk(p0 - eps * e), X, G)) / (2 * eps)
            an = np.real(np.conj(unit) * grad[k])
            assert abs(fd - an) <= 1e-10 * max(1.0, abs(an))


def test_product_param_grad_matches_central_differences():
    # Phi = P Diag(d) C(c): gradients of d and c through the recomputed intermediates
    rng = np.random.default_rng(4)
    n, m = 16, 5
    c = rng.standard_normal(n)
    d = np.exp(2j * np.pi * rng.random(n))
    idx = np.sort(rng.choice(n, m, replace=False))
    build = lambda d_, c_: O.Product(O.Partial(idx, n), O.Diag(d_), O.Circulant(c_))  # noqa: E731
    X, G = crand(n, 3), crand(m, 3)
    gd = OG.product_param_grad(build(d, c), 1, X, G)
    gc = OG.product_param_grad(build(d, c), 2, X, G)
    v = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    fd = (_loss(build(d + 0.5 * v, c), X, G) - _loss(build(d - 0.5 * v, c), X, G))
    assert abs(fd - np.real(np.vdot(gd, v))) < 1e-10 * abs(fd)
    w = rng.standard_normal(n)
    fd = (_loss(build(d, c + 0.5 * w), X, G) - _loss(build(d, c - 0.5 * w), X, G))
    assert abs(fd - np.dot(gc, w)) < 1e-10 * abs(fd)
    assert gc.dtype.kind == "f"


def _grad_circulant_convolution(X, G, real=False):          # convolution instead of correlation
    r = np.fft.ifft(np.sum(np.fft.fft(G, axis=0) * np.fft.fft(np.conj(X), axis=0), axis=1))
    return r.real if real else r


def test_planted_param_grad_mistakes_are_caught():
    g = _kv("param_grads2.txt")
    x, gg = g["x"][:, None], g["g"][:, None]
    x3 = np.array([[1.0], [2.0], [5.0]])
    g3 = np.array([[3.0], [4.0], [-1.0]])
    assert not np.allclose(_grad_circulant_convolution(x3, g3, True), OG.grad_circulant_definition(x3, g3, True))
    assert not np.allclose(OG.grad_diag(gg, x, True) * 0 + np.sum(gg * x), g["grad_d"])   # a summed, not per-entry, gradient
    # Toeplitz with the row part read in the wrong order (t[rows + j - i] off by one)
    bad = np.concatenate([OG.grad_toeplitz(x, gg, 2, 2, True)[:2], [np.sum(gg[0] * x[0])]])
    assert not np.allclose(bad, g["grad_t"])


# ----------------------------------------------------------------- Blocks and two-level Toeplitz
def test_golden_toeplitz2():
    g = _kv("toeplitz2_2x2.txt")
    T2 = O.Toeplitz2(g["t"].reshape(3, 3), 2, 2, 2, 2)
    assert np.array_equal(T2.dense(), g["T"].reshape(4, 4))
    assert np.allclose(T2.apply(g["x"]), g["y"])


@pytest.mark.parametrize("r1,c1,r2,c2", [(3, 3, 4, 4), (2, 5, 3, 2), (15, 15, 15, 15), (1, 6, 7, 1)])
def test_toeplitz2_separable_is_kron_of_toeplitz(r1, c1, r2, c2):
    # a separable generator t[k1, k2] = a[k1] b[k2] makes T2 = T(a) (x) T(b) (scipy constructors)
    a, b = crand(r1 + c1 - 1), crand(r2 + c2 - 1)
    T2 = O.Toeplitz2(np.outer(a, b), r1, c1, r2, c2)

    def sci(v, r, c):
        return sla.toeplitz(v[:r], np.concatenate([v[:1], v[r:]]))

    want = np.kron(sci(a, r1, c1), sci(b, r2, c2))
    assert rel(T2.dense(), want) < 1e-14


@pytest.mark.parametrize("r1,c1,r2,c2", [(3, 3, 4, 4), (2, 5, 3, 2), (9, 4, 5, 11)])
def test_toeplitz2_fast_route_and_adjoint(r1, c1, r2, c2):
    T2 = O.Toeplitz2(crand(r1 + c1 - 1, r2 + c2 - 1), r1, c1, r2, c2)
    D = T2.dense()
    X, Y = crand(c1 * c2, 3), crand(r1 * r2, 3)
    assert rel(T2.apply(X), D @ X) < 1e-12
    assert rel(T2.apply(Y, adjoint=True), D.conj().T @ Y) < 1e-12


def test_blocks_dense_and_apply():
    grid = [[O.Toeplitz(crand(5), 3, 3), O.Toeplitz(crand(4), 3, 2)],
            [O.Toeplitz(crand(4), 2, 3), O.Fourier(2)]]
    B = O.Blocks(grid)
    want = np.block([[grid[0][0].dense(), grid[0][1].dense()], [grid[1][0].dense(), grid[1][1].dense()]])
    assert rel(B.dense(), want) < 1e-15
    X, Y = crand(5, 2), crand(5, 2)
    assert rel(B.apply(X), want @ X) < 1e-13
    assert rel(B.apply(Y, adjoint=True), want.conj().T @ Y) < 1e-13


def test_eq7_block_is_zero_padded_two_level_circulant():
    # Eq. (7): a two-level Toeplitz block is the row/column selection of
    # (F (x) F)^H Diag(h) (F (x) F), with h the 2-D DFT of the embedded generator over L1 L2
    r1, c1, r2, c2 = 3, 4, 2, 5
    T2 = O.Toeplitz2(crand(r1 + c1 - 1, r2 + c2 - 1), r1, c1, r2, c2)
    L1, L2 = T2.L1, T2.L2
    FK = O.Kron(O.Fourier(L1), O.Fourier(L2))
    C2 = FK.dense().conj().T @ np.diag(T2.spectrum.reshape(-1) / (L1 * L2)) @ FK.dense()
    rows = [i1 * L2 + i2 for i1 in range(r1) for i2 in range(r2)]
    cols = [j1 * L2 + j2 for j1 in range(c1) for j2 in range(c2)]
    assert rel(C2[np.ix_(rows, cols)], T2.dense()) < 1e-12


# ----------------------------------------------------------------- OMP
class _DenseOp(O.Op):
    def __init__(self, M):
        self.M = np.asarray(M)
        self.rows, self.cols = self.M.shape
        self.real = self.M.dtype.kind != "c"

    def dense(self):
        return self.M

    def _apply(self, X, adjoint):
        return (self.M.conj().T if adjoint else self.M) @ X


def test_golden_omp_with_tie():
    g = _kv("omp2x3.txt")
    A = _DenseOp(g["A"].reshape(2, 3))
    x, S, res = OMP.omp(A, g["b"], 2, return_residuals=True)
    assert S == [int(v) for v in g["S"]]
    assert np.allclose(x, g["x"]) and np.allclose(res, g["res"], atol=1e-12)


def test_omp_orthonormal_exact_recovery_and_order():
    # A = F / sqrt(n) is unitary: A^H b = x0, so OMP picks the support in order of decreasing
    # |x0| and recovers x0 exactly after K steps
    n, K = 64, 6
    A = O.Product(O.Diag(np.full(n, 1 / np.sqrt(n))), O.Fourier(n))
    x0 = np.zeros(n, dtype=complex)
    supp = RNG.choice(n, K, replace=False)
    x0[supp] = np.exp(2j * np.pi * RNG.random(K)) * (2.0 ** -np.arange(K))
    x, S = OMP.omp(A, A.apply(x0), K)
    assert S == [int(j) for j in supp]
    assert rel(x, x0) < 1e-12


def test_omp_residual_orthogonal_to_selected_columns():
    n = 32
    A = O.Product(O.Partial(np.sort(RNG.choice(n, 20, replace=False)), n), O.Toeplitz(RNG.standard_normal(2 * n - 1), n, n))
    b = RNG.standard_normal(20)
    x, S, res = OMP.omp(A, b, 8, return_residuals=True)
    r = b - A.apply(x)
    AS = np.stack([OMP.column(A, j) for j in S], axis=1)
    assert np.max(np.abs(AS.T @ r)) < 1e-10 * np.linalg.norm(b)
    assert all(res[i + 1] <= res[i] + 1e-12 for i in range(len(res) - 1))
    assert len(set(S)) == len(S)


def _matching_pursuit(A, b, K):                          # no re-solve: only the new coefficient
    r, x = b.astype(float).copy(), np.zeros(A.cols)
    for _ in range(K):
        c = A.apply(r, adjoint=True)
        j = int(np.argmax(np.abs(c)))
        a = OMP.column(A, j)
        z = a @ r / (a @ a)
        x[j] += z
        r = r - z * a
    return x


def test_planted_omp_mistake_is_caught():
    g = _kv("omp2x3.txt")
    A = _DenseOp(g["A"].reshape(2, 3))
    assert not np.allclose(_matching_pursuit(A, g["b"], 2), g["x"])


# ----------------------------------------------------------------- LFSR circulant
def test_golden_lfsr3():
    g = _kv("lfsr3.txt")
    assert np.array_equal(OL.lfsr_bits(3, 0b011, 0b001, 8), g["bits"].astype(np.int64))
    C = OL.LFSRCirculant(3, 0b011, 0b001, 8)
    assert np.array_equal(C.dense()[:, 0], g["c"])


@pytest.mark.parametrize("m,a", [(5, 2), (7, 1), (10, 3)])
def test_lfsr_maximal_length_properties(m, a):
    # x^m + x^a + 1 primitive: period 2^m - 1, 2^(m-1) ones per period, two-level autocorrelation
    P = (1 << m) - 1
    bits = OL.lfsr_bits(m, 1 | (1 << a), 1, 2 * P)
    assert np.array_equal(bits[:P], bits[P:])
    assert all(not np.array_equal(bits[:P], np.roll(bits[:P], s)) for s in range(1, P))
    assert bits[:P].sum() == 1 << (m - 1)
    c = 1.0 - 2.0 * bits[:P]
    ac = np.array([c @ np.roll(c, s) for s in range(P)])
    assert ac[0] == P and np.all(ac[1:] == -1)


# ----------------------------------------------------------------- planted mistakes
class _CirculantNoConj(O.Circulant):
    def _apply(self, X, adjoint):                       # forgets the conjugate in the adjoint
        return np.fft.ifft(self.spectrum[:, None] * np.fft.fft(X.astype(complex), axis=0), axis=0)


class _ToeplitzOffByOne(O.Toeplitz):
    def dense(self):                                    # upper triangle shifted by one
        i = np.arange(self.rows)[:, None]
        j = np.arange(self.cols)[None, :]
        d = i - j
        return np.where(d >= 0, self.t[np.clip(d, 0, None)],
                        self.t[np.clip(self.rows - d, 0, len(self.t) - 1)])


class _KronSwapped(O.Kron):
    def dense(self):                                    # factors in the wrong order
        return O.Kron(*self.factors[::-1]).dense()


def _objective_no_half(A, b, x, lam):                  # drops the 1/2 of the data term
    r = A.apply(x) - b
    return float(np.vdot(r, r).real) + lam * float(np.sum(np.abs(x)))


def _objective_l2(A, b, x, lam):                       # 2-norm in place of the l1 norm
    r = A.apply(x) - b
    return 0.5 * float(np.vdot(r, r).real) + lam * float(np.linalg.norm(x))


def _lambda_forward(A, b, rel=0.01):                   # A b in place of A^T b
    return rel * float(np.max(np.abs(A.apply(b))))


def _lambda_two_norm(A, b, rel=0.01):                  # 2-norm in place of the max norm
    return rel * float(np.linalg.norm(A.apply(b, adjoint=True)))


def test_planted_lasso_mistakes_are_caught():
    (A, b, x, lam, obj, lam_b), _ = _lasso_cases()
    for wrong in (_objective_no_half, _objective_l2):
        assert abs(wrong(A, b, x, lam) - obj) > 1e-6
    for wrong in (_lambda_forward, _lambda_two_norm):
        assert abs(wrong(A, b) - lam_b) > 1e-6


def test_planted_mistakes_are_caught():
    n = 16
    with pytest.raises(AssertionError):
        A = _CirculantNoConj(crand(n))
        x, y = crand(n), crand(n)
        assert abs(np.vdot(y, A.apply(x)) - np.vdot(A.apply(y, adjoint=True), x)) < 1e-9
    with pytest.raises(AssertionError):
        t = crand(2 * n - 1)
        col, row = t[:n], np.concatenate([t[:1], t[n:]])
        assert np.array_equal(_ToeplitzOffByOne(t, n, n).dense(), sla.toeplitz(col, row))
    with pytest.raises(AssertionError):
        fs = [O.Hadamard(4), O.Fourier(4)]
        assert rel(_KronSwapped(*fs).dense(), np.kron(fs[0].dense(), fs[1].dense())) < 1e-14


# ----------------------------------------------------------------- input generators
def test_inputs_deterministic_and_snr():
    import fm_inputs as I
    a = I.fista_instance(5)
    b = I.fista_instance(5)
    assert a["n"] == b["n"] and np.array_equal(a["t"], b["t"]) and np.array_equal(a["idx"], b["idx"])
    inst = I.fista_instance(0, log2n_range=(10, 10))
    n = inst["n"]
    bb = I.fista_measurements(inst)
    A = O.Product(O.Partial(inst["idx"], n), O.Toeplitz(inst["t"].astype(np.float64), n, n))
    clean = A.apply(inst["x0"])
    snr = 20 * np.log10(np.linalg.norm(clean) / np.linalg.norm(bb.astype(np.float64) - clean))
    assert abs(snr - 30.0) < 0.01
    c, X, Y = I.circulant_tiny(n=64, k=3)
    assert X.shape == (3, 64) and X.dtype == np.complex128
