"""GPU parameter gradients (fm_param_grad, FmParamApply) against the FP64 oracle and central
differences.

Bar: relative L2 error of the gradient vector <= 1e-5 log2(L) for FP32 (L the leaf's
transform length), <= 1e-11 for complex128; central differences of the loss
Re <G, A(theta) X> (linear in theta, so exact up to rounding) to 1e-3 relative.
"""
import numpy as np
import pytest

import fm_inputs as I
import oracle as O
import oracle.gradients as OG

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1710_09578_gb300 as fm
    return fm


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def loss(A, Xg, Gg):
    Y = A.forward(Xg).to(torch.complex128)
    return torch.vdot(Gg.to(torch.complex128).flatten(), Y.flatten()).real.item()


def test_cs_operator_param_grads_full_size(fm):
    # Phi = P Diag(d) C(c) at n = 2^18 on 64 complex64 columns: gradients of the phases d and of
    # the +-1 generator c (a real parameter), with the intermediates recomputed in the backward
    c, d, idx, X, Y, G = I.cs_operator()
    n = len(c)
    P = fm.partial(idx, n)

    def build(d_t, c_t):
        D, C = fm.diag(d_t), fm.circulant(c_t)
        return fm.product(P, D, C), [D, C]

    d_t = gpu(d).requires_grad_(True)
    c_t = gpu(c.astype(np.float32)).requires_grad_(True)
    Xg, Gg = gpu(X), gpu(G)
    Yg = fm.apply_params(build, Xg, d_t, c_t)
    (Yg * Gg.conj()).real.sum().backward()
    ref = O.Product(O.Partial(idx, n), O.Diag(d), O.Circulant(c))
    want_d = OG.product_param_grad(ref, 1, X.T, G.T)
    want_c = OG.product_param_grad(ref, 2, X.T, G.T)
    tol = 1e-5 * np.log2(n)
    assert d_t.grad.dtype == torch.complex64 and c_t.grad.dtype == torch.float32
    assert rel(d_t.grad.cpu().numpy(), want_d) <= tol
    assert rel(c_t.grad.cpu().numpy(), want_c) <= tol
    # central differences along random directions of d and c
    rng = np.random.default_rng(9)
    v = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)
    eps = 0.5
    fd = (loss(build(gpu(d + eps * v), gpu(c))[0], Xg, Gg) - loss(build(gpu(d - eps * v), gpu(c))[0], Xg, Gg)) / (2 * eps)
    an = float(np.real(np.vdot(d_t.grad.cpu().numpy().astype(np.complex128), v)))
    assert abs(fd - an) <= 1e-3 * abs(an)
    w = rng.standard_normal(n)
    fd = (loss(build(gpu(d), gpu(c + eps * w))[0], Xg, Gg) - loss(build(gpu(d), gpu(c - eps * w))[0], Xg, Gg)) / (2 * eps)
    an = float(np.dot(c_t.grad.cpu().numpy().astype(np.float64), w))
    assert abs(fd - an) <= 1e-3 * abs(an)


def test_toeplitz_generator_grad_fista_size(fm):
    # A = P T(t), n = 2^12, real FP32 t of length 2n - 1 (a FISTA instance): gradient of t
    inst = I.fista_instance(0, log2n_range=(12, 12))
    n, t, idx = inst["n"], inst["t"], inst["idx"]
    rng = np.random.default_rng(10)
    X = rng.standard_normal((4, n)).astype(np.float32)
    G = rng.standard_normal((4, len(idx))).astype(np.float32)
    P = fm.partial(idx, n)

    def build(t_t):
        T = fm.toeplitz(t_t, n, n)
        return fm.product(P, T), [T]

    t_t = gpu(t).requires_grad_(True)
    Xg, Gg = gpu(X), gpu(G)
    (fm.apply_params(build, Xg, t_t) * Gg).sum().backward()
    ref = O.Product(O.Partial(idx, n), O.Toeplitz(t.astype(np.float64), n, n))
    want = OG.product_param_grad(ref, 1, X.T, G.T)
    assert t_t.grad.dtype == torch.float32
    assert rel(t_t.grad.cpu().numpy(), want.real) <= 1e-5 * np.log2(2 * n)
    w = rng.standard_normal(2 * n - 1)
    fd = (loss(build(gpu(t + 0.5 * w))[0], Xg, Gg) - loss(build(gpu(t - 0.5 * w))[0], Xg, Gg))
    an = float(np.dot(t_t.grad.cpu().numpy().astype(np.float64), w))
    assert abs(fd - an) <= 1e-3 * abs(an)


@pytest.mark.parametrize("rows,cols", [(300, 500), (700, 129), (20000, 20000)])
def test_toeplitz_complex_rectangular(fm, rows, cols):
    rng = np.random.default_rng(rows)
    t = (rng.standard_normal(rows + cols - 1) + 1j * rng.standard_normal(rows + cols - 1)).astype(np.complex64)
    X = (rng.standard_normal((3, cols)) + 1j * rng.standard_normal((3, cols))).astype(np.complex64)
    G = (rng.standard_normal((3, rows)) + 1j * rng.standard_normal((3, rows))).astype(np.complex64)
    T = fm.toeplitz(t, rows, cols)
    got = fm.param_grad(T, T, gpu(X), gpu(G)).cpu().numpy()
    want = OG.grad_toeplitz(X.T, G.T, rows, cols)
    L = 1 << int(np.ceil(np.log2(rows + cols - 1)))
    assert rel(got, want) <= 1e-5 * np.log2(L)


def test_circulant_and_diag_complex128(fm):
    c0, X0, Y0 = I.circulant_tiny()
    C = fm.circulant(c0)
    got = fm.param_grad(C, C, gpu(X0), gpu(Y0)).cpu().numpy()
    assert rel(got, OG.grad_circulant(X0.T, Y0.T)) <= 1e-11
    d = np.exp(2j * np.pi * np.random.default_rng(1).random(4096))
    D = fm.diag(d)
    A = fm.product(D, C)                       # the diagonal sees C x as its input
    got = fm.param_grad(A, D, gpu(X0), gpu(Y0)).cpu().numpy()
    want = OG.product_param_grad(O.Product(O.Diag(d), O.Circulant(c0)), 0, X0.T, Y0.T)
    assert rel(got, want) <= 1e-11


def test_param_grad_rejections(fm):
    c = np.ones(64)
    C = fm.circulant(c)
    D = fm.diag(np.ones(64))
    X = torch.zeros((1, 64), dtype=torch.complex64, device="cuda")
    with pytest.raises(fm.FmError) as e:                      # not a term of the operator
        fm.param_grad(C, D, X, X)
    assert e.value.status == 1
    with pytest.raises(fm.FmError) as e:                      # present only as an adjoint
        fm.param_grad(fm.product(D, C.H), C, X, X)
    assert e.value.status == 4
    with pytest.raises(fm.FmError) as e:                      # no parameter vector
        F = fm.fourier(64)
        fm.param_grad(F, F, X, X)
    assert e.value.status == 1
