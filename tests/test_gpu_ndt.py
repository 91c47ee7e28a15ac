"""GPU parity of the ultrasound model pieces of Sec. 3 against the FP64 oracle: two-level
Toeplitz blocks (Eq. (7)), the block matrix H = [H_ij] of them, and the compressed model
Psi H with Psi = BlkDiag of random Fourier-row selections (Eq. (9)).

Tolerances: rel-L2 per column <= 1e-5 log2(L1 L2) for complex64 (L1 L2 the two-level
embedding), <= 1e-12 for complex128.
"""
import numpy as np
import pytest

import fm_inputs as I
import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1710_09578_gb300 as fm
    return fm


RNG = np.random.default_rng(77)


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def colerr(got, want):
    got = np.asarray(got, dtype=np.complex128).reshape(want.shape)
    return float(np.max(np.linalg.norm(got - want, axis=-1) / np.linalg.norm(want, axis=-1)))


def crand(*shape, dtype=np.complex64):
    return I.cn(RNG, shape, dtype)


def both(A, ref, X, Y, tol):
    ef = colerr(A.forward(gpu(X)).cpu().numpy(), ref.apply(X.T.astype(np.complex128)).T)
    eb = colerr(A.backward(gpu(Y)).cpu().numpy(), ref.apply(Y.T.astype(np.complex128), adjoint=True).T)
    assert ef <= tol and eb <= tol, (ef, eb, tol)


def emb(r, c):
    L = 1
    while L < r + c - 1:
        L *= 2
    return L


@pytest.mark.parametrize("r1,c1,r2,c2", [(15, 15, 15, 15), (3, 4, 2, 5), (63, 63, 63, 63), (1, 9, 33, 2),
                                         (100, 40, 7, 130)])
def test_toeplitz2_complex64(fm, r1, c1, r2, c2):
    t = crand(r1 + c1 - 1, r2 + c2 - 1)
    A = fm.toeplitz2(t, r1, c1, r2, c2)
    ref = O.Toeplitz2(t.astype(np.complex128), r1, c1, r2, c2)
    both(A, ref, crand(3, c1 * c2), crand(3, r1 * r2), 1e-5 * np.log2(emb(r1, c1) * emb(r2, c2)))


def test_toeplitz2_complex128_and_real_generator(fm):
    t = crand(9, 11, dtype=np.complex128)
    A = fm.toeplitz2(t, 4, 6, 5, 7)
    both(A, O.Toeplitz2(t, 4, 6, 5, 7), crand(2, 42, dtype=np.complex128), crand(2, 20, dtype=np.complex128), 1e-12)
    tr = RNG.standard_normal((9, 11)).astype(np.float32)
    B = fm.toeplitz2(tr, 4, 6, 5, 7)
    x = RNG.standard_normal((2, 42)).astype(np.float32)
    y = B.forward(gpu(x), real_out=True)             # real generator, real input: the real part
    want = O.Toeplitz2(tr.astype(np.float64), 4, 6, 5, 7).apply(x.T.astype(np.float64)).T
    assert y.dtype == torch.float32 and colerr(y.cpu().numpy(), want) <= 1e-5 * 8


def test_ndt_blocks_model(fm):
    # H = [H_ij], 4 x 4 blocks of two-level Toeplitz 15 x 15 levels (N1 = 4, N2 = N3 = 8)
    h, X, Y = I.ndt_model()
    n1 = h.shape[0]
    grid = [[fm.toeplitz2(h[i, j], 15, 15, 15, 15) for j in range(n1)] for i in range(n1)]
    H = fm.blocks(grid)
    ref = O.Blocks([[O.Toeplitz2(h[i, j].astype(np.complex128), 15, 15, 15, 15) for j in range(n1)]
                    for i in range(n1)])
    assert H.shape == (900, 900)
    both(H, ref, X, Y, 1e-5 * 10)
    # against the dense matrix of the definition as well
    D = ref.dense()
    got = H.forward(gpu(X)).cpu().numpy()
    assert colerr(got, (D @ X.T.astype(np.complex128)).T) <= 1e-5 * 10


def test_ndt_blocks_larger_and_rectangular_grid(fm):
    h, X, Y = I.ndt_model(n1=3, n2=16, n3=16, k=2, seed=8)
    a = 31
    grid = [[fm.toeplitz2(h[i, j], a, a, a, a) for j in range(3)] for i in range(2)]   # 2 x 3 blocks
    H = fm.blocks(grid)
    ref = O.Blocks([[O.Toeplitz2(h[i, j].astype(np.complex128), a, a, a, a) for j in range(3)] for i in range(2)])
    both(H, ref, X, Y[:, :2 * a * a], 1e-5 * 12)


def test_eq7_composition_equals_toeplitz2(fm):
    # Eq. (7) coded literally with Partial, Kron, Diag, Product and Hermitian: the same operator
    r1, c1, r2, c2 = 7, 9, 6, 5
    t = crand(r1 + c1 - 1, r2 + c2 - 1, dtype=np.complex128)
    L1, L2 = emb(r1, c1), emb(r2, c2)
    ref = O.Toeplitz2(t, r1, c1, r2, c2)
    h = (ref.spectrum / (L1 * L2)).reshape(-1)                 # 2-D DFT of the embedded generator
    FK = fm.kron(fm.fourier(L1), fm.fourier(L2))
    pin = fm.partial(np.array([j1 * L2 + j2 for j1 in range(c1) for j2 in range(c2)], np.int32), L1 * L2)
    pout = fm.partial(np.array([i1 * L2 + i2 for i1 in range(r1) for i2 in range(r2)], np.int32), L1 * L2)
    H = fm.product(pout, FK.H, fm.diag(h), FK, pin.H)
    T = fm.toeplitz2(t, r1, c1, r2, c2)
    X = crand(3, c1 * c2)
    a, b = H.forward(gpu(X)).cpu().numpy(), T.forward(gpu(X)).cpu().numpy()
    assert colerr(a, ref.apply(X.T.astype(np.complex128)).T) <= 1e-5 * 8
    assert colerr(b, a) <= 1e-5 * 8


def test_compressed_model_psi_h(fm):
    # Psi H: 16 pulse-echo signals of 32 samples (a 2 x 2 block model of 8 x 32 two-level
    # Toeplitz blocks), each compressed to n_f = 2 random Fourier coefficients
    n_meas, n_t, n_f = 16, 32, 2
    rng = np.random.default_rng(12)
    hs = [[I.cn(rng, (15, 63), np.complex64) for _ in range(2)] for _ in range(2)]
    H = fm.blocks([[fm.toeplitz2(hs[i][j], 8, 8, 32, 32) for j in range(2)] for i in range(2)])
    Href = O.Blocks([[O.Toeplitz2(hs[i][j].astype(np.complex128), 8, 8, 32, 32) for j in range(2)] for i in range(2)])
    rows = I.compressed_rows(n_meas, n_t, n_f)
    Psi = fm.blkdiag(*[fm.product(fm.partial(r, n_t), fm.fourier(n_t)) for r in rows])
    Psiref = O.BlkDiag(*[O.Product(O.Partial(r, n_t), O.Fourier(n_t)) for r in rows])
    A = fm.product(Psi, H)
    ref = O.Product(Psiref, Href)
    assert A.shape == (n_meas * n_f, 512)
    both(A, ref, crand(3, 512), crand(3, n_meas * n_f), 1e-5 * 12)
