"""GPU: the LFSR circulant and the dense execution of small operators against the FP64 oracle.

Tolerances: FP32 rel-L2 1e-5 log2(n) (the fast path's bar; a dense product of n terms is
within it), complex128 1e-12; the LFSR column is checked entry by entry after rounding to +-1.
"""
import numpy as np
import pytest

import oracle as O
import oracle.lfsr as OL

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1710_09578_gb300 as fm
    return fm


RNG = np.random.default_rng(31)


def crand(*shape, dt=np.complex64):
    return (RNG.standard_normal(shape) + 1j * RNG.standard_normal(shape)).astype(dt)


def colerr(got, want):
    got = np.asarray(got, dtype=np.complex128).reshape(want.shape)
    return float(np.max(np.linalg.norm(got - want, axis=-1) / np.linalg.norm(want, axis=-1)))


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("nbits,a,n", [(3, 1, 8), (10, 3, 4096), (17, 3, 1 << 18)])
def test_lfsr_circulant(fm, nbits, a, n):
    taps = 1 | (1 << a)
    C = fm.lfsr_circulant(nbits, taps, 1, n)
    seq = OL.lfsr_sequence(nbits, taps, 1, n)
    e0 = torch.zeros((1, n), dtype=torch.complex64, device="cuda")
    e0[0, 0] = 1
    col = C.forward(e0).cpu().numpy()[0]
    assert np.array_equal(np.sign(col.real), seq)            # the first column, entry by entry
    ref = O.Circulant(seq)
    X, Y = crand(3, n), crand(3, n)
    assert colerr(C.forward(gpu(X)).cpu().numpy(), ref.apply(X.T).T) <= 1e-5 * np.log2(max(n, 2))
    assert colerr(C.backward(gpu(Y)).cpu().numpy(), ref.apply(Y.T, adjoint=True).T) <= 1e-5 * np.log2(max(n, 2))


def _leaves(fm):
    c = crand(32)
    t = crand(16 + 24 - 1)
    return [(fm.fourier(64), O.Fourier(64)), (fm.circulant(c), O.Circulant(c.astype(np.complex128))),
            (fm.toeplitz(t, 16, 24), O.Toeplitz(t.astype(np.complex128), 16, 24)),
            (fm.hadamard(5), O.Hadamard(32))]


@pytest.mark.parametrize("k", [1, 7, 300])
def test_dense_execution_matches_oracle(fm, k):
    for A, ref in _leaves(fm):
        A.set_dense(True)
        X, Y = crand(k, A.cols), crand(k, A.rows)
        tol = 1e-5 * 6
        assert colerr(A.forward(gpu(X)).cpu().numpy(), ref.apply(X.T.astype(np.complex128)).T) <= tol
        assert colerr(A.backward(gpu(Y)).cpu().numpy(), ref.apply(Y.T.astype(np.complex128), adjoint=True).T) <= tol
        A.set_dense(False)


def test_dense_complex128_inside_product_and_calibration(fm):
    c = crand(64, dt=np.complex128)
    d = crand(64, dt=np.complex128)
    C = fm.circulant(c)
    C.set_dense(True)
    A = fm.product(fm.diag(d), C)                       # the dense leaf is not fused with Diag
    ref = O.Product(O.Diag(d), O.Circulant(c))
    X = crand(5, 64, dt=np.complex128)
    assert colerr(A.forward(gpu(X)).cpu().numpy(), ref.apply(X.T).T) <= 1e-12
    r = C.calibrate_dense(4096, torch.complex64)
    assert r["ms_fast"] > 0 and r["ms_dense"] > 0 and r["dense"] == (r["ms_dense"] < r["ms_fast"])
    X = crand(9, 64)
    assert colerr(C.forward(gpu(X)).cpu().numpy(), O.Circulant(c).apply(X.T.astype(np.complex128)).T) <= 1e-5 * 6


def test_dense_rejects_large_operators(fm):
    with pytest.raises(fm.FmError) as e:
        fm.fourier(128).set_dense(True)
    assert e.value.status == 4
