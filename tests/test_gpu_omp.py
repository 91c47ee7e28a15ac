"""GPU orthogonal matching pursuit (fm_omp) against the FP64 oracle.

The picks are integer decisions taken from floating-point correlations (FP32 on the GPU,
FP64 in the oracle), so the instances have well-separated amplitudes: the support must
match exactly, in order, and x to rel-L2 1e-4 (complex64 / float32) or 1e-10 (complex128).
"""
import numpy as np
import pytest

import fm_inputs as I
import oracle as O
import oracle.omp as OMP

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1710_09578_gb300 as fm
    return fm


def sparse(n, K, rng, cplx):
    x0 = np.zeros(n, dtype=np.complex128 if cplx else np.float64)
    supp = rng.choice(n, K, replace=False)
    amp = 0.8 ** np.arange(K) * (1 + 0.5 * rng.random(K))
    ph = np.exp(2j * np.pi * rng.random(K)) if cplx else rng.choice([-1.0, 1.0], K)
    x0[supp] = amp * ph
    return x0


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - b) / np.linalg.norm(b))


def test_omp_real_toeplitz_instance(fm):
    inst = I.fista_instance(2, log2n_range=(10, 10))
    n, t, idx = inst["n"], inst["t"], inst["idx"]
    ref = O.Product(O.Partial(idx, n), O.Toeplitz(t.astype(np.float64), n, n))
    A = fm.product(fm.partial(idx, n), fm.toeplitz(t, n, n))
    rng = np.random.default_rng(21)
    x0 = sparse(n, 8, rng, False)
    b = ref.apply(x0)
    xo, So = OMP.omp(ref, b, 8)
    x, S = fm.omp(A, torch.from_numpy(b.astype(np.float32)).cuda(), 8)
    assert S.cpu().tolist() == So
    assert rel(x.cpu().numpy(), xo) <= 1e-4


def test_omp_complex_cs_operator(fm):
    c, d, idx, _, _, _ = I.cs_operator(log2n=12, k=1)
    n = len(c)
    ref = O.Product(O.Partial(idx, n), O.Diag(d), O.Circulant(c))
    A = fm.product(fm.partial(idx, n), fm.diag(d), fm.circulant(c))
    rng = np.random.default_rng(22)
    x0 = sparse(n, 12, rng, True)
    b = ref.apply(x0)
    xo, So = OMP.omp(ref, b, 12)
    x, S = fm.omp(A, torch.from_numpy(b.astype(np.complex64)).cuda(), 12)
    assert S.cpu().tolist() == So
    assert rel(x.cpu().numpy(), xo) <= 1e-4
    assert rel(x.cpu().numpy(), x0) <= 1e-4          # noise-free: the exact sparse vector


def test_omp_complex128_and_repeatable(fm):
    n = 2048
    rng = np.random.default_rng(23)
    c = I.cn(rng, (n,))
    idx = np.sort(rng.choice(n, 512, replace=False)).astype(np.int32)
    ref = O.Product(O.Partial(idx, n), O.Circulant(c))
    A = fm.product(fm.partial(idx, n), fm.circulant(c))
    x0 = sparse(n, 20, rng, True)
    b = ref.apply(x0) + 1e-3 * I.cn(rng, (512,))
    xo, So = OMP.omp(ref, b, 20)
    bg = torch.from_numpy(b).cuda()
    x, S = fm.omp(A, bg, 20)
    assert S.cpu().tolist() == So
    assert rel(x.cpu().numpy(), xo) <= 1e-10
    x2, S2 = fm.omp(A, bg, 20)
    assert torch.equal(x, x2) and torch.equal(S, S2)


def test_omp_rejections(fm):
    A = fm.fourier(64)
    b = torch.zeros(64, dtype=torch.complex64, device="cuda")
    with pytest.raises(fm.FmError) as e:
        fm.omp(A, b, 0)
    assert e.value.status == 1
    with pytest.raises(fm.FmError) as e:
        fm.omp(A, torch.zeros(64, device="cuda"), 3)     # complex operator, real b
    assert e.value.status == 3
