"""GPU parity: every operator's forward and adjoint against the FP64 oracle.

Tolerances: FP32 FFT paths rel-L2 <= 1e-5 * log2(L) per column (L the transform length);
complex128 paths <= 1e-12; Hadamard FP32 <= 1e-5 * log2(n); int8 Hadamard and row
selection bit-exact.
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


DEV = "cuda"
RNG = np.random.default_rng(2024)


def colerr(got, want):
    got = np.asarray(got, dtype=np.complex128).reshape(want.shape)
    num = np.linalg.norm(got - want, axis=-1)
    den = np.maximum(np.linalg.norm(want, axis=-1), 1e-300)
    return float(np.max(num / den))


def tol32(L):
    return 1e-5 * max(1.0, np.log2(L))


def blk(k, n, dtype):
    return I.column_block(RNG, k, n, dtype)


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def both(fm, A, ref, X, Y, tol):
    """Check forward on X ([K, cols]) and adjoint on Y ([K, rows]) against the oracle."""
    got_f = A.forward(gpu(X)).cpu().numpy()
    got_b = A.backward(gpu(Y)).cpu().numpy()
    want_f = ref.apply(X.T).T
    want_b = ref.apply(Y.T, adjoint=True).T
    ef, eb = colerr(got_f, want_f), colerr(got_b, want_b)
    assert ef <= tol and eb <= tol, (ef, eb, tol)
    return ef, eb


# ---------------------------------------------------------------- Fourier
@pytest.mark.parametrize("n", [2, 4, 8, 64, 512, 1024, 4096, 8192, 16384, 32768, 1 << 18])
@pytest.mark.parametrize("dt", [np.complex64, np.complex128])
def test_fourier(fm, n, dt):
    k = 3 if n <= 4096 else 2
    X, Y = blk(k, n, dt), blk(k, n, dt)
    tol = tol32(n) if dt == np.complex64 else 1e-12
    both(fm, fm.fourier(n), O.Fourier(n), X, Y, tol)


@pytest.mark.parametrize("n", [16, 2048, 32768])
def test_fourier_ortho_and_real_input(fm, n):
    X = blk(5, n, np.float32)
    Y = blk(5, n, np.complex64)
    both(fm, fm.fourier(n, ortho=True), O.Fourier(n, True), X, Y, tol32(n))


# ---------------------------------------------------------------- Circulant
@pytest.mark.parametrize("n", [2, 8, 64, 4096, 16384, 32768, 1 << 17])
def test_circulant_complex(fm, n):
    c = I.cn(RNG, (n,))
    k = 5 if n <= 16384 else 2
    both(fm, fm.circulant(c), O.Circulant(c), blk(k, n, np.complex64), blk(k, n, np.complex64), tol32(n))


@pytest.mark.parametrize("n", [8, 1024, 32768])
def test_circulant_real_pairs(fm, n):
    # real generator on real data: two real columns ride in one complex transform (odd K)
    c = RNG.standard_normal(n)
    both(fm, fm.circulant(c), O.Circulant(c), blk(5, n, np.float32), blk(5, n, np.float32), tol32(n))


@pytest.mark.parametrize("n,k", [(2048, 3), (8192, 2), (8192, 80)])
def test_circulant_c128_two_pass_small_tiles(fm, n, k):
    # complex128 transforms of 2^11 .. 2^13 on a few columns run the two-pass plan on
    # four-warp tiles with radix-4 passes; with 64 columns or more, whole-vector tiles
    c = I.cn(RNG, (n,))
    both(fm, fm.circulant(c), O.Circulant(c), blk(k, n, np.complex128), blk(k, n, np.complex128), 1e-12)


def test_circulant_tiny_workload_c128(fm):
    # Circulant N=4096 with K=16 complex128 columns, against the dense definition
    c, X, Y = I.circulant_tiny()
    A = fm.circulant(c)
    ref = O.Circulant(c)
    D = ref.dense()
    got_f = A.forward(gpu(X)).cpu().numpy()
    got_b = A.backward(gpu(Y)).cpu().numpy()
    assert colerr(got_f, (D @ X.T).T) <= 1e-12
    assert colerr(got_b, (D.conj().T @ Y.T).T) <= 1e-12
    # adjoint identity <C x, y> = <x, C^H y>
    lhs = np.vdot(Y, got_f)
    rhs = np.vdot(got_b, X)
    assert abs(lhs - rhs) <= 1e-10 * abs(lhs)


def test_circulant_c128_big(fm):
    n = 1 << 15
    c = I.cn(RNG, (n,))
    both(fm, fm.circulant(c), O.Circulant(c), blk(2, n, np.complex128), blk(2, n, np.complex128), 1e-12)


# ---------------------------------------------------------------- Toeplitz
@pytest.mark.parametrize("rows,cols", [(1, 1), (3, 3), (100, 37), (37, 100), (1024, 1024), (5000, 3000),
                                       (16384, 16384)])
def test_toeplitz_complex(fm, rows, cols):
    t = I.cn(RNG, (rows + cols - 1,))
    ref = O.Toeplitz(t, rows, cols)
    both(fm, fm.toeplitz(t, rows, cols), ref, blk(3, cols, np.complex64), blk(3, rows, np.complex64),
         tol32(ref.L))


@pytest.mark.parametrize("n", [1024, 8192])
def test_toeplitz_real(fm, n):
    t = (RNG.standard_normal(2 * n - 1) / np.sqrt(n)).astype(np.float32)
    ref = O.Toeplitz(t.astype(np.float64), n, n)
    both(fm, fm.toeplitz(t, n, n), ref, blk(3, n, np.float32), blk(3, n, np.float32), tol32(2 * n))


# ---------------------------------------------------------------- Hadamard
@pytest.mark.parametrize("log2n", [1, 2, 4, 7, 10, 13, 14, 15, 16, 17])
def test_hadamard_fp32(fm, log2n):
    n = 1 << log2n
    k = 5 if log2n <= 14 else 3
    X, Y = blk(k, n, np.float32), blk(k, n, np.float32)
    both(fm, fm.hadamard(log2n), O.Hadamard(n), X, Y, tol32(n))


@pytest.mark.parametrize("log2n", [3, 12, 16])
def test_hadamard_complex(fm, log2n):
    n = 1 << log2n
    both(fm, fm.hadamard(log2n), O.Hadamard(n), blk(3, n, np.complex64), blk(3, n, np.complex64), tol32(n))


@pytest.mark.parametrize("log2n", [1, 5, 14, 16])
def test_hadamard_int8_exact(fm, log2n):
    n = 1 << log2n
    X = RNG.integers(-128, 128, size=(7, n), dtype=np.int8)
    X[0] = -128                                     # extreme column: |y_0| = 128 n
    A = fm.hadamard(log2n, fm.FM_HAD_INT8)
    got = A.forward(gpu(X)).cpu().numpy()
    assert got.dtype == np.int32
    want = O.Hadamard(n).apply(X.T).T
    assert np.array_equal(got.astype(np.int64), want)
    got_b = A.backward(gpu(X)).cpu().numpy()
    assert np.array_equal(got_b.astype(np.int64), want)


@pytest.mark.parametrize("log2n", [4, 5, 7, 10, 13, 14, 15, 16])
@pytest.mark.parametrize("mode,tol", [("FM_HAD_BF16", 2e-2), ("FM_HAD_BF16X2", 1e-5)])
def test_hadamard_bf16_tensor_cores(fm, log2n, mode, tol):
    n = 1 << log2n
    A = fm.hadamard(log2n, getattr(fm, mode))
    X = blk(3, n, np.float32)
    got = A.forward(gpu(X)).cpu().numpy()
    want = O.Hadamard(n).apply(X.T.astype(np.float64)).T
    assert colerr(got, want) <= tol
    got_b = A.backward(gpu(X)).cpu().numpy()
    assert colerr(got_b, want) <= tol


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("log2n", [15, 16])
def test_hadamard_long_columns_ld_and_sum(fm, log2n, form):
    # long columns (two or four 2^14 blocks), with (form 0) and without (form 1) the L2
    # prefetch of a later column: padded leading dimensions on both sides, and a Sum whose
    # second term accumulates into the first term's output
    n = 1 << log2n

    def had(mode=None):
        H = fm.hadamard(log2n) if mode is None else fm.hadamard(log2n, mode)
        H.set_plan(n, 5, form)
        return H

    X = blk(40, n + 64, np.float32)   # more columns than the prefetch distance on small GPUs
    want = O.Hadamard(n).apply(X[:, :n].T.astype(np.float64)).T
    Yg = torch.zeros((40, n + 32), dtype=torch.float32, device=DEV)
    had().forward(gpu(X)[:, :n], out=Yg[:, :n])
    assert colerr(Yg[:, :n].cpu().numpy(), want) <= tol32(n)
    assert torch.count_nonzero(Yg[:, n:]).item() == 0
    d = RNG.standard_normal(n).astype(np.float32)
    S = fm.sum_(had(), had(), fm.diag(d))
    got = S.forward(gpu(X)[:, :n]).cpu().numpy()
    assert colerr(got, 2 * want + d * X[:, :n]) <= tol32(n)
    Xi = RNG.integers(-128, 128, size=(3, n + 64)).astype(np.int8)
    Xi[0, :n] = -128                                  # extreme column: |y_0| = 128 n
    gi = had(fm.FM_HAD_INT8).forward(gpu(Xi)[:, :n]).cpu().numpy()
    assert np.array_equal(gi.astype(np.int64), O.Hadamard(n).apply(Xi[:, :n].T.astype(np.int64)).T)


@pytest.mark.parametrize("log2n,dt", [(24, np.complex64), (22, np.complex128)])
def test_fourier_and_circulant_largest(fm, log2n, dt):
    # the largest lengths the constructors accept, through the two-pass plan
    n = 1 << log2n
    X = blk(1, n, dt)
    tol = tol32(n) if dt == np.complex64 else 1e-10
    got = fm.fourier(n).forward(gpu(X)).cpu().numpy()
    assert colerr(got, O.Fourier(n).apply(X.T).T) <= tol
    c = I.cn(RNG, (n,))
    got = fm.circulant(c).backward(gpu(X)).cpu().numpy()
    assert colerr(got, O.Circulant(c).apply(X.T, adjoint=True).T) <= tol


@pytest.mark.parametrize("log2n,k", [(17, 2), (19, 1), (22, 1), (24, 1)])
def test_hadamard_up_to_2p24(fm, log2n, k):
    # lengths above one column tile run as two passes (low 14 index bits, then the rest)
    n = 1 << log2n
    X = blk(k, n, np.float32)
    got = fm.hadamard(log2n).forward(gpu(X)).cpu().numpy()
    assert colerr(got, O.Hadamard(n).apply(X.T.astype(np.float64)).T) <= tol32(n)


def test_hadamard_long_int8_complex_and_sum(fm):
    n = 1 << 20
    Xi = RNG.integers(-128, 128, size=(2, n)).astype(np.int8)
    gi = fm.hadamard(20, fm.FM_HAD_INT8).forward(gpu(Xi)).cpu().numpy()
    assert gi.dtype == np.int32
    assert np.array_equal(gi.astype(np.int64), O.Hadamard(n).apply(Xi.T.astype(np.int64)).T)
    Xc = blk(2, 1 << 18, np.complex64)
    both(fm, fm.hadamard(18), O.Hadamard(1 << 18), Xc, Xc, tol32(1 << 18))
    X = blk(2, n, np.float32)
    got = fm.sum_(fm.hadamard(20), fm.hadamard(20)).forward(gpu(X)).cpu().numpy()   # accumulation
    assert colerr(got, 2 * O.Hadamard(n).apply(X.T.astype(np.float64)).T) <= tol32(n)


def test_hadamard_bf16_workload_full(fm):
    xf, _ = I.hadamard_block()
    want = O.Hadamard(1 << 16).apply(xf.T.astype(np.float64)).T
    for mode, tol in (("FM_HAD_BF16", 2e-2), ("FM_HAD_BF16X2", 1e-5)):
        got = fm.hadamard(16, getattr(fm, mode)).forward(gpu(xf)).cpu().numpy()
        assert colerr(got, want) <= tol, mode


@pytest.mark.parametrize("form", [0, 1])
def test_hadamard_workload_full(fm, form):
    # the 2^16 x 256 block with and without the L2 prefetch: FP32 within tolerance, int8 bit-exact
    xf, xi = I.hadamard_block()
    A = fm.hadamard(16)
    A.set_plan(1 << 16, 5, form)
    got = A.forward(gpu(xf)).cpu().numpy()
    want = O.Hadamard(1 << 16).apply(xf.T.astype(np.float64)).T
    assert colerr(got, want) <= tol32(1 << 16)
    Ai = fm.hadamard(16, fm.FM_HAD_INT8)
    Ai.set_plan(1 << 16, 5, form)
    gi = Ai.forward(gpu(xi)).cpu().numpy()
    assert np.array_equal(gi.astype(np.int64), O.Hadamard(1 << 16).apply(xi.T).T)


# ---------------------------------------------------------------- Diag, Partial
@pytest.mark.parametrize("dt", [np.float32, np.complex64, np.complex128])
def test_diag(fm, dt):
    n = 1000
    d = I.cn(RNG, (n,))
    tol = 1e-6 if dt != np.complex128 else 1e-15
    both(fm, fm.diag(d), O.Diag(d), blk(3, n, dt), blk(3, n, dt), tol)


def test_partial_bit_exact(fm):
    n = 1 << 18
    idx = np.sort(RNG.choice(n, n // 4, replace=False)).astype(np.int32)
    P = fm.partial(idx, n)
    ramp = np.arange(n, dtype=np.float32)[None, :].repeat(2, 0)
    got = P.forward(gpu(ramp)).cpu().numpy()
    assert np.array_equal(got, np.broadcast_to(idx.astype(np.float32), got.shape))
    e = np.zeros((1, n // 4), dtype=np.float32)
    e[0, 17] = 1.0
    z = P.backward(gpu(e)).cpu().numpy()[0]
    assert z[idx[17]] == 1.0 and np.count_nonzero(z) == 1


def test_partial_rejects_bad_indices(fm):
    with pytest.raises(fm.FmError):
        fm.partial(np.array([0, 3, 3], dtype=np.int32), 8)
    with pytest.raises(fm.FmError):
        fm.partial(np.array([0, 8], dtype=np.int32), 8)


# ---------------------------------------------------------------- compositions
def _pdc(n, m, seed):
    rng = np.random.default_rng(seed)
    c = np.where(rng.integers(0, 2, n) == 1, 1.0, -1.0)
    d = np.exp(2j * np.pi * rng.random(n)).astype(np.complex64)
    idx = np.sort(rng.choice(n, m, replace=False)).astype(np.int32)
    return c, d, idx


@pytest.mark.parametrize("n", [64, 4096, 1 << 16])
def test_product_pdc_fused(fm, n):
    c, d, idx = _pdc(n, n // 4, n)
    A = fm.product(fm.partial(idx, n), fm.diag(d), fm.circulant(c))
    ref = O.Product(O.Partial(idx, n), O.Diag(d), O.Circulant(c))
    both(fm, A, ref, blk(3, n, np.complex64), blk(3, n // 4, np.complex64), tol32(n))


def test_back_to_back_dependent_launches(fm):
    # Every kernel starts early and waits for its predecessor on the stream before touching
    # memory: long chains of dependent calls with no host synchronisation must give the
    # composed result.
    n, k = 1 << 16, 8
    X = blk(k, n, np.float32)
    H = fm.hadamard(16)
    bufs = [gpu(X), torch.empty((k, n), dtype=torch.float32, device=DEV)]
    for i in range(6):
        H.forward(bufs[i % 2], out=bufs[(i + 1) % 2])
    got = bufs[0].cpu().numpy().astype(np.float64)
    assert colerr(got, X.astype(np.float64) * float(n) ** 3) <= 6 * tol32(n)
    # forward, adjoint, forward of a three-pass operator, again without synchronising
    m = 1 << 18
    c, d, idx = _pdc(m, m // 4, 11)
    A = fm.product(fm.partial(idx, m), fm.diag(d), fm.circulant(c))
    ref = O.Product(O.Partial(idx, m), O.Diag(d), O.Circulant(c))
    Xc = blk(2, m, np.complex64)
    W = A.forward(A.backward(A.forward(gpu(Xc)))).cpu().numpy()
    want = ref.apply(ref.apply(ref.apply(Xc.T), adjoint=True)).T
    # a race (a pass reading its predecessor's output early) gives O(1) errors; the bound
    # leaves room for the rounding of three applies amplified by C's spread of |spectrum|
    assert colerr(W, want) <= 10 * tol32(m)


def test_graph_capture_replays_chained_launches(fm):
    # the chained launches captured into a CUDA graph (programmatic edges) and replayed give
    # the eager result bit for bit, and the oracle's within tolerance
    n = 1 << 14
    c, d, idx = _pdc(n, n // 4, 12)
    A = fm.product(fm.partial(idx, n), fm.diag(d), fm.circulant(c))
    ref = O.Product(O.Partial(idx, n), O.Diag(d), O.Circulant(c))
    H = fm.hadamard(15)
    X = gpu(blk(4, n, np.complex64))
    Xh = gpu(blk(4, 1 << 15, np.float32))
    Y = torch.empty((4, n // 4), dtype=torch.complex64, device=DEV)
    Z = torch.empty_like(X)
    Hy = torch.empty_like(Xh)
    Hz = torch.empty_like(Xh)
    A.reserve(4, torch.complex64)

    def run():
        A.forward(X, out=Y)
        A.backward(Y, out=Z)
        H.forward(Xh, out=Hy)
        H.forward(Hy, out=Hz)

    run()
    torch.cuda.synchronize()
    Z0, Hz0 = Z.clone(), Hz.clone()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        run()
    Z.zero_()
    Hz.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(Z, Z0) and torch.equal(Hz, Hz0)
    Xn = X.cpu().numpy()
    want = ref.apply(ref.apply(Xn.T), adjoint=True).T
    assert colerr(Z.cpu().numpy(), want) <= 10 * tol32(n)  # two applies, C's spread of |spectrum|
    assert colerr(Hz.cpu().numpy(), Xh.cpu().numpy().astype(np.float64) * float(1 << 15)) <= 2 * tol32(1 << 15)


def test_cs_operator_workload_full(fm):
    # Phi = P Diag(d) C at N = 2^18, M = N/4, 64 complex64 columns
    c, d, idx, X, Y, G = I.cs_operator()
    n = len(c)
    A = fm.product(fm.partial(idx, n), fm.diag(d), fm.circulant(c))
    ref = O.Product(O.Partial(idx, n), O.Diag(d), O.Circulant(c))
    ef, eb = both(fm, A, ref, X, Y, tol32(n))
    # the launch configuration the benchmark times: the split calibrated for 64 columns
    A.calibrate(64, torch.complex64)
    ef, eb = both(fm, A, ref, X, Y, tol32(n))
    # sampled rows straight from the definition
    got = A.forward(gpu(X[:2])).cpu().numpy()
    for r in [0, 777, n // 4 - 1]:
        row = ref.row(r)
        want = row @ X[:2].T.astype(np.complex128)
        assert np.all(np.abs(got[:, r] - want) <= 1e-4 * np.linalg.norm(want) + 1e-3)


def test_sum_blkdiag_nested(fm):
    n = 64
    c = I.cn(RNG, (n,))
    S = fm.sum_(fm.circulant(c), fm.hadamard(6), fm.fourier(n))
    Sr = O.Sum(O.Circulant(c), O.Hadamard(n), O.Fourier(n))
    both(fm, S, Sr, blk(3, n, np.complex64), blk(3, n, np.complex64), tol32(n))
    both(fm, S, Sr, blk(3, n, np.float32), blk(3, n, np.complex64), tol32(n))
    idx = np.array([1, 3], dtype=np.int32)
    B = fm.blkdiag(fm.fourier(4), fm.partial(idx, 5), fm.hadamard(3), fm.circulant(c))
    Br = O.BlkDiag(O.Fourier(4), O.Partial(idx, 5), O.Hadamard(8), O.Circulant(c))
    both(fm, B, Br, blk(4, Br.cols, np.complex64), blk(4, Br.rows, np.complex64), tol32(n))


@pytest.mark.parametrize("shape", [(4, 4, 2), (16, 16, 16), (8, 2, 32), (2, 1024, 4)])
def test_kron_three_factors(fm, shape):
    a, b, cc = shape
    c = I.cn(RNG, (b,))
    A = fm.kron(fm.hadamard(int(np.log2(a))), fm.circulant(c), fm.fourier(cc))
    ref = O.Kron(O.Hadamard(a), O.Circulant(c), O.Fourier(cc))
    n = a * b * cc
    both(fm, A, ref, blk(3, n, np.complex64), blk(3, n, np.complex64), tol32(n))


@pytest.mark.parametrize("dt", [np.float32, np.complex64])
@pytest.mark.parametrize("la,lb", [(1, 6), (3, 5), (5, 4), (8, 4)])
def test_kron_hadamard_strided_axis(fm, dt, la, lb):
    # Hadamard along the outer axis of Kron(H, H, Diag): a strided axis with 16 or more
    # vectors side by side (every transform length of the strided kernel), plus a Sum
    # whose second term accumulates
    d = RNG.standard_normal(4).astype(np.float32)
    A = fm.kron(fm.hadamard(la), fm.hadamard(lb), fm.diag(d))
    ref = O.Kron(O.Hadamard(1 << la), O.Hadamard(1 << lb), O.Diag(d))
    n = ref.cols
    both(fm, A, ref, blk(3, n, dt), blk(3, n, dt), tol32(n))
    X = blk(2, n, dt)
    got = fm.sum_(A, A).forward(gpu(X)).cpu().numpy()
    assert colerr(got, 2 * ref.apply(X.T.astype(np.complex128)).T) <= tol32(n)


@pytest.mark.parametrize("pair", [0, 1, 2, 3])
@pytest.mark.parametrize("la,mid,lb,ortho", [(4, 4, 6, 0), (6, 3, 4, 1), (7, 2, 6, 0), (5, 1, 5, 0), (8, 1, 6, 1),
                                          (4, 1, 8, 0)])
def test_kron_hadamard_fourier_fused(fm, la, mid, lb, ortho, pair):
    # Kron(H, middle, F) on complex64: the outer Hadamard and inner Fourier factors run as
    # one fused pass (middle = 1: no middle factor, the pass writes the output directly)
    c = I.cn(RNG, (mid,))
    # middle factor: a circulant (power-of-two length) or a diagonal (any length), or none
    pow2 = mid & (mid - 1) == 0
    mk = ([fm.circulant(c)] if pow2 else [fm.diag(c)]) if mid > 1 else []
    mr = ([O.Circulant(c)] if pow2 else [O.Diag(c)]) if mid > 1 else []
    kids = [fm.hadamard(la)] + mk + [fm.fourier(1 << lb, ortho=bool(ortho))]
    refs = [O.Hadamard(1 << la)] + mr + [O.Fourier(1 << lb, ortho=bool(ortho))]
    A = fm.kron(*kids)
    A.set_plan(A.rows, 3, pair)        # one CTA, a pair or a quad of CTAs per tile
    ref = O.Kron(*refs)
    n = ref.cols
    both(fm, A, ref, blk(3, n, np.complex64), blk(3, n, np.complex64), tol32(n))
    X = blk(2, n, np.complex64)
    got = fm.sum_(A, A).forward(gpu(X)).cpu().numpy()       # the second term accumulates (same plan)
    assert colerr(got, 2 * ref.apply(X.T).T) <= tol32(n)


def test_kron_mixed_and_nested(fm):
    idx = np.array([0, 2, 5], dtype=np.int32)
    d = I.cn(RNG, (8,))
    A = fm.kron(fm.partial(idx, 6), fm.product(fm.fourier(8), fm.diag(d)), fm.hadamard(2))
    ref = O.Kron(O.Partial(idx, 6), O.Product(O.Fourier(8), O.Diag(d)), O.Hadamard(4))
    both(fm, A, ref, blk(3, ref.cols, np.complex64), blk(3, ref.rows, np.complex64), 1e-5 * 6)
    Z = blk(2, ref.rows, np.complex64)
    got = A.H.forward(gpu(Z)).cpu().numpy()          # forward of A^H is the backward of A
    assert colerr(got, ref.apply(Z.T, adjoint=True).T) <= 1e-5 * 6


def test_kron_workload_analogue(fm):
    c, X, Y = I.kron_small()
    A = fm.kron(fm.hadamard(4), fm.circulant(c), fm.fourier(16))
    ref = O.Kron(O.Hadamard(16), O.Circulant(c), O.Fourier(16))
    D = ref.dense()
    got = A.forward(gpu(X.astype(np.complex64))).cpu().numpy()
    assert colerr(got, (D @ X.T).T) <= tol32(4096)


@pytest.mark.parametrize("pair", [0, 1, 2, 3])
def test_kron_workload_full_sampled(fm, pair):
    # Kron(H_256, C_1024, F_64) on 4 columns of length 2^24: sampled rows from the
    # definition and the adjoint identity at full size (both forms of the fused pass).
    c, X, Y = I.kron_large()
    A = fm.kron(fm.hadamard(8), fm.circulant(c), fm.fourier(64))
    A.set_plan(A.rows, 3, pair)
    ref = O.Kron(O.Hadamard(256), O.Circulant(c), O.Fourier(64))
    Xg, Yg = gpu(X), gpu(Y)
    F = A.forward(Xg)
    B = A.backward(Yg)
    lhs = torch.vdot(Yg.flatten().to(torch.complex128), F.flatten().to(torch.complex128)).item()
    rhs = torch.vdot(B.flatten().to(torch.complex128), Xg.flatten().to(torch.complex128)).item()
    assert abs(lhs - rhs) <= 1e-4 * abs(lhs)
    Fh = F.cpu().numpy()
    Xd = X.astype(np.complex128)
    for r in [0, 12345, (1 << 24) - 1, 9_000_001]:
        row = ref.row(r)
        want = row @ Xd.T
        err = np.abs(Fh[:, r] - want) / (np.linalg.norm(Fh, axis=1) / np.sqrt(1 << 24))
        assert np.all(err <= 5 * tol32(1 << 24)), err


# ---------------------------------------------------------------- autograd
def test_autograd_matches_adjoint_and_fd(fm):
    c, d, idx, X, Y, G = I.cs_operator(log2n=12, k=4)
    n = len(c)
    A = fm.product(fm.partial(idx, n), fm.diag(d), fm.circulant(c))
    ref = O.Product(O.Partial(idx, n), O.Diag(d), O.Circulant(c))
    x = gpu(X).requires_grad_(True)
    y = fm.apply(A, x)
    g = gpu(G)
    (y * g.conj()).real.sum().backward()
    want = ref.apply(G.T, adjoint=True).T
    assert colerr(x.grad.cpu().numpy(), want) <= tol32(n)
    # central differences of f(x) = Re <g, A x> along a random direction v; the map is
    # linear, so the difference quotient is exact up to rounding for any step
    v = blk(4, n, np.complex64)
    eps = 0.5
    dY = (fm.apply(A, gpu(X + eps * v)) - fm.apply(A, gpu(X - eps * v))).to(torch.complex128)
    fd = torch.vdot(g.flatten().to(torch.complex128), dY.flatten()).real.item() / (2 * eps)
    an = float(np.real(np.vdot(x.grad.cpu().numpy().astype(np.complex128), v.astype(np.complex128))))
    assert abs(fd - an) <= 1e-3 * abs(an)


def test_autograd_hadamard_real(fm):
    n = 1 << 16
    X = blk(1, n, np.float32)
    A = fm.hadamard(16)
    x = gpu(X).requires_grad_(True)
    g = blk(1, n, np.float32)
    (fm.apply(A, x) * gpu(g)).sum().backward()
    want = O.Hadamard(n).apply(g.T.astype(np.float64)).T
    assert colerr(x.grad.cpu().numpy(), want) <= tol32(n)
    # central differences on the first 2^10 coordinates of column 0
    gd = gpu(g).to(torch.float64)
    for j in [0, 5, 1023]:
        e = np.zeros_like(X)
        e[0, j] = 0.5
        dY = (fm.apply(A, gpu(X + e)) - fm.apply(A, gpu(X - e))).to(torch.float64)
        fd = (dY * gd).sum().item() / 1.0
        assert abs(fd - x.grad[0, j].item()) <= 1e-3 * max(1.0, abs(fd))


def _fd_check(fm, A, X, g, grad, v, eps=0.5, tol=1e-3):
    """Central difference of f(x) = Re <g, A x> along v against <grad, v> (the map is linear,
    so the quotient is exact up to rounding for any step)."""
    dY = (fm.apply(A, gpu(X + eps * v)) - fm.apply(A, gpu(X - eps * v))).to(torch.complex128)
    fd = torch.vdot(g.flatten().to(torch.complex128), dY.flatten()).real.item() / (2 * eps)
    an = float(np.real(np.vdot(grad.astype(np.complex128).ravel(), v.astype(np.complex128).ravel())))
    assert abs(fd - an) <= tol * abs(an), (fd, an)


def test_autograd_cs_operator_full_size(fm):
    # config 2: Phi = P Diag(d) C at n = 2^18 on 64 complex64 columns, through the calibrated
    # two-pass plan the benchmark times; gradient against the FP64 oracle's Phi^H g and central
    # differences
    c, d, idx, X, Y, G = I.cs_operator()
    n = len(c)
    A = fm.product(fm.partial(idx, n), fm.diag(d), fm.circulant(c))
    A.calibrate(X.shape[0], torch.complex64)
    x = gpu(X).requires_grad_(True)
    g = gpu(G)
    (fm.apply(A, x) * g.conj()).real.sum().backward()
    ref = O.Product(O.Partial(idx, n), O.Diag(d), O.Circulant(c))
    want = ref.apply(G.T, adjoint=True).T
    got = x.grad.cpu().numpy()
    assert colerr(got, want) <= tol32(n)
    v = blk(X.shape[0], n, np.complex64)
    _fd_check(fm, A, X, g, got, v)


def test_autograd_real_input_complex_operator(fm):
    # real x into a complex operator: the gradient is Re(A^H g), computed by the library
    # (fm_backward with a real output type)
    c, d, idx, X, Y, G = I.cs_operator(log2n=12, k=3)
    n = len(c)
    A = fm.product(fm.partial(idx, n), fm.diag(d), fm.circulant(c))
    Xr = np.ascontiguousarray(X.real).astype(np.float32)
    x = gpu(Xr).requires_grad_(True)
    g = gpu(G)
    (fm.apply(A, x) * g.conj()).real.sum().backward()
    assert x.grad.dtype == torch.float32
    ref = O.Product(O.Partial(idx, n), O.Diag(d), O.Circulant(c))
    want = ref.apply(G.T, adjoint=True).T.real
    assert colerr(x.grad.cpu().numpy(), want) <= tol32(n)
    assert torch.equal(x.grad, A.backward(g, real_out=True))


def test_autograd_kron_analogue(fm):
    # config 4's 2^12 analogue Kron(H_16, C_16, F_16): gradient against the oracle's A^H g and
    # central differences (the adjoint recomputes the mode-product intermediates)
    c, X, Y = I.kron_small()
    A = fm.kron(fm.hadamard(4), fm.circulant(c), fm.fourier(16))
    ref = O.Kron(O.Hadamard(16), O.Circulant(c), O.Fourier(16))
    Xc = X.astype(np.complex64)
    x = gpu(Xc).requires_grad_(True)
    G = blk(X.shape[0], 4096, np.complex64)
    g = gpu(G)
    (fm.apply(A, x) * g.conj()).real.sum().backward()
    want = ref.apply(G.T.astype(np.complex128), adjoint=True).T
    got = x.grad.cpu().numpy()
    assert colerr(got, want) <= tol32(4096)
    _fd_check(fm, A, Xc, g, got, blk(X.shape[0], 4096, np.complex64))


def test_autograd_kron_full_size(fm):
    # config 4 at full size, 2^24 x 4: the gradient is the library adjoint of g, and central
    # differences along a random direction agree with it
    c, X, Y = I.kron_large()
    A = fm.kron(fm.hadamard(8), fm.circulant(c), fm.fourier(64))
    x = gpu(X).requires_grad_(True)
    g = gpu(Y)
    (fm.apply(A, x) * g.conj()).real.sum().backward()
    assert torch.equal(x.grad, A.backward(g))
    v = I.cn(np.random.default_rng(41), X.shape, np.complex64)
    _fd_check(fm, A, X, g, x.grad.cpu().numpy(), v, tol=2e-3)


def test_autograd_hadamard_fd_slice(fm):
    # config 1: central differences on the first 2^10 input coordinates of column 0 -- along a
    # random direction supported on that slice, and along e_j for a spread of j in it
    n = 1 << 16
    X = blk(4, n, np.float32)
    A = fm.hadamard(16)
    x = gpu(X).requires_grad_(True)
    G = blk(4, n, np.float32)
    (fm.apply(A, x) * gpu(G)).sum().backward()
    grad = x.grad.cpu().numpy()
    gd = gpu(G).to(torch.float64)
    rng = np.random.default_rng(5)
    v = np.zeros_like(X)
    v[0, :1024] = rng.standard_normal(1024)
    dY = (fm.apply(A, gpu(X + 0.5 * v)) - fm.apply(A, gpu(X - 0.5 * v))).to(torch.float64)
    fd = (dY * gd).sum().item()
    an = float(np.dot(grad[0, :1024].astype(np.float64), v[0, :1024]))
    assert abs(fd - an) <= 1e-3 * abs(an)
    for j in range(0, 1024, 73):
        e = np.zeros_like(X)
        e[0, j] = 0.5
        dY = (fm.apply(A, gpu(X + e)) - fm.apply(A, gpu(X - e))).to(torch.float64)
        assert abs((dY * gd).sum().item() - grad[0, j]) <= 1e-3 * max(1.0, abs(grad[0, j]))


# ---------------------------------------------------------------- edge cases
def test_zero_columns_and_strided_input(fm):
    A = fm.fourier(64)
    empty = torch.empty((0, 64), dtype=torch.complex64, device=DEV)
    assert A.forward(empty).shape == (0, 64)
    X = blk(6, 128, np.complex64)
    Xg = gpu(X)[:, :64]                 # leading dimension 128 > 64
    got = A.forward(Xg).cpu().numpy()
    assert colerr(got, O.Fourier(64).apply(X[:, :64].T).T) <= tol32(64)


def test_repeat_calls_bit_identical(fm):
    n = 1 << 16
    c, d, idx = _pdc(n, n // 4, 5)
    A = fm.product(fm.partial(idx, n), fm.diag(d), fm.circulant(c))
    X = gpu(blk(3, n, np.complex64))
    a = A.forward(X)
    b = A.forward(X)
    assert torch.equal(a, b)


# ---------------------------------------------------------------- launch tracing
def test_trace_labels_and_times(fm):
    from paper_1710_09578_gb300 import _lib
    c, X, _ = I.kron_small()
    A = fm.kron(fm.hadamard(8), fm.circulant(np.tile(c, 4)), fm.fourier(64))
    Xg = gpu(blk(2, A.cols, np.complex64))
    A.forward(Xg)
    torch.cuda.synchronize()
    _lib.fm_trace_begin(16)
    before = fm.launch_count()
    A.forward(Xg)
    A.backward(Xg)
    recs = _lib.fm_trace_end()
    assert len(recs) == fm.launch_count() - before == 4      # two passes per apply
    names = [r[0] for r in recs]
    assert names[0].startswith("kron_hf_kernel<8,6>") and names[1].startswith("fft2_kernel<f32,L=2^6,strided,conv>")
    assert all(ms > 0 for _, ms in recs)
    with pytest.raises(fm.FmError):
        _lib.fm_trace_end()                                   # not on any more
