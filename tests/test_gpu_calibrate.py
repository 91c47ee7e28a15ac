"""GPU: calibration of the two-pass split (fm_calibrate / fm_set_split).

Every split the calibration may choose must give the oracle's result; the calibration must
pick one of its candidates and keep the operator correct; the JSON cache must restore a
stored choice without timing.
"""
import json

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


def colerr(got, want):
    got = np.asarray(got, dtype=np.complex128).reshape(want.shape)
    num = np.linalg.norm(got - want, axis=-1)
    den = np.maximum(np.linalg.norm(want, axis=-1), 1e-300)
    return float(np.max(num / den))


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _cs(n, seed):
    rng = np.random.default_rng(seed)
    c = np.where(rng.integers(0, 2, n) == 1, 1.0, -1.0)
    d = np.exp(2j * np.pi * rng.random(n)).astype(np.complex64)
    idx = np.sort(rng.choice(n, n // 4, replace=False)).astype(np.int32)
    return c, d, idx


def _check(A, ref, X, Y, tol):
    ef = colerr(A.forward(gpu(X)).cpu().numpy(), ref.apply(X.T).T)
    eb = colerr(A.backward(gpu(Y)).cpu().numpy(), ref.apply(Y.T, adjoint=True).T)
    assert ef <= tol and eb <= tol, (ef, eb, tol)


@pytest.mark.parametrize("n1", [32, 64, 128, 512, 2048, 8192])
def test_every_split_matches_oracle(fm, n1):
    n = 1 << 18
    c, d, idx = _cs(n, 5)
    A = fm.product(fm.partial(idx, n), fm.diag(d), fm.circulant(c))
    ref = O.Product(O.Partial(idx, n), O.Diag(d), O.Circulant(c))
    A.set_split(n, n1)
    X = I.column_block(RNG, 2, n, np.complex64)
    Y = I.column_block(RNG, 2, n // 4, np.complex64)
    _check(A, ref, X, Y, 1e-5 * 18)
    F = fm.fourier(n)
    F.set_split(n, n1)
    _check(F, O.Fourier(n), X, X, 1e-5 * 18)


def test_calibrate_picks_a_candidate_and_stays_correct(fm, tmp_path):
    n = 1 << 18
    c, d, idx = _cs(n, 6)
    A = fm.product(fm.partial(idx, n), fm.diag(d), fm.circulant(c))
    ref = O.Product(O.Partial(idx, n), O.Diag(d), O.Circulant(c))
    cache = str(tmp_path / "tune.json")
    res = A.calibrate(8, torch.complex64, cache=cache)
    assert [e["kind"] for e in res] == [0, 1, 2] and all(e["L"] == n for e in res)
    for e in res:
        assert e["value"] in e["ms"] and len(e["ms"]) >= 2
        assert all(v > 0 for v in e["ms"].values())
    X = I.column_block(RNG, 2, n, np.complex64)
    Y = I.column_block(RNG, 2, n // 4, np.complex64)
    _check(A, ref, X, Y, 1e-5 * 18)
    # a second operator restores the stored split from the cache without timing
    with open(cache) as f:
        stored = json.load(f)
    assert len(stored) == 1
    B = fm.product(fm.partial(idx, n), fm.diag(d), fm.circulant(c))
    again = B.calibrate(8, torch.complex64, cache=cache)
    assert [(e["kind"], e["value"]) for e in again] == [(e["kind"], e["value"]) for e in res]
    assert list(stored)[0].startswith(B.signature() + "|n=")
    _check(B, ref, X, Y, 1e-5 * 18)


def test_split_rules(fm):
    F = fm.fourier(1 << 16)
    with pytest.raises(fm.FmError):
        F.set_split(1 << 16, 48)          # not a power of two
    with pytest.raises(fm.FmError):
        F.set_split(1 << 16, 4)           # N2 = 2^14 above one FP64 tile
    F.set_split(1 << 12, 64)              # no transform of that length: nothing to do
    F.set_split(1 << 16, 0)               # back to the default
    # a single-tile transform has no split to tune, only its tile shape and radix schedule
    assert [e["kind"] for e in fm.fourier(1024).calibrate(4)] == [1, 2]
    with pytest.raises(fm.FmError):
        F.set_plan(1 << 16, 2, 4)         # radix cap 0 or 3 only
    with pytest.raises(fm.FmError):
        F.set_plan(1 << 16, 1, 5)         # tile shapes 0 .. 4


def _plan_cases(fm):
    rng = np.random.default_rng(40)
    c = I.cn(rng, (1024,))
    K = fm.kron(fm.hadamard(4), fm.circulant(c), fm.fourier(16))
    Kref = O.Kron(O.Hadamard(16), O.Circulant(c), O.Fourier(16))
    c2, d2, idx2 = _cs(4096, 3)
    P = fm.product(fm.partial(idx2, 4096), fm.diag(d2), fm.circulant(c2))
    Pref = O.Product(O.Partial(idx2, 4096), O.Diag(d2), O.Circulant(c2))
    F = fm.kron(fm.fourier(512), fm.fourier(32))
    Fref = O.Kron(O.Fourier(512), O.Fourier(32))
    # a two-pass transform whose first pass is 2^10 along a stride of 256 (fused twiddles)
    G = fm.fourier(1 << 18)
    G.set_split(1 << 18, 1024)
    return [(K, Kref, 1024), (P, Pref, 4096), (F, Fref, 512), (G, O.Fourier(1 << 18), 1 << 18)]


@pytest.mark.parametrize("tile,rcap", [(0, 0), (1, 0), (2, 0), (3, 0), (4, 0), (0, 3), (1, 3), (2, 3), (3, 3), (4, 3)])
def test_every_plan_choice_keeps_parity(fm, tile, rcap):
    # the compiled variants the calibration chooses among: tile shape of strided views and the
    # radix schedule, on a Kron circulant of 2^10 along a stride, a 2^12 convolution tile, a
    # 2^9 Fourier along a stride of 32 and the passes of a 2^18 Fourier transform
    for A, ref, L in _plan_cases(fm):
        A.set_plan(L, 1, tile)
        A.set_plan(L, 2, rcap)
        X = I.column_block(RNG, 3, A.cols, np.complex64)
        Y = I.column_block(RNG, 3, A.rows, np.complex64)
        _check(A, ref, X, Y, 1e-5 * 18)


@pytest.mark.parametrize("inner", [2, 4, 16, 32])
@pytest.mark.parametrize("tile", [0, 4])
def test_radix32_tiles_ragged(fm, inner, tile):
    # the radix-32 tile of 2^10 along a stride (vectors side by side, 8 per tile) with vector
    # counts that leave a partial last tile or let a tile span two outer indices, and the same
    # tile on contiguous vectors (a plain circulant on 5 columns) and at 2^9
    rng = np.random.default_rng(41)
    c = I.cn(rng, (1024,))
    K = fm.kron(fm.hadamard(1), fm.circulant(c), fm.fourier(inner))
    K.set_plan(1024, 1, tile)
    Kref = O.Kron(O.Hadamard(2), O.Circulant(c), O.Fourier(inner))
    X = I.column_block(RNG, 3, K.cols, np.complex64)
    Y = I.column_block(RNG, 3, K.rows, np.complex64)
    _check(K, Kref, X, Y, 1e-5 * 18)
    for n in (512, 1024):
        C = fm.circulant(c[:n])
        C.set_plan(n, 1, tile)
        X = I.column_block(RNG, 5, n, np.complex64)
        _check(C, O.Circulant(c[:n]), X, X, 1e-5 * 10)


@pytest.mark.parametrize("n1", [32, 64, 256, 1024, 2048])
def test_two_pass_staged_outputs(fm, n1):
    # a 2^16 Fourier transform under every split with its second pass's interleaved outputs
    # (staged through shared memory where the tile holds 16 or more rows), forward and
    # adjoint, and a Sum whose second term accumulates into the first's output
    n = 1 << 16
    F = fm.fourier(n)
    F.set_split(n, n1)
    X = I.column_block(RNG, 3, n, np.complex64)
    _check(F, O.Fourier(n), X, X, 1e-5 * 16)
    G = fm.fourier(n)
    G.set_split(n, n1)
    S = fm.sum_(F, G)
    got = S.forward(gpu(X)).cpu().numpy()
    want = 2 * O.Fourier(n).apply(X.T.astype(np.complex128)).T
    err = np.linalg.norm(got - want, axis=1) / np.linalg.norm(want, axis=1)
    assert err.max() <= 1e-5 * 16
