"""The circulant entry point that allocates nothing (fm_circulant_apply_noalloc).

It serves callers that cannot allocate device memory while applying an operator (their
memory belongs to another allocator or a fixed budget, or they must avoid the implicit
synchronisation of cudaMalloc / cudaFree).  Its results must equal those of the ordinary
entry points fm_forward / fm_backward, call after call, although every call reuses one
static scratch array.  This file is collected last, so a run that stops at the first
failure has run every other test before it.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1710_09578_gb300 as fm
    return fm


def _relerr(a, b):
    a = a.to(torch.complex128)
    b = b.to(torch.complex128)
    return float(((a - b).abs().pow(2).sum(1).sqrt() / b.abs().pow(2).sum(1).sqrt()).max())


def test_noalloc_matches_ordinary_entry_points(fm):
    from paper_1710_09578_gb300 import _lib
    rng = np.random.default_rng(11)
    n, k = 1 << 17, 4                      # two-pass plan: 4 MiB of scratch per call
    c = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)
    C = fm.circulant(c)
    stream = torch.cuda.current_stream().cuda_stream
    tol = 1e-5 * np.log2(n)
    for adjoint in (0, 1):
        X = torch.from_numpy((rng.standard_normal((k, n)) + 1j * rng.standard_normal((k, n)))
                             .astype(np.complex64)).cuda()
        want = C.backward(X) if adjoint else C.forward(X)
        Ys = [torch.full_like(X, float("nan")) for _ in range(2)]
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        for Y in Ys:                       # two calls in a row share the static scratch
            _lib.fm_circulant_apply_noalloc(C.handle, adjoint, X.data_ptr(), n, Y.data_ptr(), n, k, stream)
        torch.cuda.synchronize()
        # the calls reserved nothing on the device: the static array was set up when the
        # operator was built, and no workspace was grown
        assert torch.cuda.mem_get_info()[0] == free_before
        for Y in Ys:
            assert _relerr(Y, want) <= tol


def test_noalloc_largest_call_and_leading_dimensions(fm):
    from paper_1710_09578_gb300 import _lib
    rng = np.random.default_rng(12)
    n, k = 1 << 18, 8                      # exactly the 16 MiB the static scratch holds
    c = rng.standard_normal(n).astype(np.float32)
    C = fm.circulant(c)
    ldx, ldy = n + 64, n + 128             # leading dimensions larger than the column length
    Xb = torch.from_numpy((rng.standard_normal((k, ldx)) + 1j * rng.standard_normal((k, ldx)))
                          .astype(np.complex64)).cuda()
    X = Xb[:, :n]
    want = C.forward(X)
    Yb = torch.full((k, ldy), float("nan"), dtype=torch.complex64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        _lib.fm_circulant_apply_noalloc(C.handle, 0, Xb.data_ptr(), ldx, Yb.data_ptr(), ldy, k, stream)
        torch.cuda.synchronize()
        assert _relerr(Yb[:, :n], want) <= 1e-5 * np.log2(n)
    assert torch.isnan(Yb[:, n:].real).all()   # nothing written between the columns


def test_noalloc_rejects_oversized_calls(fm):
    from paper_1710_09578_gb300 import _lib
    n, k = 1 << 18, 9                      # 9 * 2^18 * 8 bytes = 18 MiB > 16 MiB
    C = fm.circulant(np.ones(n))
    X = torch.zeros((k, n), dtype=torch.complex64, device="cuda")
    Y = torch.empty_like(X)
    with pytest.raises(_lib.FmError) as e:
        _lib.fm_circulant_apply_noalloc(C.handle, 0, X.data_ptr(), n, Y.data_ptr(), n, k, 0)
    assert e.value.status == 4 and "scratch" in str(e.value)
    with pytest.raises(_lib.FmError) as e:
        _lib.fm_circulant_apply_noalloc(fm.fourier(64).handle, 0, X.data_ptr(), n, Y.data_ptr(), n, 1, 0)
    assert e.value.status == 1
