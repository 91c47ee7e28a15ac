"""The C ABI without a GPU: symbols, status strings, host-side validation and composition."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1710_09578_gb300 import _lib
    return _lib


def _declared():
    src = open(os.path.join(ROOT, "include", "fm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fm_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(L):
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(L.lib, n), n
    assert sorted(names) == sorted(L.EXPORTED)


def _signature(name):
    src = open(os.path.join(ROOT, "include", "fm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    m = re.search(r"fm_status\s+" + name + r"\s*\(([^;]*)\);", src)
    assert m, name
    return [" ".join(a.split()) for a in m.group(1).split(",")]


def test_fista_signature_is_the_operator_batch_form():
    # fm_fista takes the batch as operators plus one b and one x buffer per instance
    # (A, batch, b[], x[], params, report, stream)
    assert _signature("fm_fista") == [
        "const fm_op* A", "int64_t batch", "const float* const* b", "float* const* x",
        "const fm_fista_params* p", "const fm_fista_report* rep", "void* stream"]
    assert _signature("fm_fista_batch")[:5] == [
        "fm_batch B", "const float* b", "float* x", "float* y", "const fm_fista_params* p"]


def test_fista_params_layout(L):
    import ctypes
    assert ctypes.sizeof(L.fm_fista_params) == 40
    assert L.fm_fista_params.warm.offset == 32 and L.fm_fista_params.k0.offset == 36


def test_fista_host_validation(L):
    p = L.fm_fista_params(10, 20, 0.01, 1.05, 1, 0, 0, 0)
    with pytest.raises(L.FmError) as e:
        L.fm_fista([], [], [], p, None)                     # empty batch
    assert e.value.status == 1
    bad = L.fm_fista_params(-1, 20, 0.01, 1.05, 1, 0, 0, 0)
    with pytest.raises(L.FmError) as e:
        L.fm_fista([1], [8], [16], bad, None)              # negative step count
    assert e.value.status == 1
    warm = L.fm_fista_params(10, 20, 0.01, 1.05, 1, 0, 1, 5)
    rep = L.fm_fista_report(8, 8, 0, 0)
    with pytest.raises(L.FmError) as e:
        L.fm_fista([1], [8], [16], warm, rep)              # a resume goes through the batch form
    assert e.value.status == 4
    with pytest.raises(L.FmError) as e:
        L.fm_fista([1], [8], [0], p, None)                 # null x
    assert e.value.status == 1


def test_status_strings_and_version(L):
    for s in range(10):
        assert L.fm_status_string(s) and L.fm_status_string(s) != "unknown status"
    assert L.fm_status_string(99) == "unknown status"
    assert "fastmat" in L.fm_version()


def test_validation_before_any_launch(L):
    with pytest.raises(L.FmError) as e:
        L.fm_fourier(12)                      # not a power of two
    assert e.value.status == 4
    with pytest.raises(L.FmError) as e:
        L.fm_hadamard(30)
    assert e.value.status == 4
    with pytest.raises(L.FmError) as e:
        L.fm_hadamard(3, L.FM_HAD_BF16)      # BF16 tiles need n >= 16
    assert e.value.status == 4
    with pytest.raises(L.FmError) as e:
        L.fm_hadamard(4, 17)
    assert e.value.status == 1
    with pytest.raises(L.FmError) as e:
        L.fm_product([], )
    assert e.value.status == 1
    with pytest.raises(L.FmError) as e:
        L.fm_partial(0, 5, 3)                 # null pointer
    assert e.value.status == 1


def test_composition_shapes_and_dtypes(L):
    h4 = L.fm_hadamard(4)
    h3 = L.fm_hadamard(3)
    i8 = L.fm_hadamard(4, L.FM_HAD_INT8)
    try:
        assert L.fm_shape(h4) == (16, 16)
        with pytest.raises(L.FmError) as e:
            L.fm_product([h4, h3])
        assert e.value.status == 2
        with pytest.raises(L.FmError) as e:
            L.fm_sum([h4, h3])
        assert e.value.status == 2
        k = L.fm_kron([h4, h3])
        assert L.fm_shape(k) == (128, 128)
        b = L.fm_blkdiag([h4, h3])
        assert L.fm_shape(b) == (24, 24)
        hh = L.fm_hermitian(k)
        assert L.fm_shape(hh) == (128, 128)
        assert L.fm_is_real(k)
        assert L.fm_out_dtype(h4, L.FM_F32) == L.FM_F32
        assert L.fm_out_dtype(h4, L.FM_C64) == L.FM_C64
        assert L.fm_out_dtype(i8, L.FM_I8) == L.FM_I32
        with pytest.raises(L.FmError) as e:
            L.fm_out_dtype(h4, L.FM_I8)
        assert e.value.status == 3
        p = L.fm_product([k, hh])
        assert L.fm_out_dtype(p, L.FM_F32) == L.FM_F32
        # a forward call with the wrong output dtype is refused on the host
        with pytest.raises(L.FmError) as e:
            L.fm_forward(h4, 1, 16, L.FM_F32, 2, 16, L.FM_C64, 1)
        assert e.value.status == 3
        # ... and so is an output that overlaps the input
        with pytest.raises(L.FmError) as e:
            L.fm_forward(h4, 4096, 16, L.FM_F32, 4096 + 32, 16, L.FM_F32, 2)
        assert e.value.status == 5
        with pytest.raises(L.FmError) as e:
            L.fm_forward(h4, 4096, 8, L.FM_F32, 1 << 20, 16, L.FM_F32, 2)
        assert e.value.status == 2
        for h in (p, hh, b, k):
            L.fm_release(h)
    finally:
        for h in (h4, h3, i8):
            L.fm_release(h)


def test_product_releases_children_safely(L):
    a = L.fm_hadamard(2)
    b = L.fm_hadamard(2)
    p = L.fm_product([a, b])
    L.fm_release(a)
    L.fm_release(b)
    assert L.fm_shape(p) == (4, 4)   # children kept alive by the composite
    L.fm_release(p)
