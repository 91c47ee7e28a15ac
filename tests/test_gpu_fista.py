"""GPU batched FISTA (fm_fista) against the FP64 oracle, instance by instance.

Bar: ||x_gpu - x_fp64|| / ||x_fp64|| <= 1e-4 per instance after the same protocol
(lambda = 0.01 ||A^T b||_inf, L from 20 power iterations capped by max|c_hat|^2, 200 steps).
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


def _batch(fm, insts):
    ops, bs = [], []
    for inst in insts:
        n = inst["n"]
        ops.append(fm.product(fm.partial(inst["idx"], n), fm.toeplitz(inst["t"], n, n)))
        bs.append(I.fista_measurements(inst))
    B = fm.FistaBatch(ops)
    b = torch.from_numpy(np.concatenate(bs)).cuda()
    return B, b, bs


def _split(x, insts):
    out, off = [], 0
    for inst in insts:
        out.append(x[off:off + inst["n"]])
        off += inst["n"]
    return out


def _oracle(inst, b, iters=200, accel=True):
    A, lam, L = O.fista_problem(inst, b.astype(np.float64))
    x = O.fista(A, b.astype(np.float64), lam, L, iters=iters, accel=accel)
    return x, lam, L, O.objective(A, b.astype(np.float64), x, lam)


def _check(fm, insts, iters=200, accel=True, mode=0, tol=1e-4):
    B, b, bs = _batch(fm, insts)
    x, rep = B.solve(b, iters=iters, accel=accel, mode=mode, report=True)
    torch.cuda.synchronize()
    xs = _split(x.cpu().numpy(), insts)
    worst = 0.0
    for i, inst in enumerate(insts):
        xo, lam, L, obj = _oracle(inst, bs[i], iters=iters, accel=accel)
        err = np.linalg.norm(xs[i] - xo) / max(np.linalg.norm(xo), 1e-30)
        worst = max(worst, err)
        assert err <= tol, (i, inst["n"], err)
        assert abs(rep["lambda"][i].item() - lam) <= 1e-5 * lam
        assert abs(rep["L"][i].item() - L) <= 1e-4 * L
        assert abs(rep["objective"][i].item() - obj) <= 1e-4 * abs(obj)
        assert rep["status"][i].item() == 0
    return worst, x


def test_fista_mixed_sizes(fm):
    insts = [I.fista_instance(j, log2n_range=(8, 12)) for j in range(24)]
    _check(fm, insts)


def test_fista_workload_sizes_sampled(fm):
    # instances of the 4096-instance workload (n in 2^10..2^14), a sample covering every size
    insts, seen = [], {}
    j = 0
    while len(insts) < 12:
        inst = I.fista_instance(j)
        if seen.get(inst["n"], 0) < 3:
            insts.append(inst)
            seen[inst["n"]] = seen.get(inst["n"], 0) + 1
        j += 1
    _check(fm, insts)


def test_ista_mode(fm):
    insts = [I.fista_instance(j, log2n_range=(9, 11)) for j in range(6)]
    _check(fm, insts, iters=50, accel=False)


def test_per_instance_launch_mode_matches(fm):
    insts = [I.fista_instance(j, log2n_range=(8, 11)) for j in range(10)]
    B, b, _ = _batch(fm, insts)
    x0 = B.solve(b, mode=0)
    x1 = B.solve(b, mode=1)
    torch.cuda.synchronize()
    d = (x0 - x1).norm() / x0.norm()
    assert d.item() <= 1e-5


def _sized(log2n, count, start):
    """`count` workload instances of one size n = 2^log2n (seed 3, instance streams from `start`)."""
    return [I.fista_instance(start + j, log2n_range=(log2n, log2n)) for j in range(count)]


def test_fista_full_work_list_groups(fm):
    # a work-list group packs 2^14 / n equal-size instances into one tile: 17 instances of
    # n = 2^10 fill one group of 16 and start a second, 5 of n = 2^12 fill one group of 4 and
    # start a second; every instance must still match its own FP64 solve (the timed batch of
    # 4096 instances runs full groups only, apart from one partial group per size)
    insts = _sized(10, 17, 0) + _sized(12, 5, 100)
    _check(fm, insts)


def test_repeat_solves_bit_identical(fm):
    # the per-instance sums are taken in a fixed order, so a solve is reproducible bit for bit
    insts = _sized(10, 17, 0) + _sized(9, 3, 50)
    B, b, _ = _batch(fm, insts)
    x0 = B.solve(b).clone()
    x1 = B.solve(b)
    torch.cuda.synchronize()
    assert torch.equal(x0, x1)


@pytest.mark.parametrize("accel", [True, False])
def test_warm_resume_bit_identical(fm, accel):
    # K1 steps, then K2 steps resumed from (x_K1, y_K1+1, L, lambda), give the bits of K1 + K2
    # steps in one run (the resume state of the oracle's fista(..., state=...))
    insts = _sized(10, 5, 7) + _sized(12, 2, 200)
    B, b, _ = _batch(fm, insts)
    n = B.total_cols
    x_full, y_full = torch.empty(n, device="cuda"), torch.empty(n, device="cuda")
    x_full, rep_full = B.solve(b, x=x_full, y=y_full, iters=200, accel=accel, report=True)
    x, y = torch.empty(n, device="cuda"), torch.empty(n, device="cuda")
    x, rep = B.solve(b, x=x, y=y, iters=70, accel=accel, report=True)
    x, rep = B.solve(b, x=x, y=y, iters=130, accel=accel, report=rep, resume_from=70)
    torch.cuda.synchronize()
    assert torch.equal(x, x_full) and torch.equal(y, y_full)
    assert torch.equal(rep["objective"], rep_full["objective"])
    assert torch.equal(rep["L"], rep_full["L"]) and torch.equal(rep["lambda"], rep_full["lambda"])


def test_fista_per_instance_buffers(fm):
    # fm_fista: instances given as operators with their own b and x buffers
    insts = _sized(10, 3, 11) + _sized(11, 2, 300) + _sized(13, 1, 400)
    ops, bs = [], []
    for inst in insts:
        n = inst["n"]
        ops.append(fm.product(fm.partial(inst["idx"], n), fm.toeplitz(inst["t"], n, n)))
        bs.append(torch.from_numpy(I.fista_measurements(inst)).cuda())
    xs, rep = fm.fista(ops, bs, report=True)
    torch.cuda.synchronize()
    B = fm.FistaBatch(ops)
    xp = B.solve(torch.cat(bs))
    torch.cuda.synchronize()
    off = 0
    for i, inst in enumerate(insts):
        n = inst["n"]
        assert torch.equal(xs[i], xp[off:off + n])          # same kernel, same arithmetic
        off += n
        xo, lam, L, obj = _oracle(inst, bs[i].cpu().numpy())
        err = np.linalg.norm(xs[i].cpu().numpy() - xo) / np.linalg.norm(xo)
        assert err <= 1e-4, (i, err)
        assert rep["status"][i].item() == 0


def test_fista_rejects_bad_resume_and_alignment(fm):
    insts = _sized(9, 2, 0)
    B, b, _ = _batch(fm, insts)
    x = torch.zeros(B.total_cols, device="cuda")
    with pytest.raises(ValueError):
        B.solve(b, x=x, resume_from=3)                       # no y, no report
    from paper_1710_09578_gb300 import _lib
    params = _lib.fm_fista_params(10, 20, 0.01, 1.05, 1, 0, 1, 3)
    with pytest.raises(fm.FmError) as e:                      # warm start without L and lambda
        _lib.fm_fista_batch(B._b, b.data_ptr(), x.data_ptr(), x.data_ptr(), params, None)
    assert e.value.status == 1
    params = _lib.fm_fista_params(10, 20, 0.01, 1.05, 1, 0, 0, 0)
    with pytest.raises(fm.FmError) as e:                      # x not 8-byte aligned
        _lib.fm_fista_batch(B._b, b.data_ptr(), x.data_ptr() + 4, None, params, None)
    assert e.value.status == 1


def test_work_list_orders_and_tuning(fm):
    # both work-list orders solve every instance to the oracle's answer, bit for bit alike, and
    # the tuner times both and keeps one
    insts = _sized(10, 17, 0) + _sized(12, 5, 100) + _sized(9, 4, 60)
    B, b, bs = _batch(fm, insts)
    B.set_order(0)
    x0 = B.solve(b).clone()
    B.set_order(1)
    x1, rep = B.solve(b, report=True)
    torch.cuda.synchronize()
    assert torch.equal(x0, x1)
    xs = _split(x1.cpu().numpy(), insts)
    for i in (0, 16, 17, 21, 22):
        xo = _oracle(insts[i], bs[i])[0]
        assert np.linalg.norm(xs[i] - xo) / np.linalg.norm(xo) <= 1e-4
    r = B.tune(b)
    assert r["order"] in (0, 1) and all(t > 0 for t in r["ms"])
    with pytest.raises(fm.FmError):
        B.set_order(2)


def test_batch_rejects_other_operators(fm):
    with pytest.raises(fm.FmError):
        fm.FistaBatch([fm.fourier(256)])
    t = np.random.default_rng(0).standard_normal(2 * 100 - 1)
    with pytest.raises(fm.FmError):   # n not a power of two
        fm.FistaBatch([fm.product(fm.partial(np.arange(50, dtype=np.int32), 100), fm.toeplitz(t, 100, 100))])
