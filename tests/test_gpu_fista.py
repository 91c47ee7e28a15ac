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


def test_warm_resume_is_not_needed_for_repeat(fm):
    # two solves of the same batch give the same answer (state is rebuilt from scratch)
    insts = [I.fista_instance(j, log2n_range=(8, 10)) for j in range(5)]
    B, b, _ = _batch(fm, insts)
    x0 = B.solve(b).clone()
    x1 = B.solve(b)
    torch.cuda.synchronize()
    assert (x0 - x1).norm().item() <= 1e-6 * x0.norm().item()


def test_batch_rejects_other_operators(fm):
    with pytest.raises(fm.FmError):
        fm.FistaBatch([fm.fourier(256)])
    t = np.random.default_rng(0).standard_normal(2 * 100 - 1)
    with pytest.raises(fm.FmError):   # n not a power of two
        fm.FistaBatch([fm.product(fm.partial(np.arange(50, dtype=np.int32), 100), fm.toeplitz(t, 100, 100))])
