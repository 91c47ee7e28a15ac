"""Throughput of the structured-operator hot path on GB300 (one JSON line on stdout).

Step = forward + adjoint of the composed operator Kron(Hadamard 2^8, Circulant 2^10,
Fourier 2^6) on 4 complex64 columns of length N = 2^24 (512 MiB in, 512 MiB out per
apply; the largest single-GPU workload of the metric).  ``value`` is whole-job GB/s of
algorithmic bytes (read X + write Y per apply) with inputs resident in HBM; each buffer is
four times the L2, so consecutive steps read cold data without a flush.  ``e2e`` is the
same metric through the public API with pinned HOST buffers: H2D of X, forward, adjoint,
D2H of the result, pipelined over three streams so that the copies in and out of
neighbouring steps overlap each other and the compute.

``roofline`` is the dominant kernel of the step: its algorithmic bytes per launch over its
device time, measured with the library's launch tracing (CUDA events around every launch)
on the same steps after the timed region.  Every result carries its relative L2 error
against the FP64 oracle (sampled columns or instances where the oracle cannot run it all).

The other hot-path rows -- Hadamard 2^16 x 256 (FP32, int8, BF16, split BF16), the
compressed-sensing operator P Diag(d) C at 2^18 x 64, a plain 2^18 Fourier transform, the
complex128 circulant 4096 x 16 and batched FISTA (4096 instances) -- are under ``"rows"``,
with cuFFT (torch.fft) compositions of the same maps timed beside them as reference points.

``--impl reference`` times the FP64 CPU oracle on the same metric (bounded sample).
Multi-GPU: replicas only -- each rank runs its own block, no collective on the data path.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import fm_inputs as I  # noqa: E402

KRON_N = 1 << 24
KRON_K = 4
APPLY_BYTES = 2 * KRON_N * KRON_K * 8      # read X + write Y, complex64
STEP_BYTES = 2 * APPLY_BYTES               # forward + adjoint
METRIC = "fwd+adjoint apply GB/s vs HBM peak; batched FISTA solves/s at 1e-4 rel err"
WORKLOAD = "Kron(Hadamard 2^8, Circulant 2^10, Fourier 2^6), N = 2^24, 4 complex64 columns, forward + adjoint"
HAD_LOG2N, HAD_K = 16, 256
HAD_N = 1 << HAD_LOG2N
HAD_APPLY_BYTES = 2 * HAD_N * HAD_K * 4
# DRAM bytes (read + write) per launch from one ncu capture of the kernel as it is now
# (dram__bytes_read.sum + dram__bytes_write.sum); None where no current capture exists.
NCU_TRAFFIC = {
    "fwht_long_kernel": 67134464 + 22094080,
    # captured on one column of the Kron workload, scaled x4 to a 4-column launch
    "fft2_kernel<f32,L=2^10,strided,conv>": 4 * (134313472 + 91964160),
    "fft2_kernel<f32,L=2^10,strided,conv,radix=32>": 4 * (134312448 + 92168960),
    "kron_hfc_kernel<8,6,cluster=2>": 4 * (134261760 + 85114112),
}
FISTA_INSTANCES = 4096
FISTA_ITERS = 200


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# FP32 peak derived from unit counts (no measured figure exists): 152 SMs x 128 FP32 lanes
# x 2 flop per FMA x 2.07 GHz.
FP32_PEAK_DERIVED_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int, interval_ms: int = 20):
        self.index = index
        self.interval_ms = interval_ms
        self.proc = None
        # raw samples: FM_CLOCKS_DIR if set (to keep them), else the system temporary directory
        self.path = os.path.join(os.environ.get("FM_CLOCKS_DIR", tempfile.gettempdir()), f"fm_clocks_rank{index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", str(self.interval_ms)],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            # the first sample takes a moment: wait for it so that the timed region is covered
            t0 = time.time()
            while time.time() - t0 < 5.0 and os.path.getsize(self.path) == 0:
                time.sleep(0.01)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def job_throughput(t_local: float, units_local: float, pg=None, device=None):
    """Whole-job throughput of independent replicas: units of all ranks / the slowest rank's time.

    Every rank passes its own timed seconds and processed units; with a process group the
    time is max-reduced and the units sum-reduced (replicas exchange nothing else).
    """
    if pg is None:
        return units_local / t_local, t_local
    import torch
    tt = torch.tensor([t_local, units_local], dtype=torch.float64, device=device)
    tmax = tt[:1].clone()
    pg.all_reduce(tmax, op=pg.ReduceOp.MAX)
    units = tt[1:].clone()
    pg.all_reduce(units, op=pg.ReduceOp.SUM)
    return units.item() / tmax.item(), tmax.item()


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def rel_err(got, want) -> float:
    """Largest per-column relative L2 error (columns along the last axis)."""
    got = np.asarray(got, dtype=np.complex128).reshape(np.shape(want))
    want = np.asarray(want, dtype=np.complex128)
    num = np.linalg.norm(got - want, axis=-1)
    den = np.maximum(np.linalg.norm(want, axis=-1), 1e-300)
    return float(np.max(num / den))


# ------------------------------------------------------------------ oracle tasks (CPU, FP64)
# Module-level functions so that a spawn process pool can run them on the host cores.
def _kron_oracle():
    import oracle as O
    return O.Kron(O.Hadamard(256), O.Circulant(I.kron_generator()), O.Fourier(64))


def oracle_kron_apply(col: np.ndarray, adjoint: bool) -> np.ndarray:
    """One column of the headline operator, forward or adjoint, in FP64."""
    return _kron_oracle().apply(col.astype(np.complex128)[:, None], adjoint=adjoint)[:, 0]


def oracle_kron_timed(col: np.ndarray, adjoint: bool) -> float:
    """Forward or adjoint of one column of the headline operator; returns seconds taken."""
    K = _kron_oracle()
    t0 = time.perf_counter()
    K.apply(col.astype(np.complex128)[:, None], adjoint=adjoint)
    return time.perf_counter() - t0


def oracle_fista(j: int):
    """Instance j of the FISTA workload solved by the FP64 oracle (x, seconds)."""
    import oracle as O
    it = I.fista_instance(j)
    bb = I.fista_measurements(it).astype(np.float64)
    t0 = time.perf_counter()
    A, lam, L = O.fista_problem(it, bb)
    x = O.fista(A, bb, lam, L, iters=FISTA_ITERS)
    return x, time.perf_counter() - t0


def reference_arm(args, world, rank):
    """FP64 CPU oracle on the headline metric: each step applies the operator to one column
    of the workload (forward on even steps, adjoint on odd ones), a bounded sample."""
    if rank != 0:
        return
    _, X, Y = I.kron_large()
    xs = [X[0].copy(), Y[0].copy()]
    del X, Y
    for i in range(args.warmup):
        oracle_kron_apply(xs[i % 2], i % 2 == 1)
    t0 = time.perf_counter()
    for i in range(args.steps):
        oracle_kron_apply(xs[i % 2], i % 2 == 1)
    dt = time.perf_counter() - t0
    sample_bytes = 2 * KRON_N * 8                  # one column read + written
    gbs = sample_bytes * args.steps / dt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "n": KRON_N, "columns": KRON_K,
                                            "bytes_per_step": STEP_BYTES, "parallelism": "oracle on one host core"},
            "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": 1, "kind": "oracle",
                             "sample": "one of 4 columns per step (forward on even steps, adjoint on odd), "
                                       "FP64 numpy mode products"},
            "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(pool, cores, Xk):
    """The headline oracle on the host cores: one core, then every task of the sample at once."""
    t1 = oracle_kron_timed(Xk[0], False) + oracle_kron_timed(Xk[0], True)
    one = {"value": 2 * 2 * KRON_N * 8 / t1 / 1e9, "cores": 1,
           "sample": f"column 0, forward + adjoint, {t1:.1f} s"}
    tasks = [(Xk[j], adj) for j in range(KRON_K) for adj in (False, True)]
    used = min(len(tasks), cores)
    t0 = time.perf_counter()
    pool.starmap(oracle_kron_timed, tasks)
    tall = time.perf_counter() - t0
    allc = {"value": len(tasks) * 2 * KRON_N * 8 / tall / 1e9, "cores": used,
            "sample": f"all 4 columns, forward + adjoint, {len(tasks)} column applies in {tall:.1f} s"}
    return {"value": one["value"], "unit": "GB/s", "cores": 1, "kind": "oracle", "sample": one["sample"],
            "all_cores": {**allc, "unit": "GB/s", "host_cpu_count": cores}}


# ------------------------------------------------------------------ GPU helpers
def timed_loop(fn, steps, flush, stream, torch):
    """Per-step CUDA-event times; L2 flushed (outside the events) before each step."""
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for i in range(steps):
        flush.zero_()
        starts[i].record(stream)
        fn()
        ends[i].record(stream)
    torch.cuda.synchronize()
    return [s.elapsed_time(e) for s, e in zip(starts, ends)]


def _gbs_loop(fn, nbytes, steps, flush, stream, torch):
    for _ in range(3):
        fn()
    torch.cuda.synchronize()
    ts = timed_loop(fn, steps, flush, stream, torch)
    return nbytes * steps / (sum(ts) / 1e3) / 1e9


def _b2b_rotating(fns, nbytes, reps, stream, torch):
    """GB/s of algorithmic bytes for back-to-back calls cycling through buffer sets that
    together exceed L2 (no flush, no host gap)."""
    for f in fns:
        f()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(reps):
        fns[i % len(fns)]()
    e1.record(stream)
    torch.cuda.synchronize()
    return nbytes * reps / (e0.elapsed_time(e1) / 1e3) / 1e9


def trace_kernels(fm, fn, reps, torch):
    """Device time per kernel label over `reps` calls of fn, from the library's launch tracing."""
    from paper_1710_09578_gb300 import _lib
    fn()
    torch.cuda.synchronize()
    _lib.fm_trace_begin(4096)
    for _ in range(reps):
        fn()
    recs = _lib.fm_trace_end()
    per = {}
    for name, ms in recs:
        e = per.setdefault(name, {"launches": 0, "ms": 0.0})
        e["launches"] += 1
        e["ms"] += ms
    total = sum(e["ms"] for e in per.values()) or 1.0
    for e in per.values():
        e["mean_us"] = e["ms"] / e["launches"] * 1e3
        e["share"] = e["ms"] / total
    return per


def roofline_of(per, bytes_per_launch, peak, peak_src, traffic=None):
    """Roofline entry of the kernel with the largest total device time."""
    name = max(per, key=lambda k: per[k]["ms"])
    mean_s = per[name]["mean_us"] / 1e6
    achieved = bytes_per_launch / mean_s / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "kernel": name, "peak_source": peak_src,
            "algorithmic_bytes_per_launch": bytes_per_launch, "mean_launch_us": per[name]["mean_us"],
            "share_of_step": per[name]["share"]}


def _fwht_dim(T, dim, n, torch):
    """Walsh-Hadamard transform along `dim` (length n) by log2 n butterfly stages (torch ops)."""
    h = 1
    while h < n:
        sh = list(T.shape)
        T = T.reshape(sh[:dim] + [n // (2 * h), 2, h] + sh[dim + 1:])
        a, b = T.select(dim + 1, 0), T.select(dim + 1, 1)
        T = torch.stack((a + b, a - b), dim=dim + 1).reshape(sh)
        h *= 2
    return T


# ------------------------------------------------------------------ main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--rows", type=int, default=1, help="also measure the other hot-path rows")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile", default=None, choices=["hadamard", "hadamard_int8", "hadamard_bf16", "cs", "kron",
                                                        "kron1", "circulant_c128", "fista", "fourier"],
                    help="run one workload a few times and exit (for ncu captures)")
    args = ap.parse_args()
    world, rank, local = dist_init()
    if args.impl == "reference":
        reference_arm(args, world, rank)
        return

    cores = os.cpu_count() or 1
    pool = None
    if rank == 0 and world == 1 and not args.profile and not args.no_cpu_baseline:
        # the oracle's process pool, started (spawn) before the first GPU call
        pool = mp.get_context("spawn").Pool(min(cores, 2 * KRON_K))

    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1710_09578_gb300 as fm

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.profile:
        profile_run(fm, torch, dev, args.profile, args.steps)
        return
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    stream = torch.cuda.current_stream()
    props = torch.cuda.get_device_properties(dev)
    l2 = getattr(props, "L2_cache_size", 126 * 1024 * 1024)
    peak, peak_src = _peaks()

    # ---- headline: Kron(H_256, C_1024, F_64) forward + adjoint on 4 columns of 2^24
    ck, Xk, Yk = I.kron_large()
    Xh = torch.from_numpy(Xk).pin_memory()
    del Yk
    K = fm.kron(fm.hadamard(8), fm.circulant(ck), fm.fourier(64))
    X = Xh.to(dev)
    Y = torch.empty_like(X)
    Z = torch.empty_like(X)
    K.reserve(KRON_K, torch.complex64)
    # set-up: the execution plan of the operator's transforms for this column count
    kron_plan = [[e["L"], e["kind"], e["value"]] for e in K.calibrate(KRON_K, torch.complex64)]

    def step():
        K.forward(X, out=Y)
        K.backward(Y, out=Z)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    l0 = fm.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
    launches = fm.launch_count() - l0
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    t_local = e0.elapsed_time(e1) / 1e3
    rate, t_total = job_throughput(t_local, float(STEP_BYTES) * args.steps, pg, dev)
    value = rate / 1e9

    # ---- roofline of the dominant kernel: per-launch device time of the same steps, traced
    per = trace_kernels(fm, step, 5, torch)
    # every pass of the two-pass plan reads and writes the whole block once: its algorithmic
    # bytes per launch are those of one apply
    roof = roofline_of(per, APPLY_BYTES, peak, peak_src)
    roof["traffic"] = NCU_TRAFFIC.get(roof["kernel"])
    roof["kernels"] = per
    roof["apply_level"] = {"achieved": value, "frac": value / peak,
                           "note": "compulsory bytes of the whole apply over the step time (two passes per apply)"}

    # ---- accuracy of this step's results: column 0, forward and adjoint, against FP64
    y0 = Y[0].cpu().numpy()
    z0 = Z[0].cpu().numpy()
    acc = {}
    if rank == 0:
        if pool is not None:
            fy, fz = pool.starmap(oracle_kron_apply, [(Xk[0], False), (y0, True)])
        else:
            fy, fz = oracle_kron_apply(Xk[0], False), oracle_kron_apply(y0, True)
        acc = {"forward": rel_err(y0, fy), "adjoint": rel_err(z0, fz),
               "tolerance": 1e-5 * 24, "sample": "column 0 of 4; the adjoint's input is the GPU forward output"}
    cpu_line = cpu_baseline(pool, cores, Xk) if (rank == 0 and world == 1 and pool is not None) else None
    del Xk

    # ---- end to end through the public API with host buffers: every step copies its input
    # from pinned host memory, runs forward + adjoint and copies the result back.  Three
    # streams form a pipeline (host-to-device copy of step i + 1, forward + adjoint of step i,
    # device-to-host copy of step i - 1), with two input and two output buffers and events
    # between the stages, so the host link carries both directions at once while the GPU
    # computes; one operator on the compute stream.
    NB = 2
    Xe = [X, torch.empty_like(X)]
    Ze = [Z, torch.empty_like(X)]
    out_h = [torch.empty_like(Xh).pin_memory() for _ in range(NB)]
    ev = {name: [torch.cuda.Event() for _ in range(NB)] for name in ("loaded", "read", "done", "drained")}
    e2e_steps = max(6, min(30, args.steps // 10))

    def e2e_step(i, streams):
        s_in, s_cmp, s_out = streams
        k = i % NB
        with torch.cuda.stream(s_in):
            s_in.wait_event(ev["read"][k])          # the forward of step i - 2 has read Xe[k]
            Xe[k].copy_(Xh, non_blocking=True)
            ev["loaded"][k].record(s_in)
        with torch.cuda.stream(s_cmp):
            s_cmp.wait_event(ev["loaded"][k])
            s_cmp.wait_event(ev["drained"][k])      # step i - 2's result has left Ze[k]
            K.forward(Xe[k], out=Y)
            ev["read"][k].record(s_cmp)
            K.backward(Y, out=Ze[k])
            ev["done"][k].record(s_cmp)
        with torch.cuda.stream(s_out):
            s_out.wait_event(ev["done"][k])
            out_h[k].copy_(Ze[k], non_blocking=True)
            ev["drained"][k].record(s_out)

    streams = tuple(torch.cuda.Stream(dev) for _ in range(3))
    for i in range(2 * NB):
        e2e_step(i, streams)
    torch.cuda.synchronize()
    # three timed runs of e2e_steps steps each; the value is their median (all three reported:
    # on GB300 a run now and then moves the two directions one after the other, ~400 against
    # 662 GB/s)
    e2e_runs = []
    for _ in range(3):
        t0 = time.perf_counter()
        for i in range(e2e_steps):
            e2e_step(i, streams)
        torch.cuda.synchronize()
        e2e_runs.append(world * STEP_BYTES * e2e_steps / (time.perf_counter() - t0) / 1e9)
    e2e_val = sorted(e2e_runs)[1]
    e2e_ok = all(bool(torch.equal(out_h[0], o)) for o in out_h[1:])
    del Xe, Ze, out_h

    # ---- cuFFT reference point: the same map as mode-wise torch.fft and a torch FWHT
    cufft = {}
    if rank == 0:
        chat = torch.fft.fft(torch.from_numpy(ck).to(dev)).to(torch.complex64).view(1, 1, 1024, 1)

        def torch_kron(T, adj):
            T = T.view(KRON_K, 256, 1024, 64)
            T = torch.fft.ifft(T, dim=3) * 64 if adj else torch.fft.fft(T, dim=3)
            T = torch.fft.ifft((chat.conj() if adj else chat) * torch.fft.fft(T, dim=2), dim=2)
            return _fwht_dim(T, 1, 256, torch).reshape(KRON_K, KRON_N)

        Yt = torch_kron(X, False)
        Zt = torch_kron(Yt, True)
        flush = torch.empty(2 * l2, dtype=torch.uint8, device=dev)
        cufft = {"GB/s": _gbs_loop(lambda: torch_kron(torch_kron(X, False), True), STEP_BYTES, 5, flush, stream,
                                   torch),
                 "what": "torch.fft along modes 2 and 1 (spectrum product), 8 torch butterfly stages along mode 0",
                 "max_rel_diff_vs_ours": max(rel_err(Yt.cpu().numpy(), Y.cpu().numpy()),
                                             rel_err(Zt.cpu().numpy(), Z.cpu().numpy()))}
        del Yt, Zt, flush
    del X, Y, Z, K
    torch.cuda.empty_cache()

    rows = {}
    if args.rows and rank == 0:
        rows = measure_rows(fm, torch, dev, stream, l2, peak, peak_src, pool)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_total / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": KRON_N, "columns": KRON_K, "bytes_per_step": STEP_BYTES,
                       "l2": "inputs larger than L2: each 512 MiB buffer is 4x the L2, steps back to back",
                       "streams": "one stream (the operator's workspace is per operator)",
                       "plan": {"calibrated": kron_plan,
                                "format": "[L, kind (0 split, 1 tile shape, 2 radix schedule, 3 fused Kron pass), chosen value]"},
                       "parallelism": f"replicas x{world}"},
            "clocks": clk.summary(),
            "e2e": {"value": e2e_val, "unit": "GB/s", "h2d_bytes_per_step": KRON_N * KRON_K * 8,
                    "d2h_bytes_per_step": KRON_N * KRON_K * 8,
                    "pipeline": "3 streams: copy in, forward + adjoint, copy out; 2 buffers each side",
                    "steps": e2e_steps, "runs_GB/s": e2e_runs, "value_is": "median of the three runs",
                    "results_agree": e2e_ok},
            "gpu_launches": int(launches),
            "roofline": roof,
            "rel_err_vs_fp64": acc,
            "cufft_reference": cufft,
            "rows": rows,
        }
        if cpu_line is not None:
            line["cpu_baseline"] = cpu_line
        print(json.dumps(line), flush=True)
    if pool is not None:
        pool.close()
        pool.join()
    if pg:
        pg.destroy_process_group()


# ------------------------------------------------------------------ the other rows
def measure_rows(fm, torch, dev, stream, l2, peak, peak_src, pool):
    """GB/s (forward + adjoint unless stated), error against FP64 and reference points of the
    other hot-path rows."""
    import oracle as O
    rows = {}
    flush = torch.empty(2 * l2, dtype=torch.uint8, device=dev)
    xf, xi = I.hadamard_block()

    # Hadamard FP32: back to back over four rotating buffer sets (768 MiB) and with L2 flushed
    Xs = [torch.from_numpy(xf).to(dev) for _ in range(4)]
    Ys = [torch.empty_like(Xs[0]) for _ in range(4)]
    Zs = [torch.empty_like(Xs[0]) for _ in range(4)]
    A = fm.hadamard(HAD_LOG2N)
    fn = [lambda k=k: (A.forward(Xs[k], out=Ys[k]), A.backward(Ys[k], out=Zs[k])) for k in range(4)]
    rot = [0]

    def fwd_rotating():
        k = rot[0] = (rot[0] + 1) % 4
        A.forward(Xs[k], out=Ys[k])

    per = trace_kernels(fm, fwd_rotating, 50, torch)
    roof = roofline_of(per, HAD_APPLY_BYTES, peak, peak_src)
    roof["traffic"] = NCU_TRAFFIC.get(roof["kernel"])
    b2b_launch = _b2b_rotating([lambda k=k: A.forward(Xs[k], out=Ys[k]) for k in range(4)], HAD_APPLY_BYTES, 400,
                               stream, torch)
    roof["achieved_back_to_back"] = b2b_launch
    roof["frac_back_to_back"] = b2b_launch / peak
    H = O.Hadamard(HAD_N)
    cols = [0, 255]
    y = Ys[0][cols].cpu().numpy()
    rows["hadamard_2p16x256_fp32_fwd+adj"] = {
        "GB/s_back_to_back_rotating": _b2b_rotating(fn, 2 * HAD_APPLY_BYTES, 200, stream, torch),
        "GB/s": _gbs_loop(fn[0], 2 * HAD_APPLY_BYTES, 100, flush, stream, torch),
        "roofline": roof,
        "rel_err_vs_fp64": rel_err(y, H.apply(xf[cols].T.astype(np.float64)).T),
        "rel_err_sample": "columns 0 and 255 of the forward", "tolerance": 1e-5 * HAD_LOG2N}
    del Xs, Ys, Zs

    # int8 -> int32 Hadamard (exact)
    Xi = [torch.from_numpy(xi).to(dev) for _ in range(4)]
    Ai = fm.hadamard(HAD_LOG2N, fm.FM_HAD_INT8)
    Yi = [torch.empty((HAD_K, HAD_N), dtype=torch.int32, device=dev) for _ in range(4)]
    rows["hadamard_int8_fwd"] = {
        "GB/s": _gbs_loop(lambda: Ai.forward(Xi[0], out=Yi[0]), HAD_N * HAD_K * 5, 200, flush, stream, torch),
        "GB/s_back_to_back_rotating": _b2b_rotating(
            [lambda k=k: Ai.forward(Xi[k], out=Yi[k]) for k in range(4)], HAD_N * HAD_K * 5, 400, stream, torch),
        "max_abs_diff_vs_int64": int(np.max(np.abs(Yi[0][cols].cpu().numpy().astype(np.int64)
                                                   - H.apply(xi[cols].T.astype(np.int64)).T))),
        "sample": "columns 0 and 255"}
    del Xi, Yi
    # BF16 tensor-core Hadamard and its split hi + lo form (forward)
    Xf = [torch.from_numpy(xf).to(dev) for _ in range(4)]
    Yf = [torch.empty_like(Xf[0]) for _ in range(4)]
    want = H.apply(xf[cols].T.astype(np.float64)).T
    for name, mode, tol in (("hadamard_bf16_fwd", fm.FM_HAD_BF16, 2e-2), ("hadamard_bf16x2_fwd", fm.FM_HAD_BF16X2, 1e-5)):
        Ab = fm.hadamard(HAD_LOG2N, mode)
        g = _gbs_loop(lambda: Ab.forward(Xf[0], out=Yf[0]), HAD_APPLY_BYTES, 200, flush, stream, torch)
        rows[name] = {
            "GB/s": g, "frac_of_hbm": g / peak,
            "GB/s_back_to_back_rotating": _b2b_rotating(
                [lambda k=k: Ab.forward(Xf[k], out=Yf[k]) for k in range(4)], HAD_APPLY_BYTES, 400, stream, torch),
            "rel_err_vs_fp64": rel_err(Yf[0][cols].cpu().numpy(), want), "tolerance": tol}
    del Xf, Yf

    # compressed-sensing operator Phi = P Diag(d) C, N = 2^18, 64 complex64 columns
    c, d, idx, Xc, Yc, _ = I.cs_operator()
    n, m = len(c), len(idx)
    A = fm.product(fm.partial(idx, n), fm.diag(d), fm.circulant(c))
    Xg = torch.from_numpy(Xc).to(dev)
    Ygo = torch.empty((64, m), dtype=torch.complex64, device=dev)
    Zg = torch.empty((64, n), dtype=torch.complex64, device=dev)
    A.reserve(64, torch.complex64)
    tune = A.calibrate(64, torch.complex64)          # set-up: the two-pass split for 64 columns
    byts = 2 * (64 * n * 8 + 64 * m * 8 + n * 8 * 2 + m * 4)
    cs_fn = lambda: (A.forward(Xg, out=Ygo), A.backward(Ygo, out=Zg))  # noqa: E731
    g = _gbs_loop(cs_fn, byts, 50, flush, stream, torch)
    ref = O.Product(O.Partial(idx, n), O.Diag(d), O.Circulant(c))
    cs_cols = [0, 63]
    yo = Ygo[cs_cols].cpu().numpy()
    e_f = rel_err(yo, ref.apply(Xc[cs_cols].T.astype(np.complex128)).T)
    e_b = rel_err(Zg[cs_cols].cpu().numpy(), ref.apply(yo.T.astype(np.complex128), adjoint=True).T)
    # cuFFT composition of the same map
    chat = torch.fft.fft(torch.from_numpy(c).to(dev)).to(torch.complex64)
    dg = torch.from_numpy(d).to(dev)
    ig = torch.from_numpy(idx.astype(np.int64)).to(dev)

    def torch_cs():
        yy = (dg * torch.fft.ifft(chat * torch.fft.fft(Xg)))[:, ig]
        s = torch.zeros((64, n), dtype=torch.complex64, device=dev)
        s[:, ig] = yy
        return torch.fft.ifft(chat.conj() * torch.fft.fft(dg.conj() * s))

    rows["cs_PDC_2p18x64_fwd+adj"] = {
        "GB/s": g, "frac_of_hbm": g / peak, "algorithmic_bytes": byts,
        "calibrated_plan": [[e["L"], e["kind"], e["value"]] for e in tune],
        "kernels": trace_kernels(fm, cs_fn, 5, torch),
        "rel_err_vs_fp64": {"forward": e_f, "adjoint": e_b, "tolerance": 1e-5 * 18, "sample": "columns 0 and 63"},
        "cufft_reference_GB/s": _gbs_loop(torch_cs, byts, 20, flush, stream, torch),
        "cufft_reference": "P d ifft(c_hat fft(x)) and its adjoint in torch.fft / torch ops"}
    del Xg, Ygo, Zg, A

    # plain Fourier transform 2^18 on 64 columns, against torch.fft.fft
    F = fm.fourier(n)
    tuneF = F.calibrate(64, torch.complex64)
    Xg = torch.from_numpy(Xc).to(dev)
    Yg = torch.empty_like(Xg)
    fb = 2 * 64 * n * 8
    g = _gbs_loop(lambda: F.forward(Xg, out=Yg), fb, 50, flush, stream, torch)
    rows["fourier_2p18x64_fwd"] = {
        "GB/s": g, "frac_of_hbm": g / peak, "calibrated_plan": [[e["L"], e["kind"], e["value"]] for e in tuneF],
        "rel_err_vs_fp64": rel_err(Yg[cs_cols].cpu().numpy(), np.fft.fft(Xc[cs_cols].astype(np.complex128), axis=1)),
        "tolerance": 1e-5 * 18,
        "cufft_reference_GB/s": _gbs_loop(lambda: torch.fft.fft(Xg), fb, 50, flush, stream, torch)}
    del Xg, Yg, F

    # complex128 circulant N = 4096, 16 columns
    c0, X0, _ = I.circulant_tiny()
    C0 = fm.circulant(c0)
    X0g = torch.from_numpy(X0).to(dev)
    Y0 = torch.empty_like(X0g)
    Z0 = torch.empty_like(X0g)
    byts = 2 * (2 * X0.nbytes + 4096 * 16)
    fn0 = lambda: (C0.forward(X0g, out=Y0), C0.backward(Y0, out=Z0))  # noqa: E731
    eager = _gbs_loop(fn0, byts, 200, flush, stream, torch)
    # At this size a call costs more host time than GPU time: the same two calls captured once
    # in a CUDA graph and replayed give the GPU-side rate.
    Z_eager = Z0.clone()
    g0 = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g0):
        fn0()
    Z0.zero_()
    replay = _gbs_loop(g0.replay, byts, 200, flush, stream, torch)
    C0o = O.Circulant(c0)
    chat0 = torch.fft.fft(torch.from_numpy(c0).to(dev))
    tc = lambda: torch.fft.ifft(chat0.conj() * torch.fft.fft(torch.fft.ifft(chat0 * torch.fft.fft(X0g))))  # noqa: E731
    rows["circulant_c128_4096x16_fwd+adj"] = {
        "GB/s": replay, "graph": True, "GB/s_eager_calls": eager,
        "graph_matches_eager": bool(torch.equal(Z0, Z_eager)), "algorithmic_bytes": byts,
        "rel_err_vs_fp64": {"forward": rel_err(Y0.cpu().numpy(), C0o.apply(X0.T).T),
                            "adjoint": rel_err(Z0.cpu().numpy(), C0o.apply(Y0.cpu().numpy().T, adjoint=True).T),
                            "tolerance": 1e-12},
        "cufft_reference_GB/s": _gbs_loop(tc, byts, 200, flush, stream, torch)}
    del g0, X0g, Y0, Z0
    torch.cuda.empty_cache()
    rows["fista_4096"] = measure_fista(fm, torch, dev, stream, pool)
    return rows


def profile_run(fm, torch, dev, which, steps):
    """A few plain launches of one workload (warm-up included), for ncu captures."""
    if which.startswith("hadamard"):
        xf, xi = I.hadamard_block()
        mode = {"hadamard": fm.FM_HAD_FP32, "hadamard_int8": fm.FM_HAD_INT8, "hadamard_bf16": fm.FM_HAD_BF16X2}[which]
        X = torch.from_numpy(xi if mode == fm.FM_HAD_INT8 else xf).to(dev)
        A = fm.hadamard(HAD_LOG2N, mode)
        fn = lambda: A.forward(X)  # noqa: E731
    elif which == "cs":
        c, d, idx, X, _, _ = I.cs_operator()
        A = fm.product(fm.partial(idx, len(c)), fm.diag(d), fm.circulant(c))
        Xg = torch.from_numpy(X).to(dev)
        A.calibrate(Xg.shape[0], torch.complex64)   # as in the bench row
        fn = lambda: A.backward(A.forward(Xg))  # noqa: E731
    elif which == "fourier":
        _, _, _, X, _, _ = I.cs_operator()
        A = fm.fourier(X.shape[1])
        Xg = torch.from_numpy(X).to(dev)
        A.calibrate(Xg.shape[0], torch.complex64)
        fn = lambda: A.forward(Xg)  # noqa: E731
    elif which in ("kron", "kron1"):
        # kron1: column 0 only (the same kernels on a quarter of the tiles, for full captures)
        ck, Xk, _ = I.kron_large()
        if which == "kron1":
            Xk = Xk[:1].copy()
        A = fm.kron(fm.hadamard(8), fm.circulant(ck), fm.fourier(64))
        Xg = torch.from_numpy(Xk).to(dev)
        A.calibrate(Xg.shape[0], torch.complex64)   # as in the bench step
        fn = lambda: A.backward(A.forward(Xg))  # noqa: E731
    elif which == "circulant_c128":
        c0, X0, _ = I.circulant_tiny()
        A = fm.circulant(c0)
        Xg = torch.from_numpy(X0).to(dev)
        fn = lambda: A.backward(A.forward(Xg))  # noqa: E731
    else:
        insts = [I.fista_instance(j) for j in range(512)]
        ops = [fm.product(fm.partial(it["idx"], it["n"]), fm.toeplitz(it["t"], it["n"], it["n"])) for it in insts]
        b = torch.from_numpy(np.concatenate([I.fista_measurements(it) for it in insts])).to(dev)
        B = fm.FistaBatch(ops)
        fn = lambda: B.solve(b)  # noqa: E731
    # the profiled runs sit in an NVTX range (ncu --nvtx --nvtx-include "fm_profile/")
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("fm_profile")
    for _ in range(max(1, steps)):
        fn()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    print(json.dumps({"profile": which, "runs": max(1, steps), "launches": fm.launch_count()}))


def fista_operator_loop(A, b, torch, iters=FISTA_ITERS, power_iters=20):
    """One instance solved through the operator API only, FP32, one call per step: the plain
    form of the same protocol (lambda = 0.01 ||A^T b||_inf, 20 power iterations for L capped by
    nothing, 200 FISTA steps), each product a fm_forward / fm_backward launch and the update in
    torch element-wise ops on the whole GPU."""
    lam = 0.01 * A.backward(b).abs().max()
    v = torch.full((A.cols,), A.cols ** -0.5, dtype=torch.float32, device=b.device)
    for _ in range(power_iters):
        w = A.backward(A.forward(v))
        v = w / w.norm()
    L = 1.05 * A.forward(v).norm() ** 2
    x = torch.zeros_like(v)
    y = torch.zeros_like(v)
    t = 1.0
    for _ in range(iters):
        z = y - A.backward(A.forward(y) - b) / L
        xn = torch.sign(z) * torch.clamp(z.abs() - lam / L, min=0)
        tn = 0.5 * (1 + (1 + 4 * t * t) ** 0.5)
        y = xn + ((t - 1) / tn) * (xn - x)
        x, t = xn, tn
    return x


def measure_fista(fm, torch, dev, stream, pool):
    """Batched FISTA: 4096 instances, n ~ U{2^10..2^14}, 200 steps, one persistent launch
    replayed from a CUDA graph; accuracy of the timed batch on sampled instances; against the
    same protocol solved one instance at a time through the operator API, and against the
    same kernel launched once per instance."""
    insts = [I.fista_instance(j) for j in range(FISTA_INSTANCES)]
    ops = [fm.product(fm.partial(it["idx"], it["n"]), fm.toeplitz(it["t"], it["n"], it["n"])) for it in insts]
    bh = [I.fista_measurements(it) for it in insts]
    b = torch.from_numpy(np.concatenate(bh)).to(dev)
    B = fm.FistaBatch(ops)
    x = torch.empty(B.total_cols, dtype=torch.float32, device=dev)
    order = B.tune(b, x=x)                # set-up: the work-list order (also the warm-up)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        B.solve(b, x=x)
    g.replay()
    torch.cuda.synchronize()
    reps = 3
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        g.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    t_batch = e0.elapsed_time(e1) / 1e3 / reps
    xh = x.cpu().numpy()
    offs = np.concatenate([[0], np.cumsum([it["n"] for it in insts])])
    # accuracy of the timed batch: the first two instances of each size (the batch sorts
    # instances by size, so these sit in the first, full work-list group of their size)
    sample = []
    for ln in range(10, 15):
        sample += [j for j, it in enumerate(insts) if it["n"] == 1 << ln][:2]
    t0 = time.perf_counter()
    if pool is not None:
        res = pool.map(oracle_fista, sample)
    else:
        res = [oracle_fista(j) for j in sample]
    t_wall = time.perf_counter() - t0
    errs = [float(np.linalg.norm(xh[offs[j]:offs[j + 1]] - xo) / np.linalg.norm(xo)) for j, (xo, _) in zip(sample, res)]
    cpu_1core = len(sample) / sum(t for _, t in res)
    # plain FP32 form through the operator API, one instance at a time (a sample of the batch)
    ns = 16
    bs = [torch.from_numpy(bh[j]).to(dev) for j in range(ns)]
    fista_operator_loop(ops[0], bs[0], torch, iters=5, power_iters=2)
    torch.cuda.synchronize()
    e0.record(stream)
    xs_api = [fista_operator_loop(ops[j], bs[j], torch) for j in range(ns)]
    e1.record(stream)
    torch.cuda.synchronize()
    t_api = e0.elapsed_time(e1) / 1e3
    err_api = max(float(np.linalg.norm(xs_api[i].cpu().numpy() - xh[offs[i]:offs[i + 1]]) /
                        np.linalg.norm(xh[offs[i]:offs[i + 1]])) for i in range(ns))
    # the same kernel launched once per instance (one CTA per launch), on a sample
    ss = 256
    Bs = fm.FistaBatch(ops[:ss])
    bsub = b[:Bs.total_rows]
    Bs.solve(bsub, mode=1)
    torch.cuda.synchronize()
    e0.record(stream)
    Bs.solve(bsub, mode=1)
    e1.record(stream)
    torch.cuda.synchronize()
    t_single = e0.elapsed_time(e1) / 1e3
    flops = sum(FISTA_ITERS * 20.0 * it["n"] * np.log2(it["n"]) for it in insts)
    solves = FISTA_INSTANCES / t_batch
    return {"solves/s": solves, "ms_per_batch": t_batch * 1e3, "instances": FISTA_INSTANCES,
            "iterations": FISTA_ITERS, "graph": True,
            "work_list_order": {"chosen": ["largest first", "smallest first"][order["order"]],
                                "ms_largest_first": order["ms"][0], "ms_smallest_first": order["ms"][1]},
            "max_rel_err_vs_fp64": max(errs), "rel_err_sample": f"{len(sample)} instances, 2 per size, full groups",
            "tolerance": 1e-4,
            "operator_api_solves/s": ns / t_api, "operator_api_sample": ns,
            "operator_api_max_rel_diff": err_api,
            "speedup_vs_operator_api": solves / (ns / t_api),
            "per_instance_launch_solves/s": ss / t_single, "per_instance_launch_sample": ss,
            "speedup_vs_per_instance_launch": solves / (ss / t_single),
            "roofline": {"bound": "alu", "achieved": flops / t_batch / 1e12, "unit": "TFLOP/s",
                         "peak": FP32_PEAK_DERIVED_TFLOPS, "frac": flops / t_batch / 1e12 / FP32_PEAK_DERIVED_TFLOPS,
                         "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz",
                         "nominal_flops": flops, "flops_model": "20 n log2 n per instance and step (4 FFTs)"},
            "cpu_oracle_solves/s": cpu_1core, "cpu_oracle_sample": f"{len(sample)} instances, FP64 numpy, one core each",
            "cpu_oracle_all_cores_solves/s": len(sample) / t_wall,
            "cpu_oracle_all_cores": f"the same {len(sample)} instances over {1 if pool is None else pool._processes} "
                                    f"processes, {t_wall:.1f} s wall"}


if __name__ == "__main__":
    main()
