"""Benchmark of the randomized Tucker hot path on one GB300 (or N replicas).

One step = the whole path on the 512^3 FP32 smooth-field workload:
  rHKron-re (sketch, thin QR, core, FP64 truncation, relative error)
  + rSTHKron (per-mode sketch / QR / TTM, truncation, relative error)
  + the loss gradient at the rHKron-re result (dG, dU, dX).
Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_FULL = 512
RANKS = (32, 32, 32)
P_OVER = 8
SEED = 0
WORKLOAD = ("bumps512_f32: 512^3 FP32 field, sum of 200 anisotropic Gaussian bumps + 1e-4 relative noise; "
            "rHKron-re and rSTHKron at r=(32,32,32), p=8 (s=(6,7,7); S rows {5,8}); loss gradient at the rHKron-re result; "
            "Gaussian sketch factors drawn on the device (Philox4x32-10) inside every step")
METRIC = "rHKron-re + rSTHKron (+ loss gradient) wall time per step, 512^3 FP32, r=32, p=8"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            pk = json.load(fh)
        return float(pk["hbm_gbs"]), float(pk["bf16_tflops"]), "measured"
    except Exception:
        return 6800.0, 1900.0, "fallback"


KERNEL_NAMES = {
    "xpass_tc": "ttm_tf32x3_kernel (tcgen05 3xTF32 TTM streaming X: sketch/core passes and the fused residual)",
    "xpass_narrow": "ttm_fma_stream_kernel (TMA-fed FP32 FMA TTM streaming X: the narrow sketch passes)",
    "ttm_tc": "ttm_tf32x3_kernel on intermediates",
}
# DRAM traffic / algorithmic bytes of one X-streaming launch, from an ncu capture of a 384^3 FP32
# core pass (243.0 MB moved for 251.5 MB of algorithmic bytes: part of the output stays in L2;
# summarised under profiles/); traffic scales with the elements streamed.
TRAFFIC_RATIO = {"xpass_tc": 241.9 / 251.5}
TRAFFIC_NOTE = {"xpass_tc": "algorithmic bytes per launch x 0.962, the DRAM/algorithmic ratio of a 384^3 core-pass "
                            "capture"}


# ------------------------------------------------------------------ ranks (one process per GPU)

def rank_env():
    """(rank, world size, local rank) from the torchrun environment (1 process when absent)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init_ranks(world: int):
    """A gloo process group for the barrier and the timing reduction when world > 1 (the data
    path has no collective: every rank decomposes its own tensor), else None."""
    if world <= 1:
        return None
    import torch.distributed as dist
    dist.init_process_group("gloo")
    return dist


def barrier(dist) -> None:
    if dist is not None:
        dist.barrier()


def max_over_ranks(x: float, dist) -> float:
    """The slowest rank's value: the job's time is set by its last replica."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ CPU oracle leg

def oracle_step(n: int, x=None):
    """One oracle step of the workload at edge n: rHKron-re and rSTHKron with their relative errors,
    and the loss gradient at the rHKron-re result.  x: the field as a float64 host array (the GPU's
    own X, copied back), else the same recipe generated on the host (its noise then comes from the
    host generator, so it is not bit-identical to a field drawn on the device).  Returns
    (seconds, (rel_err rHKron-re, rel_err rSTHKron)); the field is built outside the timed part."""
    import numpy as np

    import oracle as O
    from paper_2211_13028_gb300 import synth

    if x is None:
        x = synth.from_fortran(synth.gaussian_bumps(n, 3, 200, SEED, 1e-4, "cpu", "f32"))
    r, p = RANKS, P_OVER
    s, _ = O.subranks_reuse(r, p)
    S, w = O.subranks_matrix(r, p)
    k = [min(n, ww) for ww in w]
    t0 = time.perf_counter()
    # the Gaussian sketch factors from the oracle's statement of the device generator (Philox4x32-10,
    # Box-Muller): rHKron-re's Phi_j from stream j, rSTHKron's Phi_{j,k} from stream 8 j + k
    om = [synth.round_to(O.gaussian_factor(n, s[j], SEED + 1, j), "f32") for j in range(3)]
    oms, done = {}, set()
    for j in range(3):
        for kk in range(3):
            if kk != j:
                cur = k[kk] if kk in done else n
                oms[(j, kk)] = synth.round_to(O.gaussian_factor(cur, int(S[j][kk]), SEED + 2, 8 * j + kk), "f32")
        done.add(j)
    a = O.rhkron(x, r, om)
    ea = O.rel_err(x, a["G"], a["U"])
    b = O.rsthkron(x, r, oms)
    eb = O.rel_err(x, b["G"], b["U"])
    O.loss_grads(x, a["G"], a["U"])
    dt = time.perf_counter() - t0
    del np
    return dt, (ea, eb)


def cpu_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


_ONE_THREAD = {k: "1" for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")}


def oracle_one_thread(n: int, timeout_s: float = 240.0):
    """The oracle step at edge n in a child process whose BLAS runs on one thread (the thread count of
    a BLAS library is fixed when it loads).  Returns (seconds, rel_errs) or None."""
    code = ("import json, sys; sys.path.insert(0, %r); import bench; "
            "print('ORACLE1', json.dumps(bench.oracle_step(%d)))" % (ROOT, n))
    try:
        r = subprocess.run([sys.executable, "-c", code], env={**os.environ, **_ONE_THREAD}, capture_output=True,
                           text=True, timeout=timeout_s)
        for ln in r.stdout.splitlines():
            if ln.startswith("ORACLE1 "):
                dt, errs = json.loads(ln[8:])
                return float(dt), tuple(errs)
    except Exception:
        pass
    return None


def cpu_baseline(xh, gpu_errs, n_one_thread: int = 256):
    """The FP64 oracle timed on the host cores: one full step of the workload at 512^3 on the GPU's own
    field (all cores), and a one-thread run of the same recipe at n_one_thread^3."""
    dt, errs = oracle_step(N_FULL, xh)
    one = oracle_one_thread(n_one_thread)
    out = dict(value=dt * 1e3, unit="ms", cores=cpu_cores(), kind="oracle",
               sample=("one full step at 512^3 (rHKron-re + rSTHKron + loss gradient) on the GPU's own field, "
                       "copied to the host; FP64 NumPy, BLAS on all %d cores" % cpu_cores()),
               same_config=True,
               oracle_rel_err=dict(rhkron=errs[0], rsthkron=errs[1]),
               gpu_rel_err=dict(rhkron=gpu_errs[0], rsthkron=gpu_errs[1]),
               abs_diff=dict(rhkron=abs(errs[0] - gpu_errs[0]), rsthkron=abs(errs[1] - gpu_errs[1])))
    if one is not None:
        out["one_thread"] = dict(ms=one[0] * 1e3, cores=1,
                                 sample="%d^3 field of the same recipe (host-drawn noise), BLAS on 1 thread"
                                        % n_one_thread,
                                 rel_err=dict(rhkron=one[1][0], rsthkron=one[1][1]))
    return out


def run_reference(args):
    """The reference arm: the FP64 oracle, as it stands, on the host cores, each timed step one full
    512^3 step of the workload (rHKron-re + rSTHKron + loss gradient).  The field is built once
    before the timed steps; the untimed warm-up steps run the same code at 128^3."""
    rank = rank_env()[0]
    if rank != 0:  # the oracle runs once, on rank 0; the other ranks exit without work
        return
    from paper_2211_13028_gb300 import synth

    n = args.ref_n
    for _ in range(args.warmup):
        oracle_step(min(n, 128))
    xh = synth.from_fortran(synth.gaussian_bumps(n, 3, 200, SEED, 1e-4, "cpu", "f32"))
    times = []
    for _ in range(args.steps):
        dt, errs = oracle_step(n, xh)
        times.append(dt)
    ms = sum(times) / len(times) * 1e3
    line = dict(metric=METRIC, value=ms, unit="ms", n_gpus=args.gpus, steps=args.steps, warmup=args.warmup,
                ms_per_step=ms, higher_is_better=False, scaling="weak", vs_baseline=None, dtype="f64",
                data="synthetic", impl="reference",
                config=dict(workload=WORKLOAD,
                            sample=("every timed step is the full 512^3 workload" if n == N_FULL else
                                    "every timed step is the workload's recipe at %d^3 (not the full size)" % n),
                            field="the recipe with its noise drawn by the host generator"),
                cpu_baseline=dict(value=ms, unit="ms", cores=cpu_cores(), kind="oracle",
                                  sample="%d^3 step (FP64 NumPy, BLAS on all cores); warm-up at %d^3"
                                         % (n, min(n, 128))),
                e2e=dict(value=ms, unit="ms", h2d_bytes_per_step=0, d2h_bytes_per_step=0),
                rel_err=dict(rhkron=errs[0], rsthkron=errs[1]))
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ clocks

class ClockSampler:
    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"])
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sms, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sms.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for nm, v in zip(names, f[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        sms.sort()
        return dict(sm_mhz=sms[len(sms) // 2] if sms else None, sm_max_mhz=mx, reasons=sorted(reasons),
                    samples=len(sms))


# ------------------------------------------------------------------ single building block (profiling)

def profile_case(args):
    """Repetitions of one building block on an n^3 FP32 field of the bench generator:
    'sketch' (tucker_sketch, s = (6,7,7)), 'core' (tucker_core, k = (49,42,42)),
    'residual' (tucker_loss with r = 32: the fused tensor-core residual) or
    'rhkron' / 'rsthkron' (all of rHKron-re / rSTHKron, r = 32, p = 8), 'backward' (dG, dU)."""
    import torch

    from paper_2211_13028_gb300 import synth
    from paper_2211_13028_gb300 import tucker as T

    dev = torch.device("cuda", 0)
    n = args.n
    X = synth.gaussian_bumps(n, 3, 200, SEED, 1e-4, dev, "f32")
    xs = 1.0
    if args.dtype == "bf16":
        X = X.to(torch.bfloat16)
    elif args.dtype == "fp8":  # per-tensor scale, q = e4m3(x * scale)
        xs = 448.0 / float(X.abs().max())
        X = (X * xs).to(torch.float8_e4m3fn)
    g = __import__("numpy").random.Generator(__import__("numpy").random.PCG64(SEED))
    if args.profile_case == "sketch":
        om = [synth.fmat(o, "f32", dev) for o in synth.sketch_factors_reuse(X.shape, (6, 7, 7), SEED + 1, "f32")]
        fn = lambda: T.tucker_sketch(X, om, scale=xs)  # noqa: E731
    elif args.profile_case == "core":
        qs = [synth.fmat(__import__("numpy").linalg.qr(g.standard_normal((n, k)))[0], "f32", dev) for k in (49, 42, 42)]
        fn = lambda: T.tucker_core(X, qs, scale=xs)  # noqa: E731
    elif args.profile_case == "backward":
        # dG and dU at an rHKron-re result (r = 32, p = 8)
        s, _ = T.tucker_subranks_reuse(RANKS, P_OVER)
        om = [synth.fmat(o, "f32", dev) for o in synth.sketch_factors_reuse(X.shape, s, SEED + 1, "f32")]
        G, U, _ = T.tucker_rhkron(X, RANKS, P_OVER, om)
        fn = lambda: T.tucker_reconstruct_backward(X, G, U, 1.0, need_dX=False)  # noqa: E731
    elif args.profile_case == "rhkron":
        # the whole of rHKron-re at r = 32, p = 8: the core sizes (49,42,42) do not depend on n
        s, _ = T.tucker_subranks_reuse(RANKS, P_OVER)
        om = [synth.fmat(o, "f32", dev) for o in synth.sketch_factors_reuse(X.shape, s, SEED + 1, "f32")]
        fn = lambda: T.tucker_rhkron(X, RANKS, P_OVER, om, scale=xs)  # noqa: E731
    elif args.profile_case == "rsthkron":
        # the whole of rSTHKron at r = 32, p = 8 (S rows {5, 8}), factors drawn on the device
        S, w = T.tucker_subranks_matrix(RANKS, P_OVER)
        k = [min(n, ww) for ww in w]
        oms = T.gaussian_factors_matrix(tuple(X.shape), S, k, [0, 1, 2], SEED + 2, torch.float32, dev)
        fn = lambda: T.tucker_rsthkron(X, RANKS, P_OVER, oms)  # noqa: E731
    else:
        G = synth.fortran(g.standard_normal((32, 32, 32)), "f32", dev)
        U = [synth.fmat(__import__("numpy").linalg.qr(g.standard_normal((n, 32)))[0], "f32", dev) for _ in range(3)]
        fn = lambda: T.tucker_loss(X, G, U)  # noqa: E731
    for _ in range(3):
        fn()
    torch.cuda.synchronize()
    T.tk_profile(True, dev)
    torch.cuda.nvtx.range_push("profile_reps")  # lets ncu select exactly these repetitions
    for _ in range(5):
        fn()
    torch.cuda.nvtx.range_pop()
    prof = T.tk_profile_read(dev)
    T.tk_profile(False, dev)
    hbm = _peaks()[0]
    out = dict(profile_case=args.profile_case, n=n, dtype=args.dtype, status=T.tk_sync_status(dev)[0], kernels={})
    for name, v in prof.items():
        ms = v["ms"] / v["launches"]
        out["kernels"][name] = dict(launches=v["launches"] // 5, us_per_launch=1e3 * ms,
                                    gbs=(v["bytes"] / v["launches"]) / (ms * 1e-3) / 1e9 if ms > 0 else 0.0,
                                    frac_hbm=((v["bytes"] / v["launches"]) / (ms * 1e-3) / 1e9) / hbm if ms > 0 else 0.0)
    print(json.dumps(out))


# ------------------------------------------------------------------ BF16 storage form (1024^3)

def run_bf16_workload(args):
    """rHKron-re at r = 64, p = 16 (s = (9,9,9)) on the 1024^3 Gaussian-bump field stored in BF16
    (X rounded once; the core pass applies Q as a BF16 hi + lo pair), timed beside the same
    decomposition of the FP32 field.  Relative errors are reported against the data each form
    consumed and against the FP32 field; the FP64 oracle is run on a 256^3 field of the same
    generator and ranks (the whole 1024^3 oracle would take minutes on the host)."""
    import numpy as np
    import torch

    import oracle as O
    from paper_2211_13028_gb300 import synth
    from paper_2211_13028_gb300 import tucker as T

    n, r, p = 1024, (64, 64, 64), 16
    # oracle leg first, before any CUDA work in this process
    n_or = args.oracle_n
    xo = synth.from_fortran(synth.gaussian_bumps(n_or, 3, 200, SEED, 1e-4, "cpu", "f32"))
    xo16 = synth.round_to(xo, "bf16")
    s, _ = O.subranks_reuse(r, p)
    om_o = synth.sketch_factors_reuse(xo.shape, s, SEED + 1, "bf16")
    t_or = time.perf_counter()
    ref = O.rhkron(xo16, r, om_o)
    t_or = time.perf_counter() - t_or
    err_or = O.rel_err(xo16, ref["G"], ref["U"])

    dev = torch.device("cuda", 0)
    T.load()
    Xo = synth.fortran(xo16, "bf16", dev)
    _, _, err_gpu_small = T.tucker_rhkron(Xo, r, p, [synth.fmat(o, "f32", dev) for o in om_o])
    del Xo
    X32 = synth.gaussian_bumps(n, 3, 200, SEED, 1e-4, dev, "f32")
    X16 = X32.to(torch.bfloat16)
    assert T.is_colmajor(X16)
    sc8 = 448.0 / float(X32.abs().max())  # FP8 storage: per-tensor scale, q = e4m3(x * scale)
    X8 = (X32 * sc8).to(torch.float8_e4m3fn)
    assert T.is_colmajor(X8)
    om = [synth.fmat(o, "f32", dev) for o in synth.sketch_factors_reuse(tuple(X32.shape), s, SEED + 1, "bf16")]
    nrm32 = float(torch.linalg.vector_norm(X32.double()))
    hbm = _peaks()[0]
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    forms = {}
    for name, X, xs in (("bf16", X16, 1.0), ("f32", X32, 1.0), ("fp8", X8, sc8)):
        for _ in range(args.warmup):
            out = T.tucker_rhkron(X, r, p, om, scale=xs)
        torch.cuda.synchronize()
        T.tk_profile(True, dev, only="xpass")  # live timing of the X-streaming kernels only
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            out = T.tucker_rhkron(X, r, p, om, async_outputs=True, scale=xs)
        e1.record()
        torch.cuda.synchronize()
        prof = T.tk_profile_read(dev)
        T.tk_profile(False, dev)
        G, U, err = out
        loss32 = T.tucker_loss(X32, G, U)
        passes = {}
        for cls in ("xpass_tc", "xpass_simt", "xpass_narrow"):
            xp = prof.get(cls)
            if not xp or xp["ms"] <= 0:
                continue
            gbs = (xp["bytes"] / xp["launches"]) / (xp["ms"] / xp["launches"] * 1e-3) / 1e9
            passes[cls] = dict(gbs=gbs, frac=gbs / hbm, launches_per_step=xp["launches"] / args.steps,
                               us_per_launch=1e3 * xp["ms"] / xp["launches"],
                               bytes_per_launch=xp["bytes"] / xp["launches"])
        tc = passes.get("xpass_tc", dict(gbs=0.0, frac=0.0, launches_per_step=0, bytes_per_launch=0.0))
        forms[name] = dict(ms=e0.elapsed_time(e1) / args.steps, rel_err_vs_own_data=err.value,
                           rel_err_vs_f32_field=float(np.sqrt(max(loss32, 0.0))) / nrm32,
                           xpass_gbs=tc["gbs"], xpass_frac=tc["frac"], xpass_launches=tc["launches_per_step"],
                           x_passes=passes)
    clk = clocks.stop()
    st, _ = T.tk_sync_status(dev)
    line = dict(
        metric="rHKron-re wall time, 1024^3 field, r=64, p=16: BF16 storage (Q hi+lo refinement) vs FP32 (and FP8)",
        value=forms["bf16"]["ms"], unit="ms", n_gpus=1, steps=args.steps, warmup=args.warmup,
        ms_per_step=forms["bf16"]["ms"], higher_is_better=False, scaling="weak", vs_baseline=None,
        dtype="bf16", data="synthetic",
        config=dict(workload=("bumps1024_bf16: 1024^3 Gaussian-bump field (the 512^3 generator at n=1024), "
                              "stored BF16 (rounded once), FP32, and FP8 E4M3 (per-tensor scale 448/amax); "
                              "rHKron-re r=(64,64,64), p=16, s=(9,9,9)"),
                    l2="X is 2 GiB (BF16) / 4 GiB (FP32) / 1 GiB (FP8), larger than L2: no flush"),
        forms=forms, speedup_bf16_over_f32=forms["f32"]["ms"] / forms["bf16"]["ms"],
        speedup_fp8_over_f32=forms["f32"]["ms"] / forms["fp8"]["ms"],
        cpu_baseline=dict(value=t_or * 1e3, unit="ms", cores=cpu_cores(), kind="oracle",
                          sample="one FP64 oracle rHKron-re on the BF16-rounded %d^3 field of the same generator"
                                 % n_or,
                          oracle_rel_err=err_or, gpu_rel_err=err_gpu_small, abs_diff=abs(err_or - err_gpu_small)),
        device_status=st, clocks=clk)
    return line


# ------------------------------------------------------------------ 4-way rSTHKron (160^4)

def run_tucker4_workload(args):
    """rSTHKron on the 160^4 FP32 four-way tensor (core 40^4 with entries N(0,1) 0.9^(index sum),
    random orthonormal factors, 1e-3 noise), uneven ranks (10,20,30,40), p = 6, modes processed
    4 -> 1; the FP64 oracle checks the same generator at a reduced edge."""
    import torch

    import oracle as O
    from paper_2211_13028_gb300 import synth
    from paper_2211_13028_gb300 import tucker as T

    r, p, order = (10, 20, 30, 40), 6, [3, 2, 1, 0]
    n_or = args.oracle_n4
    xo = synth.from_fortran(synth.tucker4_device(n_or, 40, 0.9, 1e-3, SEED, "cpu", "f32"))
    S, w = O.subranks_matrix(r, p, order)
    ko = [min(n_or, ww) for ww in w]
    oms_o = synth.sketch_factors_matrix(xo.shape, S, ko, order, SEED + 2, "f32")
    t_or = time.perf_counter()
    ref = O.rsthkron(xo, r, oms_o, order)
    t_or = time.perf_counter() - t_or
    err_or = O.rel_err(xo, ref["G"], ref["U"])

    dev = torch.device("cuda", 0)
    T.load()
    Xo = synth.fortran(xo, "f32", dev)
    _, _, err_gpu_small = T.tucker_rsthkron(Xo, r, p, {kk: synth.fmat(v, "f32", dev) for kk, v in oms_o.items()},
                                            order=order)
    del Xo
    n = 160
    X = synth.tucker4_device(n, 40, 0.9, 1e-3, SEED, dev, "f32")
    k = [min(n, ww) for ww in w]
    oms = {kk: synth.fmat(v, "f32", dev)
           for kk, v in synth.sketch_factors_matrix(tuple(X.shape), S, k, order, SEED + 2, "f32").items()}
    for _ in range(args.warmup):
        out = T.tucker_rsthkron(X, r, p, oms, order=order)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    T.tk_profile(True, dev, only="xpass")  # live timing of the X-streaming kernel only
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        out = T.tucker_rsthkron(X, r, p, oms, order=order, async_outputs=True)
    e1.record()
    torch.cuda.synchronize()
    prof = T.tk_profile_read(dev)
    T.tk_profile(False, dev)
    T.tk_profile(True, dev)  # all classes, one extra call after the timed region
    T.tucker_rsthkron(X, r, p, oms, order=order)
    prof_all = T.tk_profile_read(dev)
    T.tk_profile(False, dev)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    hbm = _peaks()[0]
    xp = prof.get("xpass_tc", dict(ms=0.0, launches=1, bytes=0.0))
    gbs = (xp["bytes"] / max(1, xp["launches"])) / (xp["ms"] / max(1, xp["launches"]) * 1e-3) / 1e9 \
        if xp["ms"] > 0 else 0.0
    tot = sum(v["ms"] for v in prof_all.values())
    line = dict(
        metric="rSTHKron wall time, 160^4 FP32, r=(10,20,30,40), p=6, order 4->1", value=ms, unit="ms",
        n_gpus=1, steps=args.steps, warmup=args.warmup, ms_per_step=ms, higher_is_better=False,
        scaling="weak", vs_baseline=None, dtype="f32", data="synthetic",
        config=dict(workload=("tucker160x4_f32: 160^4 FP32, core 40^4 N(0,1)*0.9^(index sum), orthonormal "
                              "factors, 1e-3 noise; rSTHKron r=(10,20,30,40), p=6 (l'=16,27,36,48), order 4->1"),
                    l2="X is 2.6 GB, larger than L2: no flush"),
        rel_err=out[2].value,
        xpass=dict(gbs=gbs, frac=gbs / hbm, launches_per_step=xp["launches"] / args.steps,
                   bytes_per_step=xp["bytes"] / args.steps),
        kernel_shares={kk: round(v["ms"] / tot, 4) for kk, v in sorted(prof_all.items(), key=lambda kv: -kv[1]["ms"])},
        cpu_baseline=dict(value=t_or * 1e3, unit="ms", cores=cpu_cores(), kind="oracle",
                          sample="one FP64 oracle rSTHKron on the %d^4 tensor of the same generator" % n_or,
                          oracle_rel_err=err_or, gpu_rel_err=err_gpu_small, abs_diff=abs(err_or - err_gpu_small)),
        device_status=T.tk_sync_status(dev)[0], clocks=clk)
    return line


# ------------------------------------------------------------------ Section 7.1 accuracy: SRHT vs Gaussian sketches

def run_srht_workload(args):
    """The accuracy experiment of Section 7.1 at 512^3 (a power of two, as the Walsh-Hadamard factors
    need): X = sum_i 0.4^i q1_i o q2_i o q3_i (a superdiagonal core of 40 entries decaying by 0.4
    times random orthonormal factors), rank (10,10,10), p = 5.  rHKron-re with Gaussian Kronecker
    factors and with the Kronecker-SRHT sketch, fresh random factors per trial; the deterministic
    (STHOSVD) error of this tensor is 0.4^10 in closed form.  Reports the relative errors over the
    trials and the time of one decomposition of each kind."""
    import numpy as np
    import torch

    import oracle as O
    from paper_2211_13028_gb300 import synth
    from paper_2211_13028_gb300 import tucker as T

    n, rr, p, trials = 512, (10, 10, 10), 5, args.trials
    so, _ = O.subranks_reuse(rr, p)
    # oracle leg first, before any CUDA work in this process: a 64^3 tensor of the same construction,
    # with the factors of the first GPU trial
    no = 64
    fo = [np.linalg.qr(np.random.Generator(np.random.PCG64(SEED + j)).standard_normal((no, 40)))[0] for j in range(3)]
    xo = synth.round_to(np.einsum("i,ai,bi,ci->abc", 0.4 ** np.arange(40), *fo), "f32")
    Ho = synth.sketch_factors_srht((no, no, no), so, SEED + 200, "f32")
    t_or = time.perf_counter()
    ref = O.rhkron_srht(xo, rr, Ho, SEED + 300)
    t_or = time.perf_counter() - t_or
    err_or = O.rel_err(xo, ref["G"], ref["U"])

    dev = torch.device("cuda", 0)
    T.load()
    s, _ = T.tucker_subranks_reuse(rr, p)
    gpu_o = T.tucker_rhkron_srht(synth.fortran(xo, "f32", dev), rr, p, [synth.fmat(h, "f32", dev) for h in Ho],
                                 seed=SEED + 300)[2]
    g = torch.Generator(device="cpu").manual_seed(SEED)
    facs = [torch.linalg.qr(torch.randn(n, 40, generator=g, dtype=torch.float64))[0] for _ in range(3)]
    lam = 0.4 ** torch.arange(40, dtype=torch.float64)
    X = torch.einsum("i,ai,bi,ci->cba", lam.float().to(dev), *[f.float().to(dev) for f in facs]).permute(2, 1, 0)
    # (a column-major view: the einsum writes index order (c, b, a) row-major)
    det = 0.4 ** 10
    errs = {"gaussian": [], "srht": []}
    for t in range(trials):
        om = [synth.fmat(o, "f32", dev) for o in synth.sketch_factors_reuse((n, n, n), s, SEED + 100 + t, "f32")]
        H = [synth.fmat(h, "f32", dev) for h in synth.sketch_factors_srht((n, n, n), s, SEED + 200 + t, "f32")]
        errs["gaussian"].append(T.tucker_rhkron(X, rr, p, om)[2])
        errs["srht"].append(T.tucker_rhkron_srht(X, rr, p, H, seed=SEED + 300 + t)[2])
    times = {}
    for name in ("gaussian", "srht"):
        fn = (lambda: T.tucker_rhkron(X, rr, p, om, async_outputs=True)) if name == "gaussian" else \
             (lambda: T.tucker_rhkron_srht(X, rr, p, H, seed=SEED, async_outputs=True))
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        times[name] = e0.elapsed_time(e1) / args.steps
    summ = {k: dict(median=float(np.median(v)), min=float(np.min(v)), max=float(np.max(v)),
                    median_over_deterministic=float(np.median(v) / det)) for k, v in errs.items()}
    line = dict(
        metric="rHKron-re, Section 7.1 tensor at 512^3, r=(10,10,10), p=5: Kronecker-SRHT vs Gaussian sketch",
        value=times["srht"], unit="ms", n_gpus=1, steps=args.steps, warmup=args.warmup, ms_per_step=times["srht"],
        higher_is_better=False, scaling="weak", vs_baseline=None, dtype="f32", data="synthetic",
        config=dict(workload=("srht512_f32: 512^3 FP32, superdiagonal core 0.4^i (40 entries) times random "
                              "orthonormal factors; rHKron-re r=10, p=5, s=%s; %d trials per sketch" % (list(s), trials)),
                    l2="X is 512 MiB, larger than L2: no flush"),
        ms=times, rel_err=summ, deterministic_rel_err=det,
        cpu_baseline=dict(value=t_or * 1e3, unit="ms", cores=cpu_cores(), kind="oracle",
                          sample="one FP64 oracle rHKron-re with the Kronecker-SRHT sketch on the %d^3 tensor of "
                                 "the same construction" % no,
                          oracle_rel_err=err_or, gpu_rel_err=gpu_o, abs_diff=abs(err_or - gpu_o)),
        device_status=T.tk_sync_status(dev)[0])
    return line


# ------------------------------------------------------------------ gradient descent on the loss (256^3)

def run_descent_workload(args):
    """Tucker fitting by gradient descent: rHKron-re initialisation (r = 16, p = 8) of the 256^3
    FP32 tensor (core 16^3 N(0,1), orthonormal factors, 1e-2 noise), then 50 Adam steps
    (lr 1e-3, betas (0.9, 0.999), eps 1e-8) on ||X - G x_j U_j||^2 through TuckerLoss: each step
    is one loss plus its adjoint (dG, dU; X is a constant) on the GPU and torch's Adam update."""
    import numpy as np
    import torch

    from paper_2211_13028_gb300 import synth
    from paper_2211_13028_gb300 import tucker as T

    dev = torch.device("cuda", 0)
    T.load()
    n, r, p, nsteps = 256, (16, 16, 16), 8, 50
    x = synth.tucker_tensor((n, n, n), r, seed=SEED, noise_rel=1e-2)
    X = synth.fortran(x, "f32", dev)
    nrm = float(np.linalg.norm(x))
    s, _ = T.tucker_subranks_reuse(r, p)
    om = [synth.fmat(o, "f32", dev) for o in synth.sketch_factors_reuse(x.shape, s, SEED + 1, "f32")]

    def fit():
        G0, U0, e0 = T.tucker_rhkron(X, r, p, om)
        G = G0.clone().requires_grad_(True)
        U = [u.clone().requires_grad_(True) for u in U0]
        opt = torch.optim.Adam([G] + U, lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
        for _ in range(nsteps):
            opt.zero_grad(set_to_none=False)
            loss = T.TuckerLoss.apply(X, G, *U)
            loss.backward()
            opt.step()
        return e0, loss

    for _ in range(args.warmup):
        fit()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_init = torch.cuda.Event(enable_timing=True)
    e0.record()
    G0, U0, err0 = T.tucker_rhkron(X, r, p, om)
    t_init.record()
    G = G0.clone().requires_grad_(True)
    U = [u.clone().requires_grad_(True) for u in U0]
    opt = torch.optim.Adam([G] + U, lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    for _ in range(nsteps):
        opt.zero_grad(set_to_none=False)
        loss = T.TuckerLoss.apply(X, G, *U)
        loss.backward()
        opt.step()
    e1.record()
    torch.cuda.synchronize()
    total = e0.elapsed_time(e1)
    init = e0.elapsed_time(t_init)
    final = float(np.sqrt(T.tucker_loss(X, G.detach(), [u.detach() for u in U]))) / nrm
    line = dict(
        metric="Tucker fit: rHKron-re init + 50 Adam steps on ||X - G x U||^2, 256^3 FP32, r=16", value=total,
        unit="ms", n_gpus=1, steps=1, warmup=args.warmup, ms_per_step=(total - init) / nsteps,
        higher_is_better=False, scaling="weak", vs_baseline=None, dtype="f32", data="synthetic",
        config=dict(workload=("descent256_f32: 256^3 FP32, core 16^3 N(0,1), orthonormal factors, 1e-2 noise; "
                              "rHKron-re r=16 p=8 (s=(5,5,5)); Adam lr=1e-3 betas=(0.9,0.999) eps=1e-8, 50 steps"),
                    l2="X is 64 MiB, inside L2 after the first pass of a step"),
        init_ms=init, adam_step_ms=(total - init) / nsteps, rel_err_init=err0, rel_err_final=final,
        device_status=T.tk_sync_status(dev)[0])
    return line


# ------------------------------------------------------------------ sharded rHKron-re (one field split across ranks)

def run_sharded(args):
    """One rHKron-re decomposition of the 512^3 field split along mode 3 into one slab per rank
    (Section 6.3; sharded.rhkron_sharded): each rank sketches and contracts its slab, the partial
    sketches, the mode-3 sketch rows, the partial cores and the error norms are exchanged over the
    process group (gloo, staged through host memory), and the QR and the core truncation run
    redundantly on every rank.  Total work is fixed as N grows (strong scaling)."""
    import torch

    from paper_2211_13028_gb300 import sharded, synth
    from paper_2211_13028_gb300 import tucker as T

    rank, world, local = rank_env()
    dist = init_ranks(world)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    T.load()
    r, p = RANKS, P_OVER
    X = synth.gaussian_bumps(N_FULL, 3, 200, SEED, 1e-4, dev, "f32")
    off, rows = sharded.slab_bounds(N_FULL, world, rank)
    Xs = X[..., off:off + rows]
    s, _ = T.tucker_subranks_reuse(r, p)
    om = T.gaussian_factors(tuple(X.shape), s, SEED + 1, torch.float32, dev)
    for _ in range(args.warmup):
        out = sharded.rhkron_sharded(Xs, off, N_FULL, r, p, om)
    torch.cuda.synchronize()
    whole = T.tucker_rhkron(X, r, p, om)[2] if world == 1 else None
    barrier(dist)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        out = sharded.rhkron_sharded(Xs, off, N_FULL, r, p, om)
    e1.record()
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, dist)
    if rank == 0:
        line = dict(metric="rHKron-re wall time per decomposition, 512^3 FP32 field split along mode 3 across ranks",
                    value=ms, unit="ms", n_gpus=world, steps=args.steps, warmup=args.warmup, ms_per_step=ms,
                    higher_is_better=False, scaling="strong", vs_baseline=None, dtype="f32", data="synthetic",
                    config=dict(workload="bumps512_f32 rHKron-re, r=(32,32,32), p=8, one slab of mode 3 per rank",
                                parallelism="sharded along mode 3, exchanges over gloo (host-staged)"),
                    rel_err=out[2], rel_err_whole_tensor_call=whole)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ------------------------------------------------------------------ GPU leg

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--sample", type=int, default=256, help="edge of the one-thread oracle sample")
    ap.add_argument("--ref-n", type=int, default=N_FULL,
                    help="edge of each timed step of the reference arm (default: the full 512^3 workload)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the other configurations (BF16 1024^3 vs FP32, 4-way 160^4, 256^3 descent) that "
                         "the default line carries under 'secondary'")
    ap.add_argument("--serial", action="store_true", help="run both algorithms on one stream")
    ap.add_argument("--priority", choices=["none", "rhkron", "rsthkron"], default="none",
                    help="which algorithm's stream gets the higher CUDA stream priority")
    ap.add_argument("--h2d-chunks", type=int, default=1,
                    help="pieces (copy streams) of the end-to-end run's host-to-device copy of X")
    ap.add_argument("--sm-reserve", type=int, default=16,
                    help="SMs the streaming kernels of each stream leave to the other stream's kernels")
    ap.add_argument("--sharded", action="store_true",
                    help="one rHKron-re decomposition of the 512^3 field split along mode 3, one slab per rank")
    ap.add_argument("--no-graph", action="store_true",
                    help="time the step as eager launches only (default: the step is also recorded once into a "
                         "CUDA graph and the replays are the headline)")
    ap.add_argument("--profile-case", choices=["sketch", "core", "residual", "rhkron", "rsthkron", "backward"],
                    default=None,
                    help="run one building block on an n^3 FP32 field (for ncu captures) instead of the bench")
    ap.add_argument("--n", type=int, default=384, help="edge of the --profile-case tensor")
    ap.add_argument("--dtype", choices=["f32", "bf16", "fp8"], default="f32", help="storage of the --profile-case tensor")
    ap.add_argument("--workload", choices=["bumps512_f32", "bumps1024_bf16", "tucker160x4_f32", "descent256_f32",
                                           "srht512_f32"],
                    default="bumps512_f32",
                    help="bumps512_f32: the default step; bumps1024_bf16: the BF16 storage form vs FP32; "
                         "tucker160x4_f32: 4-way rSTHKron; descent256_f32: rHKron-re init + 50 Adam steps; "
                         "srht512_f32: the Section 7.1 accuracy experiment, Kronecker-SRHT vs Gaussian sketches")
    ap.add_argument("--trials", type=int, default=20, help="random trials per sketch kind (srht512_f32)")
    ap.add_argument("--oracle-n", type=int, default=256, help="edge of the oracle check of --workload bumps1024_bf16")
    ap.add_argument("--oracle-n4", type=int, default=48, help="edge of the oracle check of --workload tucker160x4_f32")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.profile_case:
        profile_case(args)
        return
    side = {"bumps1024_bf16": run_bf16_workload, "tucker160x4_f32": run_tucker4_workload,
            "descent256_f32": run_descent_workload, "srht512_f32": run_srht_workload}
    if args.workload in side and args.impl == "native":
        print(json.dumps(side[args.workload](args)), flush=True)
        return

    if args.impl == "reference":
        run_reference(args)
        return
    if args.sharded:
        run_sharded(args)
        return

    rank, world, local = rank_env()

    import numpy as np
    import torch

    from paper_2211_13028_gb300 import synth
    from paper_2211_13028_gb300 import tucker as T

    dist = init_ranks(world)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    T.load()

    r, p = RANKS, P_OVER
    X = synth.gaussian_bumps(N_FULL, 3, 200, SEED, 1e-4, dev, "f32")
    dims = tuple(X.shape)
    s, _ = T.tucker_subranks_reuse(r, p)
    S, w = T.tucker_subranks_matrix(r, p)
    k = [min(n, ww) for n, ww in zip(dims, w)]
    torch.cuda.synchronize()

    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    # The two algorithms are independent: rHKron-re and its gradient run on one stream, rSTHKron on a
    # second, so the latency-bound small kernels of one overlap the other (--serial: one stream).
    main_s = torch.cuda.current_stream(dev)
    pa, pb = {"none": (0, 0), "rhkron": (-1, 0), "rsthkron": (0, -1)}[args.priority]
    sa = torch.cuda.Stream(dev, priority=pa) if not args.serial else main_s
    sb = torch.cuda.Stream(dev, priority=pb) if not args.serial else main_s
    use_graph = not args.no_graph and not args.serial
    # the two algorithms' streams run concurrently: each one's passes over X leave SMs to the other's
    # chains of small kernels (one stream: every SM)
    reserve = args.sm_reserve if sa is not sb else 0
    for st in {sa, sb}:
        with torch.cuda.stream(st):
            T.tk_set_sm_reserve(reserve, dev)

    def step(Xin, marks=None):
        main_s = torch.cuda.current_stream(dev)  # the recording stream when the step is captured
        if sa is not main_s:
            sa.wait_stream(main_s)
            sb.wait_stream(main_s)
        with torch.cuda.stream(sa):
            if marks:
                marks[0].record(sa)
            # fresh Gaussian sketch factors on the device (Philox4x32-10), as each decomposition draws them
            om = T.gaussian_factors(dims, s, SEED + 1, torch.float32, dev)
            # rHKron-re and the loss gradient (dG, dU, dX) at its result in one call: the gradient's
            # products come from the core's chain of TTMs and the relative error from the dX pass
            G1, U1, e1, dG, dU, dX = T.tucker_rhkron_grad(Xin, r, p, om, 1.0, async_outputs=True)
            if marks:
                marks[1].record(sa)
        with torch.cuda.stream(sb):
            if marks:
                marks[2].record(sb)
            oms = T.gaussian_factors_matrix(dims, S, k, [0, 1, 2], SEED + 2, torch.float32, dev)
            G2, U2, e2 = T.tucker_rsthkron(Xin, r, p, oms, async_outputs=True)
            if marks:
                marks[3].record(sb)
        if sa is not main_s:
            main_s.wait_stream(sa)
            main_s.wait_stream(sb)
        return (G1, U1, e1, G2, U2, e2, dG, dU, dX)

    for _ in range(args.warmup):
        out = step(X)
    torch.cuda.synchronize()
    errs = (out[2].value, out[5].value)
    dev_status, qr_info = T.tk_sync_status(dev)  # 0: every Jacobi solve converged


    # ---- device-timed region (inputs resident in HBM; X = 512 MiB > L2)
    marks = [[ev() for _ in range(4)] for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier(dist)
    torch.cuda.synchronize()
    l0 = T.tk_launch_count(dev)
    # live timing of the X-streaming tensor-core kernel only: an event pair per recorded launch
    # costs the host ~16 us, too much to time all ~290 launches of a step inside the timed region
    T.tk_profile(True, dev, only="xpass")
    t0, t1 = ev(), ev()
    t0.record()
    host_t = time.perf_counter()
    for i in range(args.steps):
        torch.cuda.nvtx.range_push("timed_step")  # lets ncu select exactly the timed launches
        step(X, marks[i])
        torch.cuda.nvtx.range_pop()
    host_ms = (time.perf_counter() - host_t) * 1e3 / args.steps  # host time to queue a step
    t1.record()
    torch.cuda.synchronize()
    prof = T.tk_profile_read(dev)
    T.tk_profile(False, dev)
    launches = T.tk_launch_count(dev) - l0
    # shares of every kernel class: one extra step after the timed region, all classes recorded
    T.tk_profile(True, dev)
    step(X)
    torch.cuda.synchronize()
    prof_all = T.tk_profile_read(dev)
    T.tk_profile(False, dev)
    ms = t0.elapsed_time(t1) / args.steps
    # ---- the same step recorded once into a CUDA graph (both streams, every launch) and replayed:
    # the launches no longer wait on the host or on per-launch queueing
    graph_ms, graph_errs = None, None
    if use_graph:
        gX = T.TuckerGraph(lambda: step(X), warmup=1)
        for _ in range(args.warmup):
            gX.replay()
        torch.cuda.synchronize()
        barrier(dist)
        g0, g1 = ev(), ev()
        g0.record()
        for _ in range(args.steps):
            gX.replay()
        g1.record()
        torch.cuda.synchronize()
        graph_ms = g0.elapsed_time(g1) / args.steps
        graph_errs = (gX.outputs[2].value, gX.outputs[5].value)
        del gX
    # ---- the roofline kernel alone: the first (X-streaming) product of tucker_core on the same field with
    # factors of the core's widths (49, 42, 42), nothing else on the GPU (5 repetitions, live event timing)
    rng_q = np.random.Generator(np.random.PCG64(SEED + 5))
    qs = [synth.fmat(np.linalg.qr(rng_q.standard_normal((N_FULL, kq)))[0], "f32", dev) for kq in (49, 42, 42)]
    T.tucker_core(X, qs)
    torch.cuda.synchronize()
    T.tk_profile(True, dev, only="xpass")
    for _ in range(5):
        T.tucker_core(X, qs)
    prof_alone = T.tk_profile_read(dev)
    T.tk_profile(False, dev)
    alone = prof_alone.get("xpass_tc")
    del qs
    barrier(dist)
    clk = clocks.stop()
    ph = [sum(marks[i][a].elapsed_time(marks[i][b]) for i in range(args.steps)) / args.steps
          for a, b in ((0, 1), (2, 3))]
    ms = max_over_ranks(ms, dist)
    if graph_ms is not None:
        graph_ms = max_over_ranks(graph_ms, dist)

    # ---- end to end through the public API with host buffers: every step copies its X from pinned
    # host memory (on a copy stream, into one of two device buffers, so step i+1's copy overlaps
    # step i's compute) and reads its results back (G, U, dG, dU and the two relative errors)
    Xh = X.detach().permute(2, 1, 0).contiguous().cpu().pin_memory()
    Xd = [torch.empty_like(X.permute(2, 1, 0).contiguous()) for _ in range(2)]
    # the host-to-device copy of a step's X in args.h2d_chunks pieces, each on its own copy stream (one
    # cudaMemcpyAsync per piece), so that several copy engines share it
    nch = max(1, args.h2d_chunks)
    css = [torch.cuda.Stream(dev) for _ in range(nch)]
    hflat = Xh.view(-1)
    bounds = [(hflat.numel() * q // nch, hflat.numel() * (q + 1) // nch) for q in range(nch)]
    copied = [[torch.cuda.Event() for _ in range(nch)] for _ in range(2)]
    consumed = [torch.cuda.Event() for _ in range(2)]

    def copy_in(b, after=None):
        dflat = Xd[b].view(-1)
        for q, cs in enumerate(css):
            with torch.cuda.stream(cs):
                if after is not None:
                    cs.wait_event(after)
                dflat[bounds[q][0]:bounds[q][1]].copy_(hflat[bounds[q][0]:bounds[q][1]], non_blocking=True)
                copied[b][q].record(cs)

    res_bytes = 0
    for b in range(2):
        Xd[b].copy_(Xh)
    gE = [T.TuckerGraph(lambda b=b: step(Xd[b].permute(2, 1, 0)), warmup=1) for b in range(2)] if use_graph else None
    torch.cuda.synchronize()
    e0, e1 = ev(), ev()
    barrier(dist)
    torch.cuda.synchronize()
    e0.record()
    for cs in css:
        cs.wait_stream(main_s)
    copy_in(0)
    hosts = []
    for i in range(args.steps):
        b = i & 1
        if i + 1 < args.steps:
            copy_in(1 - b, consumed[1 - b] if i >= 1 else None)  # after step i-1 has finished with that buffer
        for q in range(nch):
            main_s.wait_event(copied[b][q])
        if gE is not None:
            gE[b].replay()
            out = gE[b].outputs
        else:
            out = step(Xd[b].permute(2, 1, 0))
        consumed[b].record(main_s)
        host = [t.detach().to("cpu", non_blocking=True) for t in [out[0], *out[1], out[3], *out[4], out[6], *out[7]]]
        hosts.append((host, out[2], out[5]))
        res_bytes = sum(t.numel() * t.element_size() for t in host) + 16  # dX stays on the device
    e1.record()
    torch.cuda.synchronize()
    assert all(np.isfinite(h[1].value) and np.isfinite(h[2].value) for h in hosts)
    e2e_ms = e0.elapsed_time(e1) / args.steps
    e2e_ms = max_over_ranks(e2e_ms, dist)

    # ---- roofline: the kernel classes' shares come from one extra all-class step; the roofline kernel is
    # the HBM-streaming class (an X pass on the tensor cores or on the FP32 pipe) with the largest share,
    # timed live in the timed region; the dominant class overall and the runner-up are reported beside it
    hbm, bf16, peak_src = _peaks()
    peak_note = "the kernel is timed inside the step, next to the other kernels"
    step_ms_total = sum(v["ms"] for v in prof_all.values())
    ranked = sorted(prof_all.items(), key=lambda kv: -kv[1]["ms"])
    shares = {kname: round(v["ms"] / step_ms_total, 4) for kname, v in ranked}
    streaming = [kname for kname, _ in ranked if kname in ("xpass_tc", "xpass_narrow")]
    name = streaming[0] if streaming else "xpass_tc"
    d = prof.get(name, dict(ms=0.0, launches=1, bytes=0.0, flops=0.0))
    per_launch_ms = d["ms"] / max(1, d["launches"])
    ach = (d["bytes"] / max(1, d["launches"])) / (per_launch_ms * 1e-3) / 1e9 if per_launch_ms > 0 else 0.0
    ttm = [v for kname, v in prof_all.items() if kname.startswith(("ttm", "xpass"))]
    ttm_ms = sum(v["ms"] for v in ttm)
    ttm_tflops = (sum(v["flops"] for v in ttm) / (ttm_ms * 1e-3) / 1e12) if ttm_ms > 0 else 0.0
    runner = ranked[1][0] if len(ranked) > 1 else None  # the class after the dominant one
    # the same tensor-core kernel launched on part of the SMs beside a chain of small kernels (the gradient's
    # product pass and its dX pass): slower per launch by design, reported beside the roofline kernel
    isolated = None
    if alone and alone["launches"] > 0 and alone["ms"] > 0:
        a_gbs = (alone["bytes"] / alone["launches"]) / (alone["ms"] / alone["launches"] * 1e-3) / 1e9
        isolated = dict(achieved=a_gbs, frac=a_gbs / hbm, ms_per_launch=alone["ms"] / alone["launches"],
                        bytes_per_launch=alone["bytes"] / alone["launches"],
                        note="the same kernel timed alone: the X pass of tucker_core on the 512^3 field (mode 3, "
                             "42 output columns), 5 repetitions, nothing else running")
    bg = prof.get("xpass_tc_bg")
    background = None
    if bg and bg["launches"] > 0 and bg["ms"] > 0:
        bg_gbs = (bg["bytes"] / bg["launches"]) / (bg["ms"] / bg["launches"] * 1e-3) / 1e9
        background = dict(kernel_class="xpass_tc_bg", launches_per_step=bg["launches"] / args.steps,
                          bytes_per_launch=bg["bytes"] / bg["launches"], ms_per_launch=bg["ms"] / bg["launches"],
                          achieved=bg_gbs, frac=bg_gbs / hbm,
                          note="ttm_tf32x3_kernel on two thirds of the SMs (the gradient's X x_{j!=m1} Q_j^T pass "
                               "beside the core truncation, and its dX pass beside the gradient's small kernels)")

    if rank != 0:
        return
    value = graph_ms if graph_ms is not None else ms
    line = dict(
        metric=METRIC, value=value, unit="ms", n_gpus=world, steps=args.steps, warmup=args.warmup,
        ms_per_step=value,
        higher_is_better=False, scaling="weak", vs_baseline=None, dtype="f32", data="synthetic",
        config=dict(workload=WORKLOAD, l2="X is 512 MiB, larger than the 129 MB L2: no flush between steps",
                    parallelism=("replicas" if world > 1 else "single GPU"),
                    streams=("one stream" if args.serial else
                             "rHKron-re + its loss gradient (dG, dU, dX) on one stream, rSTHKron on a second, "
                             "concurrently; the streaming kernels of each leave %d SMs to the other's kernels "
                             "(tk_set_sm_reserve)" % reserve),
                    gradient=("rHKron-re and the gradient at its result in one call (tucker_rhkron_grad): the "
                              "gradient's products R x_{j!=n} U_j^T come from the core's chain of TTMs and from "
                              "one X pass (X x_{j!=m1} Q_j^T) made beside the core truncation, and rHKron-re's "
                              "relative error from the norms of the pass that forms dX; rSTHKron computes its own"),
                    launch=("the step recorded once into a CUDA graph (both streams), replayed every step"
                            if graph_ms is not None else "eager launches")),
        eager_ms_per_step=ms,
        graph_ms_per_step=graph_ms,
        graph_rel_err=(dict(rhkron=graph_errs[0], rsthkron=graph_errs[1]) if graph_errs else None),
        phases_ms=dict(rhkron_and_gradient=ph[0], rsthkron=ph[1],
                       note=("sequential" if args.serial else
                             "stream 1: rHKron-re with the loss gradient (one call); stream 2: rSTHKron; "
                             "from the eager timed steps")),
        rel_err=dict(rhkron=errs[0], rsthkron=errs[1]),
        device_status=dev_status,
        multi_ttm=dict(tflops=ttm_tflops, ms_per_step=ttm_ms, frac_of_bf16_peak=ttm_tflops / bf16),
        roofline=dict(bound="hbm",
                      kernel=KERNEL_NAMES.get(name, name), kernel_class=name, achieved=ach, peak=hbm, unit="GB/s",
                      frac=ach / hbm,
                      traffic=(TRAFFIC_RATIO[name] * d["bytes"] / max(1, d["launches"])
                               if name in TRAFFIC_RATIO else None),
                      traffic_note=TRAFFIC_NOTE.get(name),
                      peak_source=f"{peak_src} hbm_gbs (burst copy; {peak_note})",
                      bytes_per_launch=d["bytes"] / max(1, d["launches"]), ms_per_launch=per_launch_ms,
                      launches_per_step=d["launches"] / args.steps,
                      kernel_share_of_step=shares.get(name, 0.0),
                      dominant_class=dict(name=ranked[0][0], share=shares[ranked[0][0]]) if ranked else None,
                      runner_up=(dict(name=runner, share=shares[runner],
                                      bound=("hbm" if runner.startswith(("xpass", "ttm", "residual", "elementwise")) else
                                             "latency (one-CTA small-matrix kernel or short FP64 product)"))
                                 if runner else None),
                      note=("the roofline kernel is the HBM-streaming class with the largest share of the summed "
                            "kernel time (one extra all-class step); its %d launches per step are timed live with "
                            "CUDA events in the eager timed region (a recorded graph carries no per-launch events)"
                            % round(d["launches"] / args.steps)),
                      background=background, isolated=isolated),
        kernel_shares=shares,
        kernel_shares_note="all kernel classes timed in one extra step after the timed region",
        kernel_ms_per_step=step_ms_total,
        e2e=dict(value=e2e_ms, unit="ms", h2d_bytes_per_step=Xh.numel() * Xh.element_size(),
                 d2h_bytes_per_step=res_bytes,
                 note=("X copied from pinned host memory every step (%d piece(s), one copy stream each) into two "
                       "device buffers " % nch) +
                      "(step i+1's copy overlaps step i's compute); G, U, dG, dU and rel_err read back every step"
                      + ("; one recorded graph per input buffer, replayed" if gE is not None else "")),
        gpu_launches=launches,
        gpu_launches_note="kernels of the eager timed steps (the graph replays launch the same kernels per step)",
        host_queue_ms_per_step=host_ms,
        clocks=clk,
    )
    # ---- CPU baseline: the FP64 oracle on the GPU's own field at the full size (rank 0, N = 1)
    if world == 1 and not args.no_cpu_baseline:
        xh = synth.from_fortran(X)
        line["cpu_baseline"] = cpu_baseline(xh, errs, args.sample)
        del xh
    # ---- the other configurations, each a bounded run, on the same GPU after the timed regions
    if world == 1 and not args.no_secondary:
        import types
        del gE, X, Xd, Xh
        torch.cuda.empty_cache()
        sub = types.SimpleNamespace(steps=5, warmup=3, oracle_n=256, oracle_n4=48, trials=5)
        sec = {}
        for key, fn in (("bumps1024_bf16", run_bf16_workload), ("tucker160x4_f32", run_tucker4_workload),
                        ("descent256_f32", run_descent_workload)):
            t_s = time.perf_counter()
            try:
                sl = fn(sub)
                sl.pop("clocks", None)
                sl["driver_wall_s"] = time.perf_counter() - t_s
                sec[key] = sl
            except Exception as e:  # a failing side configuration must not hide the main line
                sec[key] = dict(error=repr(e))
            torch.cuda.empty_cache()
        line["secondary"] = sec
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
