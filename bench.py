"""Benchmark of one finite-temperature PEPS-VMC cooling step on GB300.

A step is the whole hot path of one stochastic-reconfiguration step (arXiv:2409.05285,
Sec. II): one Metropolis sweep of every chain, the evaluation of every chain (boundary-MPS
environments, amplitude, E_loc, O rows), and the SR update (weights, gradient, CG solve of
(G + eps) x = g with G applied to the O rows, theta update).

Headline workload (default): 8x8 open Heisenberg J=1, d^2 = 4, D = 4, chi = 16, 8192 chains,
the state after a short cooling run from the perturbed beta = 0 state; tau = 0.02, eps = 1e-4,
CG tolerance 1e-10 relative, at most 100 CG iterations; TF32 tensor-core contractions.  The O
rows (8192 x 10816 values) are larger than L2, so no L2 flush is needed between steps.  The
last warm-up step carries CUDA events around every kernel launch (kernel shares, roofline);
the timed steps run without them.

With --largest 1 (default) the line also carries `largest_workload`: the 10x10 J1-J2 D=6
chi=36 workload at 16384 samples per SR step, one warm-up and one timed step (a step takes
minutes on one GPU, so the headline's step counts do not apply to it).

With --direct the step draws every chain anew by reweighted direct sampling (App. A, Eqs.
A2-A7) instead of a sweep and weights the SR step by r_4 = rho^2 / q: workload direct6, 6x6
Heisenberg D=2 chi=16, 30000 samples per step.  With --serve the serving loop runs a mixed
request stream instead.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on a bounded
sample of the same workload.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PEPS samples/s per SR cooling step (mixed vs FP64 at <=1e-3 E/site); p50/p99 step latency"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
BLOCK_MODES = {"auto": 0, "narrow": 1, "wide": 2, "batched": 3}
# Per-SM issue rates of GB300 (sm_103): 128 FP32 FMA/clk, 2 FP64 FMA/clk; 152 SMs; 2070 MHz.
SMS, MAX_MHZ = 152, 2070.0
SU_TAU = 0.01   # step of the simple-update warm start (--su-warmup)
PEAK_FP32_TFLOPS = 128 * 2 * SMS * MAX_MHZ * 1e6 / 1e12
PEAK_FP64_TFLOPS = 2 * 2 * SMS * MAX_MHZ * 1e6 / 1e12
# dense tensor-core rates of GB300 (nominal, per GPU): TF32 1.1 PFLOP/s against BF16 2.25; a
# TF32 peak is the measured BF16 figure times this ratio
TF32_OVER_BF16 = 1.1 / 2.25

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of the dominant kernel, from one
# ncu capture of the first launches of that kernel in this bench's timed step (the timed region
# is bracketed by cudaProfilerStart/Stop, so `ncu --profile-from-start off` starts there), set
# against the algorithmic bytes of the same launches (`--launch-bytes`),
# stored with the SHA-256 of the kernel and launch-planner sources it was taken on (their code,
# comments excluded).  Once that code changes the entry no longer applies and the bench
# reports null.
NCU_TRAFFIC = {
    ("heis8", "tf32", "kb_gemm_tc"): {
        "chains": 2048,
        "launches": 100,
        "dram_bytes": 6969.22e6,        # DRAM read + write of the first 100 launches of the step
        "alg_bytes": 9975.38e6,         # algorithmic bytes of the same 100 launches
        "sources_sha256": "e7997e742bd0251c6223b3b09e0e0ea0a5c7b20f11f5fde0f50bb44526b564b0",
        "source": "ncu --profile-from-start off --clock-control none --metrics "
                  "dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum "
                  "-k regex:kb_gemm_tc -c 100 (cold cache): the first 100 launches of the timed "
                  "step at 2048 chains (shapes 100,12288,16,16,0), scaled by algorithmic bytes",
    },
    ("j1j2_10", "tf32", "kb_gemm_tc"): {
        "chains": 512,
        "launches": 100,
        "dram_bytes": 38160.7e6,
        "alg_bytes": 41258.7e6,
        "sources_sha256": "e7997e742bd0251c6223b3b09e0e0ea0a5c7b20f11f5fde0f50bb44526b564b0",
        "source": "ncu --profile-from-start off --clock-control none --metrics "
                  "dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum "
                  "-k regex:^kb_gemm_tc$ -c 100 (cold cache): the first 100 launches of the timed "
                  "step at 512 chains (default shapes, no autotune), scaled by algorithmic bytes",
    },
}
TRAFFIC_SOURCES = ("paper_2409_05285_gb300/csrc/pv_tc.cuh", "paper_2409_05285_gb300/csrc/pv_tc2.cuh",
                   "paper_2409_05285_gb300/csrc/pv_batch.cuh")


def code_text(src):
    """C++ source without comments and with whitespace runs collapsed: what the compiler sees
    of it, so that editing a comment does not invalidate a recorded measurement."""
    import re
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    return " ".join(src.split())


def sources_sha256():
    import hashlib
    h = hashlib.sha256()
    for rel in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, rel)) as f:
            h.update(code_text(f.read()).encode())
    return h.hexdigest()


def recorded_traffic(workload, precision, kernel):
    """The capture recorded for this workload and kernel (taken at the chain count it states;
    the DRAM bytes per algorithmic byte carry over to other chain counts of the same launch
    shapes), or None when there is none or the sources changed since it was taken."""
    rec = NCU_TRAFFIC.get((workload, precision, kernel))
    if rec is None or rec["sources_sha256"] != sources_sha256():
        return None
    return rec


def traffic_per_launch(rec, alg_bytes_per_launch):
    """DRAM bytes per launch of the timed steps: the captured launches' DRAM bytes per
    algorithmic byte (the same launches on both sides) times this run's algorithmic bytes per
    launch."""
    return rec["dram_bytes"] / rec["alg_bytes"] * alg_bytes_per_launch


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(ms, device="cuda"):
    """The slowest rank's time (replicas: the job ends when the last rank does)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(n_per_rank, world, ms_per_step):
    """Whole-job samples/s: every rank advances its own n chains per step (weak scaling)."""
    return world * n_per_rank / (ms_per_step / 1e3)


def rank_seed(base, rank):
    """Seed of a replica's chains and initial noise: independent chains on every rank."""
    return base + rank


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"bench_clocks_{os.getpid()}.csv")

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        self.f.close()
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
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f)
    except OSError:
        return {}


def kdelta(cum, base, acc):
    """Adds to `acc` the per-kernel sums accumulated since `base` (both updated in place)."""
    for k, v in cum.items():
        b = base.get(k, (0, 0.0, 0.0, 0.0))
        d = tuple(x - y for x, y in zip(v, b))
        a = acc.get(k, (0, 0.0, 0.0, 0.0))
        acc[k] = tuple(x + y for x, y in zip(a, d))
        base[k] = v
    return acc


def kernel_shares(ks):
    tot = sum(v[1] for v in ks.values()) or 1.0
    return {k: {"launches": v[0], "ms": round(v[1], 3), "share": round(v[1] / tot, 4)}
            for k, v in sorted(ks.items(), key=lambda kv: -kv[1][1]) if v[0] > 0}


def tf32_peak(peaks):
    """TF32 dense peak (TFLOP/s) for a kernel timed inside a long step: the measured sustained
    BF16 rate times the nominal TF32/BF16 ratio, else the recipe's fallback."""
    bf = peaks.get("bf16_tflops_sustained")
    if bf:
        return bf * TF32_OVER_BF16, "measured BF16 sustained %.1f TFLOP/s x %.3f (nominal TF32/BF16)" % (bf, TF32_OVER_BF16)
    return 1700.0 * TF32_OVER_BF16, "fallback BF16 sustained 1700 TFLOP/s x %.3f (nominal TF32/BF16)" % TF32_OVER_BF16


def kernel_roofline(kstats, peaks, prec, binding):
    """Roofline of the dominant kernel from the library's per-launch CUDA events (taken on an
    untimed step): achieved = algorithmic flops (tensor-core contractions) or bytes per launch /
    mean launch time.  The tensor-core contractions (register-staged and cp.async-pipelined)
    are bounded by the tensor pipe (TF32 peak); their HBM view (algorithmic bytes / time
    against the measured copy bandwidth) is given too."""
    total = sum(v[1] for v in kstats.values()) or 1.0
    kernels = {k: {"launches": v[0], "ms": round(v[1], 3), "share": round(v[1] / total, 4),
                   "GB_s": round(v[2] / (v[1] / 1e3) / 1e9, 1) if v[1] > 0 and v[2] > 0 else None,
                   "TFLOP_s": round(v[3] / (v[1] / 1e3) / 1e12, 2) if v[1] > 0 and v[3] > 0 else None}
               for k, v in sorted(kstats.items(), key=lambda kv: -kv[1][1])[:12]}
    if not kstats:
        return None, kernels
    name, (n, ms, nbytes, flops) = max(kstats.items(), key=lambda kv: kv[1][1])
    hbm = peaks.get("hbm_gbs")
    hpeak, hsrc = (hbm, "measured") if hbm else (6800.0, "fallback")
    if name in ("kb_gemm_tc", "kb_gemm_tc2") and flops > 0:
        peak, src = tf32_peak(peaks)
        achieved = flops / n / (ms / n / 1e3) / 1e12
        out = {"kernel": name, "bound": "tensor", "achieved": achieved, "peak": peak,
               "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
               "flops_per_launch": flops / n, "bytes_per_launch": nbytes / n,
               "mean_launch_us": ms / n * 1e3, "launches": n, "share_of_kernel_time": ms / total,
               "peak_source": src}
        if nbytes > 0:
            gbs = nbytes / n / (ms / n / 1e3) / 1e9
            out["hbm_view"] = {"achieved_GB_s": gbs, "peak_GB_s": hpeak, "frac": gbs / hpeak,
                               "peak_source": "%s HBM copy bandwidth (MEASURED_PEAKS.json)" % hsrc}
        return out, kernels
    if name == "kb_trunc" and flops > 0:
        # one-sided Jacobi SVD per chain: FMA-bound (float32, float64 in FP64 mode); its flops
        # are those of the sweeps the matrices took, counted on the device
        peak = PEAK_FP64_TFLOPS if prec == binding.PEPS_FP64 else PEAK_FP32_TFLOPS
        achieved = flops / n / (ms / n / 1e3) / 1e12
        out = {"kernel": name, "bound": "alu", "achieved": achieved, "peak": peak,
               "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
               "flops_per_launch": flops / n, "bytes_per_launch": nbytes / n,
               "mean_launch_us": ms / n * 1e3, "launches": n, "share_of_kernel_time": ms / total,
               "peak_source": "derived: %s FMA/clk/SM x 152 SMs x 2070 MHz" %
                              ("2 FP64" if prec == binding.PEPS_FP64 else "128 FP32")}
        if nbytes > 0:
            gbs = nbytes / n / (ms / n / 1e3) / 1e9
            out["hbm_view"] = {"achieved_GB_s": gbs, "peak_GB_s": hpeak, "frac": gbs / hpeak,
                               "peak_source": "%s HBM copy bandwidth (MEASURED_PEAKS.json)" % hsrc}
        return out, kernels
    if nbytes > 0:
        achieved = nbytes / n / (ms / n / 1e3) / 1e9
        return {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": hpeak,
                "unit": "GB/s", "frac": achieved / hpeak, "traffic": None,
                "bytes_per_launch": nbytes / n, "mean_launch_us": ms / n * 1e3,
                "launches": n, "share_of_kernel_time": ms / total,
                "peak_source": "%s HBM copy bandwidth (MEASURED_PEAKS.json)" % hsrc}, kernels
    peak = PEAK_FP64_TFLOPS if prec == binding.PEPS_FP64 else PEAK_FP32_TFLOPS
    achieved = flops / (ms / 1e3) / 1e12
    return {"kernel": name, "bound": "alu", "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
            "peak_source": "derived: FMA/clk/SM x 152 SMs x 2070 MHz"}, kernels


def workload_config(wl, n, ws):
    """The `config` object both arms report for a workload at n chains per GPU."""
    return {"workload": f"{wl.L}x{wl.L} OBC Heisenberg J1={wl.J1} J2={wl.J2}, d2=4, "
                        f"D={wl.D}, chi={wl.chi}, chains={n} per GPU",
            "global_batch": ws * n, "tau": wl.tau, "eps": wl.eps, "max_cg": wl.max_cg,
            "cg_tol": wl.cg_tol, "parallelism": f"replicas{ws}"}


def cooled_state(ctx, steps, tau, p_switch_t, t_start=0.0):
    """Cools the context for `steps` SR steps from imaginary time t_start (p = 1 while
    beta_obs < 0.3).  Returns the imaginary time reached."""
    t = t_start
    for _ in range(steps):
        p = 1 if 4 * t < p_switch_t else 2
        ctx.step(n_sweeps=1, p=p, tau=tau, eps=1e-4, max_cg=100, cg_tol=1e-10)
        t += tau
    return t


def run_ours(args):
    import numpy as np
    import torch

    from paper_2409_05285_gb300 import binding
    from paper_2409_05285_gb300.build import build
    from paper_2409_05285_gb300.workloads import WORKLOADS

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if rank == 0:
        build()
    if ws > 1:
        torch.distributed.barrier()
    wl = WORKLOADS[args.workload]
    prec = {"fp32": binding.PEPS_FP32, "tf32": binding.PEPS_TF32, "fp64": binding.PEPS_FP64}[args.precision]
    stream = torch.cuda.Stream()
    n = args.chains or wl.n_samples
    ctx = binding.Context(wl.L, wl.L, wl.D, wl.chi, n, J1=wl.J1, J2=wl.J2, precision=prec,
                          init_noise=wl.init_noise, seed=rank_seed(wl.seed, rank), n_blocks=args.blocks,
                          stream=ctypes_stream(stream), block_mode=BLOCK_MODES[args.block_mode])
    if args.cg_product:
        ctx.set_cg_product(args.cg_product)
    if args.graphs and args.block_mode in ("auto", "batched"):
        ctx.set_graphs(True)   # the sweep's and the evaluation's launch sequences as graphs
    t_su = 0.0
    if args.su_warmup > 0:
        # simple-update warm start (host-side, nearest-neighbour bonds) to t = su_warmup
        if wl.J2 != 0.0:
            raise SystemExit("--su-warmup: the simple-update warm start covers J1 bonds only")
        n_su = max(1, int(round(args.su_warmup / SU_TAU)))
        ctx.set_theta(binding.su_theta(wl.L, wl.L, wl.D, wl.J1, SU_TAU, n_su))
        t_su = n_su * SU_TAU
    ctx.mc_sweep(args.burn, p=1 if 4 * t_su < 0.3 else 2)
    t0 = cooled_state(ctx, args.precool, wl.tau, 0.3, t_start=t_su)
    tau, eps, max_cg, tol = wl.tau, wl.eps, wl.max_cg, wl.cg_tol
    p = 2
    ev = lambda: torch.cuda.Event(enable_timing=True)
    for _ in range(args.warmup - 1):
        ctx.step(n_sweeps=1, p=p, tau=tau, eps=eps, max_cg=max_cg, cg_tol=tol)
    # launch shapes tuned on this context's chains, or pinned (results do not depend on them)
    if args.tune:
        ctx.set_tune(*(int(v) for v in args.tune.split(",")))
        tune = ctx.autotune(reps=0)
    elif args.block_mode in ("auto", "batched") and not args.no_autotune:
        tune = ctx.autotune(reps=1)
    else:
        tune = None
    # the last warm-up step: CUDA events around every launch of the context (per-kernel time,
    # algorithmic bytes and flops, per phase) and the algorithmic flop counters; the timed
    # steps below run without them
    kstats, phase_k, prof = profiled_step(ctx, p, tau, eps, max_cg, tol, n)
    clocks = Clocks(local)
    step_ms, mc_ms, eval_ms, sr_ms, cg_its, stats = [], [], [], [], [], []
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    if args.launch_bytes:
        ctx.profile(True, gemm_only=True)
    launches0 = ctx.launches()
    e_start, e_end = ev(), ev()
    torch.cuda.profiler.start()   # the window `ncu --profile-from-start off` captures
    e_start.record(stream)
    for _ in range(args.steps):
        e0, e1, e2, e3 = ev(), ev(), ev(), ev()
        e0.record(stream)
        ctx.mc_sweep(1, p)
        e1.record(stream)
        ctx.eval_chains()
        e2.record(stream)
        st = ctx.sr_step(tau, eps=eps, max_cg=max_cg, cg_tol=tol, p=p)
        e3.record(stream)
        stats.append(st)
        cg_its.append(st["cg_iters"])
        e3.synchronize()
        mc_ms.append(e0.elapsed_time(e1))
        eval_ms.append(e1.elapsed_time(e2))
        sr_ms.append(e2.elapsed_time(e3))
        step_ms.append(e0.elapsed_time(e3))
    e_end.record(stream)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    clk = clocks.stop()
    launches = ctx.launches() - launches0
    if args.launch_bytes:
        # algorithmic bytes of every tensor-core contraction launch of the timed steps, in
        # launch order, to set against a per-launch DRAM capture of the same launches
        with open(args.launch_bytes, "w") as f:
            json.dump({"kernel": "kb_gemm_tc", "steps": args.steps,
                       "bytes": ctx.profile_launch_bytes("kb_gemm_tc")}, f)
        ctx.profile(False)
    total_ms = max_over_ranks(e_start.elapsed_time(e_end))
    ms_per_step = total_ms / args.steps
    samples_per_s = job_throughput(n, ws, ms_per_step)

    # end to end through the public API with host buffers: upload theta and the chain
    # configurations from pinned host memory, run the step, read theta' and S' back.
    th_h = torch.from_numpy(ctx.get_theta()).pin_memory()
    S_h = torch.from_numpy(ctx.get_configs()).pin_memory()
    th_np, S_np = th_h.numpy(), S_h.numpy()
    e2e_ms = []
    for _ in range(max(2, args.steps // 2)):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        ctx.set_theta(th_np)
        ctx.set_configs(S_np)
        ctx.step(n_sweeps=1, p=p, tau=tau, eps=eps, max_cg=max_cg, cg_tol=tol)
        th_np[:] = ctx.get_theta()
        S_np[:] = ctx.get_configs()
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t1) * 1e3)
    e2e_step = statistics.median(e2e_ms)

    fp64_check = None
    if prec != binding.PEPS_FP64 and not args.no_fp64_check:
        fp64_check = compare_fp64(ctx, wl, binding, min(n, args.fp64_chains), stream, torch)
    peaks = measured_peaks()
    roofline, kernels = kernel_roofline(kstats, peaks, prec, binding)
    if roofline is not None:
        rec = recorded_traffic(args.workload, args.precision, roofline["kernel"])
        if rec is not None and roofline.get("bytes_per_launch"):
            roofline["traffic"] = traffic_per_launch(rec, roofline["bytes_per_launch"])
            roofline["traffic_over_algorithmic"] = rec["dram_bytes"] / rec["alg_bytes"]
            roofline["traffic_source"] = rec["source"]
    step_sorted = sorted(step_ms)
    out = {
        "metric": METRIC,
        "value": samples_per_s,
        "unit": "samples/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_per_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {binding.PEPS_FP64: "f64", binding.PEPS_FP32: "f32",
                  binding.PEPS_TF32: "tf32 (contractions; f32 storage, f64 SR)"}[prec],
        "data": "synthetic (seeded beta=0 PEPS cooled in-run; no dataset)",
        "config": dict(workload_config(wl, n, ws), t_start=t0,
                       warm_start=(f"simple update to t={t_su:g} (tau {SU_TAU:g})" if t_su > 0
                                   else "perturbed beta=0 state"),
                       l2="inputs larger than L2 (O rows %.0f MB)" % (n * ctx.No * (8 if prec == 0 else 4) / 1e6)),
        "sr_steps_per_s": ws / (ms_per_step / 1e3),
        "latency_ms": {"p50": step_sorted[len(step_sorted) // 2],
                       "p99": step_sorted[min(len(step_sorted) - 1, int(0.99 * len(step_sorted)))]},
        "phase_ms": {"mc_sweep": statistics.mean(mc_ms), "eval": statistics.mean(eval_ms),
                     "sr_step": statistics.mean(sr_ms)},
        "cg_iters": statistics.mean(cg_its),
        "cg_resid": statistics.mean(st["cg_resid"] for st in stats),
        "sr_step_ms": statistics.mean(sr_ms),
        "eval_gflop_per_sample": prof["eval_flops"] / n / 1e9,
        "sweep_gflop_per_sample": prof["mc_flops"] / n / 1e9,
        "jacobi_sweeps_per_sample": prof["jacobi_sweeps"] / n,
        "E_site": stats[-1]["E_site"], "beta_obs": stats[-1]["beta_obs"] + 4.0 * t_su,
        "roofline": roofline,
        "kernels": kernels,
        "autotune": tune,
        "kernels_by_phase": {ph: kernel_shares(v) for ph, v in phase_k.items()},
        "kernel_stats_from": "one untimed step with CUDA events around every launch (the last warm-up step)",
        "e2e": {"value": ws * n / (e2e_step / 1e3), "unit": "samples/s",
                "h2d_bytes_per_step": int(ctx.Np * 8 + n * ctx.N),
                "d2h_bytes_per_step": int(ctx.Np * 8 + n * ctx.N)},
        "gpu_launches": launches,
        "clocks": clk,
        "fp64_check": fp64_check,
    }
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(wl, n, args.cpu_samples)
    ctx.close()
    if rank == 0 and args.largest and args.workload != "j1j2_10":
        out["largest_workload"] = largest_workload(args, binding, stream, torch, peaks)
    if ws > 1:
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


def profiled_step(ctx, p, tau, eps, max_cg, tol, n):
    """One cooling step with CUDA events around every kernel launch: per-kernel sums (launches,
    ms, algorithmic bytes and flops) over the step and per phase, and the algorithmic flop
    and Jacobi counters of the sweep and the evaluation."""
    ctx.profile(True, gemm_only=False)
    base, phase_k = {}, {"mc_sweep": {}, "eval": {}, "sr_step": {}}
    ctx.mc_sweep(1, p)
    mc_flops = ctx.counters()[0]
    phase_k["mc_sweep"] = kdelta(ctx.profile_read(), base, phase_k["mc_sweep"])
    ctx.eval_chains()
    ev_flops, jsw = ctx.counters()
    phase_k["eval"] = kdelta(ctx.profile_read(), base, phase_k["eval"])
    ctx.sr_step(tau, eps=eps, max_cg=max_cg, cg_tol=tol, p=p)
    phase_k["sr_step"] = kdelta(ctx.profile_read(), base, phase_k["sr_step"])
    ctx.profile(False)
    total = {}
    for ph in phase_k.values():
        for k, v in ph.items():
            a = total.get(k, (0, 0.0, 0.0, 0.0))
            total[k] = tuple(x + y for x, y in zip(a, v))
    return total, phase_k, {"mc_flops": mc_flops, "eval_flops": ev_flops, "jacobi_sweeps": jsw}


def largest_workload(args, binding, stream, torch, peaks):
    """The largest single-GPU workload (10x10 J1-J2 D=6 chi=36, 16384 samples per SR step,
    TF32) measured within a bounded time: one warm-up step (CUDA events around every launch:
    kernel shares and roofline), then one timed step.  One step takes minutes on one GPU, so
    the step counts of the headline line do not apply to it."""
    from paper_2409_05285_gb300.workloads import WORKLOADS
    wl = WORKLOADS["j1j2_10"]
    n = wl.n_samples
    ev = lambda: torch.cuda.Event(enable_timing=True)
    ctx = binding.Context(wl.L, wl.L, wl.D, wl.chi, n, J1=wl.J1, J2=wl.J2, precision=binding.PEPS_TF32,
                          init_noise=wl.init_noise, seed=wl.seed, stream=ctypes_stream(stream))
    if args.graphs:
        ctx.set_graphs(True)
    tau, eps, max_cg, tol = wl.tau, wl.eps, wl.max_cg, wl.cg_tol
    t0 = time.perf_counter()
    kstats, phase_k, prof = profiled_step(ctx, 1, tau, eps, max_cg, tol, n)
    warm_s = time.perf_counter() - t0
    torch.cuda.synchronize()
    e = [ev() for _ in range(4)]
    e[0].record(stream)
    ctx.mc_sweep(1, 1)
    e[1].record(stream)
    ctx.eval_chains()
    e[2].record(stream)
    st = ctx.sr_step(tau, eps=eps, max_cg=max_cg, cg_tol=tol, p=1)
    e[3].record(stream)
    e[3].synchronize()
    ms = e[0].elapsed_time(e[3])
    roofline, kernels = kernel_roofline(kstats, peaks, binding.PEPS_TF32, binding)
    if roofline is not None:
        rec = recorded_traffic("j1j2_10", "tf32", roofline["kernel"])
        if rec is not None and roofline.get("bytes_per_launch"):
            roofline["traffic"] = traffic_per_launch(rec, roofline["bytes_per_launch"])
            roofline["traffic_over_algorithmic"] = rec["dram_bytes"] / rec["alg_bytes"]
            roofline["traffic_source"] = rec["source"]
    fp64 = None
    if not args.no_fp64_check:
        fp64 = compare_fp64(ctx, wl, binding, 64, stream, torch)
    ctx.close()
    out = {"config": workload_config(wl, n, 1), "dtype": "tf32 (contractions; f32 storage, f64 SR)",
           "value": n / (ms / 1e3), "unit": "samples/s", "ms_per_step": ms,
           "sr_steps_per_s": 1e3 / ms, "steps": 1, "warmup": 1, "warmup_s": warm_s,
           "phase_ms": {"mc_sweep": e[0].elapsed_time(e[1]), "eval": e[1].elapsed_time(e[2]),
                        "sr_step": e[2].elapsed_time(e[3])},
           "cg_iters": st["cg_iters"], "E_site": st["E_site"], "beta_obs": st["beta_obs"],
           "eval_gflop_per_sample": prof["eval_flops"] / n / 1e9,
           "sweep_gflop_per_sample": prof["mc_flops"] / n / 1e9,
           "roofline": roofline, "kernels": kernels,
           "kernels_by_phase": {ph: kernel_shares(v) for ph, v in phase_k.items()},
           "fp64_check": fp64,
           "note": "p = 1 sampling from the perturbed beta = 0 state (t < 0.075); one warm-up "
                   "step of 16384 chains (kernel statistics taken on it) and one timed step"}
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(wl, n, 16)
    return out


def compare_fp64(ctx, wl, binding, m, stream, torch):
    """The mixed-precision path against the FP64 path on the same parameters and the same m chain
    configurations: amplitude and local-energy differences, and the evaluation throughput
    of both paths on those configurations."""
    import numpy as np
    th = ctx.get_theta()
    S = np.ascontiguousarray(ctx.get_configs()[:m])
    ref = binding.Context(wl.L, wl.L, wl.D, wl.chi, m, J1=wl.J1, J2=wl.J2,
                          precision=binding.PEPS_FP64, seed=wl.seed,
                          stream=ctypes_stream(stream))
    ref.set_theta(th)
    out = {}
    for name, c in (("mixed", ctx), ("fp64", ref)):
        c.eval_batch(S[: min(m, 8)], with_O=False)   # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        la, sg, es, ea, _ = c.eval_batch(S, with_O=True)
        torch.cuda.synchronize()
        out[name] = (la, sg, es + ea, m / (time.perf_counter() - t0))
    ref.close()
    la32, sg32, e32, r32 = out["mixed"]
    la64, sg64, e64, r64 = out["fp64"]
    N = wl.L * wl.L
    return {"chains": m, "max_abs_dlog_amp": float(np.max(np.abs(la32 - la64))),
            "sign_mismatch": int(np.sum(sg32 != sg64)),
            "E_site_mixed": float(np.mean(e32) / (2 * N)), "E_site_fp64": float(np.mean(e64) / (2 * N)),
            "dE_site": float(abs(np.mean(e32) - np.mean(e64)) / (2 * N)),
            "max_dEloc_site": float(np.max(np.abs(e32 - e64)) / (2 * N)),
            "eval_samples_per_s_mixed": r32, "eval_samples_per_s_fp64": r64,
            "speedup_mixed_over_fp64": r32 / r64}


def ctypes_stream(stream):
    import ctypes
    return ctypes.c_void_p(stream.cuda_stream)


def _oracle_chain(args):
    """One chain of the oracle: a Metropolis sweep then the evaluation (runs in a worker)."""
    L, D, chi, J1, J2, seed, chain, theta = args
    sys.path.insert(0, ROOT)
    import numpy as np
    from oracle import peps, sampler
    from oracle.lattice import Lattice
    lat = Lattice(L, L, D, J1=J1, J2=J2)
    S = peps.init_configs(lat, seed, chain + 1)[chain]
    S, _, _ = sampler.mc_sweep(lat, theta, S, chi, 2, seed, chain, 0)
    r = peps.eval_sample(lat, theta, S, chi)
    return S, r["log_abs"], r["e_sys"], r["e_anc"], r["O"]


def oracle_step(wl, n_samples, pool):
    """The oracle's cooling step on n_samples chains (sweep + evaluation per chain in the
    pool, then the SR update).  Returns seconds."""
    import numpy as np
    from oracle import peps, sr
    from oracle.lattice import Lattice
    lat = Lattice(wl.L, wl.L, wl.D, J1=wl.J1, J2=wl.J2)
    theta = peps.init_theta(lat, wl.seed, wl.init_noise)
    t0 = time.perf_counter()
    res = pool.map(_oracle_chain, [(wl.L, wl.D, wl.chi, wl.J1, wl.J2, wl.seed, c, theta)
                                   for c in range(n_samples)])
    S = np.array([r[0] for r in res])
    la = np.array([r[1] for r in res])
    es = np.array([r[2] for r in res])
    ea = np.array([r[3] for r in res])
    O = np.array([r[4] for r in res])
    sr.sr_step(lat, theta, S, la, es, ea, O, 2, wl.tau, wl.eps, wl.cg_tol, wl.max_cg)
    return time.perf_counter() - t0


def _one_thread_workers():
    # one BLAS thread per worker process: the pool already spans the host cores
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"


def cpu_baseline(wl, n, n_samples):
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    _one_thread_workers()
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        secs = oracle_step(wl, n_samples, pool)
    return {"value": n_samples / secs, "unit": "samples/s", "cores": cores, "kind": "oracle",
            "sample": f"{n_samples} chains of the {wl.L}x{wl.L} D={wl.D} chi={wl.chi} workload: one "
                      f"Metropolis sweep + evaluation each (spawn pool over {cores} host cores), "
                      f"then one SR step on those samples; value = samples / wall time"}


def _oracle_direct_chain(args):
    """One direct draw of the oracle (boundary-MPS form, shared down environments) and its
    evaluation (runs in a worker)."""
    L, D, chi, J1, J2, theta, u, b_d, expo, down = args
    sys.path.insert(0, ROOT)
    from oracle import direct, peps
    from oracle.lattice import Lattice
    lat = Lattice(L, L, D, J1=J1, J2=J2)
    S, lq = direct.draw_bmps(lat, theta, u, chi, b_d, expo, down=down)
    r = peps.eval_sample(lat, theta, S, chi)
    return S, lq, r["log_abs"], r["e_sys"], r["e_anc"], r["O"]


def oracle_direct_step(wl, n_samples, pool, b_d, expo, seed=0):
    """The oracle's cooling step on direct draws: the summed down environments once, then per
    sample a draw and its evaluation in the pool, then the SR update with p = 0 weights.
    Returns seconds."""
    import numpy as np
    from oracle import direct, peps, sr
    from oracle.lattice import Lattice
    lat = Lattice(wl.L, wl.L, wl.D, J1=wl.J1, J2=wl.J2)
    theta = peps.init_theta(lat, wl.seed, wl.init_noise)
    u = np.random.default_rng(seed).random((n_samples, lat.N))
    t0 = time.perf_counter()
    down = direct.summed_down_envs(lat, theta, wl.chi)
    res = pool.map(_oracle_direct_chain, [(wl.L, wl.D, wl.chi, wl.J1, wl.J2, theta, u[k], b_d, expo,
                                           down) for k in range(n_samples)])
    S = np.array([r[0] for r in res])
    lq = np.array([r[1] for r in res])
    la = np.array([r[2] for r in res])
    es = np.array([r[3] for r in res])
    ea = np.array([r[4] for r in res])
    O = np.array([r[5] for r in res])
    sr.sr_step(lat, theta, S, la, es, ea, O, 0, wl.tau, wl.eps, wl.cg_tol, wl.max_cg, log_q=lq)
    return time.perf_counter() - t0


def run_direct(args):
    """Cooling steps on reweighted direct draws (App. A, Eqs. A2-A7): per step every chain is
    replaced by an independent draw (peps_direct_draw, Philox uniforms), evaluated, and the SR
    update takes the p = 0 weights r_4 = rho^2 / q; b_d adapts between steps
    (peps_direct_next_bd).  Workload direct6 (or --workload), TF32 by default."""
    import numpy as np
    import torch

    from paper_2409_05285_gb300 import binding
    from paper_2409_05285_gb300.build import build
    from paper_2409_05285_gb300.workloads import WORKLOADS

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if rank == 0:
        build()
    if ws > 1:
        torch.distributed.barrier()
    wl = WORKLOADS[args.workload if args.workload != "heis8" else "direct6"]
    prec = {"fp32": binding.PEPS_FP32, "tf32": binding.PEPS_TF32, "fp64": binding.PEPS_FP64}[args.precision]
    stream = torch.cuda.Stream()
    n = args.chains or wl.n_samples
    N = wl.L * wl.L
    expo = wl.extra.get("exponent", 0.5)
    ctx = binding.Context(wl.L, wl.L, wl.D, wl.chi, n, J1=wl.J1, J2=wl.J2, precision=prec,
                          init_noise=wl.init_noise, seed=rank_seed(wl.seed, rank),
                          stream=ctypes_stream(stream), block_mode=binding.PEPS_BLOCKS_BATCHED)
    if args.graphs:
        ctx.set_graphs(True)
    su_t = wl.extra.get("su_t", 0.0)
    n_su = int(round(su_t / SU_TAU))
    if n_su > 0:
        ctx.su_warm_start(SU_TAU, n_su)
    tau, eps, max_cg, tol = wl.tau, wl.eps, wl.max_cg, wl.cg_tol
    b_d = wl.extra.get("b_d0", 1.0)
    for _ in range(args.warmup - 1):
        _, b_d = ctx.direct_step(b_d, expo, tau=tau, eps=eps, max_cg=max_cg, cg_tol=tol)
    # the last warm-up step with CUDA events around every launch (per-kernel time, bytes, flops)
    ctx.profile(True, gemm_only=False)
    base, phase_k = {}, {"draw": {}, "eval": {}, "sr_step": {}}
    ctx.direct_draw(None, b_d, expo)
    draw_flops, draw_jsw = ctx.counters()
    phase_k["draw"] = kdelta(ctx.profile_read(), base, phase_k["draw"])
    ctx.eval_chains()
    phase_k["eval"] = kdelta(ctx.profile_read(), base, phase_k["eval"])
    st = ctx.sr_step(tau, eps=eps, max_cg=max_cg, cg_tol=tol, p=0)
    phase_k["sr_step"] = kdelta(ctx.profile_read(), base, phase_k["sr_step"])
    ctx.profile(False)
    b_d = binding.direct_next_bd(b_d, st["diag_frac"], N)
    kstats = {}
    for ph in phase_k.values():
        for k, v in ph.items():
            a = kstats.get(k, (0, 0.0, 0.0, 0.0))
            kstats[k] = tuple(x + y for x, y in zip(a, v))

    ev = lambda: torch.cuda.Event(enable_timing=True)
    clocks = Clocks(local)
    step_ms, draw_ms, eval_ms, sr_ms, stats, bds = [], [], [], [], [], []
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = ctx.launches()
    e_start, e_end = ev(), ev()
    torch.cuda.profiler.start()   # the window `ncu --profile-from-start off` captures
    e_start.record(stream)
    for _ in range(args.steps):
        e0, e1, e2, e3 = ev(), ev(), ev(), ev()
        e0.record(stream)
        ctx.direct_draw(None, b_d, expo)
        e1.record(stream)
        ctx.eval_chains()
        e2.record(stream)
        st = ctx.sr_step(tau, eps=eps, max_cg=max_cg, cg_tol=tol, p=0)
        e3.record(stream)
        e3.synchronize()
        stats.append(st)
        bds.append(b_d)
        b_d = binding.direct_next_bd(b_d, st["diag_frac"], N)
        draw_ms.append(e0.elapsed_time(e1))
        eval_ms.append(e1.elapsed_time(e2))
        sr_ms.append(e2.elapsed_time(e3))
        step_ms.append(e0.elapsed_time(e3))
    e_end.record(stream)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    clk = clocks.stop()
    launches = ctx.launches() - launches0
    total_ms = max_over_ranks(e_start.elapsed_time(e_end))
    ms_per_step = total_ms / args.steps

    # end to end through the public API with host buffers: the step's uniforms from pinned
    # host memory (drawn on the host), log q and the step's statistics read back
    u_h = torch.empty((n, N), dtype=torch.float64).pin_memory()
    u_np = u_h.numpy()
    rng = np.random.default_rng(rank_seed(wl.seed, rank) + 1)
    e2e_ms = []
    for _ in range(max(2, args.steps // 2)):
        u_np[:] = rng.random((n, N))
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        ctx.direct_draw(u_np, b_d, expo)
        ctx.eval_chains()
        st2 = ctx.sr_step(tau, eps=eps, max_cg=max_cg, cg_tol=tol, p=0)
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t1) * 1e3)
        b_d = binding.direct_next_bd(b_d, st2["diag_frac"], N)
    e2e_step = statistics.median(e2e_ms)

    peaks = measured_peaks()
    roofline, kernels = kernel_roofline(kstats, peaks, prec, binding)
    step_sorted = sorted(step_ms)
    out = {
        "metric": "PEPS samples/s per SR cooling step on reweighted direct draws (App. A)",
        "value": job_throughput(n, ws, ms_per_step),
        "unit": "samples/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_per_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {binding.PEPS_FP64: "f64", binding.PEPS_FP32: "f32",
                  binding.PEPS_TF32: "tf32 (contractions; f32 storage, f64 SR)"}[prec],
        "data": "synthetic (seeded beta=0 PEPS cooled in-run; no dataset)",
        "config": {"workload": f"{wl.L}x{wl.L} OBC Heisenberg J1={wl.J1} J2={wl.J2}, d2=4, D={wl.D}, "
                               f"chi={wl.chi} (double layer: bond {wl.D * wl.D}), {n} direct samples "
                               f"per SR step per GPU, exponent {expo}",
                   "global_batch": ws * n, "tau": tau, "eps": eps, "max_cg": max_cg, "cg_tol": tol,
                   "warm_start": (f"simple update to t={n_su * SU_TAU:g} (tau {SU_TAU:g})" if n_su
                                  else "perturbed beta=0 state"),
                   "parallelism": f"replicas{ws}",
                   "l2": "inputs larger than L2 (O rows %.0f MB)" % (n * ctx.No * (8 if prec == 0 else 4) / 1e6)},
        "sr_steps_per_s": ws / (ms_per_step / 1e3),
        "latency_ms": {"p50": step_sorted[len(step_sorted) // 2],
                       "p99": step_sorted[min(len(step_sorted) - 1, int(0.99 * len(step_sorted)))]},
        "phase_ms": {"direct_draw": statistics.mean(draw_ms), "eval": statistics.mean(eval_ms),
                     "sr_step": statistics.mean(sr_ms)},
        "draw_gflop_per_sample": draw_flops / n / 1e9,
        "draw_jacobi_sweeps_per_sample": draw_jsw / n,
        "b_d": bds, "diag_frac": [s_["diag_frac"] for s_ in stats],
        "cg_iters": statistics.mean(s_["cg_iters"] for s_ in stats),
        "E_site": stats[-1]["E_site"], "E_err": stats[-1]["E_err"],
        "beta_obs": stats[-1]["beta_obs"],
        "roofline": roofline,
        "kernels": kernels,
        "kernels_by_phase": {ph: kernel_shares(v) for ph, v in phase_k.items()},
        "kernel_stats_from": "one untimed step with CUDA events around every launch (the last warm-up step)",
        "e2e": {"value": ws * n / (e2e_step / 1e3), "unit": "samples/s",
                "h2d_bytes_per_step": int(n * N * 8), "d2h_bytes_per_step": int(n * 8)},
        "gpu_launches": launches,
        "clocks": clk,
    }
    ctx.close()
    if rank == 0 and not args.no_cpu_baseline:
        import multiprocessing as mp
        cores = os.cpu_count() or 1
        _one_thread_workers()
        with mp.get_context("spawn").Pool(cores) as pool:
            m = max(args.cpu_samples, 150 * cores)   # ~10-20 s of oracle work
            secs = oracle_direct_step(wl, m, pool, bds[-1], expo)
        out["cpu_baseline"] = {"value": m / secs, "unit": "samples/s", "cores": cores, "kind": "oracle",
                               "sample": f"{m} direct samples of the {wl.L}x{wl.L} D={wl.D} chi={wl.chi} "
                                         f"workload: summed down environments once, a boundary-MPS draw "
                                         f"+ evaluation per sample (spawn pool over {cores} host cores), "
                                         f"then one SR step with p = 0 weights; value = samples / wall time"}
    if ws > 1:
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    import multiprocessing as mp
    from paper_2409_05285_gb300.workloads import WORKLOADS
    wl = WORKLOADS[args.workload]
    cores = os.cpu_count() or 1
    _one_thread_workers()
    ctx = mp.get_context("spawn")
    n_s = args.cpu_samples
    with ctx.Pool(cores) as pool:
        for _ in range(args.warmup):
            oracle_step(wl, min(n_s, cores), pool)
        times = [oracle_step(wl, n_s, pool) for _ in range(args.steps)]
    ms = 1e3 * statistics.mean(times)
    v = n_s / (ms / 1e3)
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "samples/s", "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": workload_config(wl, args.chains or wl.n_samples, ws),
           "cpu_baseline": {"value": v, "unit": "samples/s", "cores": cores, "kind": "oracle",
                            "sample": f"{n_s} of the workload's chains per timed step: one sweep + "
                                      f"evaluation each, then one SR step on them"},
           "e2e": {"value": v, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def serve_stream(seed, rate, window):
    """The mixed request stream of the serving workload: Poisson arrivals at `rate` per s over
    `window` s; per request L in {4, 6, 8, 10, 12}, D in {2, 4, 6}, chi = D^2, J1 = 1,
    J2 ~ U[0, 0.6], t_end ~ U[0.5, 4] (beta_obs = 4 t_end)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    out, t = [], 0.0
    while True:
        t += rng.exponential(1.0 / rate)
        if t > window:
            break
        L = int(rng.choice([4, 6, 8, 10, 12]))
        D = int(rng.choice([2, 4, 6]))
        out.append((t, dict(L1=L, L2=L, D=D, chi=D * D, J2=float(rng.uniform(0.0, 0.6)),
                            t_end=float(rng.uniform(0.5, 4.0)), seed=int(rng.integers(1 << 30)))))
    return out


def run_serve(args):
    """Serving loop under the mixed request stream (serve_stream): requests arrive at `--rate`
    per s over `--window` s and are admitted by device-memory footprint (at most --max-active
    running, each on its own context and stream); after `--duration` s from the first
    arrival the server is stopped (queued requests cancelled, running ones end after their
    current step).  Per-step latency p50/p99 and aggregate samples/s are over every step that
    finished; a request of this stream runs for tens to hundreds of SR steps of up to seconds
    each, far beyond a bounded measurement, so most requests are still running or queued when
    it ends."""
    import numpy as np
    import torch

    from paper_2409_05285_gb300 import binding
    from paper_2409_05285_gb300.build import build
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    build()
    arrivals = serve_stream(args.seed, args.rate, args.window)
    srv = binding.Server(max_active=args.max_active)
    t0 = time.perf_counter()
    ids, geo = [], {}
    for ta, kw in arrivals:
        d = ta - (time.perf_counter() - t0)
        if d > 0:
            time.sleep(d)
        if time.perf_counter() - t0 > args.duration:
            break
        rid = srv.submit(precision=binding.PEPS_TF32, n_chains=args.serve_chains, tau=args.serve_tau, **kw)
        ids.append(rid)
        geo[rid] = (kw["L1"], kw["D"])
    rest = args.duration - (time.perf_counter() - t0)
    if rest > 0:
        time.sleep(rest)
    srv.stop()
    srv.drain()
    wall = time.perf_counter() - t0
    m = srv.metrics()
    states = {}
    per_geo = {}
    for rid in ids:
        st, steps = srv.poll(rid)
        states[st] = states.get(st, 0) + 1
        g = "L%d_D%d" % geo[rid]
        per_geo.setdefault(g, 0)
        per_geo[g] += len(steps)
    srv.close()
    names = {binding.PEPS_REQ_DONE: "done", binding.PEPS_REQ_CANCELLED: "cancelled",
             binding.PEPS_REQ_FAILED: "failed", binding.PEPS_REQ_QUEUED: "queued",
             binding.PEPS_REQ_RUNNING: "running"}
    out = {"metric": "serving: per-SR-step latency p50/p99 and aggregate samples/s under a "
                     "Poisson stream of cooling requests", "value": m["samples_per_s"],
           "unit": "samples/s", "n_gpus": 1, "latency_ms": {"p50": m["p50_ms"], "p99": m["p99_ms"]},
           "steps": m["steps"], "requests": len(ids), "wall_s": wall, "higher_is_better": True,
           "request_states": {names.get(k, str(k)): v for k, v in states.items()},
           "steps_by_geometry": per_geo, "dtype": "tf32", "data": "synthetic",
           "config": {"workload": f"Poisson arrivals {args.rate}/s over {args.window} s, seed "
                                  f"{args.seed}; L in {{4,6,8,10,12}}, D in {{2,4,6}}, chi=D^2, "
                                  f"J1=1, J2~U[0,0.6], t_end~U[0.5,4]; {args.serve_chains} samples "
                                  f"per SR step, tau={args.serve_tau}",
                      "max_active": args.max_active, "measured_for_s": args.duration}}
    print(json.dumps(out))


def compare_fp64_fermion(f, wl, binding, theta, S, m, stream):
    """The fermionic mixed-precision path against the FP64 path on the same parameters and the
    same m configurations: amplitude and local-energy differences, and the evaluation
    throughput (amplitudes and local energies) of both paths."""
    import numpy as np
    t_hop, U, mu = wl.extra["t"], wl.extra["U"], wl.extra["mu"]
    S = np.ascontiguousarray(S[:m])
    ref = binding.FermionAmplitudes(wl.L, wl.L, wl.D, wl.chi, m, precision=binding.PEPS_FP64,
                                    stream=ctypes_stream(stream))
    out = {}
    for name, g in (("mixed", f), ("fp64", ref)):
        g.local_energy(theta, S[: min(m, 8)], t_hop, U, mu)    # warm-up
        t0 = time.perf_counter()
        la, sg, es, ea = g.local_energy(theta, S, t_hop, U, mu)
        out[name] = (la, sg, es + ea, m / (time.perf_counter() - t0))
    ref.close()
    la32, sg32, e32, r32 = out["mixed"]
    la64, sg64, e64, r64 = out["fp64"]
    N = wl.L * wl.L
    return {"chains": m, "max_abs_dlog_amp": float(np.max(np.abs(la32 - la64))),
            "sign_mismatch": int(np.sum(sg32 != sg64)),
            "E_site_mixed": float(np.mean(e32) / (2 * N)), "E_site_fp64": float(np.mean(e64) / (2 * N)),
            "dE_site": float(abs(np.mean(e32) - np.mean(e64)) / (2 * N)),
            "max_dEloc_site": float(np.max(np.abs(e32 - e64)) / (2 * N)),
            "eval_samples_per_s_mixed": r32, "eval_samples_per_s_fp64": r64,
            "speedup_mixed_over_fp64": r32 / r64}


def l2_flusher(stream):
    """A function that writes a 256 MB device buffer (twice the 129 MB L2) on `stream`."""
    import torch
    buf = torch.empty(64 << 20, dtype=torch.float32, device="cuda")

    def flush():
        with torch.cuda.stream(stream):
            buf.fill_(1.0)
    return flush


def _oracle_fermion_amps(args):
    """Amplitudes of a few configurations by the oracle's exact row-vector contraction of the
    signed slices (runs in a worker).  Returns (seconds, evaluations)."""
    L, D, theta, S_list = args
    sys.path.insert(0, ROOT)
    import numpy as np
    from oracle import fermion as fm
    from oracle import fermion_vmc as fv
    from paper_2409_05285_gb300.workloads import site_dims
    like = [np.zeros((16,) + d) for d in site_dims(L, L, D)]
    t0 = time.perf_counter()
    amp = fm.fpeps_amplitude_function(L, L, fv.unflatten(theta, like))
    for S in S_list:
        amp(S)
    return time.perf_counter() - t0, len(S_list)


def oracle_fermion_baseline(wl, theta, S, per_worker=6):
    """The oracle's cost per sample of the fermionic step, from a bounded sample: amplitude
    evaluations (exact row-vector contraction) timed in a spawn pool over the host cores, and
    the evaluations one sample needs (the proposals of a sweep that apply at its
    configuration, its allowed hops for E_loc, its own amplitude) counted with the oracle's
    move set.  The oracle's O rows (a sum over every virtual assignment) are left out."""
    import multiprocessing as mp
    from oracle import fermion_vmc as fv
    cores = os.cpu_count() or 1
    _one_thread_workers()
    moves = fv.moves(wl.L, wl.L)
    evals = []
    for x in S[:64]:
        app = [fv.propose(x, m) is not None for m in moves]
        hops = sum(a for a, m in zip(app, moves) if m[0] == "hop")
        evals.append(sum(app) + hops + 1)
    per_sample = float(sum(evals)) / len(evals)
    jobs = [(wl.L, wl.D, theta, [S[(w * per_worker + k) % len(S)] for k in range(per_worker)])
            for w in range(cores)]
    with mp.get_context("spawn").Pool(cores) as pool:
        pool.map(_oracle_fermion_amps, jobs[:1])          # workers warm (imports)
        t0 = time.perf_counter()
        res = pool.map(_oracle_fermion_amps, jobs)
        wall = time.perf_counter() - t0
    n_eval = sum(r[1] for r in res)
    return {"value": n_eval / wall / per_sample, "unit": "samples/s", "cores": cores,
            "kind": "oracle",
            "sample": f"{n_eval} amplitude evaluations of the {wl.L}x{wl.L} D={wl.D} workload by the "
                      f"oracle's exact row-vector contraction ({per_worker} per worker, spawn pool over "
                      f"{cores} host cores, {wall:.1f} s), scaled by {per_sample:.1f} evaluations per "
                      f"sample (applicable proposals of a sweep + allowed hops + 1); the oracle's O "
                      f"rows and SR solve are not included (a lower bound on its cost)"}


def run_fermion(args):
    """Cooling steps of the fermionic thermal state (Sec. III.B: Hubbard t = 1, U = 8, mu = 4
    on 6x6 OBC; fermionic PEPS of sixteen local states, D = 4, chi = 16): per step one
    Metropolis sweep of every chain (peps_famp_sweep: pair and hop proposals, each proposal's
    amplitude a full boundary-MPS contraction of the signed slices) and one SR step
    (peps_famp_sr_step: local energies, O rows, weights, CG, update), from the perturbed |I>
    (peps_famp_init_theta).  p = 1 while beta_obs < 0.3, then p = 2.  TF32 by default."""
    import numpy as np
    import torch

    from paper_2409_05285_gb300 import binding
    from paper_2409_05285_gb300.build import build
    from paper_2409_05285_gb300.workloads import WORKLOADS, fermion_support_configs

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if rank == 0:
        build()
    if ws > 1:
        torch.distributed.barrier()
    wl = WORKLOADS[args.workload if args.workload != "heis8" else "hubbard6"]
    if "U" not in wl.extra:
        raise SystemExit("--fermion needs a Hubbard workload (hubbard6, hubbard8), not " + wl.name)
    prec = {"fp32": binding.PEPS_FP32, "tf32": binding.PEPS_TF32, "fp64": binding.PEPS_FP64}[args.precision]
    stream = torch.cuda.Stream()
    n = args.chains or wl.n_samples
    N = wl.L * wl.L
    t_hop, U, mu = wl.extra["t"], wl.extra["U"], wl.extra["mu"]
    tau, eps, max_cg, tol = wl.tau, wl.eps, wl.max_cg, wl.cg_tol
    f = binding.FermionAmplitudes(wl.L, wl.L, wl.D, wl.chi, n, precision=prec,
                                  stream=ctypes_stream(stream))
    theta = binding.famp_init_theta(wl.L, wl.L, wl.D, wl.init_noise, rank_seed(wl.seed, rank))
    theta0 = theta.copy()
    S = fermion_support_configs(n, N, rank_seed(wl.seed, rank) + 1)
    seed = rank_seed(wl.seed, rank) + 2
    state = {"sweep": 0, "t": 0.0}

    def step(theta, S, profile=None):
        p = 1 if 4 * state["t"] < 0.3 else 2
        S, acc, _, _ = f.sweep(theta, S, p=p, n_sweeps=1, seed=seed, sweep0=state["sweep"])
        if profile is not None:
            profile["sweep"] = kdelta(f.profile_read(), profile["base"], profile["sweep"])
        theta, st = f.sr_step(theta, S, t_hop, U, mu, p=p, tau=tau, eps=eps, max_cg=max_cg, cg_tol=tol)
        if profile is not None:
            profile["sr_step"] = kdelta(f.profile_read(), profile["base"], profile["sr_step"])
        state["sweep"] += 1
        state["t"] += tau
        st["p"] = p
        st["accept"] = float(acc.sum()) / (n * f.n_moves)
        return theta, S, st

    S, _, _, _ = f.sweep(theta, S, p=1, n_sweeps=args.burn, seed=seed, sweep0=0)
    state["sweep"] = args.burn
    for _ in range(args.warmup - 1):
        theta, S, _ = step(theta, S)
    # the last warm-up step with CUDA events around every launch (per-kernel time, bytes, flops)
    f.profile(True)
    prof = {"base": {}, "sweep": {}, "sr_step": {}}
    theta, S, _ = step(theta, S, prof)
    f.profile(False)
    kstats = {}
    for ph in ("sweep", "sr_step"):
        for k, v in prof[ph].items():
            a = kstats.get(k, (0, 0.0, 0.0, 0.0))
            kstats[k] = tuple(x + y for x, y in zip(a, v))

    ev = lambda: torch.cuda.Event(enable_timing=True)
    clocks = Clocks(local)
    step_ms, sweep_ms, sr_ms, stats = [], [], [], []
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = f.launches()
    flush = l2_flusher(stream)
    torch.cuda.profiler.start()
    for _ in range(args.steps):
        e0, e1, e2 = ev(), ev(), ev()
        p = 1 if 4 * state["t"] < 0.3 else 2
        flush()
        e0.record(stream)
        S, acc, _, _ = f.sweep(theta, S, p=p, n_sweeps=1, seed=seed, sweep0=state["sweep"])
        e1.record(stream)
        theta, st = f.sr_step(theta, S, t_hop, U, mu, p=p, tau=tau, eps=eps, max_cg=max_cg, cg_tol=tol)
        e2.record(stream)
        e2.synchronize()
        state["sweep"] += 1
        state["t"] += tau
        st["p"] = p
        st["accept"] = float(acc.sum()) / (n * f.n_moves)
        stats.append(st)
        sweep_ms.append(e0.elapsed_time(e1))
        sr_ms.append(e1.elapsed_time(e2))
        step_ms.append(e0.elapsed_time(e2))
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    clk = clocks.stop()
    launches = f.launches() - launches0
    del flush
    total_ms = max_over_ranks(sum(step_ms))
    ms_per_step = total_ms / args.steps

    # end to end through the public API: each step's host theta and configurations copied in
    # (pinned host buffers), the updated theta, configurations and statistics read back
    th_h = torch.empty(theta.size, dtype=torch.float64).pin_memory().numpy()
    S_h = torch.empty(S.shape, dtype=torch.uint8).pin_memory().numpy()
    th_h[:] = theta
    S_h[:] = S
    e2e_ms = []
    for _ in range(max(2, args.steps // 2)):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        p = 1 if 4 * state["t"] < 0.3 else 2
        S2, _, _, _ = f.sweep(th_h, S_h, p=p, n_sweeps=1, seed=seed, sweep0=state["sweep"])
        th2, _ = f.sr_step(th_h, S2, t_hop, U, mu, p=p, tau=tau, eps=eps, max_cg=max_cg, cg_tol=tol)
        e2e_ms.append((time.perf_counter() - t1) * 1e3)
        th_h[:] = th2
        S_h[:] = S2
        state["sweep"] += 1
        state["t"] += tau
    e2e_step = statistics.median(e2e_ms)
    fp64_check = None
    if prec != binding.PEPS_FP64 and not args.no_fp64_check:
        fp64_check = compare_fp64_fermion(f, wl, binding, theta, S, min(n, args.fp64_chains), stream)
    np_ = theta.size
    h2d = 2 * np_ * 8 + 2 * n * N
    d2h = n * N + n * (4 + 8 + 1) + np_ * 8

    peaks = measured_peaks()
    roofline, kernels = kernel_roofline(kstats, peaks, prec, binding)
    step_sorted = sorted(step_ms)
    out = {
        "metric": "fermionic PEPS samples/s per SR cooling step (Metropolis sweep + SR, Hubbard)",
        "value": job_throughput(n, ws, ms_per_step),
        "unit": "samples/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_per_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {binding.PEPS_FP64: "f64", binding.PEPS_FP32: "f32",
                  binding.PEPS_TF32: "tf32 (contractions; f32 storage, f64 SR)"}[prec],
        "data": "synthetic (seeded perturbed |I> cooled in-run; no dataset)",
        "config": {"workload": f"{wl.L}x{wl.L} OBC Fermi-Hubbard t={t_hop} U={U} mu={mu}, d2=16 "
                               f"(fermionic PEPS), D={wl.D}, chi={wl.chi}, {n} Metropolis chains per GPU",
                   "global_batch": ws * n, "tau": tau, "eps": eps, "max_cg": max_cg, "cg_tol": tol,
                   "moves_per_sweep": f.n_moves, "parallelism": f"replicas{ws}",
                   "l2": "L2 flushed before every timed step (a 256 MB buffer written outside the "
                         "step's events; O rows %.0f MB)" % (n * (np_ // 16) * (8 if prec == binding.PEPS_FP64 else 4) / 1e6)},
        "sr_steps_per_s": ws / (ms_per_step / 1e3),
        "latency_ms": {"p50": step_sorted[len(step_sorted) // 2],
                       "p99": step_sorted[min(len(step_sorted) - 1, int(0.99 * len(step_sorted)))]},
        "phase_ms": {"sweep": statistics.mean(sweep_ms), "sr_step": statistics.mean(sr_ms)},
        "accept": statistics.mean(s_["accept"] for s_ in stats),
        "cg_iters": statistics.mean(s_["cg_iters"] for s_ in stats),
        "E_site": stats[-1]["E_site"], "E_err": stats[-1]["E_err"], "docc": stats[-1]["docc"],
        "density": stats[-1]["density"], "beta_obs": 4 * (state["t"] - tau * len(e2e_ms)),
        "fp64_check": fp64_check,
        "roofline": roofline,
        "kernels": kernels,
        "kernels_by_phase": {ph: kernel_shares(prof[ph]) for ph in ("sweep", "sr_step")},
        "kernel_stats_from": "one untimed step with CUDA events around every launch (the last warm-up step)",
        "e2e": {"value": ws * n / (e2e_step / 1e3), "unit": "samples/s",
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": launches,
        "clocks": clk,
    }
    f.close()
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = oracle_fermion_baseline(wl, theta0, S)
    if ws > 1:
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="heis8")
    ap.add_argument("--precision", default="tf32", choices=["fp32", "tf32", "fp64"])
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch shapes of the batched engine")
    ap.add_argument("--chains", type=int, default=0)
    ap.add_argument("--blocks", type=int, default=0, help="persistent blocks of the sample kernels (0 = auto)")
    ap.add_argument("--block-mode", default="auto", choices=list(BLOCK_MODES))
    ap.add_argument("--burn", type=int, default=2)
    ap.add_argument("--precool", type=int, default=2)
    ap.add_argument("--cpu-samples", type=int, default=32)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-check", action="store_true")
    ap.add_argument("--serve", action="store_true", help="serving-loop benchmark instead")
    ap.add_argument("--direct", action="store_true",
                    help="cooling steps on reweighted direct draws (workload direct6) instead")
    ap.add_argument("--fermion", action="store_true",
                    help="fermionic cooling steps (Hubbard, workload hubbard6) instead")
    ap.add_argument("--rate", type=float, default=20.0)
    ap.add_argument("--window", type=float, default=10.0, help="serving: arrival window (s)")
    ap.add_argument("--duration", type=float, default=60.0, help="serving: measured time (s)")
    ap.add_argument("--serve-chains", type=int, default=1024, help="serving: samples per SR step")
    ap.add_argument("--serve-tau", type=float, default=0.02, help="serving: imaginary-time step")
    ap.add_argument("--max-active", type=int, default=4)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--fp64-chains", type=int, default=608)
    ap.add_argument("--su-warmup", type=float, default=0.0,
                    help="start from the simple-update state at this imaginary time (J1 workloads)")
    ap.add_argument("--tune", default="",
                    help="pin the launch shapes instead of autotuning: grid_pct,db_bytes,ffma_g,kc_max[,pipelined]")
    ap.add_argument("--cg-product", type=int, default=0, choices=[0, 1, 2, 3],
                    help="CG product form: 0 automatic, 1 fused single read, 2 two passes")
    ap.add_argument("--graphs", type=int, default=1, choices=[0, 1],
                    help="replay the batched engine's launch sequences as CUDA graphs")
    ap.add_argument("--largest", type=int, default=1,
                    help="also measure the 10x10 D=6 chi=36 workload at 16384 samples (1 warm-up + 1 timed step)")
    ap.add_argument("--launch-bytes", default="",
                    help="write the per-launch algorithmic bytes of kb_gemm_tc in the timed steps to this file")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        run_reference(args)
    elif args.serve:
        run_serve(args)
    elif args.direct:
        run_direct(args)
    elif args.fermion:
        run_fermion(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
