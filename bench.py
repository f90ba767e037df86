"""Benchmark: Wiener-filter solves per second at Nside 1024 (lmax 2048) with
the hybrid dual messenger (Algorithm 2), to 1e-6 relative accuracy.

One step = one complete solve of one map, inputs resident in HBM, with the
mixed solver's default options: every cooling stage in FP32 transforms in
correction form around FP64 anchors (double-float Legendre steps), the
re-anchoring bound tied to the stage tolerance, and the tail stages
(mu <= alpha) iterated in double-float; each stage ends on the paper's
Cauchy criterion (Sect. 3).  The result reproduces the plain FP64 solve of
the same map (same stage lengths; its distance is reported).  Workload:
synthetic Gaussian sky with C_l = 1/(l(l+1)) b_l^2 (3-pixel beam), ecliptic
scan noise with hits 1-100, sigma0 set for signal-to-noise one at l = 1000,
25% mask (galactic band + 500 discs of 0.5 deg).  The data map is
synthesised on the GPU by the library's own alm2map.

Multi-GPU (torchrun, one process per GPU): independent maps per rank (weak
scaling, no collective on the data path); value = all ranks' solves / max
time over ranks.  --impl reference times the CPU oracle (plain FP64 direct
transforms) on a bounded sample of the same workload.
"""
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

METRIC = "WF solves/s to 1e-6 rel at Nside 1024"
UNIT = "solves/s"
# iterations of the plain FP64 solve of this workload (measured on the GPU:
# the FP64 oracle would take the same path), used to scale the oracle's
# per-iteration cost in the reference arm
REF_ITERATIONS = {1024: 2048, 256: 4216}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nside", type=int, default=1024)
    ap.add_argument("--eps", type=float, default=1e-6)
    ap.add_argument("--no-fp64", action="store_true",
                    help="skip the plain FP64 solve used for the comparison")
    ap.add_argument("--cpu-sample-s", type=float, default=15.0)
    ap.add_argument("--kernel-case", choices=["legendre32", "legendre64", "legendre_df64"],
                    default=None,
                    help="run only the Legendre kernels of one transform pair "
                         "(small case for profiling) and exit")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--train-maps", type=int, default=64)
    ap.add_argument("--eval-maps", type=int, default=8)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--net-channels", type=int, default=16,
                    help="learned: channels of the per-ring convolutions (<= 32)")
    ap.add_argument("--net-kernel", type=int, default=9,
                    help="learned: odd convolution width (<= 15)")
    ap.add_argument("--net-hidden", type=int, default=32,
                    help="learned: width of the l-feature MLP (<= 64)")
    ap.add_argument("--profile-solve", action="store_true",
                    help="one warm-up solve, then one solve inside the NVTX range "
                         "'solve' (for a bounded profiler launch list) and exit")
    ap.add_argument("--group-maps", type=int, default=64,
                    help="group_sht: maps per grouped transform pair")
    ap.add_argument("--workload", choices=["nside1024", "batch64", "learned", "flat512",
                                           "group_sht"],
                    default="nside1024",
                    help="batch64: 64 maps, Nside drawn from {64, 128, 256}, solved "
                         "together (maps/s); group_sht: the grouped tensor-core "
                         "transforms of --group-maps maps at --nside (256 unless given)")
    return ap.parse_args()


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if len(r) > 8 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 8 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            if len(r) > 8:
                for n, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(n)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            with open(path) as f:
                return json.load(f), "measured"
        except (OSError, ValueError):
            pass
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# DRAM bytes (read + write, ncu) of one full-band launch of the FP32 analysis
# variant the autotuner picks at Nside 1024 / lmax 2048 (an ncu capture of
# the --kernel-case legendre32 run); scaled to a live launch by its share
# of the full band's terms.  None once the kernel changes after a capture,
# and for a plan whose autotuner picked another analysis variant.
ANALYSIS_DRAM_FULL_BAND = {"nside": 1024, "bytes": 213754624.0,
                           "terms": 3140761977.0,
                           "variant": {"ana_np": 4, "ana_queue": 0, "ana_packed": 1,
                                       "ana_global_acc": 1},
                           "source": "ncu --set full, one full-band launch of the kernel "
                                     "case (dram__bytes_read.sum 137.4 MB + "
                                     "dram__bytes_write.sum 76.4 MB)"}


def analysis_variant(tuning):
    """The FP32 analysis launch variant of a plan's tuning report."""
    return {"ana_np": tuning["ana_np"][1], "ana_queue": tuning["ana_queue"],
            "ana_packed": tuning["ana_packed"], "ana_global_acc": tuning["ana_global_acc"]}


def analysis_traffic(nside, gflop, launches, variant=None):
    """Bytes per live analysis launch from the captured full-band figure."""
    ref = ANALYSIS_DRAM_FULL_BAND
    if ref["bytes"] is None or nside != ref["nside"] or not launches:
        return None
    if variant is not None and variant != ref["variant"]:
        return None
    terms_per_launch = gflop * 1e9 / 7.0 / launches
    return ref["bytes"] * terms_per_launch / ref["terms"]


def alu_peaks(wf):
    """FMA-pipe peaks measured on this device (wf_alu_peak: FMA chains in
    every thread of a grid filling every SM, fastest of 5 launches): FP32
    (the larger of scalar and packed f32x2) and FP64, in TFLOP/s, and the SM
    count the device reports."""
    f64, _, sms = wf.wf_alu_peak(0, 5)
    f32, _, _ = wf.wf_alu_peak(1, 5)
    f32x2, _, _ = wf.wf_alu_peak(2, 5)
    return {"fp32_tflops": max(f32, f32x2), "fp32_scalar_tflops": f32,
            "fp32_packed_tflops": f32x2, "fp64_tflops": f64, "num_sms": sms,
            "source": "measured live: wf_alu_peak FMA chains on every SM, best of 5"}


# FP32 flops of the double-float formulas per (l, m, ring pair) term: the
# recurrence step (product c u, product by z, difference: 28 with an FMA
# counted as 2) and two accumulations of a product (15 each)
DD_FLOPS_PER_TERM = 58.0
KERNEL_NAMES = ["legendre_analysis_f32", "legendre_synthesis_f32", "ring_step_f32",
                "legendre_synthesis_dd", "legendre_analysis_dd", "ring_step_dd"]


def kernel_rooflines(kern, alu, peaks, peak_src, args, ana_variant):
    """Per-kernel rooflines of the timed solves (wf_kernel_stats, CUDA events
    around every launch) and the dominant kernel's at the top level.
    Legendre kernels: 7 algorithmic flops per term against the measured FP32
    FMA peak (the double-float ones: the 58 FP32 flops of their formulas per
    term against the same peak, and their FP64-equivalent 7 flops per term
    beside the measured FP64 peak); ring steps: DRAM bytes they cannot avoid
    against the measured copy bandwidth."""
    total = sum(k["ms"] for k in kern) or 1.0
    rows = []
    for i, (k, name) in enumerate(zip(kern, KERNEL_NAMES)):
        if not k["ms"]:
            continue
        ms = k["ms"] / max(1, k["launches"])
        if i in (2, 5):
            r = ring_roofline(k, peaks, peak_src)
        else:
            g = k["gflop"] * (DD_FLOPS_PER_TERM / 7.0 if i in (3, 4) else 1.0)
            ach = g / (k["ms"] / 1e3) / 1e3
            r = {"bound": "alu", "achieved": ach, "peak": alu["fp32_tflops"],
                 "unit": "TFLOP/s", "frac": ach / alu["fp32_tflops"],
                 "peak_source": alu["source"] + f" ({alu['num_sms']} SMs), FP32 FMA pipe",
                 "avg_launch_ms": ms}
            if i in (3, 4):
                e = k["gflop"] / (k["ms"] / 1e3) / 1e3
                r["flops_per_term"] = DD_FLOPS_PER_TERM
                r["fp64_equivalent"] = {"achieved": e, "fp64_peak": alu["fp64_tflops"],
                                        "ratio": e / alu["fp64_tflops"]}
        r.update({"kernel": name, "launches": k["launches"], "time_share": k["ms"] / total})
        rows.append(r)
    top = dict(max(rows, key=lambda r: r["time_share"])) if rows else {}
    if top.get("kernel") == "legendre_analysis_f32":
        top["traffic"] = analysis_traffic(args.nside, kern[0]["gflop"], kern[0]["launches"],
                                          ana_variant)
        top["traffic_source"] = ANALYSIS_DRAM_FULL_BAND["source"]
        top["variant"] = ana_variant
    else:
        top.setdefault("traffic", None)
        top["traffic_source"] = "see profiles/ (one-kernel ncu captures)"
    top["kernels"] = rows
    return top


def ring_roofline(k, peaks, peak_src):
    """HBM roofline of the ring step (fold, ring FFTs, t-update): algorithmic
    bytes (ring coefficients in and out, d and sigma^2) per timed launch pair
    over its CUDA-event time."""
    if not k["ms"]:
        return None
    gbs = k["gbytes"] / (k["ms"] / 1e3)
    return {"bound": "hbm", "achieved": gbs, "unit": "GB/s", "peak": peaks["hbm_gbs"],
            "frac": gbs / peaks["hbm_gbs"], "peak_source": peak_src,
            "avg_launch_ms": k["ms"] / max(1, k["launches"]),
            "bytes_per_launch": k["gbytes"] * 1e9 / max(1, k["launches"])}


# ---------------------------------------------------------------- workload
def make_workload(nside, seed):
    import numpy as np
    import torch
    from paper_1702_08852_gb300 import inputs, wf
    p = inputs.scan_problem(nside, seed=seed, mask_fraction=0.25, discs=500,
                            disc_radius_deg=0.5, ell_star=min(1000, nside))
    dev = torch.device("cuda", torch.cuda.current_device())
    nv = torch.from_numpy(p.noise_var).to(dev)
    mk = torch.from_numpy(p.mask.astype(np.uint8)).to(dev)
    with wf.Plan(p.nside, p.lmax, p.cl) as tp:
        s = tp.alm2map(torch.from_numpy(p.alm_true).to(dev))
    d = s + torch.from_numpy(p.noise).to(dev)
    d[torch.from_numpy(p.mask).to(dev)] = 0.0
    return p, nv, mk, d


def max_over_ranks(value, dist=None, device=None):
    """The slowest rank's time (the contract's max over ranks)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_value(world, steps, total_ms):
    """Whole-job solves/s: every rank solved `steps` maps; the job took the
    slowest rank's time."""
    return world * steps / (total_ms / 1e3)


def flush_l2(buf):
    buf.add_(1.0)


# ---------------------------------------------------------------- our arm
def run_ours(args, rank, world):
    import numpy as np
    import torch
    from paper_1702_08852_gb300 import wf
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    alu = alu_peaks(wf)
    p, nv, mk, d = make_workload(args.nside, seed=3000 + rank)
    plan = wf.Plan(p.nside, p.lmax, p.cl, nv, mk, precision=wf.WF_PREC_MIXED,
                   eps_final=args.eps, timing=1, autotune=1)
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2
    for _ in range(args.warmup):
        alm, mp, st = plan.solve(d)
    for k in range(6):
        plan.kernel_stats(k, reset=True)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(dev.index)
    clocks.start()
    step_ms, stats = [], []
    for _ in range(args.steps):
        flush_l2(flush)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        alm, mp, st = plan.solve(d)
        e1.record(stream)
        torch.cuda.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        stats.append(st)
    clk = clocks.stop()
    total_ms = max_over_ranks(sum(step_ms), dist, dev)
    kern = [plan.kernel_stats(k) for k in range(6)]
    ana_variant = analysis_variant(plan.tuning())
    ms_step_mean = sum(step_ms) / len(step_ms)

    # end to end through the C ABI with host buffers (pinned)
    d_host = torch.empty(d.numel(), dtype=torch.float64, pin_memory=True)
    d_host.copy_(d.cpu())
    e2e_s = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        a_h, _, _ = plan.solve_host(d_host.numpy(), want_alm=True, want_map=False)
        e2e_s.append(time.perf_counter() - t0)

    # plain FP64 dual messenger on the same map (rank 0): the comparison the
    # speedup is quoted against, and the mixed result's distance from it;
    # beside it the mixed solver's fast configuration on the same map
    fp64, fast, cfg2, methods, flat, group = {}, {}, {}, {}, {}, {}
    if rank == 0 and not args.no_fp64:
        p64 = wf.Plan(p.nside, p.lmax, p.cl, nv, mk, precision=wf.WF_PREC_FP64,
                      eps_final=args.eps, timing=1, autotune=1)
        flush_l2(flush)
        a64, m64, s64 = p64.solve(d)
        k64 = [p64.kernel_stats(k) for k in (0, 1)]
        fp64 = {"solve_s": s64["elapsed_ms"] / 1e3, "iterations": s64["iterations"],
                "stages": s64["stages"], "solves_per_s": 1e3 / s64["elapsed_ms"],
                "final_cauchy": s64["final_cauchy"],
                "mixed_vs_fp64_rel_l2": float(torch.linalg.norm(mp - m64) /
                                               torch.linalg.norm(m64)),
                "speedup_mixed_over_fp64": (s64["elapsed_ms"] / 1e3) / (ms_step_mean / 1e3),
                "legendre_analysis_f64": {"ms": k64[0]["ms"], "gflop": k64[0]["gflop"],
                                          "tflops": k64[0]["gflop"] / k64[0]["ms"]
                                          if k64[0]["ms"] else None},
                "legendre_synthesis_f64": {"ms": k64[1]["ms"], "gflop": k64[1]["gflop"],
                                           "tflops": k64[1]["gflop"] / k64[1]["ms"]
                                           if k64[1]["ms"] else None}}
        for k in ("legendre_analysis_f64", "legendre_synthesis_f64"):
            t = fp64[k]["tflops"]
            fp64[k]["frac_of_fp64_peak"] = t / alu["fp64_tflops"] if t else None
        p64.close()
        fast = fast_mode(wf, p, nv, mk, d, m64, s64, args)
        cfg2 = config2(wf, args)
        methods = methods_comparison(wf, args)
        flat = flat_sky(wf, args)
        group = run_group(argparse.Namespace(nside=256, group_maps=64, steps=5, warmup=3),
                          0, 1)
    plan.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank != 0:
        return None

    ms_per_step = total_ms / args.steps
    value = aggregate_value(world, args.steps, total_ms)
    peaks, peak_src = measured_peaks()
    iters = [s["iterations"] for s in stats]
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 transforms; anchors and tail stages: double-float Legendre and ring FFTs",
        "data": "synthetic",
        "config": {"workload": f"Nside {args.nside} lmax {2 * args.nside} scan-noise "
                               f"25% mask, 1 map per GPU",
                   "global_batch": world, "nside": args.nside, "lmax": 2 * args.nside,
                   "eps": args.eps, "precision": "mixed",
                   "l2": "256 MB buffer written between timed steps; working set > L2",
                   "parallelism": f"replicas x{world}"},
        "solve": {"iterations_mean": sum(iters) / len(iters), "stages": stats[-1]["stages"],
                  "anchors": stats[-1]["refinements"],
                  "criterion": "last-stage Cauchy ratio < eps (Sect. 3); FP64 step from "
                               "the result passes it too",
                  "mode": "default mixed options: every stage anchored, re-anchoring "
                          "bound 100 eps_k, tail stages (mu <= alpha) in double-float",
                  "fp64_cauchy_of_result": stats[-1]["fp_residual"],
                  "converged": stats[-1]["converged"]},
        "roofline": kernel_rooflines(kern, alu, peaks, peak_src, args, ana_variant),
        "clocks": clk,
        "e2e": {"value": 1.0 / (sum(e2e_s) / len(e2e_s)), "unit": UNIT,
                "h2d_bytes_per_step": 8 * 12 * args.nside ** 2,
                "d2h_bytes_per_step": 16 * (2 * args.nside + 1) * (2 * args.nside + 2) // 2},
        "gpu_launches": None,
        "plain_fp64": fp64,
        "fast_mode": fast,
        "nside256": cfg2,
        "methods_nside256": methods,
        "flat_sky_512": flat,
        "group_sht_nside256": {k: group.get(k) for k in (
            "metric", "value", "unit", "ms_per_step", "per_map_f32", "speedup_vs_per_map_f32",
            "contraction", "vs_fp64_rel_l2", "table_build_s")} if group else {},
        "peaks": {"hbm_gbs": peaks.get("hbm_gbs"), "source": peak_src, "alu": alu},
    }
    out["gpu_launches"] = int(sum(s["kernel_launches"] for s in stats))
    out["cpu_baseline"] = cpu_baseline(args, iters[-1])
    return out


FAST_OPTS = {"anchor_eps": 3e-5, "anchor_cap_tol": 0.0, "tail_exact": 0}


def fast_mode(wf, p, nv, mk, d, m64, s64, args, reps=3):
    """The mixed solver's fast configuration (FP32 stages down to tolerance
    3e-5, then anchored; FP32 tail) on the same map: solves/s and its
    distance from the FP64 result (not the 1e-6 target: its late-stage
    Cauchy tests can end a stage an iteration or two off)."""
    import torch
    plan = wf.Plan(p.nside, p.lmax, p.cl, nv, mk, precision=wf.WF_PREC_MIXED,
                   eps_final=args.eps, autotune=1, **FAST_OPTS)
    plan.solve(d)
    ts = []
    for _ in range(reps):
        _, mp, st = plan.solve(d)
        ts.append(st["elapsed_ms"] / 1e3)
    plan.close()
    t = sum(ts) / len(ts)
    return {"options": FAST_OPTS, "solves_per_s": 1.0 / t, "solve_s": t,
            "iterations": st["iterations"],
            "vs_fp64_rel_l2": float(torch.linalg.norm(mp - m64) / torch.linalg.norm(m64)),
            "speedup_over_fp64": (s64["elapsed_ms"] / 1e3) / t}


def config2(wf, args, reps=3):
    """Nside 256 / lmax 512 scan workload: plain FP64 next to the mixed
    solver (default options), solves/s and the distance between them."""
    import torch
    p, nv, mk, d = make_workload(256, seed=3100)
    out = {"workload": "Nside 256 lmax 512 scan-noise 25% mask"}
    p64 = wf.Plan(p.nside, p.lmax, p.cl, nv, mk, precision=wf.WF_PREC_FP64,
                  eps_final=args.eps, autotune=1)
    _, m64, s64 = p64.solve(d)
    p64.close()
    pm = wf.Plan(p.nside, p.lmax, p.cl, nv, mk, precision=wf.WF_PREC_MIXED,
                 eps_final=args.eps, autotune=1)
    pm.solve(d)
    ts = []
    for _ in range(reps):
        _, mm, sm = pm.solve(d)
        ts.append(sm["elapsed_ms"] / 1e3)
    pm.close()
    t = sum(ts) / len(ts)
    out.update({"fp64_solve_s": s64["elapsed_ms"] / 1e3, "fp64_iterations": s64["iterations"],
                "mixed_solve_s": t, "mixed_solves_per_s": 1.0 / t,
                "mixed_iterations": sm["iterations"],
                "mixed_vs_fp64_rel_l2": float(torch.linalg.norm(mm - m64) /
                                              torch.linalg.norm(m64)),
                "speedup_mixed_over_fp64": (s64["elapsed_ms"] / 1e3) / t})
    return out


PAPER_FLAT_DM_S = 258.0  # Sect. 4: one core of an Intel Core i5-4690, 512^2, eps 1e-6


def flat_sky(wf, args, reps=5):
    """The paper's own workload (Sect. 3): 512^2 flat sky of 10 deg, white
    noise 64 muK^2, central 5 deg square at 10^6 N, analytic spectrum in
    place of CAMB; Algorithm 2 with 2-D FFTs to the Cauchy criterion eps.
    Reported beside the paper's 258 s (its hardware; context only)."""
    import numpy as np
    import torch
    from paper_1702_08852_gb300 import inputs
    n = 512
    side = np.deg2rad(10.0)
    om = (side / n) ** 2
    ck = inputs.flat_cl(inputs.flat_mode_ell(n, side))
    nv, _ = inputs.flat_paper_noise(n)
    rng = np.random.default_rng(4000)
    d = inputs.flat_gaussian_field(rng, ck, om) + np.sqrt(nv) * rng.standard_normal((n, n))
    dev = torch.device("cuda", torch.cuda.current_device())
    with wf.FlatPlan(n, om, ck, torch.from_numpy(nv).to(dev), eps_final=args.eps) as fp:
        dd = torch.from_numpy(d).to(dev)
        fp.solve(dd)
        ts = []
        for _ in range(reps):
            _, st = fp.solve(dd)
            ts.append(st["elapsed_ms"] / 1e3)
    t = min(ts)
    return {"workload": "flat sky 512^2, L = 10 deg, 64 muK^2, 5 deg square at 1e6 N",
            "solve_s": t, "solves_per_s": 1.0 / t, "iterations": st["iterations"],
            "stages": st["stages"], "us_per_iteration": 1e6 * t / st["iterations"],
            "kernel_launches": st["kernel_launches"],
            "paper_cpu_s": PAPER_FLAT_DM_S,
            "speedup_vs_paper_cpu": PAPER_FLAT_DM_S / t,
            "note": "the paper's time is its own CPU and CAMB spectrum: context, not a target"}


def methods_comparison(wf, args):
    """The paper's three-way comparison (Sect. 4) on the Nside 256 scan
    workload, each method to its own Cauchy criterion eps (FP64 transforms):
    the dual messenger (Algorithm 2), the standard messenger (Algorithm 1,
    lambda from 1e4 by 3/4, three-step tolerances) and PCG with the
    harmonic-diagonal preconditioner (App. C, restart 200); iterations, time
    and the App. C residual of each result."""
    p, nv, mk, d = make_workload(256, seed=3100)
    out = {"workload": "Nside 256 lmax 512 scan-noise 25% mask, FP64 transforms"}
    for name, kw in (("dual_messenger", {}),
                     ("standard_messenger", {"method": wf.WF_METHOD_MESSENGER})):
        pl = wf.Plan(p.nside, p.lmax, p.cl, nv, mk, precision=wf.WF_PREC_FP64,
                     eps_final=args.eps, autotune=1, **kw)
        alm, _, st = pl.solve(d, want_map=False)
        res = pl.residual(d, alm)
        out[name] = {"solve_s": st["elapsed_ms"] / 1e3, "iterations": st["iterations"],
                     "stages": st["stages"], "rel_res_wf": res["rel_res_wf"]}
        pl.close()
    pl = wf.Plan(p.nside, p.lmax, p.cl, nv, mk, autotune=1)
    alm, _, st = pl.pcg(d, tol=args.eps, stop_rule=wf.WF_PCG_STOP_CAUCHY, restart=200,
                        want_map=False)
    res = pl.residual(d, alm)
    out["pcg"] = {"solve_s": st["elapsed_ms"] / 1e3, "iterations": st["iterations"],
                  "converged": st["converged"], "rel_res_wf": res["rel_res_wf"]}
    pl.close()
    return out


# ---------------------------------------------------------------- oracle
class OracleSampler:
    """Times the oracle's direct FP64 transforms on bounded samples of the
    Nside workload: synthesis of k pixels and analysis of k coefficients,
    scaled to one transform pair.  The inputs are drawn once; each call of
    step() is one timed sample sized to its budget."""

    def __init__(self, nside):
        import numpy as np
        from oracle import sht
        from paper_1702_08852_gb300 import inputs
        self.sht, self.nside, self.lmax = sht, nside, 2 * nside
        cl = inputs.cl_spectrum(self.lmax, nside)
        self.rng = np.random.default_rng(1)
        self.a = inputs.random_alm(self.rng, np.maximum(cl, 1e-30))
        self.npix = 12 * nside * nside
        self.m = self.rng.standard_normal(self.npix)
        self.ls, self.ms = inputs.lm_of_slots(self.lmax)
        sht.lib()
        # calibration: seconds per pixel and per coefficient on a tiny sample
        self.t_pix, self.t_mode = self._time(8, 4)

    def _time(self, kp, ka):
        t0 = time.perf_counter()
        self.sht.alm2map_pixels(self.a, self.nside, self.lmax,
                                self.rng.integers(0, self.npix, kp))
        t_pix = (time.perf_counter() - t0) / kp
        sel = self.rng.integers(0, len(self.ls), ka)
        t0 = time.perf_counter()
        self.sht.adjoint_modes(self.m, self.nside, self.lmax, self.ls[sel], self.ms[sel])
        t_mode = (time.perf_counter() - t0) / ka
        return t_pix, t_mode

    def step(self, budget_s):
        """(seconds per SHT pair, description) from one sample of ~budget_s."""
        unit = 8 * self.t_pix + 4 * self.t_mode
        scale = max(1, int(budget_s / max(unit, 1e-4)))
        kp, ka = 8 * scale, 4 * scale
        t_pix, t_mode = self._time(kp, ka)
        self.t_pix, self.t_mode = t_pix, t_mode  # sizes the next sample
        pair_s = t_pix * self.npix + t_mode * len(self.ls)
        sample = (f"direct synthesis of {kp} pixels and analysis of {ka} coefficients "
                  f"at Nside {self.nside}, scaled to one transform pair ({pair_s:.3g} s)")
        return pair_s, sample

    def threads(self):
        return self.sht.threads()


def oracle_sample(nside, budget_s):
    """One bounded sample: (seconds per SHT pair, sample, threads)."""
    s = OracleSampler(nside)
    s.step(min(0.5, budget_s / 10))  # untimed: warms up and sizes the sample
    pair_s, sample = s.step(budget_s / 2)
    return pair_s, sample, s.threads()


def cpu_baseline(args, iterations):
    try:
        pair_s, sample, threads = oracle_sample(args.nside, args.cpu_sample_s)
    except Exception as e:  # the oracle is a measurement here, not the product
        return {"value": None, "unit": UNIT, "cores": None, "kind": "oracle",
                "sample": f"failed: {e}"}
    solve_s = pair_s * iterations
    return {"value": 1.0 / solve_s, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": sample + f"; x {iterations} iterations of the GPU solve "
                               "(extrapolated)"}


def run_reference(args, rank, world):
    """The oracle, as it stands, on the host cores: each step one timed
    bounded sample of the workload's transform pair, times the iteration
    count of the plain FP64 solve (the cpu_sample_s budget is split over
    the steps; warm-up samples are untimed).  Rank 0 only."""
    if rank != 0:
        return None
    t0 = time.perf_counter()
    sampler = OracleSampler(args.nside)
    per_step = max(0.5, args.cpu_sample_s / max(1, args.steps))
    for _ in range(args.warmup):
        sampler.step(min(0.5, per_step))
    iterations = REF_ITERATIONS.get(args.nside, 2048)
    steps_s, wall_s, sample = [], [], ""
    for _ in range(args.steps):
        t1 = time.perf_counter()
        pair_s, sample = sampler.step(per_step)
        wall_s.append(time.perf_counter() - t1)
        steps_s.append(pair_s * iterations)
    threads = sampler.threads()
    value = args.steps / sum(steps_s)
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(steps_s) / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"Nside {args.nside} lmax {2 * args.nside}, oracle "
                                   "direct transforms", "nside": args.nside},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads,
                             "kind": "oracle", "sample": f"{args.steps} samples, the last: " +
                             sample + f"; x {iterations} iterations (extrapolated)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "extrapolated": "ms_per_step is one whole solve: the timed sample's time per "
                            "transform pair x the FP64 solve's iterations",
            "measured_ms_per_step": 1e3 * sum(wall_s) / args.steps,
            "wall_s": time.perf_counter() - t0}


def run_batch(args, rank, world):
    """64 independent maps (Nside 64/128/256 drawn per map, lmax = 2 Nside,
    amplitude A x U[0.5, 2], scan noise, mask 5-40 %) solved together with
    wf_solve_batch; one step = the whole batch."""
    import numpy as np
    import torch
    from paper_1702_08852_gb300 import inputs, wf
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    probs = inputs.batch_problems(64, seed_base=3000 + 1000 * rank)
    plans, ds = [], []
    for p in probs:
        nv = torch.from_numpy(p.noise_var).to(dev)
        mk = torch.from_numpy(p.mask.astype(np.uint8)).to(dev)
        plan = wf.Plan(p.nside, p.lmax, p.cl, nv, mk, precision=wf.WF_PREC_MIXED,
                       eps_final=args.eps, autotune=1)
        s = plan.alm2map(torch.from_numpy(p.alm_true).to(dev))
        d = s + torch.from_numpy(p.noise).to(dev)
        d[torch.from_numpy(p.mask).to(dev)] = 0.0
        plans.append(plan)
        ds.append(d)
    for _ in range(args.warmup):
        wf.wf_solve_batch(plans, ds, want_alm=False)
    torch.cuda.synchronize()
    clocks = ClockSampler(dev.index)
    clocks.start()
    times, stats = [], None
    for _ in range(args.steps):
        t0 = time.perf_counter()
        alms, _, stats, ms = wf.wf_solve_batch(plans, ds, want_alm=True)
        times.append(ms)
    clk = clocks.stop()
    # each map's distance from its own plain FP64 solve (untimed)
    rels = []
    if not args.no_fp64:
        for p, plan, d, a in zip(probs, plans, ds, alms):
            nv = torch.from_numpy(p.noise_var).to(dev)
            mk = torch.from_numpy(p.mask.astype(np.uint8)).to(dev)
            with wf.Plan(p.nside, p.lmax, p.cl, nv, mk, precision=wf.WF_PREC_FP64,
                         eps_final=args.eps, autotune=1) as p64:
                _, m64, _ = p64.solve(d)
                mm = plan.alm2map(a)
            rels.append(float(torch.linalg.norm(mm - m64) / torch.linalg.norm(m64)))
    for p in plans:
        p.close()
    total_ms = max_over_ranks(sum(times))
    if rank != 0:
        return None
    nmaps = len(probs)
    ns = [p.nside for p in probs]
    return {"metric": "maps/s, 64-map batch (Nside 64/128/256), to 1e-6 (Cauchy)",
            "value": world * nmaps * args.steps / (total_ms / 1e3), "unit": "maps/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 transforms; anchors and tail stages: double-float Legendre and ring FFTs",
            "data": "synthetic",
            "config": {"workload": "64 maps, Nside in {64,128,256}, lmax = 2 Nside, "
                                   "scan noise, mask 5-40 %",
                       "nside_counts": {str(k): ns.count(k) for k in (64, 128, 256)}},
            "per_map": {"iterations_max": max(s["iterations"] for s in stats),
                        "iterations_mean": sum(s["iterations"] for s in stats) / nmaps,
                        "fp64_cauchy_max": max(s["fp_residual"] for s in stats),
                        "converged": sum(s["converged"] for s in stats),
                        "vs_fp64_rel_l2_max": max(rels) if rels else None,
                        "vs_fp64_rel_l2_mean": sum(rels) / len(rels) if rels else None},
            "gpu_launches": int(sum(s["kernel_launches"] for s in stats)),
            "clocks": clk}


def run_learned(args, rank, world):
    """Learned warm start at Nside 256 (lmax 512): train the network on
    solutions of the plain solver for --train-maps seeds of the Nside-256
    scan workload, then compare cold and warm solves on --eval-maps held-out
    seeds (iterations, time, fallback, agreement)."""
    import numpy as np
    import torch
    from paper_1702_08852_gb300 import inputs, wf, learned
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    ns = 256
    H, K, Hm = args.net_channels, args.net_kernel, args.net_hidden
    t_start = time.perf_counter()

    def make(seed):
        p = inputs.scan_problem(ns, seed=seed, mask_fraction=0.25, discs=500,
                                disc_radius_deg=0.5)
        nv = torch.from_numpy(p.noise_var).to(dev)
        mk = torch.from_numpy(p.mask.astype(np.uint8)).to(dev)
        return p, nv, mk

    samples = []
    gen_plan = None
    for i in range(args.train_maps):
        p, nv, mk = make(5000 + i)
        if gen_plan is None:
            gen_plan = wf.Plan(p.nside, p.lmax, p.cl, nv, mk, precision=wf.WF_PREC_MIXED,
                               eps_final=args.eps)
        else:
            gen_plan.set_noise(nv, mk)
            gen_plan.set_cl(p.cl)
        s = gen_plan.alm2map(torch.from_numpy(p.alm_true).to(dev))
        d = s + torch.from_numpy(p.noise).to(dev)
        d[torch.from_numpy(p.mask).to(dev)] = 0.0
        a, _, _ = gen_plan.solve(d, want_map=False)
        samples.append((nv, mk, p.cl, d, a))
    t_gen = time.perf_counter() - t_start
    net = wf.Net(gen_plan, H, K, Hm, bf16=True)
    net.set_params(learned.init_params(H, K, Hm, seed=0))
    t0 = time.perf_counter()
    hist = learned.train(net, samples, epochs=args.epochs, lr=2e-3)
    t_train = time.perf_counter() - t0
    theta = net.get_params()
    rows = []
    for i in range(args.eval_maps):
        p, nv, mk = make(9000 + i)
        gen_plan.set_noise(nv, mk)
        gen_plan.set_cl(p.cl)
        s = gen_plan.alm2map(torch.from_numpy(p.alm_true).to(dev))
        d = s + torch.from_numpy(p.noise).to(dev)
        d[torch.from_numpy(p.mask).to(dev)] = 0.0
        alpha = float(np.min(p.noise_var[~p.mask]))
        cold = wf.Plan(p.nside, p.lmax, p.cl, nv, mk, precision=wf.WF_PREC_MIXED,
                       eps_final=args.eps)
        warm = wf.Plan(p.nside, p.lmax, p.cl, nv, mk, precision=wf.WF_PREC_MIXED,
                       eps_final=args.eps, mu0=30.0 * alpha)
        wnet = wf.Net(warm, H, K, Hm, bf16=True)
        wnet.set_params(theta)
        cold.solve(d, want_map=False)          # warm-up (graph capture)
        learned.warm_solve(wnet, warm, d, cold_plan=cold)
        torch.cuda.synchronize()
        tc = time.perf_counter()
        ac, mc, sc = cold.solve(d)
        torch.cuda.synchronize()
        tc = time.perf_counter() - tc
        tw = time.perf_counter()
        aw, mw, sw, used, res = learned.warm_solve(wnet, warm, d, cold_plan=cold)
        torch.cuda.synchronize()
        tw = time.perf_counter() - tw
        rows.append({"cold_iterations": sc["iterations"], "cold_s": tc,
                     "warm_iterations": sw["iterations"], "warm_s": tw, "used_warm": used,
                     "warm_start_residual": res,
                     "warm_vs_cold_rel_l2": float(torch.linalg.norm(mw - mc) /
                                                  torch.linalg.norm(mc)),
                     "warm_fp64_cauchy": sw["fp_residual"]})
        wnet.close()
        cold.close()
        warm.close()
    net.close()
    gen_plan.close()
    if rank != 0:
        return None
    ci = sum(r["cold_iterations"] for r in rows) / len(rows)
    wi = sum(r["warm_iterations"] for r in rows) / len(rows)
    ct = sum(r["cold_s"] for r in rows) / len(rows)
    wt = sum(r["warm_s"] for r in rows) / len(rows)
    return {"metric": "learned warm start, Nside 256: held-out iterations and time to the "
                      "1e-6 criterion, warm vs cold",
            "value": ct / wt, "unit": "x (cold time / warm time)", "n_gpus": world,
            "higher_is_better": True, "data": "synthetic",
            "config": {"workload": "Nside 256 lmax 512 scan noise 25 % mask",
                       "train_maps": args.train_maps, "eval_maps": args.eval_maps,
                       "epochs": args.epochs, "net": {"channels": H, "kernel": K,
                                                      "hidden": Hm, "params": len(theta),
                                                      "weights": "bf16 (fp32 master)"},
                       "warm_mu0": "30 alpha"},
            "train": {"loss_first_epoch": hist[0], "loss_last_epoch": hist[-1],
                      "data_gen_s": t_gen, "train_s": t_train},
            "eval": {"cold_iterations_mean": ci, "warm_iterations_mean": wi,
                     "cold_s_mean": ct, "warm_s_mean": wt,
                     "fallbacks": sum(1 for r in rows if not r["used_warm"]),
                     "per_map": rows}}


def run_group(args, rank, world):
    """The grouped transforms: --group-maps maps of one geometry (Nside 256,
    lmax 512 unless --nside is given), one step = alm2map_group then
    map2alm_group of the whole group; beside it the per-map FP32 transforms
    of the same maps, and the tensor-core contraction's own roofline."""
    import numpy as np
    import torch
    from paper_1702_08852_gb300 import inputs, wf
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    ns = args.nside if args.nside != 1024 else 256
    lm, nm = 2 * ns, args.group_maps
    cl = inputs.cl_spectrum(lm, ns)
    rng = np.random.default_rng(4000 + rank)
    a = np.stack([inputs.random_alm(rng, np.maximum(cl, 1e-30)) for _ in range(nm)])
    a *= rng.uniform(0.5, 2.0, nm)[:, None]
    peaks, peak_src = measured_peaks()
    with wf.Plan(ns, lm, cl, autotune=1) as p:
        ad = torch.from_numpy(a).to(dev)
        t0 = time.perf_counter()
        mg = p.alm2map_group(ad)          # builds the tables
        build_s = time.perf_counter() - t0
        ag = p.map2alm_group(mg)
        for _ in range(args.warmup):
            p.alm2map_group(ad, mg)
            p.map2alm_group(mg, ag)
        p.group_stats(reset=True)
        torch.cuda.synchronize()
        clocks = ClockSampler(dev.index)
        clocks.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            p.alm2map_group(ad, mg)
            p.map2alm_group(mg, ag)
        e1.record()
        torch.cuda.synchronize()
        clk = clocks.stop()
        ms = e0.elapsed_time(e1)
        gs = p.group_stats(reset=True)
        # per-map FP32 transforms of the same maps (the solver's single-map path)
        m1, a1 = p.alm2map_f32(ad[0]), p.map2alm_f32(mg[0])
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record()
        for b in range(nm):
            p.alm2map_f32(ad[b], m1)
            p.map2alm_f32(mg[b], a1)
        f1.record()
        torch.cuda.synchronize()
        ms_f32 = f0.elapsed_time(f1)
        # accuracy against the per-map FP64 transforms (untimed, 8 maps)
        es, ea = [], []
        for b in range(0, nm, max(1, nm // 8)):
            mf = p.alm2map(ad[b])
            es.append(float(torch.linalg.norm(mg[b] - mf) / torch.linalg.norm(mf)))
            af = p.map2alm(mf)
            ag1 = p.map2alm_group(mf.unsqueeze(0))[0]
            ea.append(float(torch.linalg.norm(ag1 - af) / torch.linalg.norm(af)))
    total_ms = max_over_ranks(ms)
    if rank != 0:
        return None
    k_ms = gs["ms"] / max(gs["launches"], 1)
    gbps = gs["gbytes"] / (gs["ms"] * 1e-3)
    tflops = 3 * gs["gflop"] / (gs["ms"] * 1e-3) * 1e-3    # the 3 split products
    tf32_peak = 0.5 * peaks["bf16_tflops"]
    roof_h = {"bound": "hbm", "achieved": gbps, "peak": peaks["hbm_gbs"], "unit": "GB/s",
              "frac": gbps / peaks["hbm_gbs"], "traffic": None,
              "kernel": "k_group_mma (tcgen05 3xTF32)", "peak_source": peak_src,
              "algorithmic_gbytes_per_launch": gs["gbytes"] / max(gs["launches"], 1)}
    roof_t = {"bound": "tensor", "achieved": tflops, "peak": tf32_peak, "unit": "TFLOP/s",
              "frac": tflops / tf32_peak,
              "peak_source": "TF32 dense = 0.5 x the measured bf16 burst (nominal ratio)"}
    roof = roof_h if roof_h["frac"] >= roof_t["frac"] else roof_t
    steps_pairs = world * nm * args.steps
    return {"metric": f"map transform pairs/s (alm2map + map2alm), group of {nm} maps "
                      f"at Nside {ns}",
            "value": steps_pairs / (total_ms / 1e3), "unit": "pairs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "3xTF32 products, FP32 accumulation (tcgen05); FP32 ring FFTs",
            "data": "synthetic",
            "config": {"workload": f"{nm} band-limited maps, Nside {ns}, lmax {lm}",
                       "l2": "inputs larger than L2 (maps and coefficients of the group)"},
            "per_map_f32": {"pairs_per_s": nm / (ms_f32 / 1e3),
                            "ms_per_pair": ms_f32 / nm},
            "speedup_vs_per_map_f32": (ms_f32 / nm) / (total_ms / args.steps / nm),
            "contraction": {"ms_per_launch": k_ms, "launches": gs["launches"],
                            "share_of_step": gs["ms"] / total_ms,
                            "hbm": roof_h, "tensor": roof_t},
            "roofline": roof,
            "table_build_s": build_s,
            "vs_fp64_rel_l2": {"synthesis_max": max(es), "analysis_max": max(ea)},
            "gpu_launches": args.steps * (4 + 4),
            "clocks": clk}


def run_kernel_case(args):
    """One FP32 (or FP64) synthesis + analysis pair at full band on a random
    band-limited field, repeated --reps times; prints the event timings."""
    import numpy as np
    import torch
    from paper_1702_08852_gb300 import inputs, wf
    ns = args.nside
    lm = 2 * ns
    cl = inputs.cl_spectrum(lm, ns)
    a = torch.from_numpy(inputs.random_alm(np.random.default_rng(5),
                                           np.maximum(cl, 1e-30))).cuda()
    out = {}
    with wf.Plan(ns, lm, cl, autotune=1) as p:
        kc = args.kernel_case
        syn = {"legendre32": p.alm2map_f32, "legendre_df64": p.alm2map_df64}.get(kc, p.alm2map)
        ana = {"legendre32": p.map2alm_f32, "legendre_df64": p.map2alm_df64}.get(kc, p.map2alm)
        m = syn(a)
        b = ana(m)
        torch.cuda.synchronize()
        # the timed launches sit in an NVTX range (profilers can select them
        # with --nvtx-include "kernel_case/")
        torch.cuda.nvtx.range_push("kernel_case")
        for name, fn, arg, o in (("synthesis", syn, a, m), ("analysis", ana, m, b)):
            ts = []
            for _ in range(args.reps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                fn(arg, o)
                e1.record()
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            out[name + "_ms"] = min(ts)
        torch.cuda.nvtx.range_pop()
        out["terms"] = p.legendre_terms()
        t = p.tuning()
        out["variants"] = {k: t[k] for k in ("syn_np", "syn_packed", "ana_np", "ana_queue",
                                              "ana_packed")}
    print(json.dumps({"kernel_case": args.kernel_case, "nside": ns, **out}))


def run_profile_solve(args):
    """The timed configuration's solve, once untimed, then once inside the
    NVTX range 'solve' (profilers select its launches with --nvtx-include
    "solve/")."""
    import torch
    from paper_1702_08852_gb300 import wf
    p, nv, mk, d = make_workload(args.nside, seed=3000)
    plan = wf.Plan(p.nside, p.lmax, p.cl, nv, mk, precision=wf.WF_PREC_MIXED,
                   eps_final=args.eps, autotune=1)
    plan.solve(d)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("solve")
    _, _, st = plan.solve(d)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    plan.close()
    print(json.dumps({"profile_solve": args.nside, "iterations": st["iterations"],
                      "kernel_launches": st["kernel_launches"],
                      "solve_ms": st["elapsed_ms"]}))


def main():
    args = parse()
    # more hardware work queues than the default 8, so that the batch's
    # per-map streams do not share queues (read when the CUDA context is
    # created, i.e. before the first CUDA call of this process)
    os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
    if args.kernel_case:
        run_kernel_case(args)
        return
    if args.profile_solve:
        run_profile_solve(args)
        return
    if args.workload == "flat512" and args.impl != "reference":
        import torch
        from paper_1702_08852_gb300 import wf
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        print(json.dumps(flat_sky(wf, args)))
        return
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    elif args.workload == "batch64":
        out = run_batch(args, rank, world)
    elif args.workload == "learned":
        out = run_learned(args, rank, world)
    elif args.workload == "group_sht":
        out = run_group(args, rank, world)
    else:
        out = run_ours(args, rank, world)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
