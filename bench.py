#!/usr/bin/env python3
"""Throughput of the registration hot path in correspondence queries per second.

Headline workload: Welsch-robust point-to-plane ICP with Anderson acceleration
(Alg. 2) on a seeded union of 8 random ellipsoids with analytic normals:
N = 500,000 target points, M = 200,000 source points cropped to 50% overlap,
noise 0.003 x diagonal, 5% uniform outliers, random rigid motion (angle <= 25
deg, translation <= 0.1 x diagonal), identity start. Synthetic inputs stand in
for the paper's scans.

One step = one whole registration through the C ABI: target index build and
nu_min statistic, source preparation, the nu_max pass, and every fused
iteration until the last nu stage converges. Metric = M x iterations / time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs independent replicas, one per rank (weak scaling), launched by
torch.distributed.run. --impl reference times the FP64 CPU oracle on a bounded
sample of the same workload instead.

Besides the headline, the default run measures the other workloads and nests
their summaries in the same JSON line ("workloads"; --no-nested skips them):
  single_torus_p2p       workload 1: Fast ICP, torus N = M = 2,000;
  single_height_field    workload 2: Welsch point-to-point, height field
                         N = 100,000, M = 80,000;
  precision              workload 3 in the FP32 and FP16-storage modes beside
                         the FP64 reference mode, each with its error against
                         the FP64 oracle's result (tests/golden, written by the
                         oracle alone);
  symmetric              workload 3 under the Welsch-robust symmetric objective
                         (Sec. 7's proposed extension, with the source's normals)
                         beside point-to-plane: time and Eq. (13) RMSE to the
                         ground-truth motion;
  batched                workload 4: 256 pairs (M, N log-uniform in [2k, 200k],
                         variants in equal thirds) in one fricp_batch_register
                         vs the plain path one pair at a time;
  served                 workload 5: Poisson arrivals of robust requests (M, N
                         log-uniform in [1k, 1M]) at 0.9x, 1.1x and 1.5x the plain
                         path's capacity through fricp_server_* vs the plain path.
Standalone runs (one line each): --workload batched | serve (five rates) |
precision | robustness.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import pathlib
import statistics
import subprocess
import sys
import threading
import time

ROOT = pathlib.Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "corr. queries/s (M x iters/s)"
UNIT = "queries/s"
VARIANT = "p2pl_welsch"
WORKLOAD = "welsch_p2pl_aa_ellipsoids_N500000_M200000"
L2_FLUSH_BYTES = 512 << 20          # > 129 MB L2
CPU_SAMPLE_M = 20000                # cpu_baseline sample: 10% of the source points, full target
CPU_SAMPLE_ITERS = 8
REF_SAMPLE_M = 4000                 # --impl reference: 2% of the source points per step
GOLDEN3 = ROOT / "tests" / "golden" / "fullsize_config3_p2pl_welsch.json"
# Files that define the search kernel k_nn (its launch, query set-up and tree
# search); the solver's algebra (solver.cuh, linalg.cuh) and the median
# (select.cuh) are compiled into the same file but only the accumulate kernel
# calls them.
KNN_SOURCES = ["step.cu", "step_common.cuh", "fricp_internal.cuh", "obb.cuh"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="single",
                    choices=["single", "batched", "serve", "precision", "robustness"])
    ap.add_argument("--serve-requests", type=int, default=96, help="distinct requests drawn (serve)")
    ap.add_argument("--serve-seconds", type=float, default=60.0, help="arrival window per rate (serve)")
    ap.add_argument("--no-nested", action="store_true", help="headline only (skip the nested workloads)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(xs, world, device="cuda"):
    """Each value's maximum over the ranks (the slowest rank sets a replica run's
    time); with one rank the values come back unchanged."""
    if world == 1:
        return [float(x) for x in xs]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x) for x in xs], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def workload_pair():
    from paper_2007_07627_gb300 import synth
    return synth.config_pair(3)


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: str):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                smax.append(float(r[1]))
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, r[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------
# CPU oracle sample (cpu_baseline and --impl reference)
# --------------------------------------------------------------------------

def oracle_sample(pair, nu, iters=CPU_SAMPLE_ITERS, m=CPU_SAMPLE_M):
    """Alg. 2 of the FP64 oracle (exhaustive closest points) on a fixed sample
    of m source points against the full target, one nu stage of `iters`
    inner iterations."""
    import numpy as np

    import oracle
    oracle.build()
    g = np.random.default_rng(20070762)
    sel = np.sort(g.choice(pair.M, m, replace=False))
    prm = oracle.Params(variant=VARIANT, p2pl_iters_first=iters, p2pl_iters_cap=iters, nu_max=nu, nu_min=nu)
    t0 = time.perf_counter()
    r = oracle.register(pair.P[sel], pair.Q, prm, normals=pair.normals)
    dt = time.perf_counter() - t0
    return {"value": m * r["iterations"] / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "seconds": dt, "iterations": r["iterations"], "corr_passes": r["corr_passes"],
            "sample": f"FP64 oracle (exhaustive closest point, OpenMP), Alg. 2 on {m} of the {pair.M} source "
                      f"points vs the full {pair.N}-point target, one nu stage at nu={nu:.3g}, {iters} iterations"}


def reference_nu(pair, m=CPU_SAMPLE_M):
    """nu of the oracle samples: a quarter of the workload's nu_max (Sec. 5:
    3 x the median plane distance at the identity start), computed by the
    oracle on the sample. (Its nu_min is the 1e-6 floor: the target is
    noise-free, so the six-neighbour plane distances vanish; at that nu every
    weight underflows.)"""
    import numpy as np

    import oracle
    g = np.random.default_rng(20070762)
    sel = np.sort(g.choice(pair.M, m, replace=False))
    nz = oracle.normalization(pair.P.astype(np.float64), pair.Q.astype(np.float64))
    Pn, Qn = nz.fwd(pair.P[sel].astype(np.float64)), nz.fwd(pair.Q.astype(np.float64))
    idx, _, _ = oracle.closest(Pn, Qn)
    h = np.abs(np.einsum("nd,nd->n", Pn - Qn[idx], pair.normals[idx].astype(np.float64)))
    return 3.0 * float(np.median(h)) / 4.0


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    pair = workload_pair()
    nu = reference_nu(pair, REF_SAMPLE_M)
    for _ in range(args.warmup):
        oracle_sample(pair, nu, iters=1, m=REF_SAMPLE_M)
    times, its = [], []
    for _ in range(args.steps):
        s = oracle_sample(pair, nu, iters=1, m=REF_SAMPLE_M)
        times.append(s["seconds"])
        its.append(s["iterations"])
    value = REF_SAMPLE_M * statistics.mean(its) / statistics.mean(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "variant": VARIANT, "N": pair.N, "M": pair.M},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                         "sample": f"each step: Alg. 2 of the FP64 oracle, one iteration, {REF_SAMPLE_M} of "
                                   f"{pair.M} source points vs the full target, nu={nu:.3g}"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# GPU path
# --------------------------------------------------------------------------

def gpu_selector(local: int) -> str:
    """nvidia-smi -i argument for CUDA device `local` (UUID when torch exposes it)."""
    import torch
    try:
        u = str(torch.cuda.get_device_properties(local).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        return vis.split(",")[local] if vis else str(local)


def measured_peaks():
    try:
        return json.loads((ROOT / "MEASURED_PEAKS.json").read_text())
    except (OSError, ValueError):
        return None


def step_kernel_hash() -> str:
    h = hashlib.sha256()
    for f in KNN_SOURCES:
        h.update((ROOT / "paper_2007_07627_gb300" / "csrc" / f).read_bytes())
    return h.hexdigest()[:16]


def profiled_kernel(workload: str):
    """Counters of the search kernel from the committed ncu summary of
    `workload` (profiles/k_nn_<workload>.json), only if they were taken on the
    current kernel source: DRAM bytes per launch, issue-slot and L2 fractions."""
    p = ROOT / "profiles" / f"k_nn_{workload}.json"
    try:
        d = json.loads(p.read_text())
    except (OSError, ValueError):
        return {}
    if d.get("kernel_source_sha256_16") != step_kernel_hash():
        return {}
    return d


def timed_registrations(fr, q, n, p, prm, steps, warmup, flush):
    """Whole registrations (target build included) timed with CUDA events, L2
    flushed before each; returns (mean ms, last result)."""
    import torch
    for _ in range(warmup):
        t = fr.target_create(q, n)
        fr.register(t, p, params=prm)
        t.destroy()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    times = []
    r = None
    for _ in range(steps):
        flush.zero_()
        ev0.record()
        t = fr.target_create(q, n)
        r = fr.register(t, p, params=prm)
        ev1.record()
        torch.cuda.synchronize()
        times.append(ev0.elapsed_time(ev1))
        t.destroy()
    return statistics.mean(times), r


def kernel_times(fr, q, n, p, prm):
    """Per-pass device time of the search and of the accumulate/solve kernels,
    from CUDA events recorded around every launch on the library's stream."""
    t = fr.target_create(q, n)
    prm_t = fr.Params.from_buffer_copy(prm)
    prm_t.time_passes = 1
    rt = fr.register(t, p, params=prm_t)
    t.destroy()
    steps = rt["device_steps"]
    return 1e3 * rt["search_ms"] / steps, 1e3 * (rt["pass_ms"] - rt["search_ms"]) / steps, rt


def roofline_of(search_us, M, N, plane, workload):
    algo = 12 * M + (24 if plane else 12) * N
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks and "hbm_gbs" in peaks else 6800.0
    achieved = algo / (search_us * 1e-6) / 1e9
    prof = profiled_kernel(workload)
    out = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
           "traffic": prof.get("dram_bytes_per_launch"), "kernel": "k_nn<0> (closest-point search)",
           "avg_launch_us": search_us, "algorithmic_bytes_per_launch": algo,
           "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else "fallback 6.8 TB/s (of fallback)"}
    if prof:
        out["issue_active_frac"] = prof.get("issue_active_frac")
        out["l2_throughput_frac"] = prof.get("l2_throughput_frac")
        out["profile"] = prof.get("summary")
    return out


def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    nested_data = None
    if world == 1 and not args.no_nested:
        nested_data = nested_inputs()        # spawn pool, before the first CUDA call
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    import paper_2007_07627_gb300 as fr

    pair = workload_pair()
    Qd = torch.from_numpy(pair.Q).cuda()
    Nd = torch.from_numpy(pair.normals).cuda()
    Pd = torch.from_numpy(pair.P).cuda()
    prm = fr.params_default(VARIANT)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def one_step(q, n, p):
        t = fr.target_create(q, n)
        r = fr.register(t, p, params=prm)
        return t, r

    for _ in range(args.warmup):
        t, r = one_step(Qd, Nd, Pd)
        t.destroy()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    fr.counters(reset=True)
    clocks = ClockSampler(gpu_selector(local))
    clocks.start()
    times, iters, passes = [], [], []
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    for _ in range(args.steps):
        flush.zero_()                       # evict L2 between timed steps
        ev0.record()
        t, r = one_step(Qd, Nd, Pd)
        ev1.record()
        torch.cuda.synchronize()
        times.append(ev0.elapsed_time(ev1))
        iters.append(r["iterations"])
        passes.append(r["corr_passes"])
        t.destroy()
    torch.cuda.synchronize()
    launches = fr.counters(reset=True)["kernel_launches"]
    clk = clocks.stop()
    (ms,) = max_over_ranks([statistics.mean(times)], world)
    if world > 1:
        torch.distributed.barrier()
    it = statistics.mean(iters)
    value = world * pair.M * it / (ms / 1e3)

    # dominant kernel: the closest-point search, timed launch by launch with
    # CUDA events on the library's stream (an event between the search and the
    # accumulate/solve kernel of every step)
    search_us, accum_us, rt = kernel_times(fr, Qd, Nd, Pd, prm)
    roofline = roofline_of(search_us, pair.M, pair.N, True, WORKLOAD)
    roofline["accum_solve_avg_launch_us"] = accum_us

    # end to end through the public API with host buffers
    e2e_t = []
    fr.counters(reset=True)
    for _ in range(args.steps):
        t0 = time.perf_counter()
        th = fr.target_create(pair.Q, pair.normals)
        rh = fr.register(th, pair.P, params=prm)
        e2e_t.append(time.perf_counter() - t0)
        th.destroy()
    cnt = fr.counters(reset=True)
    (e2e_s,) = max_over_ranks([statistics.mean(e2e_t)], world)
    e2e = {"value": world * pair.M * rh["iterations"] / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": cnt["h2d_bytes"] // args.steps, "d2h_bytes_per_step": cnt["d2h_bytes"] // args.steps}

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample(pair, reference_nu(pair))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64 (candidate distances f32 pairs)", "data": "synthetic",
        "config": {"workload": WORKLOAD, "variant": VARIANT, "N": pair.N, "M": pair.M,
                   "iterations": it, "corr_passes": statistics.mean(passes), "device_steps": rt["device_steps"],
                   "l2": "flushed between steps", "step": "target index + nu rules + source prep + all iterations",
                   "parallelism": f"replicas x{world}"},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
    }
    if nested_data is not None:
        line["workloads"] = nested_workloads(fr, nested_data, flush, pair, (Qd, Nd, Pd), rt)
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


# --------------------------------------------------------------------------
# Nested workloads of the default run (rank 0, N = 1)
# --------------------------------------------------------------------------

NESTED_SERVE_RATES = (0.9, 1.1, 1.5)
NESTED_SERVE_SECONDS = 25.0
NESTED_SERVE_POOL = 48


def nested_inputs():
    from paper_2007_07627_gb300 import synth
    t0 = time.perf_counter()
    batch = generate(synth.batch_specs())
    serve = generate(synth.serve_specs(n=NESTED_SERVE_POOL))
    return {"batch": batch, "serve": serve, "gen_s": time.perf_counter() - t0}


def single_summary(fr, cfg, variant, over, flush, steps=5, warmup=2):
    import torch

    from paper_2007_07627_gb300 import synth
    pair = synth.config_pair(cfg)
    q, p = torch.from_numpy(pair.Q).cuda(), torch.from_numpy(pair.P).cuda()
    n = torch.from_numpy(pair.normals).cuda() if pair.normals is not None and variant.startswith("p2pl") else None
    prm = fr.params_default(variant, **over)
    ms, r = timed_registrations(fr, q, n, p, prm, steps, warmup, flush)
    s_us, a_us, _ = kernel_times(fr, q, n, p, prm)
    name = {1: "p2p_aa_torus_N2000_M2000", 2: "welsch_p2p_aa_height_field_N100000_M80000"}[cfg]
    return {"workload": name, "variant": variant, "N": pair.N, "M": pair.M, "ms_per_registration": ms,
            "queries_per_s": pair.M * r["iterations"] / (ms / 1e3), "iterations": r["iterations"],
            "device_steps": r["device_steps"], "search_us_per_pass": s_us, "accum_solve_us_per_pass": a_us,
            "roofline": roofline_of(s_us, pair.M, pair.N, False, name), "steps": steps}


def precision_summary(fr, pair, dev, flush, steps=3, warmup=1):
    """Workload 3 in each precision mode; errors against the FP64 oracle's
    whole-registration result (tests/golden, written by the oracle alone) and
    against the FP64 GPU mode."""
    import numpy as np
    Qd, Nd, Pd = dev
    gold = None
    try:
        gold = json.loads(GOLDEN3.read_text())
    except (OSError, ValueError):
        pass
    modes, ref = {}, None
    for prec in ("fp64", "fp32", "fp16"):
        prm = fr.params_default(VARIANT, precision=prec)
        ms, r = timed_registrations(fr, Qd, Nd, Pd, prm, steps, warmup, flush)
        if ref is None:
            ref = r
        diag = 1.0 / r["scale"]

        def err(R, t):
            c = (np.trace(r["R"] @ np.asarray(R).T) - 1.0) / 2.0
            return {"rotation_rad": float(np.arccos(np.clip(c, -1.0, 1.0))),
                    "t_over_diag": float(np.abs(r["t"] - np.asarray(t)).max() / diag)}
        modes[prec] = {"ms_per_registration": ms, "iterations": r["iterations"], "device_steps": r["device_steps"],
                       "queries_per_s": pair.M * r["iterations"] / (ms / 1e3),
                       "us_per_device_step": 1e3 * ms / r["device_steps"],
                       "vs_fp64_oracle": (dict(err(gold["R"], gold["t"]), iterations_oracle=gold["iterations"],
                                               energy_rel=abs(r["final_energy"] - gold["final_energy"]) /
                                               abs(gold["final_energy"])) if gold else None),
                       "vs_fp64_mode": err(ref["R"], ref["t"])}
    return {"workload": WORKLOAD, "modes": modes,
            "oracle_result": "tests/golden/fullsize_config3_p2pl_welsch.json" if gold else None}


def symmetric_summary(fr, pair, dev, flush, steps=3, warmup=1):
    """Workload 3 under the Welsch-robust symmetric objective (source normals on
    the device) beside the point-to-plane Alg. 2 it extends: time per whole
    registration and the Eq. (13) RMSE against the ground-truth motion."""
    import torch
    Qd, Nd, Pd = dev
    Sd = torch.from_numpy(pair.src_normals).cuda()
    out = {}
    for variant in ("p2pl_welsch", "sym_welsch"):
        prm = fr.params_default(variant)

        def run():
            t = fr.target_create(Qd, Nd)
            if variant == "sym_welsch":
                r = fr.register_symmetric(t, Pd, Sd, params=prm)
            else:
                r = fr.register(t, Pd, params=prm)
            return t, r
        for _ in range(warmup):
            run()[0].destroy()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        times = []
        for _ in range(steps):
            flush.zero_()
            ev0.record()
            t, r = run()
            ev1.record()
            torch.cuda.synchronize()
            times.append(ev0.elapsed_time(ev1))
            t.destroy()
        ms = statistics.mean(times)
        out[variant] = {"ms_per_registration": ms, "iterations": r["iterations"], "corr_passes": r["corr_passes"],
                        "device_steps": r["device_steps"], "line_search_trials": r["line_search_trials"],
                        "queries_per_s": pair.M * r["iterations"] / (ms / 1e3),
                        "rmse_over_diag": rmse_of(pair.P, r["R"], r["t"], pair.R_gt, pair.t_gt) / pair.diag}
    return {"workload": WORKLOAD, "steps": steps, "objectives": out}


def nested_workloads(fr, data, flush, pair, dev, rt):
    t0 = time.perf_counter()
    out = {"single_torus_p2p": single_summary(fr, 1, "p2p", dict(max_iters=100), flush, steps=10, warmup=3),
           "single_height_field": single_summary(fr, 2, "p2p_welsch", {}, flush)}
    out["precision"] = precision_summary(fr, pair, dev, flush)
    out["symmetric"] = symmetric_summary(fr, pair, dev, flush)
    out["batched"] = batched_summary(fr, data["batch"], steps=1, warmup=1)
    out["served"] = served_summary(fr, data["serve"], NESTED_SERVE_RATES, NESTED_SERVE_SECONDS)
    out["seconds"] = {"generation": data["gen_s"], "measurement": time.perf_counter() - t0}
    return out


# --------------------------------------------------------------------------
# Many-pair workloads: batched and served, each against the plain path
# --------------------------------------------------------------------------

def generate(specs):
    """Build the pairs of `specs` on a spawn process pool (before any CUDA call)."""
    import multiprocessing as mp

    from paper_2007_07627_gb300 import synth
    ctx = mp.get_context("spawn")
    with ctx.Pool(max(1, min(len(specs), os.cpu_count() or 4))) as pool:
        return pool.map(synth.make_pair, specs, chunksize=1)


def same_result(a, b) -> bool:
    import numpy as np
    return (a["iterations"] == b["iterations"] and a["corr_passes"] == b["corr_passes"]
            and np.array_equal(a["R"], b["R"]) and np.array_equal(a["t"], b["t"]))


def to_device(pairs):
    import torch
    out = []
    for v, p in pairs:
        out.append((v, torch.from_numpy(p.P).cuda(), torch.from_numpy(p.Q).cuda(),
                    torch.from_numpy(p.normals).cuda() if v == "p2pl_welsch" else None))
    torch.cuda.synchronize()
    return out


def batched_summary(fr, pairs, steps=1, warmup=1):
    """Workload 4: 256 target builds plus one fricp_batch_register, against the
    plain path (target build plus fricp_register, one pair after another) on the
    same inputs; results compared bit for bit."""
    import torch
    dev = to_device(pairs)
    prms = [fr.params_default(v) for v, _ in pairs]
    sum_m = sum(p.M for _, p in pairs)

    def batched():
        ts = [fr.target_create(q, n) for _, _, q, n in dev]
        res = fr.batch_register(ts, [p for _, p, _, _ in dev], prms)
        for t in ts:
            t.destroy()
        return res

    def plain():
        res = []
        for (v, p, q, n), prm in zip(dev, prms):
            t = fr.target_create(q, n)
            res.append(fr.register(t, p, params=prm))
            t.destroy()
        return res

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t0, r

    for _ in range(warmup):
        batched()
    fr.counters(reset=True)
    bt = []
    for _ in range(steps):
        dt, rb = timed(batched)
        bt.append(dt)
    launches = fr.counters(reset=True)["kernel_launches"] // steps
    shape = fr.batch_last_shape()
    pt, rp = timed(plain)
    iters = sum(r["iterations"] for r in rb)
    queries = sum(p.M * r["iterations"] for (_, p), r in zip(pairs, rb))
    t_b = statistics.mean(bt)
    return {
        "workload": "256 pairs, M and N log-uniform in [2k, 200k], mixed variants and surfaces",
        "queries_per_s": queries / t_b, "regs_per_s": len(pairs) / t_b, "seconds_per_batch": t_b,
        "pairs": len(pairs), "sum_M": sum_m, "sum_N": sum(p.N for _, p in pairs), "iterations_total": iters,
        "step": "256 target builds + nu rules + one batched registration", "autotuned_shape": shape,
        "plain": {"queries_per_s": sum(p.M * r["iterations"] for (_, p), r in zip(pairs, rp)) / pt,
                  "regs_per_s": len(pairs) / pt, "seconds": pt},
        "speedup_vs_plain": pt / t_b,
        "equal_results": sum(same_result(a, b) for a, b in zip(rb, rp)), "of": len(pairs),
        "gpu_launches_per_batch": launches, "steps": steps,
    }


def run_batched(args):
    from paper_2007_07627_gb300 import synth
    rank, world, local = dist_env()
    if rank != 0:
        return
    pairs = generate(synth.batch_specs())
    import torch
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    import paper_2007_07627_gb300 as fr
    clocks = ClockSampler(gpu_selector(local))
    clocks.start()
    b = batched_summary(fr, pairs, steps=args.steps, warmup=args.warmup)
    clk = clocks.stop()
    line = {"metric": "corr. queries/s (sum over pairs of M x iters / s); regs/s", "workload": "batched",
            "value": b["queries_per_s"], "unit": "queries/s", "regs_per_s": b["regs_per_s"],
            "ms_per_step": 1e3 * b["seconds_per_batch"], "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "n_gpus": 1, "data": "synthetic",
            "dtype": "f64 (candidate distances f32 pairs)", "config": {"workload": b["workload"],
                                                                      "l2": "inputs 320 MB > L2"},
            "summary": b, "clocks": clk}
    print(json.dumps(line), flush=True)


def percentile(xs, q):
    import numpy as np
    return float(np.percentile(np.asarray(xs), q)) if xs else None


def served_summary(fr, reqs, rates, window_s, seed=None):
    """Workload 5: Poisson arrivals at each rate x the plain path's capacity
    over a window of window_s seconds, each arrival one of the distinct
    requests `reqs` (drawn uniformly); every arrival is a target build plus a
    registration, timed from its arrival to its result, once through the
    serving loop (continuous batching) and once through the plain path (one at
    a time, first come first served). Served results are compared with each
    request's alone result."""
    import numpy as np
    import torch

    from paper_2007_07627_gb300 import synth
    dev = to_device(reqs)
    prms = [fr.params_default(v) for v, _ in reqs]
    n = len(reqs)

    def alone(k):
        v, p, q, nrm = dev[k]
        t = fr.target_create(q, nrm)
        r = fr.register(t, p, params=prms[k])
        t.destroy()
        return r

    alone(0)                                   # warm-up
    service, ref = [], []
    for k in range(n):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ref.append(alone(k))
        torch.cuda.synchronize()
        service.append(time.perf_counter() - t0)
    capacity = 1.0 / statistics.mean(service)
    g = np.random.default_rng(synth.CONFIG_SEEDS[5] if seed is None else seed)
    out_rates = []
    srv = fr.Server(max_slots=256, steps_per_sync=8)
    for f in rates:
        lam = f * capacity
        arr = []
        tt = 0.0
        while True:
            tt += g.exponential(1.0 / lam)
            if tt > window_s:
                break
            arr.append(tt)
        pick = g.integers(0, n, len(arr))
        na = len(arr)

        # plain path: one request at a time, first come first served
        lat_p = []
        t0 = time.perf_counter()
        for a, k in zip(arr, pick):
            now = time.perf_counter() - t0
            if now < a:
                time.sleep(a - now)
            alone(int(k))
            torch.cuda.synchronize()
            lat_p.append(time.perf_counter() - t0 - a)
        span_p = time.perf_counter() - t0

        # served path: continuous batching
        lat_s, equal = [0.0] * na, 0
        t0 = time.perf_counter()
        nxt, live, done = 0, {}, 0
        while done < na:
            now = time.perf_counter() - t0
            while nxt < na and arr[nxt] <= now:
                k = int(pick[nxt])
                v, p, q, nrm = dev[k]
                t = fr.target_create(q, nrm)
                live[srv.submit(t, p, prms[k])] = (nxt, k, t)
                nxt += 1
            if live:
                srv.step(8)
                for tk in list(live):
                    r = srv.poll(tk)
                    if r is not None:
                        a_i, k, t = live.pop(tk)
                        lat_s[a_i] = time.perf_counter() - t0 - arr[a_i]
                        equal += same_result(r, ref[k])
                        t.destroy()
                        done += 1
            elif nxt < na:
                time.sleep(max(0.0, arr[nxt] - (time.perf_counter() - t0)))
        span_s = time.perf_counter() - t0
        out_rates.append({"rate_x_capacity": f, "arrivals_per_s": lam, "arrivals": na, "window_s": window_s,
                          "served": {"regs_per_s": na / span_s, "p50_s": percentile(lat_s, 50),
                                     "p99_s": percentile(lat_s, 99), "span_s": span_s},
                          "plain": {"regs_per_s": na / span_p, "p50_s": percentile(lat_p, 50),
                                    "p99_s": percentile(lat_p, 99), "span_s": span_p},
                          "equal_results": equal, "of": na})
    srv.destroy()
    return {"workload": f"Poisson arrivals of robust requests drawn from {n} distinct ones, M and N log-uniform "
                        f"in [1k, 1M] (mean M {statistics.mean(p.M for _, p in reqs):.0f})",
            "plain_capacity_regs_per_s": capacity, "plain_mean_service_s": statistics.mean(service),
            "request": "target build + nu rules + registration (arrival to result)",
            "autotuned_shape": fr.batch_last_shape(), "rates": out_rates}


def run_serve(args):
    from paper_2007_07627_gb300 import synth
    rank, world, local = dist_env()
    if rank != 0:
        return
    reqs = generate(synth.serve_specs(n=args.serve_requests))
    import torch
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    import paper_2007_07627_gb300 as fr
    clocks = ClockSampler(gpu_selector(local))
    clocks.start()
    sv = served_summary(fr, reqs, (0.25, 0.5, 0.75, 0.9, 1.1, 1.5), args.serve_seconds)
    clk = clocks.stop()
    line = {
        "metric": "served regs/s with p50/p99 latency vs plain", "workload": "serve", "unit": "regs/s",
        "value": max(r["served"]["regs_per_s"] for r in sv["rates"]), "higher_is_better": True, "n_gpus": 1,
        "data": "synthetic", "dtype": "f64 (candidate distances f32 pairs)",
        "config": {"workload": sv["workload"]}, "summary": sv, "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def run_precision(args):
    import torch

    from paper_2007_07627_gb300 import synth
    rank, world, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    import paper_2007_07627_gb300 as fr
    pair = synth.config_pair(3)
    dev = tuple(torch.from_numpy(x).cuda() for x in (pair.Q, pair.normals, pair.P))
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    sm = precision_summary(fr, pair, dev, flush, steps=args.steps, warmup=args.warmup)
    line = {"metric": "corr. queries/s (M x iters/s) per precision mode", "workload": "precision",
            "value": sm["modes"]["fp64"]["queries_per_s"], "unit": "queries/s", "higher_is_better": True,
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": pair.N, "M": pair.M,
                       "step": "target index + nu rules + source prep + all iterations",
                       "l2": "flushed between steps"},
            "summary": sm}
    print(json.dumps(line), flush=True)


def rmse_of(P, R, t, R_gt, t_gt) -> float:
    """Eq. (13): RMSE between the computed and the ground-truth motion of P."""
    import numpy as np
    P = P.astype(np.float64)
    d = P @ (np.asarray(R_gt) - np.asarray(R)).T + (np.asarray(t_gt) - np.asarray(t))
    return float(np.sqrt((d * d).sum(axis=1).mean()))


def run_robustness(args):
    import numpy as np
    import torch

    from paper_2007_07627_gb300 import synth
    rank, world, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    import paper_2007_07627_gb300 as fr
    # stand-in for the paper's failing scan pair with 50% added outliers
    pair = synth.ellipsoid_pair(synth.CONFIG_SEEDS[3] + 100, M=40000, N=40000, overlap=1.0, noise=0.003,
                                outliers=0.5, max_angle=0.0)
    starts = synth.robustness_starts(pair)
    variants = ("p2p", "p2p_welsch", "p2pl_welsch")
    t = fr.target_create(pair.Q, pair.normals)
    Pd = torch.from_numpy(pair.P).cuda()
    cases = [(v, ang, T0) for v in variants for ang, T0 in starts]
    prms = [fr.params_default(v) for v, _, _ in cases]
    T0s = np.stack([T0 for _, _, T0 in cases])
    fr.batch_register([t] * len(cases), [Pd] * len(cases), prms, T0=T0s)     # warm-up (and autotune)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = fr.batch_register([t] * len(cases), [Pd] * len(cases), prms, T0=T0s)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    t0 = time.perf_counter()
    alone = [fr.register(t, Pd, T0=T0, params=prm) for (_, _, T0), prm in zip(cases, prms)]
    torch.cuda.synchronize()
    t_plain = time.perf_counter() - t0
    err = [rmse_of(pair.P, r["R"], r["t"], pair.R_gt, pair.t_gt) / pair.diag for r in res]
    per_angle = {v: {} for v in variants}
    for (v, ang, _), e in zip(cases, err):
        per_angle[v].setdefault(ang, []).append(e)
    alphas = [10.0 ** x for x in np.arange(-5, -0.9, 0.5)]
    recall = {v: [float(np.mean([e < a for (vv, _, _), e in zip(cases, err) if vv == v])) for a in alphas]
              for v in variants}
    # Fig. 4: fixed nu = nu_max, fixed nu = nu_min, decreasing nu (Welsch point-to-point, beta = 10 deg)
    T10 = [T0 for ang, T0 in starts if ang == 10][0]
    dyn = fr.register(t, Pd, T0=T10, params=fr.params_default("p2p_welsch"))
    fixed = {}
    for name, nu in (("nu_max", dyn["nu_max"]), ("nu_min", dyn["nu_min"])):
        r = fr.register(t, Pd, T0=T10, params=fr.params_default("p2p_welsch", nu_max=nu, nu_min=nu))
        fixed[name] = rmse_of(pair.P, r["R"], r["t"], pair.R_gt, pair.t_gt) / pair.diag
    fixed["decreasing"] = rmse_of(pair.P, dyn["R"], dyn["t"], pair.R_gt, pair.t_gt) / pair.diag
    t.destroy()
    line = {"metric": "registrations/s of the batched sweep; mean RMSE/diag per initial angle",
            "workload": "robustness", "value": len(cases) / t_batch, "unit": "regs/s", "higher_is_better": True,
            "n_gpus": 1, "data": "synthetic",
            "config": {"pair": f"ellipsoids M={pair.M} N={pair.N}, full overlap, noise 0.003 diag, 50% outliers",
                       "angles_deg": [5, 10, 20, 30, 50], "axes_per_angle": 10, "registrations": len(cases)},
            "batched_s": t_batch, "plain_s": t_plain, "speedup_vs_plain": t_plain / t_batch,
            "equal_results": sum(same_result(a, b) for a, b in zip(res, alone)), "of": len(cases),
            "mean_rmse_over_diag": {v: {str(a): float(np.mean(e)) for a, e in d.items()} for v, d in per_angle.items()},
            "alpha_recall": {"alpha": alphas, **recall},
            "nu_schedule_rmse_over_diag": fixed}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "precision":
        run_precision(args)
    elif args.workload == "robustness":
        run_robustness(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
