"""Benchmark: MPR reconstructions per second on one GB300 (and N GPUs, weak scaling).

A step is one full MPR reconstruction (Alg. mpr: initialise, G generations of crossover,
self-improvement of both populations and selection, then the aligned average) of one
synthetic 512 x 512 single-shot pattern with P = 64 (2P = 128 individuals improved per
generation), 10 generations x 200 RAAR iterations.  Inputs are synthetic (seeded), shaped
like the paper's binned pnCCD data: beamstop, detector gap, saturation, Poisson noise.

  value  : reconstructions/s with the pattern already resident on the device
  e2e    : the same through the C ABI from host buffers (upload, run, download per step)
  roofline: the dominant per-iteration kernel's algorithmic bytes / its average CUDA-event
           duration, against the measured HBM copy bandwidth
  cpu_baseline: the FP64 oracle on this host's cores over a bounded sample of the work

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time
from pathlib import Path

import numpy as np

TIMING_STRIDE = 7

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

WORKLOADS = {
    # name: (pattern recipe, seed, params)
    "ell512": ("ell512", 0, dict(pop=64, iters_per_gen=200, generations=10, algorithm=2, beta=0.9,
                                 sw_sigma=1.5, sw_threshold=0.2, sw_period=20, er_tail=10)),
    "sphere64": ("sphere64", 0, dict(pop=8, iters_per_gen=100, generations=5, algorithm=2, beta=0.9,
                                     sw_sigma=1.5, sw_threshold=0.2, sw_period=20, er_tail=10)),
}
PEAKS = ROOT / "MEASURED_PEAKS.json"
GOLDEN_ORACLE = ROOT / "tests" / "golden" / "oracle_errors.json"


def pixels_per_reconstruction(n, prm):
    return 2 * prm["pop"] * prm["iters_per_gen"] * prm["generations"] * n * n


def hbm_peak():
    try:
        d = json.loads(PEAKS.read_text())
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for l in self.proc.stdout:
            self.lines.append(l.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [c.strip() for c in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_sample(pattern, prm, seconds=15.0):
    """Time the FP64 oracle's self-improvement on a bounded sample of the workload."""
    import oracle
    n = pattern.n
    I = np.fft.ifftshift(pattern.intensities.astype(np.float64))
    mask = np.fft.ifftshift(pattern.mask)
    M = np.sqrt(I)
    cores = oracle.get_threads()
    batch = cores
    K = prm["sw_period"]
    p = oracle.make_params(**{**prm, "iters_per_gen": 2 * K, "er_tail": min(prm["er_tail"], K)})
    x = oracle.initialize(1, pattern.support0, I, mask, batch)
    S = np.broadcast_to(pattern.support0, x.shape).copy()
    a = int(pattern.support0.sum())
    t0 = time.perf_counter()
    reps = 0
    while True:
        x, S, _ = oracle.improve(x, S, M, mask, p, prm["sw_sigma"], prm["sw_threshold"], a, a)
        reps += 1
        if time.perf_counter() - t0 > seconds:
            break
    dt = time.perf_counter() - t0
    it_px = reps * batch * 2 * K * n * n
    rate = it_px / dt
    return {
        "it_px_per_s": rate,
        "value": rate / pixels_per_reconstruction(n, prm),
        "cores": cores,
        "seconds": dt,
        "sample": f"{reps} self-improvement pass(es) of {batch} individuals x {2 * K} iterations "
                  f"(RAAR + ER tail + shrink-wrap + error) at {n}x{n}; rate scaled by "
                  f"{pixels_per_reconstruction(n, prm):.3g} iteration-pixels per reconstruction",
    }


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload_config(wl, n, prm, graph):
    """The `config` object of a bench line (the same for both arms)."""
    return {"workload": f"{wl}: {n}x{n}, P={prm['pop']} (2P={2 * prm['pop']} improved), "
                        f"G={prm['generations']} x {prm['iters_per_gen']} RAAR iterations",
            "n": n, **prm, "l2": "inputs larger than L2 (run state 2P x N^2 x 25 B = "
                                 f"{2 * prm['pop'] * n * n * 25 / 2**20:.0f} MiB)",
            "graph": bool(graph)}


def rank_seed(rank):
    """Run seed of a rank: every rank reconstructs its own pattern instance (weak scaling,
    no data-path collective)."""
    return 1000 + rank


def max_over_ranks(ms, dist, device):
    """The timed region's length is the slowest rank's."""
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_value(ws, steps, ms_max):
    """Whole-job reconstructions/s: every rank completed `steps` reconstructions."""
    return ws * steps / (ms_max / 1000.0)


def run_reference(args, wl):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from paper_2409_07413_gb300 import synthetic
    name, seed, prm = WORKLOADS[wl]
    pat = synthetic.config_pattern(name, seed)
    per = max(5.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_sample(pat, prm, seconds=min(per, 3.0))
    vals, cores, sample = [], 0, ""
    for _ in range(args.steps):
        r = oracle_sample(pat, prm, seconds=per)
        vals.append(r["value"])
        cores, sample = r["cores"], r["sample"]
    v = statistics.mean(vals)
    out = {
        "impl": "reference", "metric": "MPR reconstructions/s", "value": v,
        "unit": "reconstructions/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 / v if v > 0 else None, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(wl, pat.n, prm, args.graph),
        "cpu_baseline": {"value": v, "unit": "reconstructions/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": "reconstructions/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def production_legs(spring, ctx, args):
    """The three production forms of the path, each a short leg (reported beside the headline,
    not part of it):
      precision (1024 x 1024 two-panel pattern, P = 128, 20 x 300): one reconstruction with
        FP32 storage and one with FP16 storage; and the same pattern and schedule at P = 32,
        2 generations, at the run seeds whose FP64-oracle results are stored, in both
        storages, against the oracle's mean;
      batched uneven (patterns of sides drawn from {128, 192, 256, 512}, P = 32, 5 x 200):
        same-side batches (spring_mpr_run_batch), the whole set in one call (one group per
        side, one CUDA graph), served (all submitted at once) and plain (one after another);
      serving stream (Poisson arrivals at 200/s, sides {128, 256, 512, 1024} weighted
        0.4/0.3/0.2/0.1, P = 32, 5 x 200): served (spring_submit / spring_poll) against plain
        (one at a time in arrival order), with latency percentiles."""
    import torch

    from paper_2409_07413_gb300 import batchbench, servebench, synthetic
    out = {}
    # ---- precision
    t_leg = time.perf_counter()
    pat = synthetic.config_pattern("ell1024", 0)
    prob = ctx.problem(pat.intensities, pat.mask, pat.support0)
    prm4 = dict(pop=128, iters_per_gen=300, generations=20, algorithm=2, beta=0.9, sw_sigma=1.5,
                sw_threshold=0.2, sw_period=20, er_tail=10)
    px4 = pixels_per_reconstruction(1024, prm4)
    runs = {}
    for prec in (0, 1):
        prob.run(spring.params(**dict(prm4, generations=1), seed=1, precision=prec), want_arrays=False)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = prob.run(spring.params(**prm4, seed=1000, precision=prec), want_arrays=False)
        dt = time.perf_counter() - t0
        runs["fp16_storage" if prec else "fp32"] = {
            "seconds": dt, "reconstructions_per_s": 1.0 / dt, "iteration_pixels_per_s": px4 / dt,
            "final_error_avg": r["final_error_avg"], "final_error_best": r["final_error_best"]}
    golden = json.loads(GOLDEN_ORACLE.read_text()) if GOLDEN_ORACLE.exists() else {}
    orc = {g["run_seed"]: g for k, g in golden.items() if k == "ell1024_g2" or k.startswith("ell1024_g2_r")}
    red = dict(prm4, pop=32, generations=2)
    cmp = {"params": red, "run_seeds": sorted(orc)}
    if orc:
        cmp["oracle_fp64"] = {k: float(np.mean([orc[sd][k] for sd in orc])) for k in ("final_error_avg", "final_error_best")}
        for prec in (0, 1):
            ea, eb = [], []
            for sd in sorted(orc):
                r = prob.run(spring.params(**red, seed=sd, precision=prec), want_arrays=False)
                ea.append(r["final_error_avg"])
                eb.append(r["final_error_best"])
            m = {"final_error_avg": float(np.mean(ea)), "final_error_best": float(np.mean(eb))}
            m["vs_oracle_rel"] = {k: (m[k] - cmp["oracle_fp64"][k]) / cmp["oracle_fp64"][k] for k in m}
            cmp["fp16_storage" if prec else "fp32"] = m
    prob.destroy()
    out["precision_1024"] = {"workload": "ell1024: 1024x1024, P=128, G=20 x 300 RAAR", "runs": runs,
                             "reduced_vs_oracle": cmp, "leg_seconds": time.perf_counter() - t_leg}
    # ---- batched uneven workload (a subset of the 256 patterns)
    t_leg = time.perf_counter()
    prm3 = dict(pop=32, iters_per_gen=200, generations=5, algorithm=2, beta=0.9, sw_sigma=1.5,
                sw_threshold=0.2, sw_period=20, er_tail=10)
    jobs = batchbench.make_set(0, args.batch_patterns)
    for n in batchbench.SIDES:
        spring.autotune(n, 2 * prm3["pop"])
    b = batchbench.run_set(ctx, spring, jobs, prm3, ("batched", "mixed", "served", "plain"))
    b["leg_seconds"] = time.perf_counter() - t_leg
    b["batched_over_plain"] = b["batched"]["reconstructions_per_s"] / b["plain"]["reconstructions_per_s"]
    b["mixed_over_plain"] = b["mixed"]["reconstructions_per_s"] / b["plain"]["reconstructions_per_s"]
    b["served_over_plain"] = b["served"]["reconstructions_per_s"] / b["plain"]["reconstructions_per_s"]
    out["batched_uneven"] = b
    # ---- serving stream
    t_leg = time.perf_counter()
    reqs = servebench.make_stream(0, 200.0, args.serve_seconds)
    for n in servebench.SIDES:
        spring.autotune(n, 2 * servebench.PARAMS["pop"])
    sv = {"rate_hz": 200.0, "arrivals_s": args.serve_seconds, "requests": len(reqs),
          "sizes": {str(n): int(sum(1 for r in reqs if r[1] == n)) for n in servebench.SIDES},
          "params": servebench.PARAMS}
    for mode, fn in (("served", servebench.run_served), ("plain", servebench.run_plain)):
        lat, svc, errs, sizes, span = fn(ctx, spring, reqs)
        sv[mode] = {"reconstructions_per_s": len(lat) / span, "makespan_s": span,
                    "latency": servebench.percentiles(lat), "service": servebench.percentiles(svc),
                    "mean_final_error_best": float(np.mean(errs))}
    sv["served_over_plain"] = sv["served"]["reconstructions_per_s"] / sv["plain"]["reconstructions_per_s"]
    sv["leg_seconds"] = time.perf_counter() - t_leg
    out["serving_stream"] = sv
    return out


def run_ours(args, wl):
    import torch

    from paper_2409_07413_gb300 import spring, synthetic

    ws, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (no CPU fallback)")
    torch.cuda.set_device(local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    name, seed, prm = WORKLOADS[wl]
    pat = synthetic.config_pattern(name, seed)
    n = pat.n
    p = spring.params(**prm, seed=rank_seed(rank), use_graph=int(args.graph))
    ctx = spring.Context(local)
    dI = torch.from_numpy(pat.intensities).cuda()
    dm = torch.from_numpy(pat.mask).cuda()
    dS = torch.from_numpy(pat.support0).cuda()
    prob = ctx.problem_device(dI, dm, dS)
    torch.cuda.synchronize()

    def barrier():
        if pg:
            pg.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        prob.run(p, want_arrays=False)
    # ---- device-resident timed region
    clocks = Clocks(local)
    spring.stats_reset()
    # every TIMING_STRIDE-th launch of the two iteration passes is bracketed by events: the
    # events cost device time, and a stride coprime to the 20-iteration blocks samples
    # every position of a block evenly
    spring.stats_enable_timing(True, stride=TIMING_STRIDE)
    barrier()
    clocks.start()
    l0 = spring.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    step_ms, errs = [], []
    ev0.record()
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = prob.run(p, want_arrays=False)
        step_ms.append(1000.0 * (time.perf_counter() - t0))
        errs.append((r["final_error_avg"], r["final_error_best"]))
    ev1.record()
    barrier()
    clk = clocks.stop()
    launches = spring.launch_count() - l0
    spring.stats_enable_timing(False)
    ms = ev0.elapsed_time(ev1)
    kst = {kc: spring.stats_get(kc) for kc in (spring.KC_ROW_ITER, spring.KC_COL_PM)}
    if pg:
        ms = max_over_ranks(ms, pg, "cuda")
    value = weak_value(ws, args.steps, ms)

    # ---- the same runs captured as one CUDA graph each (launch gaps removed), timed apart
    #      from the region above: launches inside a capture carry no per-kernel events
    graph_out = None
    if not args.graph and args.steps > 0:
        pgr = spring.params(**prm, seed=rank_seed(rank), use_graph=1)
        prob.run(pgr, want_arrays=False)  # warm-up
        barrier()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record()
        for _ in range(args.steps):
            prob.run(pgr, want_arrays=False)
        g1.record()
        barrier()
        gms = g0.elapsed_time(g1)
        if pg:
            gms = max_over_ranks(gms, pg, "cuda")
        graph_out = {"value": weak_value(ws, args.steps, gms), "unit": "reconstructions/s",
                     "ms_per_step": gms / args.steps}

    # ---- end to end through the C ABI from host buffers
    h2d = pat.intensities.nbytes + pat.mask.nbytes + pat.support0.nbytes
    d2h = 2 * n * n * 8 + n * n + prm["generations"] * 8 * 8 + 5 * 8
    barrier()
    te0 = time.perf_counter()
    for _ in range(max(1, args.steps)):
        hp = ctx.problem(pat.intensities, pat.mask, pat.support0)
        hp.run(p, want_arrays=True)
        hp.destroy()
    barrier()
    te = time.perf_counter() - te0
    if pg:
        te = max_over_ranks(te * 1000.0, pg, "cuda") / 1000.0
    e2e = ws * max(1, args.steps) / te

    out = None
    if rank == 0:
        peak, peak_kind = hbm_peak()
        dom = max(kst.items(), key=lambda kv: kv[1].total_ms)
        kc, st = dom
        avg_ms = st.total_ms / max(1, st.timed)
        achieved = st.bytes_per_launch / (avg_ms / 1000.0) / 1e9 if avg_ms > 0 else None
        other = kst[spring.KC_COL_PM if kc == spring.KC_ROW_ITER else spring.KC_ROW_ITER]
        oavg = other.total_ms / max(1, other.timed)
        # the kernels behind the two iteration classes depend on the path the side runs:
        # two passes (k_row / k_col*) or split passes (at 512: k_row_pair / k_col_split);
        # DRAM traffic is keyed the same way
        path = spring.get_iteration_path(n)
        knames = {2: ("row_split", "col_split")}.get(path, ("row_iter", "col_pm"))
        traffic = None
        prof = ROOT / "profiles" / "traffic.json"
        if prof.exists():
            try:
                traffic = json.loads(prof.read_text()).get(knames[kc])
            except Exception:
                traffic = None
        golden = {}
        if GOLDEN_ORACLE.exists():
            golden = json.loads(GOLDEN_ORACLE.read_text()).get(wl, {})
        cpu = None
        if ws == 1 and not args.no_cpu:
            cpu = oracle_sample(pat, prm, seconds=args.cpu_seconds)
            cpu = {k: cpu[k] for k in ("value", "cores", "sample")} | {"unit": "reconstructions/s",
                                                                        "kind": "oracle"}
        ea = [e[0] for e in errs]
        eb = [e[1] for e in errs]
        out = {
            "metric": "MPR reconstructions/s", "value": value, "unit": "reconstructions/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(wl, n, prm, args.graph),
            "iteration_pixels_per_s": value * pixels_per_reconstruction(n, prm),
            "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))},
            "error": {"final_error_avg": statistics.mean(ea), "final_error_best": statistics.mean(eb),
                      "oracle": golden or None},
            "roofline": {"bound": "hbm", "kernel": knames[kc], "iteration_path": path,
                         "achieved": achieved, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                         "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                         "bytes_per_launch": st.bytes_per_launch, "avg_launch_ms": avg_ms,
                         "launches_timed": st.timed, "timing_stride": TIMING_STRIDE,
                         "other_kernel": {"name": knames[1 - kc],
                                          "avg_launch_ms": oavg,
                                          "achieved": other.bytes_per_launch / (oavg / 1000.0) / 1e9 if oavg > 0 else None}},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e, "unit": "reconstructions/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": int(launches),
            "graph_capture": graph_out,
            "clocks": clk,
        }
        if ws == 1 and not args.no_production:
            out["production"] = production_legs(spring, ctx, args)
        print(json.dumps(out), flush=True)
    prob.destroy()
    ctx.close()
    if pg:
        pg.destroy_process_group()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="ell512", choices=sorted(WORKLOADS))
    ap.add_argument("--graph", type=int, default=0,
                    help="capture each run as one CUDA graph (per-kernel roofline timing is then "
                         "unavailable: launches inside a capture carry no events)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-production", action="store_true",
                    help="skip the precision, batched-uneven and serving legs (reported beside the headline)")
    ap.add_argument("--serve-seconds", type=float, default=2.0,
                    help="arrival window of the serving leg at 200 requests/s")
    ap.add_argument("--batch-patterns", type=int, default=64,
                    help="patterns in the batched-uneven leg")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args, args.workload)
    else:
        run_ours(args, args.workload)


if __name__ == "__main__":
    main()
