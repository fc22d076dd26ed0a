"""The paper's own timing workload: one MPR reconstruction with the default parameters of
its parameter table (Table params; Sec. "Time to solution"): P = 128, G = 100, N = 512,
Sequence of j = 40 IA (RAAR, beta 0.9) and j_ER = 40 ER iterations changing linearly over
the generations (App. "Changing values over generations"), R = 3 repetitions, j_eval = 40,
shrink-wrap sigma 2 -> 0.5 px and tau -> 2/3 tau (tau has no default in the table: 0.2 as
in the other workloads), chi = 0.5, C_p = 0.6, C_w = 0.4.

    python -m paper_2409_07413_gb300.paperbench [--runs 1] [--graph 0]

Per generation 3 x 80 + 40 = 280 iterations of 2P = 256 individuals: 1.88e12 iteration
pixels per reconstruction.  Pattern: `ell512` (seeded synthetic, 512^2).  Prints one JSON
line with wall-clock seconds per reconstruction (device synchronised), iteration-pixels/s
and the final errors.
"""
from __future__ import annotations

import argparse
import json
import time


def paper_params(spring, seed, graph=0):
    return spring.params(pop=128, generations=100, algorithm=2, beta=0.9, chi=0.5, schedule=1,
                         seq_ia=40, seq_er=40, seq_eval=40, repetitions=3, sw_sigma=2.0,
                         sw_sigma_end=0.5, sw_threshold=0.2, sw_threshold_end=0.2 * 2.0 / 3.0,
                         cw=0.4, cp=0.6, seed=seed, use_graph=graph)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--runs", type=int, default=1)
    ap.add_argument("--graph", type=int, default=0)
    ap.add_argument("--seed", type=int, default=0)
    a = ap.parse_args()
    import torch
    from paper_2409_07413_gb300 import spring, synthetic
    pat = synthetic.config_pattern("ell512", a.seed)
    ctx = spring.Context(0)
    prob = ctx.problem(pat.intensities, pat.mask, pat.support0)
    spring.autotune(512, 256)
    # warm-up: a short run with the same shapes
    warm = paper_params(spring, a.seed, a.graph)
    warm.generations = 2
    prob.run(warm, want_arrays=False)
    torch.cuda.synchronize()
    secs, errs = [], []
    for r in range(a.runs):
        t0 = time.perf_counter()
        res = prob.run(paper_params(spring, a.seed + r, a.graph), want_arrays=False)
        torch.cuda.synchronize()
        secs.append(time.perf_counter() - t0)
        errs.append((res["final_error_best"], res["final_error_avg"]))
    prob.destroy()
    ctx.close()
    iters = 100 * (3 * 80 + 40)
    px = 256 * iters * 512 * 512
    s = min(secs)
    print(json.dumps({"benchmark": "paper default workload", "P": 128, "G": 100, "N": 512,
                      "iterations_per_individual": iters, "iteration_pixels": px,
                      "seconds_per_reconstruction": secs, "reconstructions_per_s": 1.0 / s,
                      "iteration_pixels_per_s": px / s, "graph": a.graph,
                      "final_error_best_avg": errs}), flush=True)


if __name__ == "__main__":
    main()
