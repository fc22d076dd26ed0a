"""Batched uneven workload: many patterns of different sides reconstructed together.

    python -m paper_2409_07413_gb300.batchbench [--patterns 256] [--generations 5]

Patterns: sides drawn uniformly from {128, 192, 256, 512}; objects, masks and noise as the
`ellN` recipe (extent 0.25 N, 1e6-1e7 photons, beamstop, gap, saturation); P = 32 each,
G generations x 200 RAAR iterations.  Two ways to run the same set:

  served: every pattern submitted at once (spring_submit); the scheduler runs several
          populations of different sides concurrently on prioritised streams, advancing
          each a generation at a time (continuous batching);
  plain:  spring_mpr_run one pattern after another;
  batched: the patterns grouped by side, each group run K at a time with
          spring_mpr_run_batch (one launch per iteration pass over K x 2P images; K such
          that a launch covers about --batch-pixels pixels);
  mixed:  the whole set in one spring_mpr_run_batch call: one group per side sharing its
          launches, the groups as parallel branches of one CUDA graph.

--graph 1 captures each plain and batched run as one CUDA graph (instantiated and
launched inside the timed region).

Reports reconstructions/s and iteration-pixels/s of each (makespan of the whole set) and
the mean final error; all see identical requests and seeds, so the errors agree exactly
(checked pattern by pattern).
Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

SIDES = (128, 192, 256, 512)


def make_set(seed, count, variants=4, sides_from=SIDES):
    from paper_2409_07413_gb300 import synthetic
    rng = np.random.default_rng(seed)
    sides = rng.choice(sides_from, size=count)
    cache = {}
    out = []
    for i, n in enumerate(sides):
        key = (int(n), i % variants)
        if key not in cache:
            cache[key] = synthetic.config_pattern(f"ell{int(n)}", key[1])
        out.append((int(n), cache[key], 500 + i))
    return out


def run_set(ctx, spring, jobs, prm, modes=("served", "plain", "batched", "mixed"), batch_pixels=2.0 ** 26, graph=0):
    """Reconstruct the set `jobs` ((side, pattern, seed) triples) once per mode; returns the
    result dict (per mode: seconds, reconstructions/s, iteration-pixels/s, mean error)."""
    import torch
    sides = sorted({n for n, _, _ in jobs})
    work_px = sum(2 * prm["pop"] * prm["iters_per_gen"] * prm["generations"] * n * n for n, _, _ in jobs)
    out = {"benchmark": "batched uneven", "patterns": len(jobs), "graph": graph,
           "sides": {str(n): int(sum(1 for j in jobs if j[0] == n)) for n in sides}, "params": prm,
           "iteration_pixels": work_px}
    per_mode = {}
    for mode in modes:
        probs = [ctx.problem(p.intensities, p.mask, p.support0) for _, p, _ in jobs]
        torch.cuda.synchronize()
        errs = [None] * len(jobs)
        t0 = time.perf_counter()
        if mode == "mixed":  # the whole set in one call: one group per side, one CUDA graph
            rs = ctx.run_batch(probs, spring.params(**prm, use_graph=1), [j[2] for j in jobs],
                               want_arrays=False)
            for i, r in enumerate(rs):
                errs[i] = r["final_error_best"]
        elif mode == "batched":
            for n in sides:
                idx = [i for i, j in enumerate(jobs) if j[0] == n]
                K = max(1, int(batch_pixels // (2 * prm["pop"] * n * n)))
                for c in range(0, len(idx), K):
                    part = idx[c:c + K]
                    rs = ctx.run_batch([probs[i] for i in part], spring.params(**prm, use_graph=graph),
                                       [jobs[i][2] for i in part], want_arrays=False)
                    for i, r in zip(part, rs):
                        errs[i] = r["final_error_best"]
        elif mode == "served":
            tickets = [pr.submit(spring.params(**prm, seed=sd)) for pr, (_, _, sd) in zip(probs, jobs)]
            for i, t in enumerate(tickets):
                st, r = ctx.poll(t, -1, want_arrays=False)
                errs[i] = r["final_error_best"]
        else:
            for i, (pr, (_, _, sd)) in enumerate(zip(probs, jobs)):
                errs[i] = pr.run(spring.params(**prm, seed=sd, use_graph=graph),
                                 want_arrays=False)["final_error_best"]
        span = time.perf_counter() - t0
        for pr in probs:
            pr.destroy()
        per_mode[mode] = errs
        out[mode] = {"seconds": span, "reconstructions_per_s": len(jobs) / span,
                     "iteration_pixels_per_s": work_px / span, "mean_final_error_best": float(np.mean(errs))}
    ms = list(per_mode)
    out["errors_identical_across_modes"] = all(per_mode[m] == per_mode[ms[0]] for m in ms)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--patterns", type=int, default=256)
    ap.add_argument("--generations", type=int, default=5)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--modes", default="served,plain,batched,mixed")
    ap.add_argument("--batch-pixels", type=float, default=2.0 ** 26)
    ap.add_argument("--sides", default=",".join(map(str, SIDES)))
    ap.add_argument("--graph", type=int, default=0, help="1: plain and batched runs captured as CUDA graphs")
    a = ap.parse_args()
    sides = tuple(int(v) for v in a.sides.split(","))
    import torch  # noqa: F401  (device selection through the library)
    from paper_2409_07413_gb300 import spring
    prm = dict(pop=32, iters_per_gen=200, generations=a.generations, algorithm=2, beta=0.9,
               sw_sigma=1.5, sw_threshold=0.2, sw_period=20, er_tail=10)
    jobs = make_set(a.seed, a.patterns, sides_from=sides)
    ctx = spring.Context(0)
    for n in sides:  # tune each side once, outside the timed region
        spring.autotune(n, 2 * prm["pop"])
    out = run_set(ctx, spring, jobs, prm, a.modes.split(","), a.batch_pixels, a.graph)
    ctx.close()
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
