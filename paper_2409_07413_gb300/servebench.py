"""Serving benchmark: a seeded Poisson stream of single-shot patterns of mixed sizes,
reconstructed by continuous batching (spring_submit / spring_poll: requests are admitted
by HBM footprint as they arrive and their work overlaps on the GPU) and, for comparison,
by the plain path (spring_mpr_run one pattern at a time, in arrival order).

    python -m paper_2409_07413_gb300.servebench --rate 20 --duration 10

Sizes are drawn from {128, 256, 512, 1024} with weights 0.4/0.3/0.2/0.1; every request
runs P = 32, 5 generations x 200 RAAR iterations.  Latency is completion - arrival
(arrival = scheduled submission time); service time is completion - admission (served: the
library's admission and completion clocks of each request; plain: the run itself).  Both
modes see the same requests and arrival times, and report percentiles overall and per
side.  Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import threading
import time

import numpy as np

SIDES = (128, 256, 512, 1024)
WEIGHTS = (0.4, 0.3, 0.2, 0.1)
PARAMS = dict(pop=32, iters_per_gen=200, generations=5, algorithm=2, beta=0.9, sw_sigma=1.5,
              sw_threshold=0.2, sw_period=20, er_tail=10)


def make_stream(seed, rate, duration):
    from paper_2409_07413_gb300 import synthetic
    arr = synthetic.poisson_arrivals(seed, rate, duration)
    rng = np.random.default_rng(seed + 7)
    sides = rng.choice(SIDES, size=len(arr), p=WEIGHTS)
    pats = {}
    reqs = []
    for i, (t, n) in enumerate(zip(arr, sides)):
        key = (int(n), i % 4)  # four distinct patterns per side
        if key not in pats:
            pats[key] = synthetic.config_pattern(f"ell{n}", key[1])
        reqs.append((float(t), int(n), pats[key], 1000 + i))
    return reqs


def percentiles(lat):
    lat = np.asarray(lat)
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "max_s": float(lat.max())}


def run_served(ctx, spring, reqs):
    """Submit each request at its arrival time; poll all; latency = done - arrival."""
    t0 = time.monotonic()
    tickets = [None] * len(reqs)
    probs = [None] * len(reqs)

    def feeder():
        for i, (ta, n, pat, seed) in enumerate(reqs):
            d = t0 + ta - time.monotonic()
            if d > 0:
                time.sleep(d)
            pr = ctx.problem(pat.intensities, pat.mask, pat.support0)
            probs[i] = pr
            tickets[i] = pr.submit(spring.params(**PARAMS, seed=seed))

    th = threading.Thread(target=feeder)
    th.start()
    lat, svc, errs, sizes = [], [], [], []
    done = 0
    while done < len(reqs):
        for i in range(len(reqs)):
            if tickets[i] is None or tickets[i] == -1:
                continue
            st, r = ctx.poll(tickets[i], 0, want_arrays=False)
            if st == spring.OK:
                tdone = time.monotonic() - t0
                lat.append(tdone - reqs[i][0])
                svc.append(r["t_done_s"] - r["t_admit_s"])
                errs.append(r["final_error_best"])
                sizes.append(reqs[i][1])
                tickets[i] = -1
                done += 1
        time.sleep(0.0005)
    th.join()
    makespan = time.monotonic() - t0
    for pr in probs:  # after timing: freeing device memory may synchronise the device
        pr.destroy()
    return lat, svc, errs, sizes, makespan


def run_plain(ctx, spring, reqs):
    """One pattern at a time in arrival order (waiting for arrivals)."""
    t0 = time.monotonic()
    lat, svc, errs, sizes = [], [], [], []
    for (ta, n, pat, seed) in reqs:
        d = t0 + ta - time.monotonic()
        if d > 0:
            time.sleep(d)
        ts = time.monotonic()
        pr = ctx.problem(pat.intensities, pat.mask, pat.support0)
        r = pr.run(spring.params(**PARAMS, seed=seed), want_arrays=False)
        pr.destroy()
        te = time.monotonic()
        lat.append(te - t0 - ta)
        svc.append(te - ts)
        errs.append(r["final_error_best"])
        sizes.append(n)
    return lat, svc, errs, sizes, time.monotonic() - t0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--rate", type=float, default=20.0)
    ap.add_argument("--duration", type=float, default=10.0)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--modes", default="served,plain")
    a = ap.parse_args()
    import torch  # noqa: F401  (device selection through the library)
    from paper_2409_07413_gb300 import spring
    reqs = make_stream(a.seed, a.rate, a.duration)
    ctx = spring.Context(0)
    # tune every side once before timing (the autotuner runs once per side and process)
    for n in SIDES:
        spring.autotune(n, 2 * PARAMS["pop"])
    out = {"benchmark": "serving", "rate_hz": a.rate, "duration_s": a.duration, "requests": len(reqs),
           "sizes": {str(n): int(sum(1 for r in reqs if r[1] == n)) for n in SIDES}, "params": PARAMS}
    work_px = sum(2 * PARAMS["pop"] * PARAMS["iters_per_gen"] * PARAMS["generations"] * r[1] ** 2 for r in reqs)
    for mode in a.modes.split(","):
        fn = run_served if mode == "served" else run_plain
        lat, svc, errs, sizes, span = fn(ctx, spring, reqs)
        sizes = np.asarray(sizes)
        out[mode] = {"reconstructions_per_s": len(lat) / span, "makespan_s": span,
                     "iteration_pixels_per_s": work_px / span, **percentiles(lat),
                     "service": percentiles(svc),
                     "per_side": {str(n): {"latency": percentiles(np.asarray(lat)[sizes == n]),
                                           "service": percentiles(np.asarray(svc)[sizes == n])}
                                  for n in SIDES if (sizes == n).any()},
                     "mean_final_error_best": float(np.mean(errs))}
    ctx.close()
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
