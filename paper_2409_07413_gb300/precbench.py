"""Precision benchmark: one 1024 x 1024 two-panel pattern (30-row central gap, central hole
r = 24 px, 1e8 photons with Poisson noise, 200 px object) reconstructed with P = 128,
20 generations x 300 RAAR iterations, once per storage precision:

  precision 0: complex64 state and FFT intermediate (FP32 storage, FP32 math)
  precision 1: FP16 (half2) storage of the state and the FFT intermediate inside the
               iteration blocks, FP32 math

Both runs keep the Fourier-error fitness and the shrink-wrap threshold statistics in FP64
on the GPU.  The same pattern and schedule at P = 32 and 2 generations are also run in both
precisions at every run seed for which the FP64 oracle's result is stored
(tests/golden/make_oracle_errors.py; the full 20 generations take the oracle hours) and
compared seed by seed and in the mean; the GPU's spread over 16 further run seeds shows
how far single trajectories scatter.  Per result it reports time, reconstructions/s, iteration-pixels/s, the final
Fourier error (Eq. error_calc) of the average and best individual, and the error of the
aligned average against the synthetic object (aligned by spring_reshift: translation,
twin and global phase; then the best real scale, since intensities in photon counts fix the
object only up to a global factor).

    python -m paper_2409_07413_gb300.precbench [--generations 20] [--iters 300] [--pop 128]

Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import time
from pathlib import Path

import numpy as np

GOLDEN = Path(__file__).resolve().parent.parent / "tests" / "golden" / "oracle_errors.json"


def truth_error(spring, rho, truth):
    import torch
    x = torch.from_numpy(np.ascontiguousarray(rho[None], np.complex64)).cuda()
    ref = torch.from_numpy(np.ascontiguousarray(truth[None], np.complex64)).cuda()
    ones = torch.ones(truth.shape, dtype=torch.float32, device="cuda")
    al, _, _, _ = spring.spring_reshift(x, None, ref, ones)
    torch.cuda.synchronize()
    a = al[0].cpu().numpy().astype(np.complex128)
    t = truth.astype(np.complex128)
    # the data fix the object only up to a global scale (intensities are photon counts)
    c = np.real(np.vdot(a, t)) / max(np.vdot(a, a).real, 1e-300)
    return float(np.linalg.norm(c * a - t) / np.linalg.norm(t))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--pop", type=int, default=128)
    ap.add_argument("--generations", type=int, default=20)
    ap.add_argument("--iters", type=int, default=300)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--precisions", default="0,1")
    a = ap.parse_args()
    import torch
    from paper_2409_07413_gb300 import spring, synthetic
    if not torch.cuda.is_available():
        raise SystemExit("precbench needs a CUDA GPU")
    pat = synthetic.config_pattern("ell1024", a.seed)
    n = pat.n
    prm = dict(pop=a.pop, iters_per_gen=a.iters, generations=a.generations, algorithm=2, beta=0.9,
               sw_sigma=1.5, sw_threshold=0.2, sw_period=20, er_tail=10)
    ctx = spring.Context(0)
    prob = ctx.problem(pat.intensities, pat.mask, pat.support0)
    out = {"benchmark": "precision", "workload": f"ell1024: {n}x{n}, P={a.pop}, "
           f"G={a.generations} x {a.iters} RAAR iterations", "params": prm, "runs": {}}
    px = 2 * a.pop * a.iters * a.generations * n * n
    for prec in [int(v) for v in a.precisions.split(",")]:
        warm = dict(prm, generations=1)
        prob.run(spring.params(**warm, seed=a.seed + 1, precision=prec), want_arrays=False)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = prob.run(spring.params(**prm, seed=a.seed + 1000, precision=prec))
        dt = time.perf_counter() - t0
        out["runs"][str(prec)] = {
            "storage": "fp16 (half2), fp32 math" if prec else "fp32 (complex64)",
            "seconds": dt, "reconstructions_per_s": 1.0 / dt, "iteration_pixels_per_s": px / dt,
            "final_error_avg": r["final_error_avg"], "final_error_best": r["final_error_best"],
            "truth_error_of_average": truth_error(spring, r["rho_avg"], pat.truth),
        }
    # the reduced configuration the oracle has run (2 generations), at its run seeds
    golden = json.loads(GOLDEN.read_text()) if GOLDEN.exists() else {}
    orc = {g["run_seed"]: g for k, g in golden.items() if k == "ell1024_g2" or k.startswith("ell1024_g2_r")}
    red = dict(prm, pop=32, generations=2)
    keys = ("final_error_avg", "final_error_best")
    cmp = {"config": red, "run_seeds": sorted(orc),
           "oracle_fp64": {str(sd): {k: orc[sd][k] for k in keys} for sd in sorted(orc)}}
    if orc:
        cmp["oracle_fp64"]["mean"] = {k: float(np.mean([orc[sd][k] for sd in orc])) for k in keys}
    for prec in [int(v) for v in a.precisions.split(",")]:
        per = {}
        for sd in sorted(orc):
            r = prob.run(spring.params(**red, seed=sd, precision=prec))
            per[str(sd)] = {"final_error_avg": r["final_error_avg"], "final_error_best": r["final_error_best"],
                            "truth_error_of_average": truth_error(spring, r["rho_avg"], pat.truth)}
        if orc:
            per["mean"] = {k: float(np.mean([per[str(sd)][k] for sd in orc])) for k in keys}
        spread = [prob.run(spring.params(**red, seed=2000 + i, precision=prec), want_arrays=False)
                  for i in range(16)]
        per["spread_16_seeds"] = {k: {"mean": float(np.mean([r[k] for r in spread])),
                                      "std": float(np.std([r[k] for r in spread], ddof=1))} for k in keys}
        cmp[str(prec)] = per
    out["versus_oracle"] = cmp
    prob.destroy()
    ctx.close()
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
