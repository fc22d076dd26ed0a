"""Micro-benchmark of the per-iteration passes (row pass with the fused update, column
pass with the fused modulus projection) on random state.

    python -m paper_2409_07413_gb300.iterbench --n 512 --batch 128 --iters 50 --alg 2 [--precision 1]

Prints one JSON line per side with each pass's average CUDA-event time, algorithmic bytes
and GB/s (events are recorded on the launching stream around every launch).

With --cufft it also times, as a reference point only, cuFFT through torch.fft on the same
batch: the forward + inverse unitary 2D transform pair alone, and one whole RAAR iteration
written as library calls (fft2, the masked modulus projection and the update as torch
elementwise operations, ifft2).  Neither is on the library's path.
"""
from __future__ import annotations

import argparse
import json

import numpy as np


def run(n, batch, iters, alg, warm=3, precision=0):
    import torch

    from paper_2409_07413_gb300 import spring

    g = torch.Generator(device="cuda").manual_seed(n)
    x = torch.randn((batch, n, n), dtype=torch.complex64, device="cuda", generator=g)
    S = (torch.rand((batch, n, n), device="cuda", generator=g) < 0.25).to(torch.uint8)
    M = torch.rand((n, n), device="cuda", generator=g) + 0.1
    M[torch.rand((n, n), device="cuda", generator=g) < 0.05] = -1.0
    spring.spring_iterate_ex(x, S, M, alg, 0.9, 0.5, warm, precision)
    torch.cuda.synchronize()
    spring.stats_reset()
    spring.stats_enable_timing(True)
    spring.spring_iterate_ex(x, S, M, alg, 0.9, 0.5, iters, precision)
    torch.cuda.synchronize()
    spring.stats_enable_timing(False)
    out = {"n": n, "batch": batch, "iters": iters, "alg": alg, "precision": precision}
    for name, kc in (("row_iter", spring.KC_ROW_ITER), ("col_pm", spring.KC_COL_PM)):
        st = spring.stats_get(kc)
        ms = st.total_ms / max(1, st.timed)
        out[name] = {"avg_ms": ms, "bytes": st.bytes_per_launch,
                     "GBps": st.bytes_per_launch / (ms / 1e3) / 1e9 if ms > 0 else None}
    it_ms = out["row_iter"]["avg_ms"] + out["col_pm"]["avg_ms"]
    out["iteration_ms"] = it_ms
    out["iteration_px_per_s"] = batch * n * n / (it_ms / 1e3)
    return out


def run_fused(n, batch, iters, alg, warm=3):
    """The on-chip kernel: one launch of `iters` iterations (N <= 256)."""
    import torch

    from paper_2409_07413_gb300 import spring

    g = torch.Generator(device="cuda").manual_seed(n)
    x = torch.randn((batch, n, n), dtype=torch.complex64, device="cuda", generator=g)
    S = (torch.rand((batch, n, n), device="cuda", generator=g) < 0.25).to(torch.uint8)
    M = torch.rand((n, n), device="cuda", generator=g) + 0.1
    M[torch.rand((n, n), device="cuda", generator=g) < 0.05] = -1.0
    spring.spring_iterate_fused(x, S, M, alg, 0.9, 0.5, warm)
    torch.cuda.synchronize()
    spring.stats_reset()
    spring.stats_enable_timing(True)
    spring.spring_iterate_fused(x, S, M, alg, 0.9, 0.5, iters)
    torch.cuda.synchronize()
    spring.stats_enable_timing(False)
    st = spring.stats_get(spring.KC_FUSED)
    ms = st.total_ms / max(1, st.timed)
    return {"n": n, "batch": batch, "iters": iters, "alg": alg, "path": "on-chip", "launch_ms": ms,
            "iteration_ms": ms / iters, "iteration_px_per_s": batch * n * n * iters / (ms / 1e3)}


def run_cufft(n, batch, iters, warm=3, beta=0.9):
    """cuFFT reference (torch.fft): the transform pair, and a RAAR iteration from library calls."""
    import torch

    g = torch.Generator(device="cuda").manual_seed(n)
    x = torch.randn((batch, n, n), dtype=torch.complex64, device="cuda", generator=g)
    S = torch.rand((batch, n, n), device="cuda", generator=g) < 0.25
    M = torch.rand((n, n), device="cuda", generator=g) + 0.1
    meas = torch.rand((n, n), device="cuda", generator=g) >= 0.05

    def pair(v):
        return torch.fft.ifft2(torch.fft.fft2(v, norm="ortho"), norm="ortho")

    def iteration(v):
        X = torch.fft.fft2(v, norm="ortho")
        a = X.abs()
        Y = torch.where(meas & (a > 0), X * (M / torch.where(a > 0, a, torch.ones_like(a))), X)
        m = torch.fft.ifft2(Y, norm="ortho")
        return torch.where(S, m, beta * v + (1 - 2 * beta) * m)

    out = {"n": n, "batch": batch, "iters": iters, "reference": "cuFFT via torch.fft"}
    for name, fn in (("fft_pair", pair), ("library_iteration", iteration)):
        y = x
        for _ in range(warm):
            y = fn(y)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(iters):
            y = fn(y)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / iters
        out[name] = {"ms": ms, "px_per_s": batch * n * n / (ms / 1e3)}
    return out


def sweep(n, batch, iters, alg):
    """Time every (row, column) launch variant of side n; returns the list of results."""
    from paper_2409_07413_gb300 import spring
    saved = spring.get_kernel_variant(n)
    res = []
    try:
        for rv in range(7):
            for cv in range(11):
                spring.set_kernel_variant(n, rv, cv)
                r = run(n, batch, iters, alg)
                r["variant"] = [rv, cv]
                res.append(r)
    finally:
        spring.set_kernel_variant(n, *saved)
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, nargs="+", default=[512])
    ap.add_argument("--batch", type=int, default=128)
    ap.add_argument("--iters", type=int, default=50)
    ap.add_argument("--alg", type=int, default=2)
    ap.add_argument("--precision", type=int, default=0, help="0: FP32 storage, 1: FP16 storage")
    ap.add_argument("--sweep", action="store_true", help="time every launch variant")
    ap.add_argument("--fused", action="store_true", help="also time the on-chip kernel (N <= 256)")
    ap.add_argument("--cufft", action="store_true", help="also time the cuFFT reference (torch.fft)")
    ap.add_argument("--variant", type=int, nargs=2, default=None, metavar=("ROW", "COL"),
                    help="launch-shape variants of the two passes (default: the built-in defaults)")
    ap.add_argument("--path", type=int, default=None,
                    help="iteration path: 0 two passes, 1 on chip (N <= 256), 2 split passes (192-1024); "
                         "with --variant or --sweep and no --path, 0 (the variants are shapes of the two passes)")
    a = ap.parse_args()
    if (a.variant or a.sweep) and a.path is None:
        a.path = 0
    if a.variant or a.path is not None:
        from paper_2409_07413_gb300 import spring
        for n in a.n:
            if a.variant:
                spring.set_kernel_variant(n, *a.variant)
            if a.path is not None:
                spring.set_iteration_path(n, a.path)
    for n in a.n:
        b = a.batch if a.batch > 0 else max(1, (128 * 512 * 512) // (n * n))
        if a.sweep:
            for r in sweep(n, b, a.iters, a.alg):
                print(json.dumps({"n": n, "variant": r["variant"], "row_ms": r["row_iter"]["avg_ms"],
                                  "row_GBps": r["row_iter"]["GBps"], "col_ms": r["col_pm"]["avg_ms"],
                                  "col_GBps": r["col_pm"]["GBps"]}), flush=True)
        else:
            print(json.dumps(run(n, b, a.iters, a.alg, precision=a.precision)), flush=True)
        if a.fused and n <= 256:
            print(json.dumps(run_fused(n, b, a.iters, a.alg)), flush=True)
        if a.cufft:
            print(json.dumps(run_cufft(n, b, a.iters)), flush=True)


if __name__ == "__main__":
    main()
