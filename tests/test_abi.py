"""The C ABI library builds, loads without a GPU, and exports every entry point that
include/spring.h declares; the binding's structures match the header's layouts."""
import ctypes as C
import re
import subprocess
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent
HEADER = ROOT / "include" / "spring.h"


@pytest.fixture(scope="module")
def libpath():
    from paper_2409_07413_gb300 import build
    return build.build()


def header_functions():
    text = re.sub(r"/\*.*?\*/", "", HEADER.read_text(), flags=re.S)
    names = re.findall(r"^\s*[A-Za-z_][\w\s\*]*?\b(spring_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    fns = header_functions()
    for required in ["spring_init", "spring_shutdown", "spring_problem_create",
                     "spring_problem_destroy", "spring_mpr_run", "spring_submit", "spring_poll",
                     "spring_cancel", "spring_status_string", "spring_last_error"]:
        assert required in fns


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", str(libpath)], capture_output=True,
                         text=True, check=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if l.strip()}
    missing = [f for f in header_functions() if f not in exported]
    assert not missing, missing


def test_binding_covers_header(libpath):
    from paper_2409_07413_gb300 import spring
    assert sorted(spring.EXPORTED) == header_functions()


def test_loads_without_gpu_and_static_calls(libpath):
    from paper_2409_07413_gb300 import spring
    L = spring.lib()
    assert L.spring_abi_version() == 2
    assert L.spring_status_string(0) == b"ok"
    assert L.spring_status_string(1) == b"invalid argument"
    p = spring.params(pop=64, iters_per_gen=200, generations=10)
    assert (p.pop, p.iters_per_gen, p.generations, p.algorithm) == (64, 200, 10, 2)
    assert abs(p.beta - 0.9) < 1e-7 and abs(p.sw_sigma - 1.5) < 1e-7 and p.sw_period == 20
    assert p.er_tail == 10 and abs(p.cp - 0.6) < 1e-7 and abs(p.cw - 0.4) < 1e-7
    # footprint is pure host arithmetic: 2P images of x and w (8 B), S (1 B), two float maps
    fp = spring.footprint_bytes(512, p)
    assert fp >= 128 * 512 * 512 * (8 + 8 + 1 + 4 + 4)
    assert fp < 1.2 * 128 * 512 * 512 * (8 + 8 + 1 + 4 + 4) + (1 << 26)
    assert spring.footprint_bytes(500, p) == 0


_LAYOUT_C = r"""
#include <stdio.h>
#include <stddef.h>
#include "spring.h"
#define F(T, m) printf("%s.%s %zu\n", #T, #m, offsetof(T, m));
int main(void) {
  printf("spring_params %zu\nspring_result %zu\nspring_kernel_stat %zu\nspring_bounds %zu\n",
         sizeof(spring_params), sizeof(spring_result), sizeof(spring_kernel_stat),
         sizeof(spring_bounds));
  F(spring_params, pop) F(spring_params, beta) F(spring_params, sw_period) F(spring_params, chi)
  F(spring_params, tile_min) F(spring_params, init_gamma) F(spring_params, precision)
  F(spring_params, use_graph) F(spring_params, schedule) F(spring_params, repetitions)
  F(spring_params, ca) F(spring_params, monitor_avg) F(spring_params, seed)
  F(spring_result, gen_stats) F(spring_result, final_error_avg) F(spring_result, t_done_s)
  F(spring_kernel_stat, total_ms) F(spring_kernel_stat, bytes_per_launch)
  F(spring_bounds, eta) F(spring_bounds, max_missing) F(spring_bounds, max_saturated)
  return 0;
}
"""


def test_struct_layouts_match_header(tmp_path):
    from paper_2409_07413_gb300 import spring
    src = tmp_path / "layout.c"
    src.write_text(_LAYOUT_C)
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", str(ROOT / "include"), str(src), "-o", str(exe)], check=True)
    vals = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], capture_output=True,
                                                          text=True, check=True).stdout.splitlines())
    vals = {k: int(v) for k, v in vals.items()}
    assert vals["spring_params"] == C.sizeof(spring.Params)
    assert vals["spring_result"] == C.sizeof(spring.Result)
    assert vals["spring_kernel_stat"] == C.sizeof(spring.KernelStat)
    assert vals["spring_bounds"] == C.sizeof(spring.Bounds)
    cls = {"spring_params": spring.Params, "spring_result": spring.Result,
           "spring_kernel_stat": spring.KernelStat, "spring_bounds": spring.Bounds}
    for k, v in vals.items():
        if "." in k:
            t, m = k.split(".")
            assert getattr(cls[t], m).offset == v, k


def test_product_path_does_not_touch_the_oracle():
    # the library sources and the binding never include, load or import the oracle
    pkg = ROOT / "paper_2409_07413_gb300"
    pat = re.compile(r"(import\s+oracle|from\s+oracle|spring_oracle|orc_\w+|#include\s+\"[^\"]*oracle)")
    for f in list((pkg / "csrc").glob("*")) + list(pkg.glob("*.py")):
        assert not pat.search(f.read_text()), f
