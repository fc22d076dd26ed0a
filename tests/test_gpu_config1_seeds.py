"""End to end at the 64 x 64 workload (P = 8, 5 x 100 RAAR): the GPU's final errors against
the FP64 oracle's over the same 8000 run seeds of one pattern, with the plain 2% bar on the
mean: |mean_gpu - mean_oracle| <= 0.02 mean_oracle, for the error of the average
reconstruction and for the best individual, with no allowance for sampling.

Single trajectories are not expected to agree (HIO/RAAR and the GA amplify FP32 rounding),
so the comparison is between the two distributions over seeds.  The error of the average
scatters by about 19% of its mean from seed to seed; over 8000 seeds the standard error of
each mean is about 0.2%, so the 2% bar stands at several standard errors of the difference
and a real bias of 2% would not hide in the sampling.  The oracle's values are stored in
tests/golden/oracle_sphere64_seeds.json (written by tests/golden/make_oracle_errors.py
--seeds, which calls only the oracle)."""
import json
from pathlib import Path

import numpy as np
import pytest

from paper_2409_07413_gb300 import synthetic

pytestmark = pytest.mark.gpu

GOLDEN = Path(__file__).resolve().parent / "golden" / "oracle_sphere64_seeds.json"


@pytest.fixture(scope="module")
def sp():
    import torch
    from paper_2409_07413_gb300 import spring
    assert torch.cuda.is_available()
    return spring


def test_sphere64_seeds_within_two_percent(sp):
    gold = json.loads(GOLDEN.read_text())
    s0, s1 = gold["run_seeds"]
    seeds = list(range(s0, s1))
    prm = gold["params"]
    pat = synthetic.config_pattern(gold["workload"], gold["pattern_seed"])
    ctx = sp.Context(0)
    try:
        prob = ctx.problem(pat.intensities, pat.mask, pat.support0)
        p = sp.params(**prm)
        ea, eb = [], []
        for i in range(0, len(seeds), 100):
            chunk = seeds[i:i + 100]
            for r in ctx.run_batch([prob] * len(chunk), p, chunk, want_arrays=False):
                ea.append(r["final_error_avg"])
                eb.append(r["final_error_best"])
        prob.destroy()
    finally:
        ctx.close()
    ga, gb = np.array(ea), np.array(eb)
    oa, ob = np.array(gold["final_error_avg"]), np.array(gold["final_error_best"])
    assert len(ga) == len(oa) == len(seeds) and np.isfinite(ga).all() and np.isfinite(gb).all()
    for name, g, o in (("average", ga, oa), ("best", gb, ob)):
        se = np.sqrt(g.var(ddof=1) / len(g) + o.var(ddof=1) / len(o))
        se_paired = np.std(g - o, ddof=1) / np.sqrt(len(g))  # the same run seeds on both sides
        rel = (g.mean() - o.mean()) / o.mean()
        print(f"sphere64 x {len(g)} seeds, error of the {name}: gpu {g.mean():.5f} oracle {o.mean():.5f} "
              f"({100 * rel:+.2f}%; standard error of the difference {100 * se / o.mean():.2f}% unpaired, "
              f"{100 * se_paired / o.mean():.2f}% paired by seed)")
        assert abs(rel) <= 0.02, (name, rel)
