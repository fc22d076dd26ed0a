"""Whole runs on the split passes against whole runs on the two passes (iteration paths 2 and
0) at 384 x 384 (Q = 3), 512 x 512 (Q = 2) and 1024 x 1024 (Q = 8): the same patterns and
run seeds, many of them, and the means of the final errors (of the average reconstruction
and of the best individual) within the plain 2% of each other.  Both paths compute the same unnormalised 2D transform pair in
another order of summation; single trajectories part after a few iterations (HIO/RAAR and
the GA amplify rounding), so the comparison is between the two distributions over seeds.
With a short schedule the runs take milliseconds, so enough seeds fit that the standard
error of the difference stays far under the bar."""
import numpy as np
import pytest

from paper_2409_07413_gb300 import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sp():
    import torch
    from paper_2409_07413_gb300 import spring
    assert torch.cuda.is_available()
    return spring


CASES = {
    "ell384": (dict(pop=16, iters_per_gen=100, generations=4, er_tail=10, sw_period=20), 200),
    "ell512": (dict(pop=16, iters_per_gen=100, generations=4, er_tail=10, sw_period=20), 200),
    "ell1024": (dict(pop=8, iters_per_gen=100, generations=3, er_tail=10, sw_period=20), 100),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_split_runs_match_two_pass_runs_over_seeds(sp, name):
    kw, nseeds = CASES[name]
    pat = synthetic.config_pattern(name, 0)
    n = pat.n
    seeds = list(range(500, 500 + nseeds))
    ctx = sp.Context(0)
    saved = sp.get_iteration_path(n)
    res = {}
    try:
        prob = ctx.problem(pat.intensities, pat.mask, pat.support0)
        p = sp.params(**kw)
        for path in (0, 2):
            sp.set_iteration_path(n, path)
            out = []
            for i in range(0, nseeds, 50):
                chunk = seeds[i:i + 50]
                out += ctx.run_batch([prob] * len(chunk), p, chunk, want_arrays=False)
            res[path] = out
        prob.destroy()
    finally:
        sp.set_iteration_path(n, saved)
        ctx.close()
    for key in ("final_error_avg", "final_error_best"):
        two = np.array([r[key] for r in res[0]])
        split = np.array([r[key] for r in res[2]])
        assert np.isfinite(two).all() and np.isfinite(split).all()
        se = np.sqrt(two.var(ddof=1) / len(two) + split.var(ddof=1) / len(split))
        rel = (split.mean() - two.mean()) / two.mean()
        print(f"{name} x {nseeds} seeds, {key}: split {split.mean():.5f} two passes {two.mean():.5f} "
              f"({100 * rel:+.2f}%; standard error of the difference {100 * se / two.mean():.2f}%)")
        assert abs(rel) <= 0.02, (key, rel)
