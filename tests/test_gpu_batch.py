"""Batched runs of several patterns (same-side patterns share one launch per iteration pass
over all their populations, the GA steps pattern by pattern; patterns of different sides
run as concurrent groups, in one CUDA graph when captured): each pattern's result equals
its own single run with the same seed bit for bit, in every iteration path and schedule."""
import numpy as np
import pytest

from paper_2409_07413_gb300 import synthetic

pytestmark = pytest.mark.gpu

KEYS = ("rho_avg", "rho_best", "support_avg", "gen_stats", "final_error_avg", "final_error_best")


@pytest.fixture(scope="module")
def sp():
    import torch
    from paper_2409_07413_gb300 import spring
    assert torch.cuda.is_available()
    return spring


@pytest.fixture(scope="module")
def ctx(sp):
    c = sp.Context(0)
    yield c
    c.close()


def problems(ctx, name, K):
    out = []
    for q in range(K):
        pat = synthetic.config_pattern(name, 10 + q)
        out.append(ctx.problem(pat.intensities, pat.mask, pat.support0))
    return out


def same(a, b):
    for k in KEYS:
        assert np.array_equal(np.asarray(a[k]), np.asarray(b[k]), equal_nan=True), k


BASE = dict(pop=4, iters_per_gen=40, generations=3, algorithm=2, beta=0.9, sw_sigma=1.5,
            sw_threshold=0.2, sw_period=20, er_tail=5)


@pytest.mark.parametrize("name", ["sphere64", "ell128", "ell256"])
@pytest.mark.parametrize("graph", [0, 1])
def test_batch_equals_single_runs(sp, ctx, name, graph):
    K = 3
    probs = problems(ctx, name, K)
    seeds = [5, 17, 5]  # a repeated seed on a different pattern must not couple the two
    p = sp.params(**BASE, use_graph=graph)
    batch = ctx.run_batch(probs, p, seeds)
    for q in range(K):
        single = probs[q].run(sp.params(**BASE, seed=seeds[q]))
        same(batch[q], single)
    assert not np.array_equal(batch[0]["rho_avg"], batch[2]["rho_avg"])
    for pr in probs:
        pr.destroy()


@pytest.mark.parametrize("extra", [dict(schedule=1, repetitions=3, seq_ia=10, seq_er=5, seq_eval=5),
                                   dict(ca=0.3, monitor_avg=1),
                                   dict(algorithm=1, sw_sigma_end=1.0, sw_threshold_end=0.1)])
def test_batch_equals_single_runs_in_every_schedule(sp, ctx, extra):
    K = 2
    probs = problems(ctx, "ell128", K)
    seeds = [3, 4]
    kw = {**BASE, **extra}
    batch = ctx.run_batch(probs, sp.params(**kw), seeds)
    for q in range(K):
        same(batch[q], probs[q].run(sp.params(**kw, seed=seeds[q])))
    for pr in probs:
        pr.destroy()


def test_batch_of_one_is_a_run(sp, ctx):
    pr = problems(ctx, "ell192", 1)[0]
    p = sp.params(**BASE, precision=1)  # a batch of one keeps every option
    same(ctx.run_batch([pr], p, [9])[0], pr.run(sp.params(**BASE, precision=1, seed=9)))
    pr.destroy()


@pytest.mark.parametrize("graph", [0, 1])
def test_mixed_side_batch_equals_single_runs(sp, ctx, graph):
    # problems of four sides in one call: one group per side sharing its launches, the groups
    # concurrent on their own streams (with use_graph, parallel branches of one CUDA graph);
    # every result is the problem's single run bit for bit, in the callers' order
    names = ["ell128", "sphere64", "ell192", "ell128", "ell96", "sphere64"]
    probs = []
    for q, name in enumerate(names):
        pat = synthetic.config_pattern(name, 30 + q)
        probs.append(ctx.problem(pat.intensities, pat.mask, pat.support0))
    seeds = [11, 12, 13, 14, 15, 16]
    batch = ctx.run_batch(probs, sp.params(**BASE, use_graph=graph), seeds)
    for q in range(len(names)):
        same(batch[q], probs[q].run(sp.params(**BASE, seed=seeds[q])))
    for pr in probs:
        pr.destroy()


def test_batch_invalid_arguments(sp, ctx):
    a = problems(ctx, "sphere64", 2)
    b = problems(ctx, "ell128", 1)
    with pytest.raises(sp.SpringError) as e:  # mixed sides keep the batch's restrictions
        ctx.run_batch([a[0], b[0]], sp.params(**BASE, precision=1), [1, 2])
    assert e.value.status == sp.E_INVALID
    with sp.Context(0) as other:  # problems of another context
        pat = synthetic.config_pattern("sphere64", 3)
        c = other.problem(pat.intensities, pat.mask, pat.support0)
        with pytest.raises(sp.SpringError) as e:
            ctx.run_batch([a[0], c], sp.params(**BASE), [1, 2])
        assert e.value.status == sp.E_INVALID
        c.destroy()
    for bad in (dict(precision=1), dict(mode=1)):
        with pytest.raises(sp.SpringError) as e:
            ctx.run_batch(a, sp.params(**BASE, **bad), [1, 2])
        assert e.value.status == sp.E_INVALID, bad
    with pytest.raises(sp.SpringError):
        ctx.run_batch([], sp.params(**BASE), [])
    for pr in a + b:
        pr.destroy()


def test_batch_of_bounded_and_plain_problems(sp, ctx):
    # the gathered modulus arrays carry each problem's own upper bounds (Eq. pm_bounds)
    pats = [synthetic.config_pattern("ell128", s) for s in (20, 21, 22)]
    probs = [ctx.problem(pats[0].intensities, pats[0].mask, pats[0].support0, saturated=pats[0].saturated,
                         bounds=sp.bounds()),
             ctx.problem(pats[1].intensities, pats[1].mask, pats[1].support0),
             ctx.problem(pats[2].intensities, pats[2].mask, pats[2].support0, bounds=sp.bounds(eta=1.0))]
    seeds = [7, 8, 9]
    batch = ctx.run_batch(probs, sp.params(**BASE), seeds)
    for q in range(3):
        same(batch[q], probs[q].run(sp.params(**BASE, seed=seeds[q])))
    for pr in probs:
        pr.destroy()
