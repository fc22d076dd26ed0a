"""End-to-end MPR on the GPU (through the C ABI) against the FP64 oracle, determinism,
graph capture, and serving (continuous batching: a result is the same alone and in the
mix; admission by HBM footprint; cancel; error paths)."""
import time

import numpy as np
import pytest

import oracle
from paper_2409_07413_gb300 import synthetic

pytestmark = pytest.mark.gpu

C1 = dict(pop=8, iters_per_gen=100, generations=5, algorithm=2, beta=0.9, sw_sigma=1.5,
          sw_threshold=0.2, sw_period=20, er_tail=10)


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


def aligned_rel_error(rho, truth):
    # aligned (translation, twin, global phase), then scaled by the best real factor: the
    # photon-count intensities fix the object only up to a global scale
    al, _, _, _ = oracle.reshift(rho.astype(np.complex128), None, truth, np.ones(truth.shape, np.uint8))
    c = np.real(np.vdot(al, truth)) / max(np.vdot(al, al).real, 1e-300)
    return np.linalg.norm(c * al - truth) / np.linalg.norm(truth)


def test_mpr_sphere64_matches_oracle_statistically(sp, ctx):
    # HIO/RAAR trajectories diverge from FP64 at the FP32 rate (see the operator tests), so
    # the end-to-end comparison is over seeds: the mean final error within 2 % of the
    # oracle's (widened by two standard errors of the difference of the two means), and
    # the same median recovery of the object (up to translation / twin / phase)
    eg, eo, rg, ro = [], [], [], []
    ea, oa = [], []
    for seed in range(16):
        pat = synthetic.config_pattern("sphere64", seed)
        prob = ctx.problem(pat.intensities, pat.mask, pat.support0)
        r = prob.run(sp.params(**C1, seed=seed))
        prob.destroy()
        o = oracle.mpr_run(pat.intensities, pat.mask, pat.support0, seed=seed, **C1)
        eg.append(r["final_error_best"])
        ea.append(r["final_error_avg"])
        eo.append(o["final_error_best"])
        oa.append(o["final_error_avg"])
        rg.append(aligned_rel_error(r["rho_avg"], pat.truth))
        ro.append(aligned_rel_error(o["rho_avg"], pat.truth))
        assert np.isfinite(r["gen_stats"][:, [0, 1, 2, 4, 5, 6, 7]]).all()
        assert 0 <= r["gen_stats"][:, 5].min() and r["gen_stats"][:, 5].max() <= 1
    eg, eo = np.array(eg), np.array(eo)
    se = np.sqrt(eg.var(ddof=1) / len(eg) + eo.var(ddof=1) / len(eo))
    print(f"mean E gpu {eg.mean():.4f} oracle {eo.mean():.4f} (se {se:.4f}); median recovery "
          f"gpu {np.median(rg):.4f} oracle {np.median(ro):.4f}")
    assert abs(eg.mean() - eo.mean()) <= 0.02 * eo.mean() + 2.0 * se
    ea, oa = np.array(ea), np.array(oa)  # the error of the average reconstruction, same bar
    sea = np.sqrt(ea.var(ddof=1) / len(ea) + oa.var(ddof=1) / len(oa))
    assert abs(ea.mean() - oa.mean()) <= 0.02 * oa.mean() + 2.0 * sea, (ea.mean(), oa.mean(), sea)
    assert abs(np.median(rg) - np.median(ro)) <= 0.05


@pytest.mark.parametrize("name", ["sphere64", "ell96", "ell128", "ell192", "ell256", "ell384", "ell512",
                                  "ell768", "ell1024"])
def test_mpr_runs_at_every_side(sp, ctx, name):
    # a short run at each supported side exercises every kernel of the run at that side
    pat = synthetic.config_pattern(name, 0)
    prob = ctx.problem(pat.intensities, pat.mask, pat.support0)
    r = prob.run(sp.params(pop=4, iters_per_gen=40, generations=2, er_tail=5, seed=3))
    prob.destroy()
    assert 0 < r["final_error_best"] < 1.5 and np.isfinite(r["final_error_avg"])
    assert r["support_avg"].sum() > 0 and np.isfinite(r["rho_avg"]).all()


def test_mpr_ell96_matches_oracle_statistically(sp, ctx):
    # a side of the form 3 x 2^k with a gap and saturation: the same bar as at 64
    eg, eo = [], []
    ea, oa = [], []
    for seed in range(12):
        pat = synthetic.config_pattern("ell96", seed)
        prob = ctx.problem(pat.intensities, pat.mask, pat.support0)
        r = prob.run(sp.params(**C1, seed=seed))
        prob.destroy()
        o = oracle.mpr_run(pat.intensities, pat.mask, pat.support0, seed=seed, **C1)
        eg.append(r["final_error_best"])
        ea.append(r["final_error_avg"])
        eo.append(o["final_error_best"])
        oa.append(o["final_error_avg"])
        assert np.isfinite(r["rho_avg"]).all()
    eg, eo = np.array(eg), np.array(eo)
    se = np.sqrt(eg.var(ddof=1) / len(eg) + eo.var(ddof=1) / len(eo))
    print(f"ell96: mean E gpu {eg.mean():.4f} oracle {eo.mean():.4f} (se {se:.4f})")
    assert abs(eg.mean() - eo.mean()) <= 0.02 * eo.mean() + 2.0 * se
    ea, oa = np.array(ea), np.array(oa)  # the error of the average reconstruction, same bar
    sea = np.sqrt(ea.var(ddof=1) / len(ea) + oa.var(ddof=1) / len(oa))
    assert abs(ea.mean() - oa.mean()) <= 0.02 * oa.mean() + 2.0 * sea, (ea.mean(), oa.mean(), sea)


def test_replacement_and_average_error_behave_as_described(sp, ctx):
    # Sec. "Monitoring the reconstruction process" (qualitative), the GPU's runs: about half
    # of the new individuals replace their parents in the first generations, and the error
    # of the average reconstruction falls over the run (the oracle shows the same)
    rep, eavg = [], []
    for seed in range(8):
        pat = synthetic.config_pattern("sphere64", seed)
        prob = ctx.problem(pat.intensities, pat.mask, pat.support0)
        st = prob.run(sp.params(**C1, seed=seed, monitor_avg=1), want_arrays=False)["gen_stats"]
        prob.destroy()
        rep.append(st[:, 5])
        eavg.append(st[:, 3])
    rep, eavg = np.array(rep), np.array(eavg)
    assert 0.25 <= rep[:, :2].mean() <= 0.75
    assert eavg[:, -1].mean() < eavg[:, 0].mean()


def test_mpr_deterministic_and_graph_identical(sp, ctx):
    pat = synthetic.config_pattern("sphere64", 3)
    prob = ctx.problem(pat.intensities, pat.mask, pat.support0)
    a = prob.run(sp.params(**C1, seed=5))
    b = prob.run(sp.params(**C1, seed=5))
    g = prob.run(sp.params(**C1, seed=5, use_graph=1))
    prob.destroy()
    for k in ("rho_avg", "rho_best", "support_avg", "gen_stats"):
        assert np.array_equal(a[k], b[k], equal_nan=True), k
        assert np.array_equal(a[k], g[k], equal_nan=True), k


def test_problem_from_device_equals_host(sp, ctx):
    import torch
    pat = synthetic.config_pattern("sphere64", 1)
    p1 = ctx.problem(pat.intensities, pat.mask, pat.support0)
    p2 = ctx.problem_device(torch.from_numpy(pat.intensities).cuda(), torch.from_numpy(pat.mask).cuda(),
                            torch.from_numpy(pat.support0).cuda())
    torch.cuda.synchronize()
    a = p1.run(sp.params(**C1, seed=2))
    b = p2.run(sp.params(**C1, seed=2))
    p1.destroy()
    p2.destroy()
    assert np.array_equal(a["rho_avg"], b["rho_avg"])


def _serve(ctx, sp, jobs, poll_us=-1):
    probs, tickets = [], []
    for (name, seed, prm) in jobs:
        pat = synthetic.config_pattern(name, seed)
        pr = ctx.problem(pat.intensities, pat.mask, pat.support0)
        probs.append(pr)
        tickets.append(pr.submit(sp.params(**prm)))
    res = []
    for t in tickets:
        st, r = ctx.poll(t, poll_us)
        assert st == sp.OK
        res.append(r)
    for pr in probs:
        pr.destroy()
    return res


def test_serving_alone_equals_in_mix(sp, ctx):
    job = ("ell128", 0, dict(C1, pop=6, seed=11))
    alone = _serve(ctx, sp, [job])[0]
    mix = [("ell192", 1, dict(C1, pop=5, seed=1)), job, ("sphere64", 2, dict(C1, seed=2)),
           ("ell256", 3, dict(C1, pop=4, generations=3, seed=3))]
    in_mix = _serve(ctx, sp, mix)[1]
    for k in ("rho_avg", "rho_best", "support_avg", "gen_stats"):
        assert np.array_equal(alone[k], in_mix[k], equal_nan=True), k
    assert in_mix["t_submit_s"] <= in_mix["t_admit_s"] <= in_mix["t_done_s"]


def test_serving_batches_same_side_requests(sp, monkeypatch):
    # one cohort at a time: a first request runs while five requests of one side and one set
    # of parameters (different patterns and seeds) queue behind it; they are then admitted
    # together as one cohort, and each result equals the request's run alone bit for bit
    monkeypatch.setenv("SPRING_MAX_ACTIVE", "1")
    jobs = [("ell256", 9, dict(C1, pop=16, seed=90))] + \
        [("ell128", q, dict(C1, pop=6, seed=100 + q)) for q in range(5)]
    with sp.Context(0) as c:
        res = _serve(c, sp, jobs)
        cohorts, admitted = c.serving_stats()
    assert admitted == 6 and cohorts <= 3, (cohorts, admitted)
    monkeypatch.delenv("SPRING_MAX_ACTIVE")
    with sp.Context(0) as c:
        for (name, seed, prm), got in zip(jobs, res):
            pat = synthetic.config_pattern(name, seed)
            pr = c.problem(pat.intensities, pat.mask, pat.support0)
            alone = pr.run(sp.params(**prm))
            pr.destroy()
            for k in ("rho_avg", "rho_best", "support_avg", "gen_stats"):
                assert np.array_equal(alone[k], got[k], equal_nan=True), (name, seed, k)
            assert alone["final_error_avg"] == got["final_error_avg"]


def test_serving_admits_by_footprint(sp):
    p = sp.params(**C1, seed=1)
    fp = sp.footprint_bytes(64, p)
    with sp.Context(0, hbm_budget_bytes=int(1.5 * fp)) as c:  # room for one request at a time
        res = _serve(c, sp, [("sphere64", s, dict(C1, seed=s)) for s in range(3)])
    # requests ran one after another: each admitted after the previous finished
    for a, b in zip(res, res[1:]):
        assert b["t_admit_s"] >= a["t_done_s"] - 1e-6


def test_serving_rejects_oversized_and_cancel(sp):
    p = sp.params(**C1, seed=1)
    fp = sp.footprint_bytes(64, p)
    with sp.Context(0, hbm_budget_bytes=int(1.5 * fp)) as c:
        pat = synthetic.config_pattern("sphere64", 0)
        pr = c.problem(pat.intensities, pat.mask, pat.support0)
        with pytest.raises(sp.SpringError) as e:
            pr.submit(sp.params(**dict(C1, pop=64)))
        assert e.value.status == sp.E_NOMEM
        t1 = pr.submit(p)
        t2 = pr.submit(p)  # waits for memory behind t1
        c.cancel(t2)
        with pytest.raises(sp.SpringError) as e:
            pr.destroy()  # still referenced by unfinished tickets
        assert e.value.status == sp.E_BUSY
        st, r = c.poll(t1, -1)
        assert st == sp.OK and r["final_error_best"] > 0
        with pytest.raises(sp.SpringError) as e:
            c.poll(t2, -1)
        assert e.value.status == sp.E_CANCELLED
        with pytest.raises(sp.SpringError) as e:
            c.poll(t2, 0)
        assert e.value.status == sp.E_NOT_FOUND
        pr.destroy()


def test_invalid_arguments(sp, ctx):
    pat = synthetic.config_pattern("sphere64", 0)
    pr = ctx.problem(pat.intensities, pat.mask, pat.support0)
    for bad in (dict(pop=3), dict(iters_per_gen=30), dict(er_tail=50), dict(algorithm=3),
                dict(beta=0.0), dict(cp=1.5), dict(precision=2)):
        with pytest.raises(sp.SpringError) as e:
            pr.run(sp.params(**{**C1, **bad}))
        assert e.value.status == sp.E_INVALID, bad
    pr.destroy()
    with pytest.raises(sp.SpringError):
        ctx.problem(np.zeros((100, 100), np.float32), np.ones((100, 100), np.uint8),
                    np.ones((100, 100), np.uint8))
