"""The whole run against the oracle in lockstep, one generation at a time.

Each generation starts both sides from the same parent population (the GPU's, after the
previous generation; for generation 1 the oracle's initial densities rounded to complex64)
and runs it once: Crossover, the areas of Alg. improve, Improve of both populations,
Select (Alg. mpr) through spring_mpr_step on the GPU and orc_mpr_step in FP64.  Compared
element by element, per generation:

- the GA's integer decisions, bit for bit: the parents of every new individual, the parent
  whose area is alpha_best, alpha_best, alpha_all and alpha_eval, and Select's replacement
  flags (wherever the two errors Select compares are not a near-tie);
- every individual's error after Improve, in both populations;
- the surviving densities and supports; the generation's monitors (best, mean and worst
  error, O_d, replacement, Gamma, density sum and spread, and E(avg) when monitored).

The floating-point bars.  HIO/RAAR with the positivity constraint amplify a relative change
of 1e-7 to order one within a few tens of iterations of a fresh start (a pixel whose Re m
sits at zero switches between the two branches of the update), so the generations here are
short: 12 iterations, in blocks of 4 with the three support updates, the last two ER.
Within such a generation nearly every individual's error agrees with the oracle's to the
operator-level FP32 drift (1e-6 .. 1e-5), but a support pixel whose smoothed value is
within FP32 rounding of the threshold, or of the alpha-th largest value, may fall the other
way; that moves the individual's error by about 1 / alpha (1e-3 .. 1e-2) and is not an
error of either side.  So the errors are held to two bars: their median over the case's
generations and individuals within MEDIAN_TOL (any mistake in the order or the inputs of the
steps shifts every individual far beyond it), and each one within MAX_TOL.  Measured on
GB300 over 8 patterns x 4 generations x 16 individuals: median 1.0e-6, 90th percentile
2.1e-5, largest 1.1e-2; every area and every replacement decision equal."""
import numpy as np
import pytest

import oracle
from paper_2409_07413_gb300 import synthetic

pytestmark = pytest.mark.gpu

MEDIAN_TOL = 1e-4    # median relative error deviation of a case
MAX_TOL = 3e-2       # any single individual's relative error deviation
X_MEDIAN_TOL = 1e-3  # median density rel L2 deviation (individuals Select kept alike)
X_MAX_TOL = 0.1
S_MAX_FRAC = 0.01    # support pixels that may differ in one individual

BASE = dict(pop=8, generations=4, iters_per_gen=12, sw_period=4, er_tail=2, algorithm=2, beta=0.9,
            sw_sigma=1.5, sw_threshold=0.2, chi=0.5, cw=0.4, cp=0.6, tile_min=4, tile_max=0)

CASES = [
    ("sphere64", 0, dict(seed=31)),
    ("sphere64", 4, dict(seed=32, schedule=1, repetitions=3, seq_ia=3, seq_er=1, seq_eval=2)),
    ("sphere64", 5, dict(seed=33, ca=0.3, monitor_avg=1)),
    ("sphere64", 6, dict(seed=35, algorithm=1, beta=0.8, chi=1.0)),
    ("sphere64", 7, dict(seed=36, chi=1.0)),
    ("ell96", 3, dict(seed=41)),
    ("ell128", 2, dict(seed=40)),
    ("ell192", 1, dict(seed=34)),
]


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


def _rel(a, b):
    return np.abs(a - b) / np.maximum(np.abs(b), 1e-300)


@pytest.mark.parametrize("recipe,pseed,extra", CASES, ids=[f"{c[0]}-{i}" for i, c in enumerate(CASES)])
def test_generation_lockstep(sp, ctx, recipe, pseed, extra):
    kw = {**BASE, **extra}
    P, G = kw["pop"], kw["generations"]
    pat = synthetic.config_pattern(recipe, pseed)
    n = pat.n
    I = np.fft.ifftshift(pat.intensities.astype(np.float64))
    mask = np.fft.ifftshift(pat.mask)
    x0 = oracle.initialize(kw["seed"], pat.support0, I, mask, P).astype(np.complex64)
    st = {"generation": 0, "pop_x": x0, "pop_S": np.repeat(pat.support0[None], P, axis=0),
          "pop_err": np.full(P, np.inf)}
    prob = ctx.problem(pat.intensities, pat.mask, pat.support0)
    p = sp.params(**kw)
    d_err_all, d_x_all = [], []
    try:
        for g in range(1, G + 1):
            go, gt = prob.step(p, st)
            oo, ot = oracle.mpr_step(pat.intensities, pat.mask,
                                     {**st, "pop_x": st["pop_x"].astype(np.complex128)}, **kw)
            assert go["generation"] == oo["generation"] == g
            # integer decisions of the GA: bit for bit
            assert np.array_equal(gt["parents"], ot["parents"]), g
            assert gt["best"] == ot["best"], g
            assert np.array_equal(gt["areas"], ot["areas"]), (g, gt["areas"], ot["areas"])
            # errors of both improved populations
            d_err = np.concatenate([_rel(gt[k], ot[k]) for k in ("err_parents", "err_new")])
            d_err_all.append(d_err)
            assert d_err.max() <= MAX_TOL, (g, d_err.max())
            # Select: the same decision wherever the pair is not a near-tie
            gap = np.abs(ot["err_new"] - ot["err_parents"]) / ot["err_parents"]
            clear = gap > 2 * MAX_TOL
            assert np.array_equal(gt["replaced"][clear], ot["replaced"][clear]), g
            assert np.array_equal(gt["replaced"].astype(bool), gt["err_new"] < gt["err_parents"]), g
            # the surviving population, where both sides kept the same individual
            same = gt["replaced"] == ot["replaced"]
            for q in np.nonzero(same)[0]:
                dx = np.linalg.norm(go["pop_x"][q] - oo["pop_x"][q]) / np.linalg.norm(oo["pop_x"][q])
                d_x_all.append(dx)
                assert dx <= X_MAX_TOL, (g, q, dx)
                assert np.mean(go["pop_S"][q] != oo["pop_S"][q]) <= S_MAX_FRAC, (g, q)
                assert _rel(go["pop_err"][q], oo["pop_err"][q]) <= MAX_TOL, (g, q)
            # the generation's monitors
            gs, os_ = gt["gen_stats"], ot["gen_stats"]
            assert np.all(_rel(gs[0:3], os_[0:3]) <= MAX_TOL), (g, gs[0:3], os_[0:3])
            assert gs[5] == pytest.approx(gt["replaced"].mean(), abs=1e-12)
            if same.all():
                assert gs[5] == os_[5]
                if np.argmin(go["pop_err"]) == np.argmin(oo["pop_err"]):  # O_d = N^2 / area of the best
                    assert _rel(gs[4], os_[4]) <= S_MAX_FRAC * os_[4], (g, gs[4], os_[4])
                assert _rel(gs[6], os_[6]) <= 1e-2, (g, gs[6], os_[6])  # Gamma
                assert _rel(gs[7], os_[7]) <= 1e-2, (g, gs[7], os_[7])  # mean |sum rho|
                assert abs(gs[8] - os_[8]) <= 1e-2, (g, gs[8], os_[8])  # relative spread
                if kw.get("monitor_avg") and g < G:
                    assert _rel(gs[3], os_[3]) <= 5e-2, (g, gs[3], os_[3])
            st = go
    finally:
        prob.destroy()
    d_err_all = np.concatenate(d_err_all)
    med_x = float(np.median(d_x_all)) if d_x_all else 0.0
    print(f"lockstep {recipe}/{pseed} {extra}: error deviation median {np.median(d_err_all):.1e}, "
          f"max {d_err_all.max():.1e}; density median {med_x:.1e}")
    assert np.median(d_err_all) <= MEDIAN_TOL
    assert med_x <= X_MEDIAN_TOL


def test_step_chain_equals_run(sp, ctx):
    """spring_mpr_step chained after generation 1 reproduces spring_mpr_run's population."""
    kw = {**BASE, "iters_per_gen": 60, "sw_period": 20, "er_tail": 5, "generations": 3, "seed": 7}
    pat = synthetic.config_pattern("sphere64", 2)
    prob = ctx.problem(pat.intensities, pat.mask, pat.support0)
    p = sp.params(**kw)
    try:
        ref = prob.run_until(p, kw["generations"])
        st = prob.run_until(p, 1)
        for g in range(2, kw["generations"] + 1):
            st, tr = prob.step(p, st)
            assert st["generation"] == g
        for k in ("pop_x", "pop_S", "pop_err"):
            assert np.array_equal(st[k], ref[k]), k
    finally:
        prob.destroy()


def test_step_arguments(sp, ctx):
    pat = synthetic.config_pattern("sphere64", 0)
    prob = ctx.problem(pat.intensities, pat.mask, pat.support0)
    p = sp.params(**{**BASE, "seed": 1})
    try:
        st = prob.run_until(p, 1)
        for g0 in (-1, BASE["generations"]):
            with pytest.raises(sp.SpringError) as e:
                prob.step(p, {**st, "generation": g0})
            assert e.value.status == sp.E_INVALID
    finally:
        prob.destroy()
