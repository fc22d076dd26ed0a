"""Checkpoint / resume of a run's population (spring_mpr_run_until, spring_mpr_resume) and
the every-generation monitor of the average reconstruction."""
import numpy as np
import pytest

from paper_2409_07413_gb300 import synthetic

pytestmark = pytest.mark.gpu

C1 = dict(pop=8, iters_per_gen=100, generations=5, algorithm=2, beta=0.9, sw_sigma=1.5,
          sw_threshold=0.2, sw_period=20, er_tail=10, seed=7)


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


@pytest.mark.parametrize("extra", [dict(), dict(mode=1), dict(use_graph=1), dict(precision=1),
                                   dict(schedule=1, repetitions=3, seq_ia=20, seq_er=10, seq_eval=10),
                                   dict(ca=0.3, monitor_avg=1)])
@pytest.mark.parametrize("g_stop", [1, 3])
def test_split_run_equals_whole_run(sp, ctx, extra, g_stop):
    pat = synthetic.config_pattern("sphere64", 2)
    prob = ctx.problem(pat.intensities, pat.mask, pat.support0)
    p = sp.params(**{**C1, **extra})
    whole = prob.run(p)
    state = prob.run_until(p, g_stop)
    assert state["generation"] == g_stop and np.isfinite(state["pop_err"]).all()
    part = prob.resume(p, state)
    prob.destroy()
    for k in ("rho_avg", "rho_best", "support_avg"):
        assert np.array_equal(whole[k], part[k]), k
    assert whole["final_error_avg"] == part["final_error_avg"]
    assert whole["final_error_best"] == part["final_error_best"]
    assert np.array_equal(whole["gen_stats"][g_stop:], part["gen_stats"][g_stop:], equal_nan=True)
    assert np.isnan(part["gen_stats"][:g_stop]).all()


def test_checkpoint_arguments(sp, ctx):
    pat = synthetic.config_pattern("sphere64", 0)
    prob = ctx.problem(pat.intensities, pat.mask, pat.support0)
    p = sp.params(**C1)
    for g in (0, 6):
        with pytest.raises(sp.SpringError) as e:
            prob.run_until(p, g)
        assert e.value.status == sp.E_INVALID
    state = prob.run_until(p, 2)
    for g in (-1, 5):
        with pytest.raises(sp.SpringError) as e:
            prob.resume(p, {**state, "generation": g})
        assert e.value.status == sp.E_INVALID
    prob.destroy()


def test_monitor_average_every_generation(sp, ctx):
    pat = synthetic.config_pattern("ell128", 3)
    prob = ctx.problem(pat.intensities, pat.mask, pat.support0)
    a = prob.run(sp.params(**C1))
    b = prob.run(sp.params(**C1, monitor_avg=1))
    prob.destroy()
    assert np.array_equal(a["rho_avg"], b["rho_avg"])  # monitoring changes nothing
    assert np.isfinite(b["gen_stats"][:, 3]).all()
    assert np.isnan(a["gen_stats"][:-1, 3]).all()
    assert b["gen_stats"][-1, 3] == b["final_error_avg"]


@pytest.mark.parametrize("name", ["sphere64", "ell256"])
def test_density_sum_monitors_match_the_population(sp, ctx, name):
    # gen_stats columns 7 and 8 of generation g (Sec. "Crossover averaging": the mean of
    # |sum rho| over the population and its population standard deviation relative to the
    # mean) against numpy on the population saved after generation g of the same run
    pat = synthetic.config_pattern(name, 1)
    prob = ctx.problem(pat.intensities, pat.mask, pat.support0)
    p = sp.params(**C1)
    whole = prob.run(p)
    assert whole["gen_stats"].shape == (C1["generations"], 9)
    for g in (2, C1["generations"]):
        state = prob.run_until(p, g)
        sums = np.abs(state["pop_x"].astype(np.complex128).reshape(C1["pop"], -1).sum(axis=1))
        row = whole["gen_stats"][g - 1]
        assert abs(row[7] - sums.mean()) <= 1e-5 * sums.mean(), g
        assert abs(row[8] - sums.std() / sums.mean()) <= 1e-4 * row[8] + 1e-7, g
    prob.destroy()
