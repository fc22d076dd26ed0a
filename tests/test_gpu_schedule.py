"""The paper's Sequence schedule, the independent-reconstruction mode and crossover
averaging on the GPU against the FP64 oracle (operators on identical state; runs
statistically over seeds) and against the GPU's own config-style schedule where the two
coincide (bit for bit)."""
import numpy as np
import pytest

import oracle
from paper_2409_07413_gb300 import synthetic

pytestmark = pytest.mark.gpu

TOL = 1e-5


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


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


def c64(x):
    return np.ascontiguousarray(x, dtype=np.complex64)


def rel(a, b):
    return np.linalg.norm(np.asarray(a, np.complex128) - b) / max(np.linalg.norm(b), 1e-300)


def population(seed, P, n):
    rng = np.random.default_rng(seed)
    obj = np.zeros((n, n))
    obj[n // 4: n // 2, n // 3: n // 2 + 3] = 1.0
    x = np.stack([np.roll(obj, (int(rng.integers(n)), int(rng.integers(n))), (0, 1))
                  * np.exp(1j * rng.uniform(-3, 3)) + 0.3 * (rng.standard_normal((n, n))
                  + 1j * rng.standard_normal((n, n))) for _ in range(P)])
    S = (np.abs(x) > 0.5).astype(np.uint8)
    M, mask = synthetic.random_modulus(seed, n, masked_frac=0.05)
    err = rng.uniform(0.1, 1.0, P)
    return x, S, M, mask, err


@pytest.mark.parametrize("n", [64, 256])
def test_average_moduli_matches_oracle(sp, n):
    P = 6
    x, S, M, mask, err = population(n, P, n)
    Menc = np.where(mask > 0, M, -1.0).astype(np.float32)
    got = host(sp.spring_average_moduli(dev(c64(x)), dev(S), dev(err), dev(Menc)))
    ref = oracle.average_moduli(c64(x), S, mask, int(np.argmin(err)))
    assert rel(got, ref) < TOL


@pytest.mark.parametrize("n", [64, 192, 512])
@pytest.mark.parametrize("ca", [0.2, 1.0])
def test_crossover_ca_matches_oracle(sp, n, ca):
    P = 6
    x, S, M, mask, _ = population(3 * n, P, n)
    Menc = np.where(mask > 0, M, -1.0).astype(np.float32)
    mavg = np.random.default_rng(n).uniform(0.2, 2.0, (n, n)).astype(np.float32)
    nx, nS, par = sp.spring_crossover_ca(dev(c64(x)), dev(S), dev(Menc), 17, 3, ca, dev(mavg))
    rx, rS, rpar = oracle.crossover(c64(x), S, mask, 17, 3, 0.4, 0.6, 4, 0, ca=ca,
                                    Mavg=mavg.astype(np.float64))
    assert np.array_equal(host(par), rpar)
    assert np.array_equal(host(nS), rS)
    assert rel(host(nx), rx) < TOL


C1 = dict(pop=8, generations=4, algorithm=2, beta=0.9, sw_sigma=1.5, sw_threshold=0.2,
          iters_per_gen=100, sw_period=20, er_tail=10)
PAPER = dict(C1, schedule=1, repetitions=3, seq_ia=20, seq_er=10, seq_eval=10)


def statistical(sp, ctx, gpu_kw, orc_kw, seeds=10, name="sphere64"):
    eg, eo = [], []
    ea, oa = [], []
    for seed in range(seeds):
        pat = synthetic.config_pattern(name, seed)
        prob = ctx.problem(pat.intensities, pat.mask, pat.support0)
        r = prob.run(sp.params(**gpu_kw, seed=seed))
        prob.destroy()
        o = oracle.mpr_run(pat.intensities, pat.mask, pat.support0, seed=seed, **orc_kw)
        eg.append(r["final_error_best"])
        ea.append(r["final_error_avg"])
        eo.append(o["final_error_best"])
        oa.append(o["final_error_avg"])
        assert np.isfinite(r["rho_avg"]).all()
    eg, eo = np.array(eg), np.array(eo)
    se = np.sqrt(eg.var(ddof=1) / len(eg) + eo.var(ddof=1) / len(eo))
    print(f"mean E gpu {eg.mean():.4f} oracle {eo.mean():.4f} (se {se:.4f})")
    assert abs(eg.mean() - eo.mean()) <= 0.02 * eo.mean() + 2.0 * se
    ea, oa = np.array(ea), np.array(oa)  # the error of the average reconstruction, same bar
    sea = np.sqrt(ea.var(ddof=1) / len(ea) + oa.var(ddof=1) / len(oa))
    assert abs(ea.mean() - oa.mean()) <= 0.02 * oa.mean() + 2.0 * sea, (ea.mean(), oa.mean(), sea)
    return eg, eo


def test_paper_schedule_matches_oracle_statistically(sp, ctx):
    statistical(sp, ctx, PAPER, PAPER)


def test_independent_mode_matches_oracle_statistically(sp, ctx):
    kw = dict(C1, mode=1)
    statistical(sp, ctx, kw, kw)


def test_crossover_averaging_run_matches_oracle_statistically(sp, ctx):
    kw = dict(C1, ca=0.3)
    statistical(sp, ctx, kw, kw)


def test_paper_schedule_reduces_to_config_schedule_on_gpu(sp, ctx):
    pat = synthetic.config_pattern("sphere64", 6)
    prob = ctx.problem(pat.intensities, pat.mask, pat.support0)
    base = dict(pop=4, generations=1, algorithm=2, beta=0.9, sw_sigma=1.5, sw_threshold=0.2, seed=3)
    a = prob.run(sp.params(**base, iters_per_gen=60, sw_period=20, er_tail=0))
    b = prob.run(sp.params(**base, schedule=1, repetitions=3, seq_ia=20, seq_er=0, seq_eval=0))
    er = dict(base, generations=3, algorithm=0)
    c = prob.run(sp.params(**er, iters_per_gen=40, sw_period=20, er_tail=0))
    d = prob.run(sp.params(**er, schedule=1, repetitions=2, seq_ia=0, seq_er=20, seq_eval=0))
    prob.destroy()
    for k in ("rho_avg", "rho_best", "gen_stats"):
        assert np.array_equal(a[k], b[k], equal_nan=True), k
        assert np.array_equal(c[k], d[k], equal_nan=True), k


def test_independent_mode_replaces_nothing_and_is_deterministic(sp, ctx):
    pat = synthetic.config_pattern("ell128", 1)
    prob = ctx.problem(pat.intensities, pat.mask, pat.support0)
    kw = dict(C1, mode=1, generations=3, seed=2)
    a = prob.run(sp.params(**kw))
    g = prob.run(sp.params(**kw, use_graph=1))
    prob.destroy()
    assert (a["gen_stats"][:, 5] == 0).all()
    assert np.array_equal(a["rho_avg"], g["rho_avg"])
    assert a["final_error_best"] == a["gen_stats"][-1, 0]


def test_schedule_and_mode_validation(sp, ctx):
    pat = synthetic.config_pattern("sphere64", 0)
    prob = ctx.problem(pat.intensities, pat.mask, pat.support0)
    for bad in (dict(schedule=2), dict(mode=2), dict(schedule=1, repetitions=1),
                dict(schedule=1, seq_ia=0, seq_er=0), dict(ca=1.5), dict(schedule=1, seq_eval=-1)):
        with pytest.raises(sp.SpringError) as e:
            prob.run(sp.params(**{**C1, **bad}))
        assert e.value.status == sp.E_INVALID, bad
    prob.destroy()
