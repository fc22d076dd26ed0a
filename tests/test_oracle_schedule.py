"""Pins of the oracle's paper-default schedule (App. "Changing values over generations",
"The algorithms sequence"), the independent-reconstruction mode (Alg. randomsearch,
Alg. normalimprove) and crossover averaging (App. "Crossover averaging": Eqs. avgint1,
avgint2, crossavg), against closed forms, exact rational arithmetic, compositions of the
already pinned primitives, and bit-identity where two schedules coincide."""
from fractions import Fraction

import numpy as np
import pytest

from paper_2409_07413_gb300 import synthetic


def half_up(q: Fraction) -> int:
    return int((2 * q.numerator + q.denominator) // (2 * q.denominator))


@pytest.mark.parametrize("j,jer,G", [(40, 40, 100), (80, 20, 7), (3, 0, 4), (1, 5, 2), (40, 40, 1)])
def test_sequence_counts_exact(orc, j, jer, G):
    for g in range(1, G + 1):
        t = Fraction(g - 1, G - 1) if G > 1 else Fraction(0)
        ia, er = orc.sequence_counts(j, jer, g, G)
        assert ia == half_up(j * (1 - t))
        assert er == jer + half_up(j * t)
    # endpoints: all IA at the start, only ER at the end
    assert orc.sequence_counts(j, jer, 1, G) == (j, jer)
    if G > 1:
        assert orc.sequence_counts(j, jer, G, G) == (0, j + jer)


KW = dict(pop=4, generations=1, algorithm=2, beta=0.9, sw_sigma=1.5, sw_threshold=0.2, chi=0.5, seed=5)


def test_paper_schedule_reduces_to_config_schedule_g1(orc):
    # one generation, Sequence = K RAAR and no ER, no EvalSequence: the same steps as the
    # configs' blocks of K with no ER tail
    pat = synthetic.config_pattern("sphere64", 1)
    a = orc.mpr_run(pat.intensities, pat.mask, pat.support0, iters_per_gen=60, sw_period=20, er_tail=0, **KW)
    b = orc.mpr_run(pat.intensities, pat.mask, pat.support0, schedule=1, repetitions=3, seq_ia=20, seq_er=0,
                    seq_eval=0, **KW)
    assert a["final_error_best"] == b["final_error_best"]
    assert np.array_equal(a["rho_avg"], b["rho_avg"])


def test_paper_schedule_reduces_to_config_schedule_er(orc):
    # with ER as the IA and no IA iterations the counts are constant over generations
    pat = synthetic.config_pattern("sphere64", 2)
    kw = dict(KW, generations=3, algorithm=0)
    a = orc.mpr_run(pat.intensities, pat.mask, pat.support0, iters_per_gen=40, sw_period=20, er_tail=0, **kw)
    b = orc.mpr_run(pat.intensities, pat.mask, pat.support0, schedule=1, repetitions=2, seq_ia=0, seq_er=20,
                    seq_eval=0, **kw)
    assert np.array_equal(a["gen_stats"], b["gen_stats"], equal_nan=True)
    assert np.array_equal(a["rho_avg"], b["rho_avg"])


def test_paper_schedule_changes_over_generations(orc):
    pat = synthetic.config_pattern("sphere64", 3)
    kw = dict(KW, generations=4)
    a = orc.mpr_run(pat.intensities, pat.mask, pat.support0, schedule=1, repetitions=3, seq_ia=20, seq_er=10,
                    seq_eval=10, **kw)
    st = a["gen_stats"]
    assert np.isfinite(st[:, [0, 1, 2, 4, 5, 6, 7]]).all()
    assert (st[:, 0] <= st[:, 1]).all() and (st[:, 1] <= st[:, 2]).all()


def test_independent_mode_is_the_composition_of_primitives(orc):
    # Alg. randomsearch with the configs' blocks: per generation, blocks of K IA iterations
    # each followed by UpdateSupport, the last er_tail iterations ER, the error before the
    # last UpdateSupport; the output is the best individual and the aligned average
    pat = synthetic.config_pattern("sphere64", 4)
    P, G, K, it, tail = 4, 2, 20, 40, 5
    r = orc.mpr_run(pat.intensities, pat.mask, pat.support0, mode=1, iters_per_gen=it, sw_period=K,
                    er_tail=tail, **dict(KW, pop=P, generations=G))
    I = np.fft.ifftshift(pat.intensities.astype(np.float64))
    mk = np.fft.ifftshift(pat.mask)
    M = np.sqrt(np.maximum(I, 0.0))
    x = orc.initialize(KW["seed"], pat.support0, I, mk, P)
    S = np.broadcast_to(pat.support0, x.shape).copy()
    err = None
    for _ in range(G):
        for _blk in range(it // K - 1):
            x = orc.iterate(x, S, M, mk, 2, 0.9, 0.5, K)
            S = orc.update_support(x, 1.5, 0.2)
        x = orc.iterate(x, S, M, mk, 2, 0.9, 0.5, K - tail)
        x = orc.iterate(x, S, M, mk, 0, 0.9, 0.5, tail)
        err = orc.fourier_error(x, S, M, mk)
        S = orc.update_support(x, 1.5, 0.2)
    b = int(np.argmin(err))
    assert r["final_error_best"] == err[b]
    assert np.array_equal(r["rho_best"], x[b])
    avg, _ = orc.average(x, S, mk, b)
    assert np.array_equal(r["rho_avg"], avg)
    assert (r["gen_stats"][:, 5] == 0).all()  # nothing is replaced


def test_average_moduli_bounds_and_copies(orc):
    rng = np.random.default_rng(7)
    n, P = 32, 5
    x = rng.standard_normal((P, n, n)) + 1j * rng.standard_normal((P, n, n))
    S = (rng.random((P, n, n)) < 0.5).astype(np.uint8)
    mask = np.ones((n, n), np.uint8)
    Mavg = orc.average_moduli(x, S, mask, 0)
    avg, _ = orc.average(x, S, mask, 0)
    mdot = np.abs(np.fft.fft2(avg, norm="ortho"))
    mdd = np.abs(np.fft.fft2(x, norm="ortho")).mean(axis=0)
    assert np.allclose(Mavg, 0.5 * (mdot + mdd), rtol=1e-12, atol=1e-12)
    assert (mdot <= mdd + 1e-12).all()  # the paper's inequality (triangle inequality)
    # copies of one object, shifted, phased and twinned: both estimates are its moduli
    y = x[0]
    cp = np.stack([y, np.roll(y, (3, -5), (0, 1)) * np.exp(0.7j),
                   np.conj(np.roll(y[::-1, ::-1], (1, 1), (0, 1))), y * np.exp(-2.0j)])
    Mc = orc.average_moduli(cp, np.ones(cp.shape, np.uint8), mask, 0)
    assert np.allclose(Mc, np.abs(np.fft.fft2(y, norm="ortho")), rtol=1e-10, atol=1e-10)


def test_crossover_averaging_formula(orc):
    rng = np.random.default_rng(8)
    n, P = 32, 6
    x = rng.standard_normal((P, n, n)) + 1j * rng.standard_normal((P, n, n))
    S = (rng.random((P, n, n)) < 0.5).astype(np.uint8)
    mask = (rng.random((n, n)) > 0.1).astype(np.uint8)
    Mavg = rng.uniform(0.5, 2.0, (n, n))
    # C_a = 0 is the plain crossover, bit for bit
    a0 = orc.crossover(x, S, mask, 11, 2, 0.4, 0.6, 4, 4)
    a1 = orc.crossover(x, S, mask, 11, 2, 0.4, 0.6, 4, 4, ca=1e-300 * 0.0, Mavg=Mavg)
    assert np.array_equal(a0[0], a1[0])
    # map = 1 everywhere, C_w = 0: the new individual is parent a (aligned) with its moduli
    # blended towards Mavg by C_a and its phases kept (Eq. crossavg)
    ca = 0.3
    plain, _, _ = orc.crossover(x, S, mask, 11, 2, 0.0, 1.0, 4, 4)
    got, _, _ = orc.crossover(x, S, mask, 11, 2, 0.0, 1.0, 4, 4, ca=ca, Mavg=Mavg)
    A = np.fft.fft2(plain, norm="ortho")
    a = np.abs(A)
    want = np.fft.ifft2(A / a * (ca * Mavg + (1 - ca) * a), norm="ortho")
    assert np.abs(got - want).max() < 1e-10 * np.abs(want).max()


def test_mpr_with_crossover_averaging_runs(orc):
    pat = synthetic.config_pattern("sphere64", 5)
    kw = dict(KW, generations=3, iters_per_gen=40, sw_period=20, er_tail=5)
    a = orc.mpr_run(pat.intensities, pat.mask, pat.support0, **kw)
    b = orc.mpr_run(pat.intensities, pat.mask, pat.support0, ca=0.2, **kw)
    assert np.isfinite(b["gen_stats"][:, [0, 1, 2]]).all()
    assert a["final_error_best"] != b["final_error_best"]  # the averaging takes part


def test_monitor_average_every_generation(orc):
    # monitoring the average reconstruction does not change the run; its error is finite
    # every generation and the last one is the final average's error
    pat = synthetic.config_pattern("sphere64", 6)
    kw = dict(KW, generations=3, iters_per_gen=40, sw_period=20, er_tail=5)
    a = orc.mpr_run(pat.intensities, pat.mask, pat.support0, **kw)
    b = orc.mpr_run(pat.intensities, pat.mask, pat.support0, monitor_avg=1, **kw)
    assert np.array_equal(a["rho_avg"], b["rho_avg"])
    assert np.isfinite(b["gen_stats"][:, 3]).all()
    assert np.isnan(a["gen_stats"][:-1, 3]).all()
    assert b["gen_stats"][-1, 3] == b["final_error_avg"]
    assert (b["gen_stats"][:, 3] >= 0).all() and (b["gen_stats"][:, 3] <= 2).all()


def test_replacement_and_average_error_behave_as_described(orc):
    # Sec. "Monitoring the reconstruction process" (qualitative): in the first generations
    # about half of the new individuals replace their parents, and the error of the
    # average reconstruction falls over the run (8 seeds of the 64 x 64 workload)
    kw = dict(pop=8, iters_per_gen=100, generations=5, algorithm=2, beta=0.9, sw_sigma=1.5,
              sw_threshold=0.2, sw_period=20, er_tail=10, monitor_avg=1)
    rep, eavg = [], []
    for seed in range(8):
        pat = synthetic.config_pattern("sphere64", seed)
        st = orc.mpr_run(pat.intensities, pat.mask, pat.support0, seed=seed, **kw)["gen_stats"]
        rep.append(st[:, 5])
        eavg.append(st[:, 3])
    rep, eavg = np.array(rep), np.array(eavg)
    assert 0.25 <= rep[:, :2].mean() <= 0.75
    assert eavg[:, -1].mean() < eavg[:, 0].mean()
