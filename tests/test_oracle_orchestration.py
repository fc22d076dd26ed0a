"""Pins of the oracle's orchestration: the order of the steps inside Improve (Alg. improve),
one generation of Alg. mpr, and the sphere draws of Initialize (App. "Initialization of the
starting densities").

The operators themselves are pinned in test_oracle_pins.py.  Here the oracle's composed
routines (orc_improve, orc_mpr_step, orc_mpr_run) are checked bit for bit against the same
steps composed by hand in the order the paper gives, and the hand composition is shown to
be sensitive to the order (swapping UpdateSupportSize(alpha_best) and
UpdateSupportSize(alpha_eval) changes the result), so that a reordering inside the oracle
cannot pass."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2409_07413_gb300 import synthetic


def _dft_inputs(pat):
    I = np.fft.ifftshift(pat.intensities.astype(np.float64))
    mask = np.fft.ifftshift(pat.mask)
    M = np.sqrt(np.maximum(I, 0.0))
    return I, mask, M


def _improve_by_hand(x, S, M, mask, kw, sigma, tau, a_best, a_eval):
    """Alg. improve for one individual, step by step (schedule 0 of the configs, or the
    paper's Sequence for schedule 1), from the pinned primitives."""
    x = x.copy()
    alg, beta, chi = kw["algorithm"], kw["beta"], kw["chi"]
    if kw.get("schedule", 0) == 1:
        R = kw["repetitions"]
        segs = [(kw["seq_ia"], kw["seq_er"])] * R
        eval_er = kw["seq_eval"]
    else:
        K, it = kw["sw_period"], kw["iters_per_gen"]
        R = it // K
        segs = [(K, 0)] * (R - 1) + [(it - (R - 1) * K - kw["er_tail"], 0)]
        eval_er = kw["er_tail"]
    for blk, (ia, er) in enumerate(segs, start=1):
        x = oracle.iterate(x, S, M, mask, alg, beta, chi, ia)
        x = oracle.iterate(x, S, M, mask, 0, beta, chi, er)
        if blk <= R - 2:
            S = oracle.update_support(x, sigma, tau)
        elif blk == R - 1:
            S = oracle.update_support_size(x, sigma, a_best)
        else:
            S = oracle.update_support_size(x, sigma, a_eval)
    x = oracle.iterate(x, S, M, mask, 0, beta, chi, eval_er)
    e = oracle.fourier_error(x, S, M, mask)
    S = oracle.update_support(x, sigma, tau)
    return x, S, e


IMPROVE_CASES = [
    dict(algorithm=2, beta=0.9, chi=0.5, iters_per_gen=60, sw_period=20, er_tail=5),
    dict(algorithm=1, beta=0.8, chi=1.0, iters_per_gen=70, sw_period=20, er_tail=7),
    dict(algorithm=2, beta=0.9, chi=0.5, schedule=1, repetitions=4, seq_ia=6, seq_er=4, seq_eval=5),
]


@pytest.mark.parametrize("kw", IMPROVE_CASES)
def test_improve_follows_the_paper_order(kw):
    pat = synthetic.config_pattern("sphere64", 3)
    I, mask, M = _dft_inputs(pat)
    x0 = oracle.initialize(11, pat.support0, I, mask, 2)[0]
    S0 = pat.support0
    sigma, tau = 1.5, 0.2
    a_best = int(S0.sum()) // 3
    a_eval = int(S0.sum()) // 2
    prm = oracle.make_params(**kw)
    xo, So, eo = oracle.improve(x0, S0, M, mask, prm, sigma, tau, a_best, a_eval)
    xh, Sh, eh = _improve_by_hand(x0, S0, M, mask, kw, sigma, tau, a_best, a_eval)
    assert np.array_equal(xo.reshape(xh.shape), xh) and np.array_equal(So.reshape(Sh.shape), Sh)
    assert eo[0] == eh
    # the composition is sensitive to the order of the two area-matched updates
    xs, Ss, es = _improve_by_hand(x0, S0, M, mask, kw, sigma, tau, a_eval, a_best)
    assert es != eh and not np.array_equal(xs, xh)


def _alpha_eval(g, G, a_best, a_all):
    v = Fraction(g, G) * a_best + (1 - Fraction(g, G)) * a_all
    return int(v + Fraction(1, 2)) if v.denominator != 1 else int(v)  # halves up


def _initial_state(pat, I, mask, P, seed):
    x = oracle.initialize(seed, pat.support0, I, mask, P)
    return {"generation": 0, "pop_x": x, "pop_S": np.repeat(pat.support0[None], P, axis=0),
            "pop_err": np.full(P, np.inf)}


STEP_KW = dict(pop=6, generations=3, iters_per_gen=60, sw_period=20, er_tail=5, algorithm=2, beta=0.9,
               sw_sigma=1.5, sw_threshold=0.2, chi=0.5, cw=0.4, cp=0.6, tile_min=4, tile_max=0, seed=21)


def test_generation_follows_alg_mpr():
    """One generation of orc_mpr_step = Crossover of the parents, the areas of Alg. improve
    from the parents (alpha_best of the lowest-error parent, alpha_all of the union, the
    rounded mix alpha_eval), Improve of both populations, Select with strict <."""
    pat = synthetic.config_pattern("sphere64", 1)
    I, mask, M = _dft_inputs(pat)
    kw = STEP_KW
    P, G = kw["pop"], kw["generations"]
    st = _initial_state(pat, I, mask, P, kw["seed"])
    for g in (1, 2):
        out, tr = oracle.mpr_step(pat.intensities, pat.mask, st, **kw)
        # by hand
        px, pS, pe = st["pop_x"], st["pop_S"], st["pop_err"]
        nx, nS, par = oracle.crossover(px, pS, mask, kw["seed"], g, kw["cw"], kw["cp"], kw["tile_min"],
                                       kw["tile_max"])
        best = 0 if g == 1 else int(np.argmin(pe))
        a_best = int(pS[best].sum())
        a_all = int(np.any(pS, axis=0).sum())
        a_eval = _alpha_eval(g, G, a_best, a_all)
        prm = oracle.make_params(**kw)
        xp, Sp, ep = oracle.improve(px.copy(), pS, M, mask, prm, 1.5, 0.2, a_best, a_eval)
        xn, Sn, en = oracle.improve(nx, nS, M, mask, prm, 1.5, 0.2, a_best, a_eval)
        repl, cnt = oracle.select(ep, en)
        r = repl.astype(bool)
        assert np.array_equal(tr["parents"], par)
        assert tr["best"] == best and list(tr["areas"]) == [a_best, a_all, a_eval]
        assert np.array_equal(tr["err_parents"], ep) and np.array_equal(tr["err_new"], en)
        assert np.array_equal(tr["replaced"], repl) and tr["gen_stats"][5] == cnt / P
        assert np.array_equal(out["pop_x"], np.where(r[:, None, None], xn, xp))
        assert np.array_equal(out["pop_S"], np.where(r[:, None, None], Sn, Sp))
        assert np.array_equal(out["pop_err"], np.where(r, en, ep))
        # a swapped pair of areas would give other errors
        _, _, ep_sw = oracle.improve(px.copy(), pS, M, mask, prm, 1.5, 0.2, a_eval, a_best)
        if a_eval != a_best:
            assert not np.array_equal(ep_sw, ep)
        st = out


@pytest.mark.parametrize("extra", [dict(), dict(schedule=1, repetitions=3, seq_ia=8, seq_er=6, seq_eval=5),
                                   dict(ca=0.3, monitor_avg=1), dict(mode=1)])
def test_step_chain_equals_run(extra):
    """orc_mpr_step chained from the initial population reproduces orc_mpr_run."""
    pat = synthetic.config_pattern("sphere64", 2)
    I, mask, _ = _dft_inputs(pat)
    kw = {**STEP_KW, **extra}
    P, G = kw["pop"], kw["generations"]
    run = oracle.mpr_run(pat.intensities, pat.mask, pat.support0, keep_population=True, **kw)
    st = _initial_state(pat, I, mask, P, kw["seed"])
    for g in range(1, G + 1):
        st, tr = oracle.mpr_step(pat.intensities, pat.mask, st, **kw)
        row = run["gen_stats"][g - 1]
        if g == G:  # the run's last row carries E(avg) of the final average
            row = row.copy()
            row[3] = np.nan
        assert np.array_equal(tr["gen_stats"], row, equal_nan=True), g
    assert st["generation"] == G
    assert np.array_equal(st["pop_x"], run["pop_x"])
    assert np.array_equal(st["pop_S"], run["pop_S"])
    assert np.array_equal(st["pop_err"], run["pop_err"])


def test_step_rejects_bad_generation():
    pat = synthetic.config_pattern("sphere64", 2)
    I, mask, _ = _dft_inputs(pat)
    st = _initial_state(pat, I, mask, 6, 1)
    for g0 in (-1, 3):
        with pytest.raises(ValueError):
            oracle.mpr_step(pat.intensities, pat.mask, {**st, "generation": g0}, **STEP_KW)


def test_initialize_sphere_diameters_and_centres():
    """App. "Initialization of the starting densities": each sphere's diameter is uniform in
    [0.2, 0.9] of the side of the initial support's bounding square, and its centre is
    uniform over the positions that keep the whole sphere inside that square.  One sphere
    per individual on a full-image support (side 64): the disc of nonzero pixels gives the
    diameter (from its area) and the centre (its centroid)."""
    n, P = 64, 600
    S0 = np.ones((n, n), np.uint8)
    I = np.ones((n, n))
    mask = np.ones((n, n), np.uint8)
    x = oracle.initialize(5, S0, I, mask, P, n_spheres=1, gamma=1.0, phi_max=0.0)
    rr, cc = np.mgrid[0:n, 0:n]
    D, u_y, u_x = [], [], []
    for p in range(P):
        nz = np.abs(x[p]) > 0
        cnt = nz.sum()
        d = 2.0 * np.sqrt(cnt / np.pi)
        rows, cols = np.nonzero(nz)
        ext_r, ext_c = rows.max() - rows.min() + 1, cols.max() - cols.min() + 1
        # a whole disc, not one cut off by the square's edge: equal extents in both axes,
        # both close to the diameter from the area
        assert abs(ext_r - ext_c) <= 2 and abs(ext_r - d) <= 2.5, (p, ext_r, ext_c, d)
        cy, cx = rr[nz].mean(), cc[nz].mean()
        D.append(d)
        if n - d > 8:  # the centre's free range is wide enough to resolve
            u_y.append((cy - d / 2) / (n - d))
            u_x.append((cx - d / 2) / (n - d))
    D = np.array(D) / n
    assert abs(D.min() - 0.2) < 0.03 and abs(D.max() - 0.9) < 0.03
    assert abs(D.mean() - 0.55) < 0.03  # uniform on [0.2, 0.9]
    for u in (np.array(u_y), np.array(u_x)):
        assert u.min() > -0.1 and u.max() < 1.1
        assert u.min() < 0.1 and u.max() > 0.9 and abs(u.mean() - 0.5) < 0.06
