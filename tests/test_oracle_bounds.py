"""Pins of the oracle's upper bounds for missing intensities (App. "Constraining
intensities at large scattering angles": Eqs. avgint, stdint, upperbound, pm_bounds)
against an independent numpy restatement, closed forms and projector invariants."""
import numpy as np
import pytest

from paper_2409_07413_gb300 import synthetic


def rand_c(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def ring_index(n):
    # distance from the detector centre (pixel (n/2, n/2)) rounded to the nearest pixel
    y, x = np.mgrid[0:n, 0:n]
    return np.rint(np.hypot(y - n // 2, x - n // 2)).astype(np.int64)


def numpy_bounds(I, mask, sat, eta, max_missing, max_saturated):
    """Restatement with numpy's mean and (population) standard deviation per ring."""
    n = I.shape[0]
    q = ring_index(n)
    U = np.full((n, n), -1.0)
    for r in np.unique(q):
        ring = q == r
        meas = ring & (mask > 0)
        if not meas.any():
            continue
        if (ring & (mask == 0)).sum() > max_missing * ring.sum():
            continue
        if (ring & (sat > 0)).sum() > max_saturated * ring.sum():
            continue
        mu, sd = I[meas].mean(), I[meas].std()
        free = ring & (mask == 0) & (sat == 0)
        U[free] = np.sqrt(mu + eta * sd)
    return U


def gapped(seed, n=32):
    rng = np.random.default_rng(seed)
    I = rng.gamma(2.0, 50.0, (n, n))
    mask = np.ones((n, n), np.uint8)
    mask[n // 2 - 1: n // 2 + 1, :] = 0                     # 2-row gap
    mask[(ring_index(n) <= 2)] = 0                           # central hole
    sat = np.zeros((n, n), np.uint8)
    sat[rng.random((n, n)) < 0.01] = 1                       # a few saturated pixels
    mask[sat > 0] = 0
    return I, mask, sat


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("eta", [0.0, 1.5])
def test_upper_bounds_match_numpy_restatement(orc, seed, eta):
    I, mask, sat = gapped(seed)
    U = orc.upper_bounds(I, mask, sat, eta, 0.2, 0.05)
    ref = numpy_bounds(I, mask, sat, eta, 0.2, 0.05)
    assert np.array_equal(U >= 0, ref >= 0)
    assert np.abs(U - ref).max() < 1e-10 * ref.max()
    # bounds only where the pixel is missing and unsaturated; some rings have bounds,
    # the central hole (every ring pixel missing) has none
    assert (U[mask > 0] < 0).all() and (U[sat > 0] < 0).all()
    assert (U >= 0).any()
    assert (U[ring_index(32) <= 1] < 0).all()


def test_upper_bounds_isotropic_closed_form(orc):
    # I constant on every ring: sigma = 0 and the bound is sqrt of the ring's value
    n = 32
    q = ring_index(n)
    I = 100.0 / (1.0 + q) ** 2
    mask = np.ones((n, n), np.uint8)
    mask[n // 2, :] = 0  # one missing row: at most 2 of >= 8 ring pixels for rings >= 2
    U = orc.upper_bounds(I, mask, None, 1.5, 0.2, 0.05)
    free = (mask == 0) & (q >= 2)
    assert np.abs(U[free] - np.sqrt(I[free])).max() < 1e-14 * np.sqrt(I).max()


def test_upper_bounds_validity_thresholds(orc):
    I, mask, sat = gapped(3)
    # no ring qualifies when no missing pixel is tolerated; every ring with a measured
    # pixel qualifies for the missing fraction when all are tolerated
    assert (orc.upper_bounds(I, mask, sat, 1.5, 0.0, 1.0) < 0).all()
    U1 = orc.upper_bounds(I, mask, None, 1.5, 1.0, 1.0)
    q = ring_index(32)
    has_meas = np.isin(q, np.unique(q[mask > 0]))
    assert ((U1 >= 0) == ((mask == 0) & has_meas)).all()
    # a ring whose saturated fraction exceeds the limit loses its bounds
    r10 = q == 10
    idx = np.flatnonzero(r10 & (mask > 0))[:4]
    sat2, mask2 = sat.copy(), mask.copy()
    sat2[r10] = 0
    sat2.flat[idx] = 1
    mask2.flat[idx] = 0
    cnt = r10.sum()
    free10 = r10 & (mask2 == 0) & (sat2 == 0)
    assert free10.any()
    ok = orc.upper_bounds(I, mask2, sat2, 1.5, 1.0, 4.5 / cnt)   # 4 saturated <= 4.5: kept
    off = orc.upper_bounds(I, mask2, sat2, 1.5, 1.0, 3.5 / cnt)  # 4 saturated > 3.5: dropped
    assert (ok[free10] >= 0).all() and (ok[sat2 > 0] < 0).all()
    assert (off[r10] < 0).all()


def spectrum_bounds(n, rng):
    mask = (rng.random((n, n)) > 0.2).astype(np.uint8)
    U = np.where(mask == 0, rng.uniform(0.2, 1.5, (n, n)), -1.0)
    U[rng.random((n, n)) < 0.3] = -1.0  # missing pixels without a bound
    return mask, U


def test_pm_bounds_definition(orc):
    rng = np.random.default_rng(4)
    n = 32
    x = rand_c(rng, n, n)
    M = rng.uniform(0.1, 2.0, (n, n))
    mask, U = spectrum_bounds(n, rng)
    out = orc.project_modulus_ub(x, M, mask, U)
    X = np.fft.fft2(x, norm="ortho")
    Y = np.fft.fft2(out, norm="ortho")
    a = np.abs(X)
    bound = (mask == 0) & (U >= 0) & (a > U)
    ref = np.where(mask > 0, X * M / a, np.where(bound, X * U / np.where(a > 0, a, 1), X))
    assert np.abs(Y - ref).max() < 1e-12 * np.abs(ref).max()
    assert bound.any() and ((mask == 0) & (U >= 0) & ~bound).any()
    # idempotent, and the bound holds after projection
    out2 = orc.project_modulus_ub(out, M, mask, U)
    assert np.abs(out2 - out).max() < 1e-12 * np.abs(out).max()
    assert (np.abs(Y)[(mask == 0) & (U >= 0)] <= U[(mask == 0) & (U >= 0)] * (1 + 1e-12)).all()


def test_pm_bounds_without_bounds_is_pm_full(orc):
    rng = np.random.default_rng(5)
    n = 32
    x = rand_c(rng, 2, n, n)
    M = rng.uniform(0.1, 2.0, (n, n))
    mask, _ = spectrum_bounds(n, rng)
    none = np.full((n, n), -1.0)
    assert np.array_equal(orc.project_modulus_ub(x, M, mask, none), orc.project_modulus(x, M, mask))
    S = (rng.random((2, n, n)) < 0.4).astype(np.uint8)
    a = orc.iterate(x.copy(), S, M, mask, 2, 0.9, 1.0, 3, U=none)
    b = orc.iterate(x.copy(), S, M, mask, 2, 0.9, 1.0, 3)
    assert np.array_equal(a, b)


def test_iterate_with_bounds_is_bounded_projection(orc):
    # one RAAR step with bounds = update with m = P_M(bounded) x
    rng = np.random.default_rng(6)
    n = 32
    x = rand_c(rng, n, n)
    M = rng.uniform(0.1, 2.0, (n, n))
    mask, U = spectrum_bounds(n, rng)
    S = (rng.random((n, n)) < 0.4).astype(np.uint8)
    m = orc.project_modulus_ub(x, M, mask, U)
    ref = np.where(S > 0, m, 0.9 * x + (1 - 1.8) * m)
    got = orc.iterate(x.copy(), S, M, mask, 2, 0.9, 1.0, 1, U=U)
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()


def test_mpr_run_bounds_off_paths_agree(orc):
    # bounds that never qualify (no missing pixel tolerated) reproduce the unbounded run
    pat = synthetic.config_pattern("ell128", 0)
    kw = dict(pop=4, iters_per_gen=40, generations=2, er_tail=5, seed=2)
    a = orc.mpr_run(pat.intensities, pat.mask, pat.support0, **kw)
    b = orc.mpr_run(pat.intensities, pat.mask, pat.support0, saturated=pat.saturated, ub_eta=1.5,
                    ub_max_missing=-1.0, **kw)
    c = orc.mpr_run(pat.intensities, pat.mask, pat.support0, saturated=pat.saturated, ub_eta=1.5, **kw)
    assert a["final_error_best"] == b["final_error_best"]
    assert np.array_equal(a["rho_avg"], b["rho_avg"])
    assert c["final_error_best"] != a["final_error_best"]  # the bounds take part
