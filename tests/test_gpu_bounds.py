"""Upper bounds for missing intensities on the GPU (Eqs. avgint, stdint, upperbound,
pm_bounds) against the FP64 oracle: the encoded modulus array, the bounded projection in
every column-pass variant, bounded iterations at every side, and end-to-end MPR."""
import numpy as np
import pytest

import oracle
from paper_2409_07413_gb300 import synthetic

pytestmark = pytest.mark.gpu

TOL = 1e-5
SIDES = [64, 96, 128, 192, 256, 384, 512, 768, 1024]


@pytest.fixture(scope="module")
def sp():
    import torch
    from paper_2409_07413_gb300 import spring
    assert torch.cuda.is_available()
    return spring


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


def decode(M):
    """(M, mask, U) of the oracle from an encoded float32 modulus array."""
    M64 = M.astype(np.float64)
    mask = (M64 >= 0).astype(np.uint8)
    U = np.where(M64 <= -2.0, -2.0 - M64, -1.0)
    return np.where(mask > 0, M64, 0.0), mask, U


def bounded_modulus(seed, n, masked_frac=0.2, bound_frac=0.7):
    """Random encoded modulus: measured, missing with a bound, missing and free."""
    rng = np.random.default_rng(seed)
    M = rng.uniform(0.1, 2.0, (n, n))
    miss = rng.random((n, n)) < masked_frac
    bnd = miss & (rng.random((n, n)) < bound_frac)
    U = rng.uniform(0.0, 2.0, (n, n))  # comparable to |F x| (~1.4) of the unit-variance state
    enc = np.where(miss, np.where(bnd, -2.0 - U, -1.0), M).astype(np.float32)
    return enc


@pytest.mark.parametrize("name", ["sphere64", "ell128", "ell256", "ell512", "ell1024"])
def test_modulus_encode_matches_oracle(sp, name):
    pat = synthetic.config_pattern(name, 1)
    n = pat.n
    sat = pat.saturated if pat.saturated is not None else np.zeros((n, n), np.uint8)
    b = sp.bounds()
    M = host(sp.spring_modulus_encode(dev(pat.intensities), dev(pat.mask), dev(sat), b))
    Uc = oracle.upper_bounds(pat.intensities.astype(np.float64), pat.mask, sat, float(np.float32(b.eta)),
                             float(np.float32(b.max_missing)), float(np.float32(b.max_saturated)))
    U = np.fft.ifftshift(Uc)
    I = np.fft.ifftshift(pat.intensities)
    mk = np.fft.ifftshift(pat.mask)
    # measured moduli bit-exact (correctly rounded FP32 square root)
    assert np.array_equal(M[mk > 0], np.sqrt(I[mk > 0]).astype(np.float32))
    # the same pixels carry bounds; decoded bounds within FP32 rounding of -2 - U
    assert np.array_equal(M <= -2.0, U >= 0)
    sel = U >= 0
    assert sel.any() or name == "sphere64"
    got = -2.0 - M[sel].astype(np.float64)
    assert (np.abs(got - U[sel]) <= 2.0 ** -23 * (2.0 + U[sel])).all()
    assert (M[(mk == 0) & ~sel] == -1.0).all()
    # no bounds requested: the plain encoding
    M0 = host(sp.spring_modulus_encode(dev(pat.intensities), dev(pat.mask), None, None))
    assert np.array_equal(M0, np.where(mk > 0, M, -1.0).astype(np.float32))


@pytest.mark.parametrize("n", SIDES)
def test_project_modulus_bounded(sp, n):
    x, _ = synthetic.population_state(n + 3, 3, n)
    enc = bounded_modulus(n, n)
    out = host(sp.spring_project_modulus(dev(c64(x)), dev(enc)))
    M, mask, U = decode(enc)
    ref = oracle.project_modulus_ub(c64(x), M, mask, U)
    assert rel(out, ref) < TOL
    # the bounds bind somewhere and hold after the projection
    Y = np.fft.fft2(out.astype(np.complex128), norm="ortho")
    X = np.fft.fft2(c64(x).astype(np.complex128), norm="ortho")
    b = (mask == 0) & (U >= 0)
    assert (np.abs(X)[:, b] > U[b]).any()
    assert (np.abs(Y)[:, b] <= U[b] * (1 + 1e-4) + 1e-4).all()


@pytest.mark.parametrize("n", SIDES)
@pytest.mark.parametrize("alg", [0, 1, 2])
def test_iterate_bounded(sp, n, alg):
    x, S = synthetic.population_state(5 * n + alg, 2, n, support_frac=0.3)
    enc = bounded_modulus(3 * n, n)
    xg = dev(c64(x))
    sp.spring_iterate(xg, dev(S), dev(enc), alg, 0.9, 1.0, 1)
    M, mask, U = decode(enc)
    ref = oracle.iterate(c64(x), S, M, mask, alg, 0.9, 1.0, 1, U=U)
    assert rel(host(xg), ref) < TOL


@pytest.mark.parametrize("n", [256, 512])
def test_bounded_projection_in_every_column_variant(sp, n):
    B = 2
    x, S = synthetic.population_state(9 * n, B, n, support_frac=0.3)
    enc = bounded_modulus(9 * n, n)
    M, mask, U = decode(enc)
    ref = oracle.iterate(c64(x), S, M, mask, 2, 0.9, 1.0, 1, U=U)
    saved = sp.get_kernel_variant(n)
    try:
        for cv in range(10):
            sp.set_kernel_variant(n, saved[0], cv)
            xg = dev(c64(x))
            sp.spring_iterate(xg, dev(S), dev(enc), 2, 0.9, 1.0, 1)
            assert rel(host(xg), ref) < TOL, cv
    finally:
        sp.set_kernel_variant(n, *saved)


def test_iterate_bounded_fp16_storage(sp):
    n = 512
    x, S = synthetic.population_state(41, 2, n, support_frac=0.3)
    enc = bounded_modulus(41, n)
    M, mask, U = decode(enc)
    ref = oracle.iterate(c64(x), S, M, mask, 2, 0.9, 1.0, 1, U=U)
    xg = dev(c64(x))
    sp.spring_iterate_ex(xg, dev(S), dev(enc), 2, 0.9, 1.0, 1, 1)
    assert rel(host(xg), ref) < 3e-3  # one iteration of binary16 storage (~1e-3)


C1 = dict(pop=8, iters_per_gen=100, generations=5, algorithm=2, beta=0.9, sw_sigma=1.5,
          sw_threshold=0.2, sw_period=20, er_tail=10)


@pytest.fixture(scope="module")
def ctx(sp):
    c = sp.Context(0)
    yield c
    c.close()


def test_mpr_bounded_matches_oracle_statistically(sp, ctx):
    # gapped 128 x 128 patterns: mean final error over seeds within 2 % of the oracle's,
    # widened by two standard errors of the difference of the means
    eg, eo, eu = [], [], []
    ea, oa = [], []
    for seed in range(12):
        pat = synthetic.config_pattern("ell128", seed)
        prob = ctx.problem(pat.intensities, pat.mask, pat.support0, saturated=pat.saturated,
                           bounds=sp.bounds())
        r = prob.run(sp.params(**C1, seed=seed))
        prob.destroy()
        o = oracle.mpr_run(pat.intensities, pat.mask, pat.support0, saturated=pat.saturated,
                           seed=seed, ub_eta=1.5, **C1)
        eg.append(r["final_error_best"])
        ea.append(r["final_error_avg"])
        eo.append(o["final_error_best"])
        oa.append(o["final_error_avg"])
        assert np.isfinite(r["rho_avg"]).all()
    eg, eo = np.array(eg), np.array(eo)
    se = np.sqrt(eg.var(ddof=1) / len(eg) + eo.var(ddof=1) / len(eo))
    print(f"bounded: mean E gpu {eg.mean():.4f} oracle {eo.mean():.4f} (se {se:.4f})")
    assert abs(eg.mean() - eo.mean()) <= 0.02 * eo.mean() + 2.0 * se
    ea, oa = np.array(ea), np.array(oa)  # the error of the average reconstruction, same bar
    sea = np.sqrt(ea.var(ddof=1) / len(ea) + oa.var(ddof=1) / len(oa))
    assert abs(ea.mean() - oa.mean()) <= 0.02 * oa.mean() + 2.0 * sea, (ea.mean(), oa.mean(), sea)


def test_bounded_problem_changes_the_run(sp, ctx):
    pat = synthetic.config_pattern("ell256", 0)
    kw = dict(pop=4, iters_per_gen=40, generations=2, er_tail=5, seed=3)
    p0 = ctx.problem(pat.intensities, pat.mask, pat.support0)
    p1 = ctx.problem(pat.intensities, pat.mask, pat.support0, saturated=pat.saturated, bounds=sp.bounds())
    p2 = ctx.problem(pat.intensities, pat.mask, pat.support0, bounds=sp.bounds(eta=0.0))
    a, b, c = p0.run(sp.params(**kw)), p1.run(sp.params(**kw)), p2.run(sp.params(**kw))
    for p in (p0, p1, p2):
        p.destroy()
    assert not np.array_equal(a["rho_avg"], b["rho_avg"])
    assert np.array_equal(a["rho_avg"], c["rho_avg"])  # eta <= 0: no bounds


def test_bounds_invalid_arguments(sp, ctx):
    pat = synthetic.config_pattern("sphere64", 0)
    with pytest.raises(Exception):
        ctx.problem(pat.intensities, pat.mask, pat.support0, bounds=sp.bounds(max_missing=-1.0))
    with pytest.raises(Exception):
        ctx.problem(pat.intensities, pat.mask, pat.support0, bounds=sp.bounds(eta=float("inf")))
