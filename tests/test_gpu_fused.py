"""The on-chip whole-iteration kernel (one thread-block cluster per image, N <= 256)
against the FP64 oracle, bit-identity with the two-pass path on the same transform plan,
and end-to-end runs on either path."""
import numpy as np
import pytest

import oracle
from paper_2409_07413_gb300 import synthetic

pytestmark = pytest.mark.gpu

TOL = 1e-5
SMALL = [64, 128, 192, 256]


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


def menc(M, mask):
    return np.where(mask > 0, M, -1.0).astype(np.float32)


@pytest.mark.parametrize("n", SMALL)
@pytest.mark.parametrize("alg", [0, 1, 2])
@pytest.mark.parametrize("chi", [0.5, 1.0])
def test_fused_one_iteration_matches_oracle(sp, n, alg, chi):
    x, S = synthetic.population_state(11 * n + alg, 3, n, support_frac=0.3)
    M, mask = synthetic.random_modulus(11 * n, n, masked_frac=0.1)
    xg = dev(c64(x))
    sp.spring_iterate_fused(xg, dev(S), dev(menc(M, mask)), alg, 0.9, chi, 1)
    ref = oracle.iterate(c64(x), S, M.astype(np.float32).astype(np.float64), mask, alg, 0.9, chi, 1)
    assert rel(host(xg), ref) < TOL


@pytest.mark.parametrize("n", SMALL)
def test_fused_equals_two_pass_bitwise(sp, n):
    # same plan in both directions (row variant 0, column variant 0): the same bits after
    # several iterations, with bounds in M, for every algorithm
    B, k = 5, 7
    x, S = synthetic.population_state(13 * n, B, n, support_frac=0.3)
    rng = np.random.default_rng(n)
    M, mask = synthetic.random_modulus(13 * n, n, masked_frac=0.2)
    enc = menc(M, mask)
    bnd = (mask == 0) & (rng.random((n, n)) < 0.5)
    enc = np.where(bnd, -2.0 - rng.uniform(0, 2, (n, n)), enc).astype(np.float32)
    saved = sp.get_kernel_variant(n)
    try:
        sp.set_kernel_variant(n, 0, 0)
        for alg in (0, 1, 2):
            a, b = dev(c64(x)), dev(c64(x))
            sp.spring_iterate(a, dev(S), dev(enc), alg, 0.9, 0.5, k)
            sp.spring_iterate_fused(b, dev(S), dev(enc), alg, 0.9, 0.5, k)
            ha, hb = host(a), host(b)
            assert np.isfinite(hb).all()
            assert np.array_equal(ha, hb), (alg, rel(hb, ha.astype(np.complex128)))
    finally:
        sp.set_kernel_variant(n, *saved)


def test_fused_rejects_large_sides(sp):
    x = dev(np.zeros((1, 512, 512), np.complex64))
    with pytest.raises(sp.SpringError):
        sp.spring_iterate_fused(x, dev(np.zeros((1, 512, 512), np.uint8)),
                                dev(np.ones((512, 512), np.float32)), 2, 0.9, 0.5, 1)


C1 = dict(pop=8, iters_per_gen=100, generations=5, algorithm=2, beta=0.9, sw_sigma=1.5,
          sw_threshold=0.2, sw_period=20, er_tail=10)


@pytest.fixture(scope="module")
def ctx(sp):
    c = sp.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("name", ["sphere64", "ell128", "ell192", "ell256"])
def test_run_on_either_path_is_identical(sp, ctx, name):
    pat = synthetic.config_pattern(name, 2)
    n = pat.n
    prob = ctx.problem(pat.intensities, pat.mask, pat.support0)
    saved, spath = sp.get_kernel_variant(n), sp.get_iteration_path(n)
    try:
        sp.set_kernel_variant(n, 0, 0)
        sp.set_iteration_path(n, 0)
        a = prob.run(sp.params(**C1, seed=4))
        sp.set_iteration_path(n, 1)
        b = prob.run(sp.params(**C1, seed=4))
        g = prob.run(sp.params(**C1, seed=4, use_graph=1))
    finally:
        sp.set_kernel_variant(n, *saved)
        sp.set_iteration_path(n, spath)
        prob.destroy()
    for k in ("rho_avg", "rho_best", "support_avg", "gen_stats"):
        assert np.array_equal(a[k], b[k], equal_nan=True), k
        assert np.array_equal(b[k], g[k], equal_nan=True), k


def test_fused_run_matches_oracle_statistically(sp, ctx):
    saved = sp.get_iteration_path(64)
    eg, eo = [], []
    ea, oa = [], []
    try:
        sp.set_iteration_path(64, 1)
        for seed in range(10):
            pat = synthetic.config_pattern("sphere64", seed)
            prob = ctx.problem(pat.intensities, pat.mask, pat.support0)
            r = prob.run(sp.params(**C1, seed=seed))
            prob.destroy()
            o = oracle.mpr_run(pat.intensities, pat.mask, pat.support0, seed=seed, **C1)
            eg.append(r["final_error_best"])
            ea.append(r["final_error_avg"])
            eo.append(o["final_error_best"])
            oa.append(o["final_error_avg"])
    finally:
        sp.set_iteration_path(64, saved)
    eg, eo = np.array(eg), np.array(eo)
    se = np.sqrt(eg.var(ddof=1) / len(eg) + eo.var(ddof=1) / len(eo))
    assert abs(eg.mean() - eo.mean()) <= 0.02 * eo.mean() + 2.0 * se
    ea, oa = np.array(ea), np.array(oa)  # the error of the average reconstruction, same bar
    sea = np.sqrt(ea.var(ddof=1) / len(ea) + oa.var(ddof=1) / len(oa))
    assert abs(ea.mean() - oa.mean()) <= 0.02 * oa.mean() + 2.0 * sea, (ea.mean(), oa.mean(), sea)
