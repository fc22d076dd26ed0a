"""Edge cases of the operators on the GPU: empty batches, zero iteration counts,
unsupported sides, and the degenerate inputs the method has (a zero state, a fully
unmeasured modulus, an empty support), each against the FP64 oracle."""
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


def test_empty_batches_and_zero_iterations(sp):
    n = 128
    x0 = dev(np.zeros((0, n, n), np.complex64))
    S0 = dev(np.zeros((0, n, n), np.uint8))
    M = dev(np.ones((n, n), np.float32))
    sp.spring_fft2(x0)
    sp.spring_iterate(x0, S0, M, 2, 0.9, 0.5, 5)
    sp.spring_iterate_ex(x0, S0, M, 2, 0.9, 0.5, 5, 1)
    assert host(sp.spring_smooth(x0, 1.5)).shape == (0, n, n)
    x, S = synthetic.population_state(1, 2, n)
    xg = dev(c64(x))
    sp.spring_iterate(xg, dev(S), M, 2, 0.9, 0.5, 0)
    assert np.array_equal(host(xg), c64(x))  # no iteration: untouched


@pytest.mark.parametrize("n", [32, 48, 100, 320, 576, 1536, 2048])
def test_unsupported_sides_are_rejected(sp, n):
    x = dev(np.zeros((1, n, n), np.complex64))
    with pytest.raises(sp.SpringError) as e:
        sp.spring_fft2(x)
    assert e.value.status == sp.E_INVALID
    with pytest.raises(sp.SpringError):
        sp.spring_iterate(x, dev(np.zeros((1, n, n), np.uint8)), dev(np.ones((n, n), np.float32)),
                          2, 0.9, 0.5, 1)


@pytest.mark.parametrize("n", [64, 512])
def test_zero_state_takes_phase_zero(sp, n):
    # F x = 0 everywhere: every measured value becomes M with phase 0 (then unmeasured stay 0)
    M, mask = synthetic.random_modulus(n, n, masked_frac=0.1)
    Menc = np.where(mask > 0, M, -1.0).astype(np.float32)
    x = np.zeros((2, n, n), np.complex64)
    got = host(sp.spring_project_modulus(dev(x), dev(Menc)))
    ref = oracle.project_modulus(x.astype(np.complex128), M.astype(np.float32).astype(np.float64), mask)
    assert rel(got, ref) < TOL
    err = host(sp.spring_fourier_error(dev(x), dev(np.ones((2, n, n), np.uint8)), dev(Menc)))
    assert np.allclose(err, 1.0, rtol=1e-12)  # E = 1 for x = 0


@pytest.mark.parametrize("alg", [0, 1, 2])
def test_nothing_measured_and_empty_support(sp, alg):
    # no measured pixel: P_M is the identity, so m = x and the update acts on x alone;
    # with an empty support every pixel is outside the constraint set
    n = 128
    x, S = synthetic.population_state(3, 2, n)
    nothing = np.full((n, n), -1.0, np.float32)
    xg = dev(c64(x))
    sp.spring_iterate(xg, dev(S), dev(nothing), alg, 0.9, 1.0, 1)
    ref = oracle.iterate(c64(x), S, np.zeros((n, n)), np.zeros((n, n), np.uint8), alg, 0.9, 1.0, 1)
    assert rel(host(xg), ref) < TOL
    M, mask = synthetic.random_modulus(4, n)
    Menc = np.where(mask > 0, M, -1.0).astype(np.float32)
    empty = np.zeros((2, n, n), np.uint8)
    yg = dev(c64(x))
    sp.spring_iterate(yg, dev(empty), dev(Menc), alg, 0.9, 1.0, 1)
    ref = oracle.iterate(c64(x), empty, M.astype(np.float32).astype(np.float64), mask, alg, 0.9, 1.0, 1)
    got = host(yg)
    if alg == 0:
        assert not got.any()  # ER keeps nothing outside the support
    else:
        assert rel(got, ref) < TOL


def test_bounded_wait_times_out_and_the_device_stays_usable(sp):
    # failure detection without a fault: a block waits on a barrier that nothing completes,
    # gives up after 2^20 cycles, records the timed-out wait, and the library reports it
    assert sp.check_wait_timeout(1 << 20) == sp.E_TIMEOUT
    assert "timed out" in sp.last_error()
    assert sp.check_wait_timeout(0) == sp.E_INVALID
    # the context is still usable and the status word was cleared: a transform afterwards
    # matches the oracle, and a whole run completes without a timeout status
    x, _ = synthetic.population_state(5, 2, 64)
    xg = dev(c64(x))
    sp.spring_fft2(xg)
    assert rel(host(xg), oracle.fft2(c64(x))) < TOL
    pat = synthetic.config_pattern("sphere64", 0)
    ctx = sp.Context(0)
    prob = ctx.problem(pat.intensities, pat.mask, pat.support0)
    r = prob.run(sp.params(pop=4, iters_per_gen=40, generations=2, er_tail=5, seed=1), want_arrays=False)
    prob.destroy()
    ctx.close()
    assert np.isfinite(r["final_error_best"])
