"""The allocation-free GetError entry point (for callers that cannot call cudaMalloc)
gives the allocating entry point's results, call after call, through the C ABI.

This file is collected last so that a run stopping at the first failure has already run
every other test; it also passes alone in a fresh process."""
import numpy as np
import pytest

from paper_2409_07413_gb300 import synthetic

pytestmark = pytest.mark.gpu
TOL = 1e-5  # the operator tolerance of the other GPU tests


def _inputs(seed, b, n):
    import torch
    x, S = synthetic.population_state(seed, b, n, support_frac=0.3)
    M, mask = synthetic.random_modulus(seed, n, masked_frac=0.1)
    Menc = np.where(mask > 0, M, -1.0).astype(np.float32)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return dev(x.astype(np.complex64)), dev(S), dev(Menc)


def test_noalloc_matches_allocating_entry_point_on_consecutive_calls():
    import torch
    from paper_2409_07413_gb300 import spring
    # two calls in a row with different sizes: the fixed scratch keeps the first call's
    # contents, which must not leak into the second result
    for seed, n, b in [(1, 512, 7), (2, 192, 3), (3, 1024, 1)]:
        x, S, M = _inputs(seed, b, n)
        ref = spring.spring_fourier_error(x, S, M)
        got = torch.empty(b, dtype=torch.float64, device="cuda")
        spring.spring_fourier_error_noalloc(x, S, M, got)
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        assert np.all(np.abs(g - r) <= TOL * np.abs(r)), (n, b, g, r)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_2409_07413_gb300 import spring
    x, S, M = _inputs(4, 8, 512)  # 8 x 512 x 512 complex64 = 16 MiB + partial sums
    err = torch.empty(8, dtype=torch.float64, device="cuda")
    with pytest.raises(spring.SpringError) as e:
        spring.spring_fourier_error_noalloc(x, S, M, err)
    assert e.value.status == spring.E_INVALID
    assert "maximum" in str(e.value)
