"""The allocation-free entry point dotpe_dist_marg_eval_noalloc.

Callers that cannot allocate device memory when they call (a host
application whose own caching allocator has reserved the device's memory, or
a latency-bound loop that must not pay for cudaMalloc/cudaFree) use this
variant: its scratch is a static device array instead of cudaMalloc'ed memory.  The test calls it
through the C ABI and checks it against the allocating dotpe_dist_marg_eval,
on two calls in a row with different inputs (so that a stale scratch array
would show), and checks that an oversized request is refused.  It creates
its own context so that it runs the same alone or after the other tests.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _inputs(rng, n, u_min):
    x = rng.uniform(-30.0, 60.0, n)
    s = np.exp(rng.uniform(-10.0, 4.0, n))
    hh = (s / u_min) ** 2
    return (x * np.sqrt(hh)).astype(np.float32), hh.astype(np.float32)


def test_noalloc_matches_allocating_entry_point_twice():
    import __graft_entry__ as ge
    ge.build()
    import paper_2507_16022_gb300 as dp
    ctx = dp.dotpe_create(0)
    try:
        rng = np.random.default_rng(11)
        for n, u_min in ((200_000, 2.0), (70_001, 9.5)):
            dh, hh = _inputs(rng, n, u_min)
            ref = dp.dotpe_dist_marg_eval(ctx, dh, hh, u_min)
            got = dp.dotpe_dist_marg_eval_noalloc(ctx, dh, hh, u_min)
            # same device function on the same inputs; the table tolerance of the parity tests
            assert got.shape == ref.shape
            assert np.all(np.isfinite(got))
            np.testing.assert_allclose(got, ref, rtol=0, atol=1e-4)
        with pytest.raises(dp.DotpeError) as ei:
            big = np.zeros(dp.DIST_MARG_NOALLOC_MAX + 1, np.float32)
            dp.dotpe_dist_marg_eval_noalloc(ctx, big, big + 1.0, 2.0)
        assert ei.value.status == dp.DOTPE_E_INVALID
        assert "allocation-free limit" in str(ei.value)
    finally:
        dp.dotpe_destroy(ctx)
