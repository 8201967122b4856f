"""rks_eval_xc_noalloc (collected last): the allocation-free variant of
rks_eval_xc gives the same results as the allocating entry, on two calls in a
row, with a smaller call after a larger one (stale scratch beyond n must not
leak into the outputs), at the size limit, and rejects n above the limit.

Tolerance: exact.  Both entries run the same kernel on the same inputs, so the
outputs are bit-identical; the B3LYP values themselves are pinned against the
oracle in test_gpu_parity.py::test_xc_kernel."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

g = pytest.importorskip("paper_2311_01135_gb300")


def _inputs(n, seed):
    rng = np.random.default_rng(seed)
    rho = 10.0 ** rng.uniform(-9, 3, n)
    sigma = rho ** (8 / 3) * 10.0 ** rng.uniform(-4, 2.5, n)
    return rho, sigma


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_noalloc_matches_allocating_entry(prec):
    p = g.RKS_FP64 if prec == "fp64" else g.RKS_MIXED
    with g.Context() as c:
        for n, seed in ((5000, 1), (5000, 2), (g.RKS_XC_NOALLOC_MAX, 3), (37, 4)):
            rho, sigma = _inputs(n, seed)
            ref = c.eval_xc(rho, sigma, p)
            for _ in range(2):
                got = c.eval_xc_noalloc(rho, sigma, p)
                for a, b in zip(got, ref):
                    np.testing.assert_array_equal(a, b)


def test_noalloc_rejects_sizes_beyond_the_scratch():
    with g.Context() as c:
        rho, sigma = _inputs(g.RKS_XC_NOALLOC_MAX + 1, 5)
        with pytest.raises(g.RKSError) as e:
            c.eval_xc_noalloc(rho, sigma)
        assert e.value.code == g.RKS_EINVAL
        assert "RKS_XC_NOALLOC_MAX" in str(e.value)
        # the context stays usable
        r, s = _inputs(16, 6)
        np.testing.assert_array_equal(c.eval_xc_noalloc(r, s)[0], c.eval_xc(r, s)[0])
