"""Host-side arithmetic of bench.py that feeds reported figures (no GPU)."""
import importlib.util
import os
from math import comb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_m2l_flops_per_pair_closed_form():
    # The Taylor recurrence of degree k costs 3 flops per nonzero index component,
    # 2 more per component >= 2 and 1 for the scaling.  Over the C(k+2, 2)
    # multi-indices of degree k these are 3*C(k+1, 2), 3*C(k, 2) and C(k+2, 2)
    # components; r^2, 1/r^2 and 1/r add 7.  The (alpha, beta) pairs with
    # |alpha| + |beta| <= p are the monomials of degree <= p in 6 variables,
    # C(p+6, 6), one FMA (2 flops) each.
    b = _bench()
    for p in range(1, 9):
        rec = 7 + sum(9 * comb(k + 1, 2) + 6 * comb(k, 2) + comb(k + 2, 2) for k in range(1, p + 1))
        assert b.m2l_flops_per_pair(p) == rec + 2 * comb(p + 6, 6), p
    assert b.m2l_flops_per_pair(6) == 2652


def test_fmm_levels_refined_follows_the_chunks():
    b = _bench()
    assert [b._fmm_levels_refined(n) for n in (1, 6, 8, 9, 10, 12, 13, 16, 17, 21, 22)] == \
        [8, 8, 8, 12, 12, 12, 16, 16, 21, 21, 21]
    # uniform 2^20 (6 levels) and Plummer 2^20 (10 levels), mixed precision
    assert b._fmm_kernels_per_instance(6, True) == 2 + 1 + 40 + 40 + 1 + 1 + 1 + 1 + 6 + 2 + 10 + 2 + 5 + 1
    assert b._fmm_kernels_per_instance(10, False) == 2 + 1 + 40 + 60 + 1 + 1 + 1 + 10 + 2 + 10 + 2 + 9 + 1
