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


def test_atomic_roofline_weighted_harmonic_peak():
    # the peak of a mix of two atomic kinds is the weighted harmonic mean of their rates:
    # the units need d/r_d + a/r_a seconds for d decrements and a accumulates
    b = _bench()
    ceil = {"join_decrement": 40e9, "accumulate": 10e9}
    r = b._atomic_roofline("k", tasks=1000, decrements=800, accumulates=200, kernel_ms=1e-3, ceil=ceil)
    assert abs(r["peak"] - 1000 / (800 / 40 + 200 / 10)) < 1e-9      # Gop/s
    assert abs(r["achieved"] - 1000 / 1e-6 / 1e9) < 1e-9
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    assert r["atomics_per_launch"] == 1000 and r["tasks_per_s"] == 1000 / 1e-6
    # one kind only: the peak is that kind's rate
    r1 = b._atomic_roofline("k", 10, 10, 0, 1.0, ceil)
    assert abs(r1["peak"] - 40.0) < 1e-9


def test_clock_summary_median_and_rejection_reasons():
    b = _bench()
    s = b.ClockSampler(0)
    # index, sm, max sm, power, active, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
    s.samples = [["0", "2070", "2070", "900", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
                 ["0", "1980", "2070", "1390", "0x4", "Not Active", "Not Active", "Not Active", "Active"],
                 ["0", "2070", "2070", "910", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
                 ["garbage"]]
    out = s.summary()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]
    s.samples.append(["0", "1500", "2070", "1400", "0x40", "Not Active", "Active", "Not Active", "Not Active"])
    assert "hw_thermal_slowdown" in s.summary()["reasons"]
    assert b.ClockSampler(0).summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_gpus_flag_disagreeing_with_world_size_exits_2():
    import json
    import subprocess
    import sys
    env = dict(os.environ, WORLD_SIZE="1", RANK="0", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--gpus", "2"], env=env,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 2
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert "WORLD_SIZE=1" in line["error"]


def test_serve_trace_is_seeded_and_mixes_four_kinds():
    b = _bench()
    a1, r1 = b._serve_trace(2000, 5000.0)
    a2, r2 = b._serve_trace(2000, 5000.0)
    assert list(a1) == list(a2) and r1 == r2
    assert all(a1[i] <= a1[i + 1] for i in range(len(a1) - 1))
    kinds = {k for k, _ in r1}
    assert kinds == {"fib", "nqueens", "kclique", "uts"}
    for k, x in r1:
        lo, hi = {"fib": (20, 32), "nqueens": (8, 12), "kclique": (10, 14), "uts": (100, 2000)}[k]
        assert lo <= x <= hi
    # mean inter-arrival time of a Poisson stream at 5000 req/s
    assert abs((a1[-1] - a1[0]) / (len(a1) - 1) - 1 / 5000.0) < 0.1 / 5000.0
