"""Host-side logic that needs no GPU: the seeded workload generators (their
distributions and determinism, the interval counts they promise) and the
benchmark's roofline selection from a per-category profile."""
import os
import sys

import numpy as np

from paper_1203_4031_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_serving_requests_follow_their_distribution_and_seed():
    a = W.serving_requests(count=400, nmin=128, nmax=4096, rate=20.0)
    b = W.serving_requests(count=400, nmin=128, nmax=4096, rate=20.0)
    assert a == b                                   # seeded, reproducible
    n = np.array([r["n"] for r in a])
    assert n.min() >= 128 and n.max() <= 4096
    # log-uniform: the median of log n sits near the middle of [log 128, log 4096]
    mid = 0.5 * (np.log(128) + np.log(4096))
    assert abs(np.median(np.log(n)) - mid) < 0.35
    k = np.array([r["count"] for r in a])
    assert k.min() >= 8 and k.max() <= 64
    assert all(r["m0"] == int(np.ceil(1.5 * r["count"])) for r in a)
    herm = np.mean([r["hermitian"] for r in a])
    assert 0.4 < herm < 0.6                         # 50/50 kinds
    t = np.array([r["t_arrival"] for r in a])
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1.0 / 20.0) < 0.2 / 20.0   # Poisson at 20/s


def test_batched_problem_intervals_hold_their_counts():
    probs = W.batched_generalized(count=4, nmin=64, nmax=160)
    again = W.batched_generalized(count=4, nmin=64, nmax=160)
    for p, q in zip(probs, again):
        assert np.array_equal(p.A, q.A) and np.array_equal(p.B, q.B)
        w = p.spectrum
        k = int(((w >= p.emin) & (w <= p.emax)).sum())
        assert 10 <= k <= 40
        assert p.m0 == int(np.ceil(1.5 * k))
        assert np.allclose(p.A, p.A.T) and np.allclose(p.B, p.B.T)
        assert np.linalg.eigvalsh(p.B).min() > 0    # B positive definite


def _bench():
    sys.path.insert(0, ROOT)
    import bench

    return bench


def test_roofline_picks_the_sliced_gemms_when_they_dominate():
    bench = _bench()
    prof = {"lu_update_gemm": (100, 50.0, 1e12), "solve_gemm": (200, 40.0, 5e11), "lu_panel": (128, 30.0, 0.0),
            "reduced_eig": (4, 20.0, 1e9), "other": (1, 0.1, 0.0)}
    tc = (300, 80.0, 1.5e12, 4.0e13)        # launches, ms, useful flops, issued bf16 flops
    r = bench.roofline(prof, tc, "fp64")
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert abs(r["achieved"] - 4.0e13 / 0.080 / 1e12) < 1e-9
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    assert abs(r["useful_fp64_tflops"] - 1.5e12 / 0.080 / 1e12) < 1e-9


def test_roofline_falls_back_to_the_dominant_alu_category():
    bench = _bench()
    prof = {"lu_update_gemm": (10, 5.0, 1e11), "solve_gemm": (10, 5.0, 1e11), "lu_panel": (128, 30.0, 0.0),
            "reduced_eig": (4, 60.0, 1.2e10), "other": (1, 0.1, 0.0)}
    tc = (20, 10.0, 2e11, 5e12)
    r = bench.roofline(prof, tc, "mixed")
    assert r["kernel"] == "reduced_eig" and r["bound"] == "alu"
    assert abs(r["achieved"] - 1.2e10 / 0.060 / 1e12) < 1e-12
