"""The benchmark's roofline accounting on CPU: every phase's `achieved` is the
method's algorithmic work (section 4.3's counts: the sketch 2 s m n flop, the
QR 2 s n^2 - 2 n^3 / 3 flop, the SVD of the triangle 11 n^3 flop, one fused
pass 8 m n bytes) divided by the phase's CUDA-event time, and `frac` is that
over the measured peak named in `peak_source`.  Values are recomputed here
from the per-phase times, so a line's fractions can be checked from its own
numbers."""
import os
import sys
from types import SimpleNamespace

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

bench = pytest.importorskip("bench")

PEAKS = {"hbm_gbs": 6785.5, "bf16_tflops": 1902.3, "bf16_tflops_sustained": 1707.9}
FP64 = 1.25


def _info(**kw):
    base = dict(s=4000, t_sketch_ms=300.0, t_sketch_gemm_ms=273.0, t_qr_ms=60.0,
                t_jacobi_ms=372.0, t_pass_ms=437.0, n_pass=95, jacobi_sweeps=10,
                jacobi_sweeps_df=0)
    base.update(kw)
    return base


def _args(**kw):
    base = dict(m=1_000_000, n=2000, sketch="tc", iter="x2")
    base.update(kw)
    return SimpleNamespace(**base)


def test_phase_work_counts_and_fractions():
    m, n, s = 1_000_000, 2000, 4000
    ph = bench.phase_rooflines([_info(), _info()], _args(), PEAKS, FP64)
    sk = ph["sketch"]
    assert sk["achieved"] == pytest.approx(2.0 * s * m * n / 0.273 / 1e12)
    assert sk["frac"] == pytest.approx(sk["achieved"] / PEAKS["bf16_tflops_sustained"])
    assert sk["slice_products_tflops"] == pytest.approx(15 * sk["achieved"])
    qr = ph["qr"]
    assert qr["achieved"] == pytest.approx((2.0 * s * n * n - 2.0 * n ** 3 / 3.0) / 0.060 / 1e12)
    assert qr["frac"] == pytest.approx(qr["achieved"] / FP64)
    svd = ph["svd"]
    assert svd["achieved"] == pytest.approx(11.0 * n ** 3 / 0.372 / 1e12)
    assert svd["sweeps"] == 10
    ps = ph["passes"]
    assert ps["ms_each"] == pytest.approx(437.0 / 95)
    assert ps["achieved"] == pytest.approx(8.0 * m * n / (437.0 / 95 * 1e-3) / 1e9)
    assert ps["frac"] == pytest.approx(ps["achieved"] / PEAKS["hbm_gbs"])
    assert ps["bytes_streamed_per_pass"] == pytest.approx(8.0 * m * n)
    # the dominant phase is the one with the largest device time per solve
    assert max(ph, key=lambda k: ph[k]["ms"]) == "passes"


def test_phase_times_are_means_over_the_timed_solves():
    ph = bench.phase_rooflines([_info(t_jacobi_ms=400.0), _info(t_jacobi_ms=600.0)], _args(),
                               PEAKS, FP64)
    assert ph["svd"]["ms"] == pytest.approx(500.0)
    assert max(ph, key=lambda k: ph[k]["ms"]) == "svd"


def test_fp64_and_fp32_modes_use_their_own_units():
    ph = bench.phase_rooflines([_info(t_sketch_ms=14900.0)], _args(sketch="f64", iter="f32"),
                               PEAKS, FP64)
    sk = ph["sketch"]
    assert sk["bound"] == "alu" and sk["peak"] == FP64
    assert sk["achieved"] == pytest.approx(2.0 * 4000 * 1_000_000 * 2000 / 14.9 / 1e12)
    # an FP32 pass streams 4 bytes per element; achieved stays the method's 8 m n
    ps = ph["passes"]
    assert ps["bytes_streamed_per_pass"] == pytest.approx(4.0 * 1_000_000 * 2000)
    assert ps["achieved"] == pytest.approx(8.0 * 1_000_000 * 2000 / (437.0 / 95 * 1e-3) / 1e9)


def test_a_shard_counts_its_own_rows():
    ph = bench.phase_rooflines([_info()], _args(), PEAKS, FP64, m_local=250_000)
    assert ph["passes"]["achieved"] == pytest.approx(8.0 * 250_000 * 2000 / (437.0 / 95 * 1e-3)
                                                     / 1e9)
