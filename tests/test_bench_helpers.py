"""Host-side helpers of bench.py: the launch count it reports as gpu_launches and the
FP64 leg's arithmetic label follow the plan's configuration (no GPU needed)."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def info(**kw):
    base = dict(prec=0, epsilon=1e-5, flags=0, legendre_restart=64, legendre_table_bytes=0, legendre_df32_mmin=0,
                mmax=4096, point_weight_bytes=0)
    base.update(kw)
    return base


def test_kernel_launches_per_plan_kind():
    # restarted FP32 recursion: two coefficient preparations, fixed-point spreading bound
    assert bench.kernel_launches(info(), "fp32") == (2 + 3 + 1) + (1 + 3 + 1)
    # Legendre tables: one preparation
    assert bench.kernel_launches(info(legendre_restart=0, legendre_table_bytes=1 << 30), "fp32") == 5 + 5
    # FP32 below 1e-5 (double-float recursion, float spreading tiles): no bound kernel
    assert bench.kernel_launches(info(legendre_restart=0, epsilon=5e-6), "fp32") == 5 + 4
    # deterministic plans: their own fixed-point path (not counted here)
    assert bench.kernel_launches(info(flags=2), "fp32") == 6 + 4
    # FP64, restarted double-float recursion for every order: one Legendre launch per direction
    f64 = info(prec=1, epsilon=1e-10, legendre_restart=128, point_weight_bytes=1)
    assert bench.kernel_launches(f64, "fp64") == 5 + 5
    # FP64 with FP64 low orders: two Legendre launches per direction
    assert bench.kernel_launches(info(prec=1, epsilon=1e-12, legendre_restart=0, legendre_df32_mmin=256),
                                 "fp64") == 6 + 6


def test_fp64_arithmetic_label():
    lab = bench.fp64_arithmetic(info(prec=1, epsilon=1e-10, legendre_restart=128, point_weight_bytes=1))
    assert "every order" in lab and "double-float interpolation" in lab
    lab = bench.fp64_arithmetic(info(prec=1, epsilon=1e-12, legendre_restart=0, legendre_df32_mmin=5121))
    assert "m < 5121" in lab and "FP64 interpolation" in lab
