"""Tensor-core Legendre synthesis (tcgen05, split TF32) of 16 or more spin-0 maps.

lens_synthesis with nmaps >= 16 on a spin-0 FP32 plan with the restarted
recursion runs the Legendre step of up to 64 maps at a time on the tensor
cores.  Each map must equal its own CUDA-core synthesis (same recursion values,
products at FP32 level, FP32 accumulation in another order) and the oracle.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2304_10431_gb300 import LensPlan
from paper_2304_10431_gb300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0") if torch.cuda.is_available() else None


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def maps_alm(L, nm, seed):
    cl = W.cmb_cl(L, 0.8 * L)
    return np.stack([W.draw_alm(cl, L, seed + 7 * b)[None] for b in range(nm)])  # [nm][1][nalm]


@pytest.mark.parametrize("L,nm", [(300, 16), (300, 40), (300, 64), (700, 17), (129, 70)])
def test_tensor_core_synthesis_matches_cuda_cores_and_oracle(L, nm):
    n = 20000
    th, ph, _ = W.random_points(n, 31 + L)
    th[:3] = [0.0, math.pi, 0.5 * math.pi]
    plan = LensPlan(L, th, ph, spin=0, epsilon=1e-5, precision="fp32", device=DEV)
    assert plan.info()["legendre_restart"] > 0
    a = maps_alm(L, nm, 100)
    ta = torch.as_tensor(a, dtype=plan.complex_dtype, device=DEV)
    tc = plan.synthesis(ta).cpu().numpy()
    plan.status()
    plan.set_tensor_cores(False)
    ref = plan.synthesis(ta).cpu().numpy()
    # two FP32 evaluations of the same sums (FP32 recursion values; split-TF32 products and
    # tensor-core accumulation order against FP32 FMAs): agree to a few 1e-6
    for b in range(nm):
        assert rel(tc[b], ref[b]) < 4e-6, (b, rel(tc[b], ref[b]))
    s = np.arange(0, n, 157)
    for b in (0, nm // 2, nm - 1):
        orc = O.synthesis(L, L, 0, th[s], ph[s], a[b])
        assert rel(tc[b][:, s], orc) <= 1e-5
    plan.close()


def test_plan_usable_after_tensor_core_call():
    """After a 16-map tensor-core call (which allocates its workspace) the plan's status is clean and its
    single-map Legendre step still matches the oracle's direct sums at lmax 1024."""
    L = 1024
    th, ph, _ = W.random_points(64, 5)
    plan = LensPlan(L, th, ph, spin=0, epsilon=1e-5, precision="fp32", device=DEV)
    a = maps_alm(L, 16, 300)
    ta = torch.as_tensor(a, dtype=plan.complex_dtype, device=DEV)
    plan.synthesis(ta)  # first call with 16 maps allocates the workspace and runs the tensor-core step
    plan.status()
    nt = plan.info()["ntheta"]
    rows = np.array(sorted(set([0, 1, 2, 3, 50, 300, nt // 4, nt // 2, nt - 2, nt - 1])))
    single = plan.ring_synthesis(ta[0]).cpu().numpy()
    orc = O.ring_coeffs(L, L, 0, rows * math.pi / (nt - 1), a[0]).T
    assert rel(single[:, rows], orc) < 2e-6
    plan.close()


def test_tensor_core_off_and_small_batches():
    th, ph, _ = W.random_points(3000, 8)
    plan = LensPlan(200, th, ph, spin=0, epsilon=1e-5, precision="fp32", device=DEV)
    a = maps_alm(200, 15, 7)
    ta = torch.as_tensor(a, dtype=plan.complex_dtype, device=DEV)
    m15 = plan.synthesis(ta).cpu().numpy()  # 15 maps: CUDA-core groups
    one = plan.synthesis(ta[3]).cpu().numpy()
    assert rel(m15[3], one) < 1e-6
    plan.close()
