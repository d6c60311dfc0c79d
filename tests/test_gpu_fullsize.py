"""Full-size parity at the headline workload (lmax 4096, HEALPix Nside 2048,
50,331,648 points), in the plan configuration the benchmark times (FP32 plans with
the restarted FP32 Legendre recursion) and with Legendre-table plans, at the
two other full-size workloads: spin-2 lensing at lmax 2048 / Nside 1024
(12,582,912 points) and the paper-scale run at lmax 5120 / Nside 2048 with the
epsilon sweep 1e-4 (FP32) and 1e-6 .. 1e-12 (FP64), and at a point of the
Fig. 4 scan, lmax 8192 / Nside 4096 (201,326,592 points).  Each case states the
relative L2 error (eps_eff), the largest error relative to the largest value
and the rms error.

The oracle cannot evaluate all 50M outputs, so:
  * forward: 256 sampled outputs (rings near both poles and the equator) are
    compared one by one; the sample's relative L2 error must be <= epsilon;
  * adjoint: the input map is non-zero only on the sampled points, so the
    oracle's adjoint over those points is the exact full a_lm vector, compared
    in relative L2.
Points: HEALPix centres displaced by independent 2.5 arcmin offsets (the
density and locality of the lensed geometry), phase chi of lensing size.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2304_10431_gb300 import LensPlan
from paper_2304_10431_gb300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0") if torch.cuda.is_available() else None
LMAX, NSIDE = 4096, 2048


@pytest.fixture(scope="module")
def geometry():
    th0, ph0 = W.healpix_centres(NSIDE)
    th, ph, chi = W.displaced_points(th0, ph0, 2.5, seed=3000)
    n = th.size
    rng = np.random.default_rng(17)
    sample = np.unique(np.concatenate([rng.integers(0, 40000, 64), rng.integers(n - 40000, n, 64),
                                       rng.integers(n // 2 - 200000, n // 2 + 200000, 128)]))
    return th, ph, chi, sample


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def stats(a, b):
    """Relative L2 (Sect. 4's eps_eff), max|err| / max|ref| and rms error / rms ref."""
    d = np.abs(np.asarray(a) - np.asarray(b))
    return {"eps_eff": rel(a, b), "max_rel": float(d.max() / np.abs(b).max()),
            "rms_err": float(np.sqrt(np.mean(d ** 2))), "rms_ref": float(np.sqrt(np.mean(np.abs(b) ** 2)))}


_REF = {}


def _sample(n, rng):
    """Indices near both poles and the equator (ring order)."""
    return np.unique(np.concatenate([rng.integers(0, 40000, 64), rng.integers(n - 40000, n, 64),
                                     rng.integers(n // 2 - 200000, n // 2 + 200000, 128)]))


def _check(lmax, th, ph, chi, s, spin, prec, eps, l_damp, seed, precise=False):
    """Forward on the sample vs the oracle; adjoint of a map supported on the sample
    (whose exact a_lm the oracle computes) vs the oracle (double-double harmonics
    when precise)."""
    nc = 1 if spin == 0 else 2
    cl = W.cmb_cl(lmax, l_damp)
    a = np.stack([W.draw_alm(cl, lmax, seed + k, spin=spin) for k in range(nc)])
    plan = LensPlan(lmax, th, ph, chi if spin else None, spin=spin, epsilon=eps, precision=prec, device=DEV)
    m = plan.synthesis(torch.as_tensor(a, dtype=plan.complex_dtype, device=DEV))
    got = m[:, torch.as_tensor(s, device=DEV)].cpu().numpy()
    y = np.random.default_rng(5).standard_normal((nc, s.size))
    key = (lmax, spin, seed, s.size, float(th[s[0]]), precise)
    if key not in _REF:  # the oracle's values depend on the inputs only, not on the plan
        _REF[key] = (O.synthesis(lmax, lmax, spin, th[s], ph[s], a, chi[s] if spin else None, precise=precise),
                     O.adjoint(lmax, lmax, spin, th[s], ph[s], y, chi[s] if spin else None, precise=precise))
    ref, aref = _REF[key]
    ymap = torch.zeros(nc, th.size, dtype=plan.real_dtype, device=DEV)
    ymap[:, torch.as_tensor(s, device=DEV)] = torch.as_tensor(y, dtype=plan.real_dtype, device=DEV)
    at = plan.adjoint(ymap).cpu().numpy()
    plan.close()
    del m, ymap
    torch.cuda.empty_cache()
    sf, sa = stats(got, ref), stats(at, aref)
    print("lmax %d spin %d %s eps %.0e: fwd eps_eff %.2e max %.2e rms %.2e | adj eps_eff %.2e max %.2e rms %.2e"
          % (lmax, spin, prec, eps, sf["eps_eff"], sf["max_rel"], sf["rms_err"], sa["eps_eff"], sa["max_rel"],
             sa["rms_err"]))
    # the largest single error relative to the largest value, stated and bounded loosely: forward
    # 3 epsilon; adjoint 10 (FP32) / 20 (FP64) epsilon: its errors are heavier-tailed over the a_lm
    k = 6.0 if precise else 1.0
    ka = 10.0 if prec == "fp32" else 20.0
    assert sf["max_rel"] <= 3 * eps * k and sa["max_rel"] <= ka * eps * k, (sf, sa)
    return rel(got, ref), rel(at, aref)


@pytest.mark.parametrize("spin,prec,eps,tables", [(0, "fp32", 1e-5, True), (2, "fp32", 1e-5, True),
                                                 (0, "fp32", 1e-5, False), (2, "fp32", 1e-5, False),
                                                 (0, "fp64", 1e-10, False)])
def test_headline_sampled(geometry, spin, prec, eps, tables):
    """The benchmark's FP32 plans (restarted recursion), plans with Legendre tables and the FP64 plan,
    at the same points."""
    th, ph, chi, s = geometry
    nc = 1 if spin == 0 else 2
    cl = W.cmb_cl(LMAX, 0.73 * LMAX)
    a = np.stack([W.draw_alm(cl, LMAX, 1000 + k, spin=spin) for k in range(nc)])
    plan = LensPlan(LMAX, th, ph, chi if spin else None, spin=spin, epsilon=eps, precision=prec,
                    legendre_tables=tables, device=DEV)
    m = plan.synthesis(torch.as_tensor(a, dtype=plan.complex_dtype, device=DEV))
    got = m[:, torch.as_tensor(s, device=DEV)].cpu().numpy()
    y = np.random.default_rng(5).standard_normal((nc, s.size))
    key = ("headline", spin)
    if key not in _REF:  # the oracle's values depend on the inputs only, not on the plan
        _REF[key] = (O.synthesis(LMAX, LMAX, spin, th[s], ph[s], a, chi[s] if spin else None),
                     O.adjoint(LMAX, LMAX, spin, th[s], ph[s], y, chi[s] if spin else None))
    ref, aref = _REF[key]
    assert rel(got, ref) <= eps
    # adjoint of a map supported on the sample: exact full a_lm from the oracle
    ymap = torch.zeros(nc, th.size, dtype=plan.real_dtype, device=DEV)
    ymap[:, torch.as_tensor(s, device=DEV)] = torch.as_tensor(y, dtype=plan.real_dtype, device=DEV)
    at = plan.adjoint(ymap).cpu().numpy()
    assert rel(at, aref) <= eps
    sf, sa = stats(got, ref), stats(at, aref)
    print("headline spin %d %s%s: fwd eps_eff %.2e max %.2e rms %.2e | adj eps_eff %.2e max %.2e rms %.2e"
          % (spin, prec, " tables" if tables else "", sf["eps_eff"], sf["max_rel"], sf["rms_err"], sa["eps_eff"],
             sa["max_rel"], sa["rms_err"]))
    assert sf["max_rel"] <= 3 * eps and sa["max_rel"] <= (10 if prec == "fp32" else 20) * eps, (sf, sa)
    plan.close()
    del m, ymap
    torch.cuda.empty_cache()


@pytest.mark.parametrize("prec,eps", [("fp32", 1e-5), ("fp64", 1e-10)])
def test_spin2_lmax2048_nside1024(prec, eps):
    th0, ph0 = W.healpix_centres(1024)
    th, ph, chi = W.displaced_points(th0, ph0, 2.5, seed=3001)
    s = _sample(th.size, np.random.default_rng(18))
    fwd, adj = _check(2048, th, ph, chi, s, 2, prec, eps, 1500.0, 1100)
    assert fwd <= eps and adj <= eps, (fwd, adj)


@pytest.fixture(scope="module")
def geometry_5120():
    th0, ph0 = W.healpix_centres(NSIDE)
    th, ph, chi = W.displaced_points(th0, ph0, 2.5, seed=3002)
    return th, ph, chi, _sample(th.size, np.random.default_rng(19))


@pytest.mark.parametrize("spin", [0, 2])
@pytest.mark.parametrize("prec,eps", [("fp32", 1e-4), ("fp64", 1e-6), ("fp64", 1e-8), ("fp64", 1e-10)])
def test_lmax5120_epsilon_sweep(geometry_5120, spin, prec, eps):
    th, ph, chi, s = geometry_5120
    fwd, adj = _check(5120, th, ph, chi, s, spin, prec, eps, 0.73 * 5120, 1200)
    print("lmax 5120 spin %d %s eps %.0e: fwd %.2e adj %.2e" % (spin, prec, eps, fwd, adj))
    assert fwd <= eps and adj <= eps, (fwd, adj)


@pytest.mark.parametrize("spin", [0, 2])
def test_lmax5120_epsilon_1e12_at_the_fp64_floor(geometry_5120, spin):
    """epsilon 1e-12 at lmax 5120.  FP64 arithmetic itself limits the result here:
    against double-double harmonics the FP64 direct-summation oracle is off by
    1.0e-12 (forward) and 3.7e-12 (adjoint) on near-pole points, and the GPU plan
    reaches the same level (9.0e-13 / 3.9e-12, unchanged at epsilon 1e-13).  So this
    case is checked against the double-double oracle (48 sampled points; the
    double-double sums are 8x dearer), with bounds at that measured floor: forward
    within 1.5e-12, adjoint within 6e-12."""
    th, ph, chi, s = geometry_5120
    n = th.size
    rng = np.random.default_rng(19)
    s48 = np.unique(np.concatenate([rng.integers(0, 40000, 16), rng.integers(n - 40000, n, 16),
                                    rng.integers(n // 2 - 200000, n // 2 + 200000, 16)]))
    fwd, adj = _check(5120, th, ph, chi, s48, spin, "fp64", 1e-12, 0.73 * 5120, 1200, precise=True)
    print("lmax 5120 spin %d fp64 eps 1e-12 (double-double oracle): fwd %.2e adj %.2e" % (spin, fwd, adj))
    assert fwd <= 1.5e-12 and adj <= 6e-12, (fwd, adj)


@pytest.fixture(scope="module")
def geometry_8192():
    """Nside 4096 (201M points), where the lmax 8192 transforms pick two-CTA FFT clusters by size."""
    th0, ph0 = W.healpix_centres(4096)
    th, ph, chi = W.displaced_points(th0, ph0, 2.5, seed=3003)
    n = th.size
    rng = np.random.default_rng(21)
    s = np.unique(np.concatenate([rng.integers(0, 160000, 16), rng.integers(n - 160000, n, 16),
                                  rng.integers(n // 2 - 800000, n // 2 + 800000, 32)]))
    return th, ph, chi, s


@pytest.mark.parametrize("spin", [0, 2])
@pytest.mark.parametrize("prec,eps", [("fp32", 1e-5), ("fp64", 1e-10)])
def test_scan_point_lmax8192_nside4096(geometry_8192, spin, prec, eps):
    """A point of the paper's Fig. 4 scan: lmax 8192 on Nside 4096, 64 sampled outputs near both poles
    and the equator (the FFT vectors there exceed one CTA's shared memory and run on clusters)."""
    th, ph, chi, s = geometry_8192
    nc = 1 if spin == 0 else 2
    cl = W.cmb_cl(8192, 0.73 * 8192)
    a = np.stack([W.draw_alm(cl, 8192, 1300 + k, spin=spin) for k in range(nc)])
    plan = LensPlan(8192, th, ph, chi if spin else None, spin=spin, epsilon=eps, precision=prec, device=DEV)
    inf = plan.info()
    assert max(inf["n1"], inf["n2"], inf["ntheta_fft"]) * (8 if prec == "fp32" else 16) > 150000  # beyond one CTA
    plan.close()
    torch.cuda.empty_cache()
    fwd, adj = _check(8192, th, ph, chi, s, spin, prec, eps, 0.73 * 8192, 1300)
    assert fwd <= eps and adj <= eps, (fwd, adj)
