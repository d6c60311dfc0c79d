"""Restarted FP32 Legendre recursion (FP32 plans, epsilon >= 1e-5) against the oracle.

The FP32 plans' default recursion keeps an FP32 state and is reset every K
degrees to values computed at plan creation; rings near the poles use
Reinsch's difference form.  These cases run at band limits where several
restarts happen (the degree loop restarts at lf + K k), on rings on both sides
of the Reinsch/plain boundary, and compare with the FP64 oracle and with the
double-float recursion of the same plan geometry.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2304_10431_gb300 import LensError, LensPlan
from paper_2304_10431_gb300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0") if torch.cuda.is_available() else None


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def make_alm(L, spin, seed):
    nc = 1 if spin == 0 else 2
    cl = W.cmb_cl(L, 0.8 * L)
    return np.stack([W.draw_alm(cl, L, seed + k, spin=spin) for k in range(nc)])


def ring_rows(nt):
    """Rings near both poles, around the Reinsch/plain boundary (cos theta ~ 0.7) and the equator."""
    j = set(range(0, 6)) | set(range(nt - 6, nt)) | set(range(nt // 2 - 3, nt // 2 + 4))
    jb = int(round(math.acos(0.7) / math.pi * (nt - 1)))
    j |= set(range(max(jb - 70, 0), jb + 70, 7)) | set(range(0, nt, max(nt // 40, 1)))
    return np.array(sorted(j))


@pytest.mark.parametrize("spin", [0, 2])
@pytest.mark.parametrize("K", [8, 64])
def test_restarted_ring_synthesis_vs_oracle(spin, K):
    L = 700
    th, ph, chi = W.random_points(100, 3)
    plan = LensPlan(L, th, ph, chi, spin=spin, epsilon=1e-5, precision="fp32", legendre_restart=K, device=DEV)
    inf = plan.info()
    assert inf["legendre_restart"] == K and inf["restart_bytes"] > 0
    a = make_alm(L, spin, 5)
    ring = plan.ring_synthesis(torch.as_tensor(a, dtype=plan.complex_dtype, device=DEV)).cpu().numpy()
    nt = inf["ntheta"]
    rows = ring_rows(nt)
    ref = O.ring_coeffs(L, L, spin, rows * math.pi / (nt - 1), a).T
    got = ring[:, rows]
    assert rel(got, ref) < 2e-6
    # per ring: no ring band is far off (near-pole rings included)
    per = np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0).clip(1e-300)
    assert per.max() < 2e-5


@pytest.mark.parametrize("spin", [0, 2])
def test_restarted_ring_adjoint_vs_oracle(spin):
    """Adjoint Legendre step with restarts: the exact transpose of the oracle's ring synthesis."""
    L = 400
    th, ph, chi = W.random_points(10, 3)
    plan = LensPlan(L, th, ph, chi, spin=spin, epsilon=1e-5, precision="fp32", device=DEV)
    assert plan.info()["legendre_restart"] == 64
    nt = plan.info()["ntheta"]
    ncol = (L + 1) if spin == 0 else 2 * L + 1
    rng = np.random.default_rng(4)
    r = np.zeros((ncol, nt), complex)
    rows = ring_rows(nt)
    r[:, rows] = rng.standard_normal((ncol, len(rows))) + 1j * rng.standard_normal((ncol, len(rows)))
    if spin == 0:
        r[0] = r[0].real
    at = plan.ring_adjoint(torch.as_tensor(r, dtype=plan.complex_dtype, device=DEV)).cpu().numpy()
    # oracle transpose through <F(a), r> = <a, F^T r> on a few random a
    em = W.alm_m_of_index(L)
    for seed in (1, 2):
        a = make_alm(L, spin, 40 + seed)
        F = O.ring_coeffs(L, L, spin, rows * math.pi / (nt - 1), a).T
        if spin == 0:
            wr = np.where(np.arange(ncol) == 0, 1.0, 2.0)[:, None]
            lhs = np.sum(wr * (F * np.conj(r[:, rows])).real)
        else:
            lhs = np.sum((F * np.conj(r[:, rows])).real)
        rhs = np.sum(np.where(em == 0, 1.0, 2.0) * (a * np.conj(at)).real)
        assert abs(lhs - rhs) <= 2e-6 * np.linalg.norm(F) * np.linalg.norm(r)


@pytest.mark.parametrize("spin", [0, 2])
def test_restarted_full_transform_vs_oracle(spin):
    L, n = 300, 20000
    th, ph, chi = W.random_points(n, 17 + spin)
    th[:4] = [0.0, math.pi, 0.5 * math.pi, 1e-9]
    plan = LensPlan(L, th, ph, chi, spin=spin, epsilon=1e-5, precision="fp32", device=DEV)
    assert plan.info()["legendre_restart"] == 64
    a = make_alm(L, spin, 11)
    m = plan.synthesis(torch.as_tensor(a, dtype=plan.complex_dtype, device=DEV)).cpu().numpy()
    sel = np.arange(0, n, 25)
    ref = O.synthesis(L, L, spin, th[sel], ph[sel], a, chi[sel])
    assert rel(m[:, sel], ref) <= 1e-5
    y = np.zeros((1 if spin == 0 else 2, n))
    y[:, sel] = np.random.default_rng(L).standard_normal((y.shape[0], len(sel)))
    at = plan.adjoint(torch.as_tensor(y, dtype=plan.real_dtype, device=DEV)).cpu().numpy()
    aref = O.adjoint(L, L, spin, th[sel], ph[sel], y[:, sel], chi[sel])
    assert rel(at, aref) <= 1e-5


@pytest.mark.parametrize("spin", [0, 1, 2])
def test_restart_matches_double_float_recursion(spin):
    """Same geometry, restarted FP32 recursion vs df32 recursion, forward and adjoint (lmax 1024)."""
    L, n = 1024, 200000
    th, ph, chi = W.random_points(n, 5)
    a = make_alm(L, spin, 21)
    y = np.random.default_rng(3).standard_normal((1 if spin == 0 else 2, n))
    out = {}
    for rs in (0, -1):
        plan = LensPlan(L, th, ph, chi, spin=spin, epsilon=1e-5, precision="fp32", legendre_restart=rs, device=DEV)
        assert plan.info()["legendre_restart"] == (64 if rs == 0 else 0)
        m = plan.synthesis(torch.as_tensor(a, dtype=plan.complex_dtype, device=DEV)).cpu().numpy()
        at = plan.adjoint(torch.as_tensor(y, dtype=plan.real_dtype, device=DEV)).cpu().numpy()
        out[rs] = (m, at)
        plan.close()
    assert rel(out[0][0], out[-1][0]) < 3e-6
    assert rel(out[0][1], out[-1][1]) < 3e-6


@pytest.mark.parametrize("spin,grad,det", [(2, True, False), (0, False, True), (2, False, True), (2, True, True)])
def test_restart_variants_vs_oracle(spin, grad, det):
    """Gradient-only and deterministic plans run the same restarted kernels."""
    L, n = 260, 8000
    th, ph, chi = W.random_points(n, 9)
    plan = LensPlan(L, th, ph, chi, spin=spin, epsilon=1e-5, precision="fp32", grad_only=grad, deterministic=det,
                    device=DEV)
    assert plan.info()["legendre_restart"] == 64
    a = make_alm(L, spin, 31)
    if grad:
        a = a.copy()
        a[1] = 0
    ain = a[:1] if grad else a
    m = plan.synthesis(torch.as_tensor(ain, dtype=plan.complex_dtype, device=DEV)).cpu().numpy()
    ref = O.synthesis(L, L, spin, th, ph, a, chi)
    assert rel(m, ref) <= 1e-5
    y = np.random.default_rng(6).standard_normal(ref.shape)
    at = plan.adjoint(torch.as_tensor(y, dtype=plan.real_dtype, device=DEV)).cpu().numpy()
    aref = O.adjoint(L, L, spin, th, ph, y, chi)
    if grad:
        aref = aref[:1]
    assert rel(at, aref) <= 1e-5
    if det:
        at2 = plan.adjoint(torch.as_tensor(y, dtype=plan.real_dtype, device=DEV)).cpu().numpy()
        assert np.array_equal(at, at2)


def test_grouped_synthesis_with_restarts():
    L, n = 500, 30000
    th, ph, chi = W.random_points(n, 12)
    for spin, nm in ((0, 4), (2, 2)):
        plan = LensPlan(L, th, ph, chi, spin=spin, epsilon=1e-5, precision="fp32", device=DEV)
        a = np.stack([make_alm(L, spin, 60 + 3 * b) for b in range(nm)])
        ta = torch.as_tensor(a, dtype=plan.complex_dtype, device=DEV)
        grouped = plan.synthesis(ta).cpu().numpy()
        plan.set_grouping(False)
        single = plan.synthesis(ta).cpu().numpy()
        assert rel(grouped, single) < 1e-6
        plan.close()


def test_restart_selection_and_errors():
    th, ph, chi = W.random_points(50, 1)
    assert LensPlan(300, th, ph, chi, epsilon=1e-5, device=DEV).info()["legendre_restart"] == 64
    assert LensPlan(300, th, ph, chi, epsilon=5e-6, device=DEV).info()["legendre_restart"] == 0
    assert LensPlan(300, th, ph, chi, epsilon=1e-5, legendre_restart=-1, device=DEV).info()["legendre_restart"] == 0
    assert LensPlan(300, th, ph, chi, epsilon=5e-6, legendre_restart=32, device=DEV).info()["legendre_restart"] == 32
    assert LensPlan(300, th, ph, chi, epsilon=1e-5, legendre_tables=True, device=DEV).info()["legendre_restart"] == 0
    # FP64 plans: double-float restarts every 128 degrees for epsilon >= 5e-11, none below or when the
    # FP64 orders are set explicitly
    p64 = LensPlan(300, th, ph, chi, epsilon=1e-8, precision="fp64", device=DEV).info()
    assert p64["legendre_restart"] == 128 and p64["legendre_df32_mmin"] == 0
    assert LensPlan(300, th, ph, chi, epsilon=1e-12, precision="fp64", device=DEV).info()["legendre_restart"] == 0
    assert LensPlan(300, th, ph, chi, epsilon=1e-10, precision="fp64", legendre_restart=-1,
                    device=DEV).info()["legendre_restart"] == 0
    assert LensPlan(300, th, ph, chi, epsilon=1e-10, precision="fp64", legendre_df32_mmin=32,
                    device=DEV).info()["legendre_restart"] == 0
    for bad in (3, 48, 8192, -2):
        with pytest.raises(LensError):
            LensPlan(300, th, ph, chi, epsilon=1e-5, legendre_restart=bad, device=DEV)
    # no restart degree below lmax + 1 - 8 - 64: the table is empty and the kernels run the plain FP32 recursion
    p = LensPlan(60, th, ph, chi, epsilon=1e-5, device=DEV)
    assert p.info()["legendre_restart"] == 64 and p.info()["restart_bytes"] == 0


# ------------------------------------------------ FP64 plans: restarted double-float recursion
@pytest.mark.parametrize("spin", [0, 2])
@pytest.mark.parametrize("K", [0, 16])
def test_fp64_restarted_ring_synthesis_vs_oracle(spin, K):
    """FP64 plans (epsilon >= 5e-11) run every order in double-float, reset to the FP64
    recursion's values every 16 (m < 16), 64 (m < 128) or 128 degrees (K = 0), or every K degrees:
    ring synthesis against the oracle and against the same plan geometry without restarts (FP64 low
    orders, double-float above); the adjoint against the latter."""
    L = 700
    th, ph, chi = W.random_points(100, 3)
    plan = LensPlan(L, th, ph, chi, spin=spin, epsilon=1e-10, precision="fp64", legendre_restart=K, device=DEV)
    inf = plan.info()
    assert inf["legendre_restart"] == (K or 128) and inf["restart_bytes"] > 0 and inf["legendre_df32_mmin"] == 0
    ref_plan = LensPlan(L, th, ph, chi, spin=spin, epsilon=1e-10, precision="fp64", legendre_restart=-1, device=DEV)
    assert ref_plan.info()["legendre_restart"] == 0 and ref_plan.info()["legendre_df32_mmin"] > 0
    a = make_alm(L, spin, 15)
    ta = torch.as_tensor(a, dtype=plan.complex_dtype, device=DEV)
    ring = plan.ring_synthesis(ta).cpu().numpy()
    nt = inf["ntheta"]
    rows = ring_rows(nt)
    ref = O.ring_coeffs(L, L, spin, rows * math.pi / (nt - 1), a).T
    # measured at lmax 700 (spin 0): 2e-12 with the default intervals (K = 128 for every order: 3e-11)
    assert rel(ring[:, rows], ref) < 5e-12
    per = np.linalg.norm(ring[:, rows] - ref, axis=0) / np.linalg.norm(ref, axis=0).clip(1e-300)
    assert per.max() < 1e-10
    assert rel(ring, ref_plan.ring_synthesis(ta).cpu().numpy()) < 5e-12
    rng = np.random.default_rng(4)
    r = rng.standard_normal(ring.shape) + 1j * rng.standard_normal(ring.shape)
    tr = torch.as_tensor(r, dtype=plan.complex_dtype, device=DEV)
    got = plan.ring_adjoint(tr).cpu().numpy()
    want = ref_plan.ring_adjoint(tr).cpu().numpy()
    # two double-float evaluations (the reference plan runs its low orders in FP64): measured 1.4e-12
    assert rel(got, want) < 5e-12
    plan.close()
    ref_plan.close()


@pytest.mark.parametrize("spin,grad", [(0, False), (2, False), (2, True)])
def test_fp64_restarted_transform_vs_oracle(spin, grad):
    """Whole forward and adjoint of a restarted FP64 plan (lmax 1100, restarts at K = 128 past the
    jump) against the oracle's direct sums at sampled points, epsilon 1e-10."""
    L, n = 1100, 30000
    th, ph, chi = W.random_points(n, 70 + spin)
    th[:4] = [0.0, math.pi, 1e-3, math.pi - 1e-3]
    plan = LensPlan(L, th, ph, chi if spin else None, spin=spin, epsilon=1e-10, precision="fp64",
                    grad_only=grad, device=DEV)
    assert plan.info()["legendre_restart"] == 128
    a = make_alm(L, spin, 21)
    if grad:
        a = a[:1]
    m = plan.synthesis(torch.as_tensor(a, dtype=plan.complex_dtype, device=DEV)).cpu().numpy()
    s = np.r_[0:4, 4:n:97]
    af = a if not grad else np.concatenate([a, np.zeros_like(a)])
    orc = O.synthesis(L, L, spin, th[s], ph[s], af, chi[s] if spin else None)
    assert rel(m[:, s], orc) < 1e-10
    # adjoint of a sparse map against the oracle's adjoint of the same map
    nc = 1 if spin == 0 else 2
    y = np.zeros((nc, n))
    y[:, s] = np.random.default_rng(9).standard_normal((nc, len(s)))
    got = plan.adjoint(torch.as_tensor(y, dtype=plan.real_dtype, device=DEV)).cpu().numpy()
    want = O.adjoint(L, L, spin, th[s], ph[s], y[:, s], chi[s] if spin else None)
    if grad:
        want = want[:1]
    assert rel(got, want) < 1e-10
    plan.close()
