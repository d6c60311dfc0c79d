"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances: the relative L2 error over all outputs (Sect. 4's eps_eff, also
applied to a_lm for the adjoint) must not exceed the requested epsilon: 1e-5
for FP32 plans, 1e-10 for FP64 plans.  The adjoint identity holds to 1e-12
(FP64) with the real-field inner product.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2304_10431_gb300 import LensError, LensPlan, pointing
from paper_2304_10431_gb300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0") if torch.cuda.is_available() else None
PRECS = [("fp32", 1e-5), ("fp64", 1e-10)]


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def make_alm(L, spin, seed, ld=None, mmax=None):
    nc = 1 if spin == 0 else 2
    cl = W.cmb_cl(L, ld or max(0.8 * L, 2.0))
    return np.stack([W.draw_alm(cl, L, seed + k, mmax=mmax, spin=spin) for k in range(nc)])


def gpu_alm(plan, a):
    return torch.as_tensor(a, dtype=plan.complex_dtype, device=DEV)


def gpu_map(plan, m):
    return torch.as_tensor(m, dtype=plan.real_dtype, device=DEV)


# ---------------------------------------------------------------- Legendre step
@pytest.mark.parametrize("spin", [0, 1, 2])
@pytest.mark.parametrize("prec,eps", PRECS)
def test_ring_synthesis_vs_oracle(spin, prec, eps):
    L = 70
    th, ph, chi = W.random_points(100, 3)
    plan = LensPlan(L, th, ph, chi, spin=spin, epsilon=eps, precision=prec, device=DEV)
    a = make_alm(L, spin, 5)
    ring = plan.ring_synthesis(gpu_alm(plan, a)).cpu().numpy()
    nt = plan.info()["ntheta"]
    ref = O.ring_coeffs(L, L, spin, np.arange(nt) * math.pi / (nt - 1), a).T
    assert rel(ring, ref) < (1e-13 if prec == "fp64" else 2e-6)


@pytest.mark.parametrize("spin", [0, 2])
@pytest.mark.parametrize("prec,eps", PRECS)
def test_ring_adjoint_is_transpose(spin, prec, eps):
    L = 70
    th, ph, chi = W.random_points(10, 3)
    plan = LensPlan(L, th, ph, chi, spin=spin, epsilon=eps, precision=prec, device=DEV)
    a = make_alm(L, spin, 8)
    F = plan.ring_synthesis(gpu_alm(plan, a)).cpu().numpy()
    rng = np.random.default_rng(1)
    r = rng.standard_normal(F.shape) + 1j * rng.standard_normal(F.shape)
    if spin == 0:
        r[0] = r[0].real
    at = plan.ring_adjoint(torch.as_tensor(r, dtype=plan.complex_dtype, device=DEV)).cpu().numpy()
    em = W.alm_m_of_index(L)
    if spin == 0:  # stored columns are m >= 0 of a Hermitian set: weight 2 for m > 0 on both sides
        wr = np.where(np.arange(F.shape[0]) == 0, 1.0, 2.0)[:, None]
        lhs = np.sum(wr * (F * np.conj(r)).real)
    else:
        lhs = np.sum((F * np.conj(r)).real)
    rhs = np.sum(np.where(em == 0, 1.0, 2.0) * (a * np.conj(at)).real)
    assert abs(lhs - rhs) <= (1e-12 if prec == "fp64" else 1e-5) * np.linalg.norm(F) * np.linalg.norm(r)


# ---------------------------------------------------------------- full operator
CASES = [  # (lmax, npoints, spin)
    (1, 37, 0), (2, 64, 2), (17, 999, 0), (17, 999, 1), (33, 3001, 2), (70, 4099, 0), (70, 4099, 2), (70, 2500, 3),
]


@pytest.mark.parametrize("L,n,spin", CASES)
@pytest.mark.parametrize("prec,eps", PRECS)
def test_forward_and_adjoint_vs_oracle(L, n, spin, prec, eps):
    th, ph, chi = W.random_points(n, 100 + L + spin)
    th[:4] = [0.0, math.pi, 0.5 * math.pi, 1e-9]
    ph[:4] = [7.0, -1.0, 2 * math.pi, 0.0]
    plan = LensPlan(L, th, ph, chi, spin=spin, epsilon=eps, precision=prec, device=DEV)
    a = make_alm(L, spin, 11)
    m = plan.synthesis(gpu_alm(plan, a)).cpu().numpy()
    ref = O.synthesis(L, L, spin, th, ph, a, chi)
    assert rel(m, ref) <= eps
    y = np.random.default_rng(L).standard_normal(ref.shape)
    at = plan.adjoint(gpu_map(plan, y)).cpu().numpy()
    aref = O.adjoint(L, L, spin, th, ph, y, chi)
    assert rel(at, aref) <= eps
    if spin == 0:
        assert np.all(at[0, W.alm_m_of_index(L) == 0].imag == 0)


@pytest.mark.parametrize("spin", [0, 2])
def test_adjoint_identity_fp64(spin):
    L, n = 96, 20000
    th, ph, chi = W.random_points(n, 4)
    plan = LensPlan(L, th, ph, chi, spin=spin, epsilon=1e-12, precision="fp64", device=DEV)
    rng = np.random.default_rng(2)
    nc = 1 if spin == 0 else 2
    x = rng.standard_normal((nc, plan.nalm)) + 1j * rng.standard_normal((nc, plan.nalm))
    em, ell = W.alm_m_of_index(L), W.alm_l_of_index(L)
    x[:, em == 0] = x[:, em == 0].real
    x[:, ell < spin] = 0
    y = rng.standard_normal((nc, n))
    ax = plan.synthesis(gpu_alm(plan, x)).cpu().numpy()
    aty = plan.adjoint(gpu_map(plan, y)).cpu().numpy()
    lhs = np.sum(ax * y)
    rhs = np.sum(np.where(em == 0, 1.0, 2.0) * (x * np.conj(aty)).real)
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(ax) * np.linalg.norm(y)


@pytest.mark.parametrize("prec,eps", PRECS)
def test_config1_lensed_healpix(prec, eps):
    """Spin-0 lensing, lmax 128, HEALPix Nside 64 (49,152 points) deflected by the
    gradient of phi (phi lmax 128, 2.5 arcmin rms), both directions."""
    L, nside = 128, 64
    th0, ph0 = W.healpix_centres(nside)
    phi_lm = W.draw_alm(W.phi_cl(L), L, 2000)
    th, ph, chi = O.deflected_points(th0, ph0, phi_lm, L)
    a = W.draw_alm(W.cmb_cl(L, 100.0), L, 1000)[None]
    plan = LensPlan(L, th, ph, chi, spin=0, epsilon=eps, precision=prec, device=DEV)
    m = plan.synthesis(gpu_alm(plan, a)).cpu().numpy()
    ref = O.synthesis(L, L, 0, th, ph, a)
    assert rel(m, ref) <= eps
    at = plan.adjoint(gpu_map(plan, ref)).cpu().numpy()
    aref = O.adjoint(L, L, 0, th, ph, ref)
    assert rel(at, aref) <= eps


def test_spin2_lensed_healpix_with_phase():
    """Spin-2 Q/U at deflected HEALPix points (Nside 32) with the lensing phase chi."""
    L, nside = 80, 32
    th0, ph0 = W.healpix_centres(nside)
    th, ph, chi = O.deflected_points(th0, ph0, W.draw_alm(W.phi_cl(L), L, 2001), L)
    a = make_alm(L, 2, 1001)
    for prec, eps in PRECS:
        plan = LensPlan(L, th, ph, chi, spin=2, epsilon=eps, precision=prec, device=DEV)
        m = plan.synthesis(gpu_alm(plan, a)).cpu().numpy()
        ref = O.synthesis(L, L, 2, th, ph, a, chi)
        assert rel(m, ref) <= eps


@pytest.mark.parametrize("spin", [0, 1, 2])
@pytest.mark.parametrize("mmin", [1, 57])
def test_fp64_plan_df32_orders(spin, mmin):
    """FP64 plans run orders m >= legendre_df32_mmin in double-float: same accuracy bar."""
    L, n = 160, 4000
    th, ph, chi = W.random_points(n, 31 + spin)
    plan = LensPlan(L, th, ph, chi, spin=spin, epsilon=1e-10, precision="fp64", legendre_df32_mmin=mmin,
                    device=DEV)
    a = make_alm(L, spin, 17)
    ring = plan.ring_synthesis(gpu_alm(plan, a)).cpu().numpy()
    nt = plan.info()["ntheta"]
    rref = O.ring_coeffs(L, L, spin, np.arange(nt) * math.pi / (nt - 1), a).T
    assert rel(ring, rref) < 1e-11  # double-float recursion: ~2^-45 per step, amplified at low m
    m = plan.synthesis(gpu_alm(plan, a)).cpu().numpy()
    ref = O.synthesis(L, L, spin, th, ph, a, chi)
    assert rel(m, ref) <= 1e-10
    y = np.random.default_rng(spin).standard_normal(ref.shape)
    at = plan.adjoint(gpu_map(plan, y)).cpu().numpy()
    assert rel(at, O.adjoint(L, L, spin, th, ph, y, chi)) <= 1e-10


@pytest.mark.parametrize("spin", [0, 2])
def test_fp64_without_point_weights(spin):
    """FP64 plans evaluate the kernel taps in every call when the per-point weight table is not kept
    (above 48 GB, or point_weights = -1): same results as with the table, and the oracle's."""
    L, n = 160, 6000
    th, ph, chi = W.random_points(n, 51 + spin)
    kw = dict(spin=spin, epsilon=1e-10, precision="fp64", device=DEV)
    p0 = LensPlan(L, th, ph, chi, point_weights=-1, **kw)
    p1 = LensPlan(L, th, ph, chi, point_weights=1, **kw)
    assert p0.info()["point_weight_bytes"] == 0 and p1.info()["point_weight_bytes"] == 16 * p1.info()["W"] * n
    a = make_alm(L, spin, 23)
    m0 = p0.synthesis(gpu_alm(p0, a)).cpu().numpy()
    m1 = p1.synthesis(gpu_alm(p1, a)).cpu().numpy()
    ref = O.synthesis(L, L, spin, th, ph, a, chi)
    assert rel(m0, ref) <= 1e-10 and rel(m0, m1) <= 1e-12
    y = np.random.default_rng(spin + 5).standard_normal(ref.shape)
    a0 = p0.adjoint(gpu_map(p0, y)).cpu().numpy()
    a1 = p1.adjoint(gpu_map(p1, y)).cpu().numpy()
    assert rel(a0, O.adjoint(L, L, spin, th, ph, y, chi)) <= 1e-10 and rel(a0, a1) <= 1e-12
    with pytest.raises(LensError):
        LensPlan(L, th, ph, chi, point_weights=2, **kw)


# ---------------------------------------------------------------- edge cases
def test_mmax_below_lmax():
    L, mmax, n = 40, 17, 1500
    th, ph, chi = W.random_points(n, 21)
    for spin in (0, 2):
        a = make_alm(L, spin, 3, mmax=mmax)
        plan = LensPlan(L, th, ph, chi, spin=spin, mmax=mmax, epsilon=1e-10, precision="fp64", device=DEV)
        m = plan.synthesis(gpu_alm(plan, a)).cpu().numpy()
        assert rel(m, O.synthesis(L, mmax, spin, th, ph, a, chi)) <= 1e-10
        y = np.random.default_rng(0).standard_normal(m.shape)
        at = plan.adjoint(gpu_map(plan, y)).cpu().numpy()
        assert rel(at, O.adjoint(L, mmax, spin, th, ph, y, chi)) <= 1e-10


def test_lmax_zero_and_empty_points():
    th, ph, _ = W.random_points(50, 1)
    plan = LensPlan(0, th, ph, spin=0, epsilon=1e-10, precision="fp64", device=DEV)
    a = torch.tensor([[2.0 + 5.0j]], dtype=torch.complex128, device=DEV)
    m = plan.synthesis(a).cpu().numpy()
    assert np.allclose(m, 2.0 / math.sqrt(4 * math.pi), atol=1e-14, rtol=0)
    e = LensPlan(8, np.zeros(0), np.zeros(0), spin=2, epsilon=1e-5, device=DEV)
    out = e.synthesis(torch.zeros(2, e.nalm, dtype=torch.complex64, device=DEV))
    assert out.shape == (2, 0)
    at = e.adjoint(torch.zeros(2, 0, dtype=torch.float32, device=DEV)).cpu().numpy()
    assert np.all(at == 0)


def test_domain_errors():
    with pytest.raises(LensError) as ex:
        LensPlan(8, np.array([0.1, 3.5]), np.array([0.0, 0.0]), device=DEV)
    assert ex.value.status == 2
    with pytest.raises(LensError) as ex:
        LensPlan(8, np.array([0.1, np.nan]), np.array([0.0, 0.0]), device=DEV)
    assert ex.value.status == 2
    with pytest.raises(LensError) as ex:
        LensPlan(8, np.array([0.1]), np.array([np.inf]), device=DEV)
    assert ex.value.status == 2
    with pytest.raises(LensError) as ex:
        LensPlan(8, np.array([0.1]), np.array([0.0]), epsilon=1e-7, precision="fp32", device=DEV)
    assert ex.value.status == 3
    with pytest.raises(LensError) as ex:  # FP32 floor: measured eps_eff 1.2e-6 at lmax 4096
        LensPlan(8, np.array([0.1]), np.array([0.0]), epsilon=1.5e-6, precision="fp32", device=DEV)
    assert ex.value.status == 3
    LensPlan(8, np.array([0.1]), np.array([0.0]), epsilon=2e-6, precision="fp32", device=DEV).close()


def test_batch_and_host_entry_points():
    L, n = 40, 2000
    th, ph, chi = W.random_points(n, 5)
    plan = LensPlan(L, th, ph, chi, spin=2, epsilon=1e-10, precision="fp64", device=DEV)
    a = np.stack([make_alm(L, 2, 40 + i) for i in range(3)])
    mb = plan.synthesis(gpu_alm(plan, a)).cpu().numpy()
    for i in range(3):
        mi = plan.synthesis(gpu_alm(plan, a[i])).cpu().numpy()
        assert np.array_equal(mb[i], mi)
    mh = plan.synthesis_host(torch.as_tensor(a)).numpy()
    assert np.array_equal(mh, mb)
    ab = plan.adjoint(gpu_map(plan, mb)).cpu().numpy()
    ah = plan.adjoint_host(torch.as_tensor(mb)).numpy()
    # spreading accumulates with atomics: equal up to the order of FP64 additions
    assert rel(ah, ab) < 1e-14


def test_repeated_calls_identical_forward():
    L, n = 64, 5000
    th, ph, chi = W.random_points(n, 6)
    plan = LensPlan(L, th, ph, chi, spin=0, epsilon=1e-5, precision="fp32", device=DEV)
    a = gpu_alm(plan, make_alm(L, 0, 9))
    m1 = plan.synthesis(a).cpu().numpy()
    m2 = plan.synthesis(a).cpu().numpy()
    assert np.array_equal(m1, m2)  # the forward path has no atomics


# ---------------------------------------------------------------- pointing / deflection
def test_pointing_vs_oracle():
    rng = np.random.default_rng(3)
    th0, ph0 = W.healpix_centres(16)
    at = rng.normal(size=th0.size) * 1e-3
    ap = rng.normal(size=th0.size) * 1e-3
    at[:5] = 0.0
    ap[:5] = 0.0
    t = [torch.as_tensor(x, device=DEV) for x in (th0, ph0, at, ap)]
    t2, p2, c2 = (x.cpu().numpy() for x in pointing(*t))
    r2 = O.pointing(th0, ph0, at, ap)
    assert np.max(np.abs(t2 - r2[0])) < 1e-13
    assert np.max(np.abs(np.angle(np.exp(1j * (p2 - r2[1]))))) < 1e-12
    assert np.max(np.abs(c2 - r2[2])) < 1e-12


def test_deflection_field_on_gpu():
    """Eq. "deflect": spin-1 synthesis of sqrt(L(L+1)) phi_LM at undeflected points."""
    L, nside = 64, 32
    th0, ph0 = W.healpix_centres(nside)
    phi_lm = W.draw_alm(W.phi_cl(L), L, 7)
    ell = W.alm_l_of_index(L)
    g = np.stack([phi_lm * np.sqrt(ell * (ell + 1.0)), 0 * phi_lm])
    plan = LensPlan(L, th0, ph0, spin=1, epsilon=1e-10, precision="fp64", device=DEV)
    a = plan.synthesis(gpu_alm(plan, g)).cpu().numpy()
    ref = O.synthesis(L, L, 1, th0, ph0, g)
    assert rel(a, ref) <= 1e-10


@pytest.mark.parametrize("cl", [2, 4])
@pytest.mark.parametrize("spin,prec,eps", [(0, "fp32", 1e-5), (2, "fp32", 1e-5), (0, "fp64", 1e-10),
                                           (2, "fp64", 1e-10)])
def test_cluster_fft_matches_single_cta(spin, prec, eps, cl):
    """FFT vectors split over a cluster of two or four CTAs (distributed shared memory),
    forced at a size where one CTA would do, give the single-CTA results and the oracle's."""
    L = 300
    th, ph, chi = W.random_points(40000, 321)
    nc = 1 if spin == 0 else 2
    a = np.stack([W.draw_alm(W.cmb_cl(L, 200.0), L, 900 + k, spin=spin) for k in range(nc)])
    y = np.random.default_rng(4).standard_normal((nc, th.size))
    out = {}
    for c in (1, cl):
        plan = LensPlan(L, th, ph, chi if spin else None, spin=spin, epsilon=eps, precision=prec, fft_cluster=c,
                        device=DEV)
        out[c] = (plan.synthesis(gpu_alm(plan, a)).cpu().numpy(),
                  plan.adjoint(torch.as_tensor(y, dtype=plan.real_dtype, device=DEV)).cpu().numpy())
        plan.close()
    tol = 1e-6 if prec == "fp32" else 1e-13
    assert rel(out[cl][0], out[1][0]) <= tol and rel(out[cl][1], out[1][1]) <= tol
    s = np.arange(0, th.size, 157)
    ref = O.synthesis(L, L, spin, th[s], ph[s], a, chi[s] if spin else None)
    assert rel(out[cl][0][:, s], ref) <= eps


@pytest.mark.parametrize("tables", [False, True])
@pytest.mark.parametrize("spin", [0, 1, 2])
def test_grouped_synthesis_matches_per_map(spin, tables):
    """FP32 plans synthesise several maps per call with one Legendre recursion
    shared by four (then two) maps; every map equals its own call (the same
    arithmetic per map: bit-identical where the rings-per-thread setting is the
    same, else up to which negligible degrees a warp skips) and the oracle."""
    L, n = 200, 30000
    th, ph, chi = W.random_points(n, 77 + spin)
    plan = LensPlan(L, th, ph, chi if spin else None, spin=spin, epsilon=1e-5, precision="fp32",
                    legendre_tables=tables, device=DEV)
    a = np.stack([make_alm(L, spin, 500 + 3 * i) for i in range(7)])
    single = np.stack([plan.synthesis(gpu_alm(plan, a[i])).cpu().numpy() for i in range(7)])
    for nm in (2, 3, 4, 5, 7):
        got = plan.synthesis(gpu_alm(plan, a[:nm])).cpu().numpy()
        for i in range(nm):
            assert rel(got[i], single[i]) <= 1e-6, (nm, i)
    vjp_g = plan.adjoint_vjp(gpu_alm(plan, a[:4])).cpu().numpy()
    plan.set_grouping(False)
    vjp_1 = plan.adjoint_vjp(gpu_alm(plan, a[:4])).cpu().numpy()
    assert rel(vjp_g, vjp_1) <= 1e-6
    assert np.array_equal(plan.synthesis(gpu_alm(plan, a[:3])).cpu().numpy(), single[:3])
    s = np.arange(0, n, 293)
    plan.set_grouping(True)
    got = plan.synthesis(gpu_alm(plan, a[:4])).cpu().numpy()
    for i in (0, 3):
        ref = O.synthesis(L, L, spin, th[s], ph[s], a[i], chi[s] if spin else None)
        assert rel(got[i][:, s], ref) <= 1e-5
    plan.close()


@pytest.mark.parametrize("spin", [1, 2, 3])
@pytest.mark.parametrize("prec,eps", PRECS)
def test_grad_only_matches_full_and_oracle(spin, prec, eps):
    """LENS_GRAD_ONLY (Sect. 4, vanishing curl): synthesis of G alone equals the
    full transform with C = 0, and the adjoint returns the full adjoint's G;
    both against the oracle.  Odd spins exercise the (-1)^s terms."""
    L, n = 100, 20000
    th, ph, chi = W.random_points(n, 90 + spin)
    full = LensPlan(L, th, ph, chi, spin=spin, epsilon=eps, precision=prec, device=DEV)
    grad = LensPlan(L, th, ph, chi, spin=spin, epsilon=eps, precision=prec, grad_only=True, device=DEV)
    assert grad.alm_ncomp == 1 and grad.info()["alm_ncomp"] == 1 and grad.info()["flags"] == 1
    a = make_alm(L, spin, 600)
    a[1] = 0.0
    mf = full.synthesis(gpu_alm(full, a)).cpu().numpy()
    mg = grad.synthesis(gpu_alm(grad, a[:1])).cpu().numpy()
    tol = 1e-6 if prec == "fp32" else 1e-13
    assert rel(mg, mf) <= tol
    s = np.arange(0, n, 97)
    assert rel(mg[:, s], O.synthesis(L, L, spin, th[s], ph[s], a, chi[s])) <= eps
    y = np.random.default_rng(spin).standard_normal((2, n))
    af = full.adjoint(gpu_map(full, y)).cpu().numpy()
    ag = grad.adjoint(gpu_map(grad, y)).cpu().numpy()
    assert ag.shape == (1, full.nalm) and rel(ag[0], af[0]) <= tol
    k = np.arange(0, n, 41)
    assert rel(grad.adjoint(gpu_map(grad, np.where(np.isin(np.arange(n), k), y, 0.0))).cpu().numpy()[0],
               O.adjoint(L, L, spin, th[k], ph[k], y[:, k], chi[k])[0]) <= eps
    full.close()
    grad.close()


def test_grad_only_needs_spin():
    th, ph, _ = W.random_points(10, 1)
    with pytest.raises(LensError) as ex:
        LensPlan(8, th, ph, spin=0, grad_only=True, device=DEV)
    assert ex.value.status == 1


@pytest.mark.parametrize("spin,grad", [(0, False), (2, False), (2, True)])
@pytest.mark.parametrize("prec,eps", PRECS)
def test_deterministic_adjoint_is_bit_reproducible(spin, grad, prec, eps):
    """LENS_DETERMINISTIC: the atomics of the spreading and of the adjoint
    Legendre step add 64-bit fixed-point integers, so repeated adjoints are
    bit-identical; they agree with the floating-point adjoint to rounding and
    with the oracle to epsilon.  A NaN in the map makes the whole output NaN."""
    L, n = 200, 200000
    th, ph, chi = W.random_points(n, 300 + spin)
    kw = dict(spin=spin, epsilon=eps, precision=prec, grad_only=grad, device=DEV)
    det = LensPlan(L, th, ph, chi if spin else None, deterministic=True, **kw)
    ref = LensPlan(L, th, ph, chi if spin else None, **kw)
    assert det.info()["flags"] == (2 | (1 if grad else 0))
    nc = 1 if spin == 0 else 2
    y = np.random.default_rng(7).standard_normal((nc, n))
    outs = [det.adjoint(gpu_map(det, y)).cpu().numpy() for _ in range(3)]
    assert all(np.array_equal(outs[0], o) for o in outs[1:])
    a_ref = ref.adjoint(gpu_map(ref, y)).cpu().numpy()
    # FP64 (epsilon >= 5e-11): the atomic path's spreading taps are double-float products (~2^-46
    # relative), the deterministic path's FP64 ones: measured 5e-13
    assert rel(outs[0], a_ref) <= (1e-6 if prec == "fp32" else 2e-12)
    k = np.arange(0, n, 499)
    ys = np.zeros_like(y)
    ys[:, k] = y[:, k]
    got = det.adjoint(gpu_map(det, ys)).cpu().numpy()
    orc = O.adjoint(L, L, spin, th[k], ph[k], y[:, k], chi[k] if spin else None)
    assert rel(got, orc[:1] if grad else orc) <= eps
    a = make_alm(L, spin, 77)[: det.alm_ncomp]
    assert np.array_equal(det.synthesis(gpu_alm(det, a)).cpu().numpy(), ref.synthesis(gpu_alm(ref, a)).cpu().numpy())
    y[0, 123] = np.nan
    assert np.all(np.isnan(det.adjoint(gpu_map(det, y)).cpu().numpy()))
    det.close()
    ref.close()


@pytest.mark.parametrize("spin,grad,det", [(0, False, False), (1, False, False), (2, False, False), (2, True, False),
                                           (2, False, True), (0, False, True)])
def test_legendre_tables_match_recursion(spin, grad, det):
    """FP32 plans with Legendre tables (values of the monic functions computed
    once at plan creation, non-negligible entries only) give the recursion's
    results: the stored values are the recursion's own, so the synthesis agrees
    to ~1e-7 and the adjoint to FP32 reduction order; both meet epsilon against
    the oracle.  lmax 300 has long evanescent stretches near the poles."""
    L, n = 300, 30000
    th, ph, chi = W.random_points(n, 410 + spin)
    kw = dict(spin=spin, epsilon=1e-5, precision="fp32", grad_only=grad, deterministic=det, device=DEV)
    tab = LensPlan(L, th, ph, chi if spin else None, legendre_tables=True, **kw)
    # the tables hold the double-float recursion's values: compare with that recursion
    rec = LensPlan(L, th, ph, chi if spin else None, legendre_restart=-1, **kw)
    inf = tab.info()
    nnp = (inf["ntheta"] + 1) // 2
    dense = ((nnp + 3) // 4 * 4) * tab.nalm * (8 if spin else 4)
    assert 0.3 * dense < inf["legendre_table_bytes"] < dense and rec.info()["legendre_table_bytes"] == 0
    a = make_alm(L, spin, 91)[: tab.alm_ncomp]
    mt = tab.synthesis(gpu_alm(tab, a)).cpu().numpy()
    mr = rec.synthesis(gpu_alm(rec, a)).cpu().numpy()
    assert rel(mt, mr) <= 1e-6
    s = np.arange(0, n, 113)
    full = a if not grad else np.stack([a[0], 0 * a[0]])
    assert rel(mt[:, s], O.synthesis(L, L, spin, th[s], ph[s], full, chi[s] if spin else None)) <= 1e-5
    nc = 1 if spin == 0 else 2
    y = np.random.default_rng(12).standard_normal((nc, n))
    at = tab.adjoint(gpu_map(tab, y)).cpu().numpy()
    ar = rec.adjoint(gpu_map(rec, y)).cpu().numpy()
    assert rel(at, ar) <= 1e-6
    if det:
        assert np.array_equal(at, tab.adjoint(gpu_map(tab, y)).cpu().numpy())
    k = np.arange(0, n, 293)
    ys = np.zeros_like(y)
    ys[:, k] = y[:, k]
    orc = O.adjoint(L, L, spin, th[k], ph[k], y[:, k], chi[k] if spin else None)
    assert rel(tab.adjoint(gpu_map(tab, ys)).cpu().numpy(), orc[:1] if grad else orc) <= 1e-5
    tab.close()
    rec.close()


def test_legendre_tables_edge_cases():
    """Tables at tiny band limits, mmax < lmax, spin = lmax; FP64 plans refuse them."""
    for L, mmax, spin in [(1, 1, 0), (2, 2, 2), (7, 3, 1), (40, 10, 2), (33, 33, 0)]:
        th, ph, chi = W.random_points(500, L)
        tab = LensPlan(L, th, ph, chi if spin else None, spin=spin, mmax=mmax, legendre_tables=True, device=DEV)
        rec = LensPlan(L, th, ph, chi if spin else None, spin=spin, mmax=mmax, device=DEV)
        a = make_alm(L, spin, 5, mmax=mmax)
        assert rel(tab.synthesis(gpu_alm(tab, a)).cpu().numpy(), rec.synthesis(gpu_alm(rec, a)).cpu().numpy()) <= 1e-6
        y = np.random.default_rng(L).standard_normal((1 if spin == 0 else 2, 500))
        assert rel(tab.adjoint(gpu_map(tab, y)).cpu().numpy(), rec.adjoint(gpu_map(rec, y)).cpu().numpy()) <= 1e-6
        tab.close()
        rec.close()
    th, ph, _ = W.random_points(10, 1)
    with pytest.raises(LensError) as ex:
        LensPlan(16, th, ph, precision="fp64", epsilon=1e-10, legendre_tables=True, device=DEV)
    assert ex.value.status == 1


def test_legendre_tables_status_clean():
    """The table kernels' bounded waits never give up on a healthy device."""
    th, ph, chi = W.random_points(5000, 3)
    plan = LensPlan(500, th, ph, chi, spin=2, legendre_tables=True, device=DEV)
    a = make_alm(500, 2, 1)
    for _ in range(3):
        m = plan.synthesis(gpu_alm(plan, a))
        plan.adjoint(m)
    plan.status()
    plan.close()


def test_async_host_entry_points_on_two_streams():
    """lens_*_host_async: enqueued on a stream, results equal to the synchronous host
    calls once the stream is synchronised; two plans on two streams overlap."""
    L, n = 64, 20000
    th, ph, chi = W.random_points(n, 8)
    p0 = LensPlan(L, th, ph, spin=0, epsilon=1e-5, precision="fp32", device=DEV)
    p2 = LensPlan(L, th, ph, chi, spin=2, epsilon=1e-5, precision="fp32", device=DEV)
    a0 = torch.as_tensor(make_alm(L, 0, 3), dtype=torch.complex64).pin_memory()
    a2 = torch.as_tensor(make_alm(L, 2, 4), dtype=torch.complex64).pin_memory()
    y2 = torch.as_tensor(np.random.default_rng(1).standard_normal((2, n)), dtype=torch.float32).pin_memory()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    m0 = p0.synthesis_host(a0, stream=s1, sync=False)
    b2 = p2.adjoint_host(y2, stream=s2, sync=False)
    m2 = p2.synthesis_host(a2, stream=s2, sync=False)
    s1.synchronize()
    s2.synchronize()
    assert np.array_equal(m0.numpy(), p0.synthesis_host(a0).numpy())
    assert np.array_equal(m2.numpy(), p2.synthesis_host(a2).numpy())
    assert rel(b2.numpy(), p2.adjoint_host(y2).numpy()) <= 1e-6
    p0.close()
    p2.close()


def test_bounded_wait_reports_timeout():
    """The bulk-copy waits of the table kernels are bounded: a wait on an
    mbarrier that no copy completes gives up (~10 ms limit here) and sets the
    status bit instead of hanging; the device stays usable afterwards."""
    import time
    from paper_2304_10431_gb300 import _native
    t0 = time.perf_counter()
    assert _native.load().lens_selftest_bounded_wait(None) == 0
    assert time.perf_counter() - t0 < 10.0
    th, ph, _ = W.random_points(100, 2)
    plan = LensPlan(16, th, ph, legendre_tables=True, device=DEV)
    plan.synthesis(gpu_alm(plan, make_alm(16, 0, 1)))
    plan.status()
    plan.close()


@pytest.mark.parametrize("spin", [0, 2])
def test_doubling_and_theta_transform_are_exact(spin):
    """Sect. 3: only the NUFFT is approximate.  The torus coefficients c_k of the
    doubled ring functions (FP64 plan) reproduce the ring functions at arbitrary
    theta in [0, pi] -- off the equiangular rings -- to rounding, against the
    oracle's direct sums sum_l a_lm lambda_lm(theta)."""
    L = 60
    th, ph, chi = W.random_points(10, 4)
    plan = LensPlan(L, th, ph, chi, spin=spin, epsilon=1e-12, precision="fp64", device=DEV)
    a = make_alm(L, spin, 31)
    c = plan.torus_coefficients(gpu_alm(plan, a)).cpu().numpy()
    t = np.random.default_rng(9).uniform(0.0, math.pi, 41)
    k = np.arange(-L, L + 1)
    F = c @ np.exp(1j * np.outer(k, t))  # [ncol, ntheta']
    ref = O.ring_coeffs(L, L, spin, t, a).T
    assert rel(F, ref) <= 1e-13
    plan.close()
