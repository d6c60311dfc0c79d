"""Pins of the FP64 oracle to facts outside itself.

Each test checks the oracle against something it does not share code with:
textbook closed forms, scipy's spherical harmonics, symbolic derivation from
the spin-raising operator (sympy), Wigner's explicit sum in 30-digit mpmath,
Gauss-Legendre quadrature exactness, finite differences, the adjoint identity
and the geometry of great circles.  A dropped term, a wrong sign, a wrong
index or a transposed operand in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2304_10431_gb300 import workloads as W

FOURPI = 4.0 * math.pi


def _lam(l, m, s, t):
    return O.slambda(l, m, s, t)[l]


# ----------------------------------------------------------- closed forms
def test_spin0_closed_forms():
    """Textbook low-l harmonics with the Condon-Shortley phase (Y_lm(theta, 0))."""
    for t in [1e-3, 0.3, 1.1, 2.0, math.pi - 1e-2]:
        c, s = math.cos(t), math.sin(t)
        ref = {
            (0, 0): 1 / math.sqrt(FOURPI),
            (1, 0): math.sqrt(3 / FOURPI) * c,
            (1, 1): -math.sqrt(3 / (8 * math.pi)) * s,
            (2, 0): math.sqrt(5 / (16 * math.pi)) * (3 * c * c - 1),
            (2, 1): -math.sqrt(15 / (8 * math.pi)) * s * c,
            (2, 2): math.sqrt(15 / (32 * math.pi)) * s * s,
            (3, 3): -math.sqrt(35 / (64 * math.pi)) * s ** 3,
        }
        for (l, m), v in ref.items():
            assert abs(_lam(l, m, 0, t) - v) < 1e-15


def test_spin2_closed_forms():
    """Textbook spin-2 harmonics at l = 2 (Goldberg convention)."""
    for t in [0.2, 0.9, 1.7, 2.8]:
        c = math.cos(t)
        ref = {
            (2, 2, 2): math.sqrt(5 / (64 * math.pi)) * (1 - c) ** 2,
            (2, 2, -2): math.sqrt(5 / (64 * math.pi)) * (1 + c) ** 2,
            (2, 2, 0): math.sqrt(15 / (32 * math.pi)) * (1 - c * c),
            (-2, 2, 2): math.sqrt(5 / (64 * math.pi)) * (1 + c) ** 2,
        }
        for (s, l, m), v in ref.items():
            assert abs(_lam(l, m, s, t) - v) < 1e-15, (s, l, m)


def test_scipy_spin0():
    """Spin 0 against scipy.special.sph_harm_y (independent library routine) up to l = 300."""
    from scipy.special import sph_harm_y
    rng = np.random.default_rng(7)
    L = 300
    for t in list(rng.uniform(0, math.pi, 6)) + [1e-4, math.pi - 1e-4]:
        for m in [0, 1, 7, 64, 150, 299]:
            v = O.slambda(L, m, 0, t)
            ell = np.arange(m, L + 1)
            ref = sph_harm_y(ell, m, t, 0.0).real
            assert np.max(np.abs(v[m:] - ref)) < 1e-12
            assert np.all(v[:m] == 0.0)


def test_sympy_eth_definition():
    """Spin +-1, +-2 from the spin-raising / lowering operators, derived symbolically."""
    sp = pytest.importorskip("sympy")
    th, ph = sp.symbols("theta phi", real=True)

    def eth(e, s):
        return -(sp.sin(th)) ** s * (sp.diff(sp.sin(th) ** (-s) * e, th)
                                     + sp.I / sp.sin(th) * sp.diff(sp.sin(th) ** (-s) * e, ph))

    def ethbar(e, s):
        return -(sp.sin(th)) ** (-s) * (sp.diff(sp.sin(th) ** s * e, th)
                                        - sp.I / sp.sin(th) * sp.diff(sp.sin(th) ** s * e, ph))

    def sY(s, l, m):
        e = sp.Ynm(l, m, th, ph).expand(func=True)
        if s >= 0:
            for k in range(s):
                e = eth(e, k)
            return sp.sqrt(sp.factorial(l - s) / sp.factorial(l + s)) * e
        for k in range(-s):
            e = ethbar(e, -k)
        return (-1) ** (-s) * sp.sqrt(sp.factorial(l + s) / sp.factorial(l - s)) * e

    t0 = 0.77
    for s in [1, 2, -1, -2]:
        for l in range(abs(s), 4):
            for m in range(-l, l + 1):
                ref = complex(sY(s, l, m).subs({th: t0, ph: 0}).evalf(25))
                assert abs(ref.imag) < 1e-14
                assert abs(_lam(l, m, s, t0) - ref.real) < 1e-14, (s, l, m)


def _wigner_d(j, m1, m2, beta, mp):
    tot = mp.mpf(0)
    for k in range(0, 2 * j + 1):
        a1, a2, a3, a4 = j + m2 - k, k, m1 - m2 + k, j - m1 - k
        if min(a1, a2, a3, a4) < 0:
            continue
        tot += ((-1) ** (m1 - m2 + k) * mp.cos(beta / 2) ** (2 * j + m2 - m1 - 2 * k)
                * mp.sin(beta / 2) ** (m1 - m2 + 2 * k)
                / (mp.factorial(a1) * mp.factorial(a2) * mp.factorial(a3) * mp.factorial(a4)))
    return mp.sqrt(mp.factorial(j + m1) * mp.factorial(j - m1) * mp.factorial(j + m2)
                   * mp.factorial(j - m2)) * tot


def _slam_mp(s, l, m, t, mp):
    return (-1) ** s * mp.sqrt((2 * l + 1) / (4 * mp.pi)) * _wigner_d(l, m, -s, mp.mpf(t), mp)


def test_wigner_explicit_sum():
    """Recursion vs Wigner's explicit sum at 30 digits (s = -2..2, l <= 20)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    L = 20
    for t in [0.05, 0.9, 2.2, 3.1]:
        for s in [-2, -1, 0, 1, 2]:
            for m in [-20, -7, -2, -1, 0, 1, 2, 5, 13, 20]:
                v = O.slambda(L, m, s, t)
                for l in range(L + 1):
                    ref = float(_slam_mp(s, l, m, t, mp)) if l >= max(abs(m), abs(s)) else 0.0
                    assert abs(v[l] - ref) < 5e-14 * max(1.0, abs(ref)), (s, l, m, t)


def test_pole_values():
    """d^l_{m,m'}(0) = delta_{m,m'} and d^l_{m,m'}(pi) = (-1)^{l-m'} delta_{m,-m'}."""
    L = 50
    for s in [0, 1, 2, -2]:
        for m in range(0, 6):
            v0 = O.slambda(L, m, s, 0.0)
            vp = O.slambda(L, m, s, math.pi)
            for l in range(max(m, abs(s)), L + 1):
                nrm = math.sqrt((2 * l + 1) / FOURPI)
                want0 = (-1) ** m * nrm if m == -s else 0.0
                wantp = (-1) ** l * nrm if m == s else 0.0
                assert abs(v0[l] - want0) < 1e-13
                assert abs(vp[l] - wantp) < 1e-13


def test_high_l_underflow_region():
    """Large m: exact zeros where sin^m underflows; O(1) values past the turning point.

    Reference: mpmath's arbitrary-precision associated Legendre function,
    normalised as sqrt((2l+1)/4pi (l-m)!/(l+m)!) P_l^m(cos theta).
    """
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 60
    v = O.slambda(2000, 1500, 0, 0.01)
    assert np.all(np.isfinite(v)) and np.all(v == 0.0)  # sin^1500(0.01) ~ 1e-3000

    def ref(l, m, t):
        nrm = mp.sqrt((2 * l + 1) / (4 * mp.pi) * mp.factorial(l - m) / mp.factorial(l + m))
        return float(nrm * mp.legenp(l, m, mp.cos(t)))

    v = O.slambda(2000, 300, 0, 0.3)
    for l in [1200, 1600, 2000]:
        assert abs(v[l] - ref(l, 300, 0.3)) < 1e-11
    # start value ~1e-316 (below the double range); the l = 4096 value is O(1)
    v = O.slambda(4096, 3000, 0, 0.9)
    for l in [3900, 4096]:
        r = ref(l, 3000, 0.9)
        assert abs(r) > 1e-3
        assert abs(v[l] - r) < 1e-11


def test_double_double_harmonics_against_mpmath():
    """The double-double mode (used where FP64's own rounding, ~1e-12 at l ~ 5000,
    would reach the target) against mpmath at l up to 4096: correct to ~1e-16 where
    the FP64 recursion is off by up to ~1e-12; spin-2 values against the FP64 mode."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50

    def ref(l, m, t):
        nrm = mp.sqrt((2 * l + 1) / (4 * mp.pi) * mp.factorial(l - m) / mp.factorial(l + m))
        return float(nrm * mp.legenp(l, m, mp.cos(t)))

    worst64, worstdd = 0.0, 0.0
    for m, t in [(0, 0.3), (30, 1.0), (500, 2.0), (1200, 0.9)]:
        vd = O.slambda(4096, m, 0, t, precise=True)
        v6 = O.slambda(4096, m, 0, t)
        for l in [4096, 4095, 4089]:
            r = ref(l, m, t)
            worstdd = max(worstdd, abs(vd[l] - r) / abs(r))
            worst64 = max(worst64, abs(v6[l] - r) / abs(r))
    assert worstdd <= 1e-15 and worst64 > 10 * worstdd, (worstdd, worst64)
    for s in (2, -2):
        vd = O.slambda(300, 7, s, 1.3, precise=True)
        v6 = O.slambda(300, 7, s, 1.3)
        assert np.max(np.abs(vd - v6)) <= 1e-13 * np.max(np.abs(v6))


@pytest.mark.parametrize("spin", [0, 2])
def test_double_double_transforms_match_fp64_mode(spin):
    """Same conventions in both modes: synthesis and adjoint agree to FP64 rounding
    at a small band limit (the e^{im phi} recurrence and the start values included)."""
    L = 40
    th, ph, chi = W.random_points(60, 12)
    nc = 1 if spin == 0 else 2
    a = np.stack([W.draw_alm(W.cmb_cl(L, 30.0), L, 50 + k, spin=spin) for k in range(nc)])
    c = chi if spin else None
    m6 = O.synthesis(L, L, spin, th, ph, a, c)
    md = O.synthesis(L, L, spin, th, ph, a, c, precise=True)
    assert np.linalg.norm(md - m6) <= 1e-14 * np.linalg.norm(m6)
    y = np.random.default_rng(3).standard_normal((nc, th.size))
    a6 = O.adjoint(L, L, spin, th, ph, y, c)
    ad = O.adjoint(L, L, spin, th, ph, y, c, precise=True)
    assert np.linalg.norm(ad - a6) <= 1e-14 * np.linalg.norm(a6)


# ----------------------------------------------------------- quadrature
@pytest.mark.parametrize("s", [0, 1, 2, -2])
def test_gauss_legendre_orthonormality(s):
    """2 pi sum_j w_j s lambda_lm s lambda_l'm = delta_ll' (GL exact for the polynomial degree)."""
    L = 32
    x, w = np.polynomial.legendre.leggauss(L + 1)
    th = np.arccos(x)
    for m in [0, 1, 2, 5, 17, 32]:
        lam = np.stack([O.slambda(L, m, s, t) for t in th])  # [ring, l]
        l0 = max(m, abs(s))
        G = 2 * math.pi * (lam[:, l0:].T * w) @ lam[:, l0:]
        assert np.max(np.abs(G - np.eye(L + 1 - l0))) < 1e-13


@pytest.mark.parametrize("spin", [0, 2])
def test_zero_deflection_is_standard_sht(spin):
    """Synthesis on a GL grid + quadrature-weighted adjoint returns the input a_lm."""
    L = 16
    t, p, wq = W.gauss_legendre_grid(L + 1, 2 * L + 2)
    nc = 1 if spin == 0 else 2
    cl = W.cmb_cl(L, 100.0)
    a = np.stack([W.draw_alm(cl, L, 11 + k, spin=spin) for k in range(nc)])
    m = O.synthesis(L, L, spin, t, p, a)
    b = O.adjoint(L, L, spin, t, p, m * wq[None, :])
    assert np.max(np.abs(b - a)) < 1e-12 * np.max(np.abs(a))


# ----------------------------------------------------------- assembly
def test_bruteforce_forward_mpmath():
    """Full forward (m<0 terms, real-field symmetry, -e^{i s chi}) vs 30-digit brute force."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    L = 6
    t, p, chi = W.random_points(12, 5)
    rng = np.random.default_rng(3)
    for spin in [0, 2]:
        nc = 1 if spin == 0 else 2
        a = rng.standard_normal((nc, W.nalm(L))) + 1j * rng.standard_normal((nc, W.nalm(L)))
        em, ell = W.alm_m_of_index(L), W.alm_l_of_index(L)
        a[:, em == 0] = a[:, em == 0].real
        a[:, ell < spin] = 0
        got = O.synthesis(L, L, spin, t, p, a, chi)
        for i in range(t.size):
            tot = mp.mpc(0)
            for k in range(ell.size):
                l, m = int(ell[k]), int(em[k])
                if l < spin:
                    continue
                for mm in ([m] if m == 0 else [m, -m]):
                    sgn = (-1) ** m if mm < 0 else 1
                    if spin == 0:
                        c = a[0, k] if mm >= 0 else np.conj(a[0, k]) * sgn
                    else:
                        g = a[0, k] if mm >= 0 else np.conj(a[0, k]) * sgn
                        cc = a[1, k] if mm >= 0 else np.conj(a[1, k]) * sgn
                        c = g + 1j * cc
                    y = _slam_mp(spin, l, mm, t[i], mp) * mp.expj(mm * p[i])
                    tot += mp.mpc(c) * y
            if spin == 0:
                assert abs(float(tot.real) - got[0, i]) < 1e-13
                assert abs(float(tot.imag)) < 1e-12
            else:
                z = -mp.expj(spin * chi[i]) * tot
                assert abs(float(z.real) - got[0, i]) < 1e-13
                assert abs(float(z.imag) - got[1, i]) < 1e-13


@pytest.mark.parametrize("spin", [0, 1, 2])
def test_adjoint_dot_product(spin):
    """<A x, y> = <x, A^T y> with the real-field a_lm inner product (m > 0 counted twice)."""
    L, n = 40, 500
    t, p, chi = W.random_points(n, 9)
    rng = np.random.default_rng(spin)
    nc = 1 if spin == 0 else 2
    a = rng.standard_normal((nc, W.nalm(L))) + 1j * rng.standard_normal((nc, W.nalm(L)))
    em, ell = W.alm_m_of_index(L), W.alm_l_of_index(L)
    a[:, em == 0] = a[:, em == 0].real
    a[:, ell < spin] = 0
    y = rng.standard_normal((nc, n))
    lhs = np.sum(O.synthesis(L, L, spin, t, p, a, chi) * y)
    aty = O.adjoint(L, L, spin, t, p, y, chi)
    wgt = np.where(em == 0, 1.0, 2.0)
    rhs = np.sum(wgt * (a * np.conj(aty)).real)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)
    if spin == 0:
        assert np.all(aty[0, em == 0].imag == 0.0)


def test_ring_coeffs_match_synthesis():
    """Summing the ring Fourier coefficients over m reproduces the point synthesis."""
    L = 30
    t, p, chi = W.random_points(40, 4)
    for spin in [0, 2]:
        nc = 1 if spin == 0 else 2
        a = np.stack([W.draw_alm(W.cmb_cl(L, 20.0), L, 30 + k, spin=spin) for k in range(nc)])
        F = O.ring_coeffs(L, L, spin, t, a)
        if spin == 0:
            m = np.arange(L + 1)
            w = np.where(m == 0, 1.0, 2.0)
            T = np.sum(w * (F * np.exp(1j * m * p[:, None])).real, axis=1)
            ref = O.synthesis(L, L, 0, t, p, a)[0]
            assert np.max(np.abs(T - ref)) < 1e-13
        else:
            m = np.arange(-L, L + 1)
            z = np.sum(F * np.exp(1j * m * p[:, None]), axis=1) * np.exp(1j * spin * chi)
            ref = O.synthesis(L, L, spin, t, p, a, chi)
            assert np.max(np.abs(z.real - ref[0])) < 1e-13
            assert np.max(np.abs(z.imag - ref[1])) < 1e-13


# ----------------------------------------------------------- deflection
def test_deflection_is_gradient():
    """Sect. 3 Eq. "deflect": the spin-1 transform of sqrt(L(L+1)) phi_LM equals grad phi."""
    L = 24
    phi_lm = W.draw_alm(W.phi_cl(L), L, 2024)
    ell = W.alm_l_of_index(L)
    t, p, _ = W.random_points(30, 6)
    t = np.clip(t, 0.2, math.pi - 0.2)
    G = phi_lm * np.sqrt(ell * (ell + 1.0))
    a = O.synthesis(L, L, 1, t, p, np.stack([G, 0 * G]))
    h = 1e-3

    def f(tt, pp):
        return O.synthesis(L, L, 0, tt, pp, phi_lm)[0]

    # 4th-order central differences
    dth = (-f(t + 2 * h, p) + 8 * f(t + h, p) - 8 * f(t - h, p) + f(t - 2 * h, p)) / (12 * h)
    dph = (-f(t, p + 2 * h) + 8 * f(t, p + h) - 8 * f(t, p - h) + f(t, p - 2 * h)) / (12 * h)
    scale = np.max(np.abs(a))
    assert np.max(np.abs(a[0] - dth)) < 1e-8 * scale
    assert np.max(np.abs(a[1] - dph / np.sin(t))) < 1e-8 * scale


# ----------------------------------------------------------- pointing
def _basis(t, p):
    n = np.array([np.sin(t) * np.cos(p), np.sin(t) * np.sin(p), np.cos(t)])
    et = np.array([np.cos(t) * np.cos(p), np.cos(t) * np.sin(p), -np.sin(t)])
    ep = np.array([-np.sin(p), np.cos(p), 0.0])
    return n, et, ep


def test_pointing_geometry():
    rng = np.random.default_rng(12)
    n = 200
    t = rng.uniform(0.05, math.pi - 0.05, n)
    p = rng.uniform(0, 2 * math.pi, n)
    at = rng.normal(size=n) * 3e-3
    ap = rng.normal(size=n) * 3e-3
    t2, p2, chi = O.pointing(t, p, at, ap)
    for i in range(n):
        nv, et, ep = _basis(t[i], p[i])
        n2, et2, ep2 = _basis(t2[i], p2[i])
        a = math.hypot(at[i], ap[i])
        # the unlensed direction lies at geodesic distance |alpha|
        assert abs(math.acos(np.clip(nv @ n2, -1, 1)) - a) < 1e-12
        # parallel transport of e_theta(n) along the geodesic (rotation about n x d)
        d = (at[i] * et + ap[i] * ep) / a
        k = np.cross(nv, d)
        k /= np.linalg.norm(k)
        v = et * math.cos(a) + np.cross(k, et) * math.sin(a) + k * (k @ et) * (1 - math.cos(a))
        ang = math.atan2(v @ ep2, v @ et2)
        assert abs(chi[i] + ang) < 1e-12
        # first order: chi ~ alpha_phi cot(theta)
        assert abs(chi[i] - ap[i] / math.tan(t[i])) < 50 * a * a / math.sin(t[i]) ** 2
    # reversal: going back from n' along the reversed geodesic undoes chi
    tt = np.empty(n); pp = np.empty(n); cr = np.empty(n)
    for i in range(n):
        nv, et, ep = _basis(t[i], p[i])
        a = math.hypot(at[i], ap[i])
        d = (at[i] * et + ap[i] * ep) / a
        tp = -math.sin(a) * nv + math.cos(a) * d
        n2, et2, ep2 = _basis(t2[i], p2[i])
        r = O.pointing(np.array([t2[i]]), np.array([p2[i]]), np.array([-a * (tp @ et2)]),
                       np.array([-a * (tp @ ep2)]))
        tt[i], pp[i], cr[i] = r[0][0], r[1][0], r[2][0]
    assert np.max(np.abs(tt - t)) < 1e-12
    assert np.max(np.abs(np.angle(np.exp(1j * (pp - p))))) < 1e-10
    assert np.max(np.abs(cr + chi)) < 1e-12


def test_pointing_special_cases():
    t = np.array([0.4, 1.0, 2.5, math.pi / 2])
    p = np.array([0.3, 5.0, 1.0, 2.0])
    # zero deflection
    t2, p2, chi = O.pointing(t, p, np.zeros(4), np.zeros(4))
    assert np.all(t2 == t) and np.allclose(p2, p) and np.all(chi == 0)
    # meridian deflection: phi and chi unchanged
    t2, p2, chi = O.pointing(t, p, np.full(4, 0.01), np.zeros(4))
    assert np.allclose(t2, t + 0.01, atol=1e-14) and np.allclose(p2, p, atol=1e-14)
    assert np.max(np.abs(chi)) < 1e-14
    # along the equator: stays on it, no rotation
    t2, p2, chi = O.pointing(np.array([math.pi / 2]), np.array([1.0]), np.zeros(1), np.array([0.2]))
    assert abs(t2[0] - math.pi / 2) < 1e-14 and abs(p2[0] - 1.2) < 1e-14 and abs(chi[0]) < 1e-14


def _phi_scaled(L, seed, rms):
    """phi_LM with rms deflection `rms` radians (large, so that the exponential-map
    Jacobian and the transport holonomy contribute visibly)."""
    phi = W.draw_alm(W.phi_cl(L), L, seed)
    ell = W.alm_l_of_index(L).astype(float)
    w = np.where(W.alm_m_of_index(L) > 0, 2.0, 1.0)
    return phi * rms / np.sqrt(np.sum(w * ell * (ell + 1) * np.abs(phi) ** 2) / (4 * math.pi))


@pytest.mark.parametrize("spin", [0, 2])
def test_phi_gradient_matches_finite_differences(spin):
    """d/dphi of L = sum g . A(phi) x (Eq. "deflect", pointing, Eq. "forward"/"forwardpol"):
    the oracle's chain rule against Richardson-extrapolated central differences of the
    oracle's own forward model, 0.3 rad rms deflection, complex directions (including
    imaginary parts at m = 0, which must get zero gradient)."""
    L = 12
    th0, ph0, _ = W.random_points(300, 4)
    phi = _phi_scaled(L, 9, 0.3)
    nc = 1 if spin == 0 else 2
    x = np.stack([W.draw_alm(W.cmb_cl(L, 8.0), L, 30 + k, spin=spin) for k in range(nc)])
    g = np.random.default_rng(1).standard_normal((nc, th0.size))
    grad = O.phi_gradient(L, spin, th0, ph0, phi, L, x, g)
    assert np.all(grad[W.alm_m_of_index(L) == 0].imag == 0)

    def loss(p):
        return float(np.sum(g * O.lensed_forward(L, spin, th0, ph0, p, L, x)))

    for k in range(3):
        rng = np.random.default_rng(100 + k)
        d = rng.standard_normal(phi.size) + 1j * rng.standard_normal(phi.size)
        t = 1e-5
        fd1 = (loss(phi + t * d) - loss(phi - t * d)) / (2 * t)
        fd2 = (loss(phi + 0.5 * t * d) - loss(phi - 0.5 * t * d)) / t
        fd = (4 * fd2 - fd1) / 3
        an = float(np.sum(grad.real * d.real + grad.imag * d.imag))
        assert abs(an - fd) <= 1e-8 * abs(fd), (k, an, fd)


def test_eth_coefficients_against_derivatives():
    """eth / ethbar coefficient maps of a spin-2 field: with eth = -(D_theta + i D_phi)
    and ethbar = -(D_theta - i D_phi) (covariant derivatives; D_theta is the plain
    theta derivative along a meridian), the spin-3 and spin-1 syntheses of
    eth_coeffs must give d_theta P = -(eth P + ethbar P) / 2, checked against a
    fourth-order central difference in theta."""
    L = 10
    th = np.array([0.4, 1.1, 1.9, 2.6])
    ph = np.array([0.2, 2.0, 4.0, 5.5])
    x = np.stack([W.draw_alm(W.cmb_cl(L, 6.0), L, 40 + k, spin=2) for k in range(2)])
    up = O.synthesis(L, L, 3, th, ph, O.eth_coeffs(L, 2, x))
    dn = O.synthesis(L, L, 1, th, ph, O.eth_coeffs(L, 2, x, lower=True))
    h = 1e-5

    def P(t):
        q = O.synthesis(L, L, 2, t, ph, x)
        return q[0] + 1j * q[1]

    dth = (8 * (P(th + h) - P(th - h)) - (P(th + 2 * h) - P(th - 2 * h))) / (12 * h)
    got = -0.5 * ((up[0] + 1j * up[1]) + (dn[0] + 1j * dn[1]))
    assert np.max(np.abs(got - dth)) <= 1e-8 * np.max(np.abs(dth))


def test_magnification_is_the_area_ratio_of_the_remapping():
    """App. B's determinant formula against the area ratio of the pointing map
    n -> n' computed by central differences of the oracle's own deflection and
    pointing (0.05 rad rms deflection, so |A| - 1 is a few per cent)."""
    L = 16
    phi = _phi_scaled(L, 21, 0.05)
    th = np.array([0.5, 1.0, 1.6, 2.2, 2.8])
    ph = np.array([0.3, 2.0, 4.0, 5.0, 1.0])
    det = O.magnification(th, ph, phi, L)
    h = 1e-5

    def npv(t, p):
        t2, p2, _ = O.deflected_points(t, p, phi, L)
        return np.stack([np.sin(t2) * np.cos(p2), np.sin(t2) * np.sin(p2), np.cos(t2)], axis=-1)

    dt = (npv(th + h, ph) - npv(th - h, ph)) / (2 * h)
    dp = (npv(th, ph + h) - npv(th, ph - h)) / (2 * h)
    n2 = npv(th, ph)
    area = np.abs(np.sum(np.cross(dt, dp) * n2, axis=-1)) / np.sin(th)
    assert np.max(np.abs(det - 1)) > 1e-3  # the test is not trivial
    assert np.max(np.abs(det - area)) <= 1e-8, (det, area)
