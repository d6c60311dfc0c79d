"""FP64 CPU oracle for the lensing SHT pair of arXiv:2304.10431 (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never touches it.

The arithmetic lives in ``oracle.c`` (plain C, OpenMP over points or over m):
direct summation of spin-weighted spherical harmonics at every point, i.e.
Sect. 2's forward operator (Eq. "forward" for spin 0, Eq. "forwardpol" for
spin s>0) and its adjoint (Eq. "adjoint"; the spin-s pair and G/C split that
follow Eq. "forwardpol"), plus the pointing formula of Sect. 3 with the spin
phase chi = beta - beta' of Fig. 1.  Every function below is a thin ctypes
marshaller; see ``oracle.c`` for the definitions and conventions.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` with gcc (-O2, OpenMP, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        i64, i32, dp = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
        lib.oracle_nalm.restype = i64
        lib.oracle_nalm.argtypes = [i32, i32]
        lib.oracle_slambda.restype = i32
        lib.oracle_slambda.argtypes = [i32, i32, i32, ctypes.c_double, dp]
        lib.oracle_ring_coeffs.restype = i32
        lib.oracle_ring_coeffs.argtypes = [i32, i32, i32, i64, dp, dp, dp]
        lib.oracle_synthesis.restype = i32
        lib.oracle_synthesis.argtypes = [i32, i32, i32, i64, dp, dp, dp, dp, dp]
        lib.oracle_adjoint.restype = i32
        lib.oracle_adjoint.argtypes = [i32, i32, i32, i64, dp, dp, dp, dp, dp]
        for name in ("oracle_synthesis_dd", "oracle_adjoint_dd"):
            getattr(lib, name).restype = i32
            getattr(lib, name).argtypes = [i32, i32, i32, i64, dp, dp, dp, dp, dp]
        lib.oracle_slambda_dd.restype = i32
        lib.oracle_slambda_dd.argtypes = [i32, i32, i32, ctypes.c_double, dp]
        lib.oracle_pointing.restype = i32
        lib.oracle_pointing.argtypes = [i64, dp, dp, dp, dp, dp, dp, dp]
        lib.oracle_num_threads.restype = i32
        lib.oracle_num_threads.argtypes = []
        _lib = lib
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def nalm(lmax: int, mmax: int | None = None) -> int:
    """Number of a_lm with 0 <= m <= mmax, m <= l <= lmax."""
    return int(_load().oracle_nalm(lmax, lmax if mmax is None else mmax))


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def slambda(lmax: int, m: int, spin: int, theta: float, precise: bool = False) -> np.ndarray:
    """spin lambda_{l,m}(theta) for l = 0..lmax, so that sY_lm = slambda * e^{i m phi}.

    precise=True runs the start value and recursion in double-double (~106 bits)."""
    out = np.zeros(lmax + 1)
    fn = _load().oracle_slambda_dd if precise else _load().oracle_slambda
    rc = fn(lmax, m, spin, float(theta), _ptr(out))
    if rc:
        raise ValueError("oracle_slambda: bad arguments")
    return out


def ring_coeffs(lmax: int, mmax: int, spin: int, theta, alm) -> np.ndarray:
    """Coefficients of e^{i m phi} of the (pre-phase) field at each theta.

    spin 0: [n, mmax+1] complex, sum_l a_lm lambda_lm.
    spin s: [n, 2 mmax+1] complex (column m + mmax), -sum_l (G + iC)_lm s lambda_lm.
    """
    theta = _f64(theta)
    alm = _c128(alm)
    ncol = mmax + 1 if spin == 0 else 2 * mmax + 1
    out = np.zeros((theta.size, ncol), dtype=np.complex128)
    rc = _load().oracle_ring_coeffs(lmax, mmax, spin, theta.size, _ptr(theta), _ptr(alm), _ptr(out))
    if rc:
        raise ValueError("oracle_ring_coeffs: bad arguments")
    return out


def synthesis(lmax: int, mmax: int, spin: int, theta, phi, alm, chi=None, precise: bool = False) -> np.ndarray:
    """Forward lensing operator by direct summation.

    alm: [ncomp, nalm] complex (spin 0: [1, nalm] or [nalm]); returns [ncomp, npts]
    (spin 0: T; spin s: Q, U).  Imaginary parts of the m = 0 entries are ignored.
    precise=True evaluates the harmonics in double-double (for targets near 1e-12
    at lmax ~ 5000, where the FP64 recursion's own rounding reaches ~1e-12).
    """
    theta, phi = _f64(theta), _f64(phi)
    chi = None if chi is None else _f64(chi)
    ncomp = 1 if spin == 0 else 2
    alm = _c128(alm).reshape(ncomp, -1).copy()
    if alm.shape[1] != nalm(lmax, mmax):
        raise ValueError("alm has the wrong size")
    # real fields (a_{l,-m} = (-1)^m conj a_lm) have real m = 0 coefficients; an
    # imaginary part there is outside the domain and ignored, as by the library
    alm[:, :lmax + 1] = alm[:, :lmax + 1].real
    out = np.zeros((ncomp, theta.size))
    fn = _load().oracle_synthesis_dd if precise else _load().oracle_synthesis
    rc = fn(lmax, mmax, spin, theta.size, _ptr(theta), _ptr(phi), _ptr(chi), _ptr(alm), _ptr(out))
    if rc:
        raise ValueError("oracle_synthesis: bad arguments")
    return out


def adjoint(lmax: int, mmax: int, spin: int, theta, phi, m, chi=None, precise: bool = False) -> np.ndarray:
    """Adjoint lensing operator by direct summation; returns [ncomp, nalm] complex.
    precise=True as for synthesis."""
    theta, phi = _f64(theta), _f64(phi)
    chi = None if chi is None else _f64(chi)
    ncomp = 1 if spin == 0 else 2
    m = _f64(m).reshape(ncomp, -1)
    if m.shape[1] != theta.size:
        raise ValueError("map has the wrong size")
    out = np.zeros((ncomp, nalm(lmax, mmax)), dtype=np.complex128)
    fn = _load().oracle_adjoint_dd if precise else _load().oracle_adjoint
    rc = fn(lmax, mmax, spin, theta.size, _ptr(theta), _ptr(phi), _ptr(chi), _ptr(m), _ptr(out))
    if rc:
        raise ValueError("oracle_adjoint: bad arguments")
    return out


def pointing(theta, phi, alpha_theta, alpha_phi):
    """Unlensed angles (theta', phi') and spin phase chi from the deflection field."""
    theta, phi = _f64(theta), _f64(phi)
    at, ap = _f64(alpha_theta), _f64(alpha_phi)
    t2, p2, chi = np.zeros_like(theta), np.zeros_like(theta), np.zeros_like(theta)
    _load().oracle_pointing(theta.size, _ptr(theta), _ptr(phi), _ptr(at), _ptr(ap), _ptr(t2), _ptr(p2),
                            _ptr(chi))
    return t2, p2, chi


def deflected_points(theta, phi, phi_lm, lmax_phi: int):
    """Lensed geometry from a lensing potential: Sect. 3, Eq. "deflect" then the pointing formula.

    The deflection alpha_theta + i alpha_phi is the spin-1 forward operator
    (Eq. "forwardpol" with s = 1, chi = 0) applied to G_LM = sqrt(L(L+1)) phi_LM,
    C_LM = 0, which equals - sum sqrt(L(L+1)) phi_LM 1Y_LM.
    """
    L = np.arange(lmax_phi + 1)
    ell = np.concatenate([L[m:] for m in range(lmax_phi + 1)])
    g = _c128(phi_lm) * np.sqrt(ell * (ell + 1.0))
    alm = np.stack([g, np.zeros_like(g)])
    a = synthesis(lmax_phi, lmax_phi, 1, theta, phi, alm)
    return pointing(theta, phi, a[0], a[1])


# ---------------------------------------------------------------- differentiation
# Gradient of a real loss L(d) of the lensed map d = A(phi) x with respect to
# the lensing potential phi_LM.  The paper gives the forward model (Sect. 2
# Eqs. "forward" / "forwardpol", Eq. "deflect", the pointing formula of
# Sect. 3 and chi of Fig. 1) but not its derivative; the chain rule below is
# written out step by step and pinned by central finite differences of that
# forward model (tests/test_oracle_pins.py).
#
# With P = Q + iU = e^{i s chi} sf(n') (sf = -sum (G + iC) sY, or sum a Y for
# s = 0) and a tangent perturbation dalpha of the deflection at n, in the
# frame of n parallel-transported along the geodesic:
#   dP = -1/2 [conj(v) A + v B] + i s c dalpha_perp P,
#   v = J dalpha,  J = ah ah^T + (sin a / a)(1 - ah ah^T)   (exponential map),
#   A = e^{i(s+1)chi} (eth sf)(n'),  B = e^{i(s-1)chi} (ethbar sf)(n')
#   (spin 0: B = conj(A)),  c = (1 - cos a) / a  (holonomy of the transport),
# a = |alpha|, ah = alpha / a, dalpha_perp the component of dalpha along i ah.
# Hence, for g = dL/dQ + i dL/dU (real dL/dd for s = 0):
#   dL/dalpha = J Y + K i ah,  Y = -1/2 [conj(g) A + g conj(B)],
#   K = -s c Im(conj(g) P),
# and dL/dphi_LM = sqrt(L(L+1)) w_m [adjoint_1(dL/dalpha)]_G at the undeflected
# points (w_0 = 1, w_m = 2: real-field coefficients appear for +m and -m).

def _ell(lmax: int) -> np.ndarray:
    return np.concatenate([np.arange(m, lmax + 1) for m in range(lmax + 1)]).astype(np.float64)


def _mweight(lmax: int) -> np.ndarray:
    return np.concatenate([np.full(lmax + 1 - m, 1.0 if m == 0 else 2.0) for m in range(lmax + 1)])


def eth_coeffs(lmax: int, spin: int, alm, lower: bool = False) -> np.ndarray:
    """Coefficients [G, C] of eth sf (spin s+1) or, lower=True, ethbar sf (spin s-1 >= 1).

    eth sY_lm = sqrt((l-s)(l+s+1)) s+1Y_lm, ethbar sY_lm = -sqrt((l+s)(l-s+1)) s-1Y_lm, and
    sf = -sum (G + iC) sY (s > 0) or sum a Y (s = 0).
    """
    ell = _ell(lmax)
    alm = _c128(alm).reshape(1 if spin == 0 else 2, -1)
    if spin == 0:
        if lower:
            raise ValueError("ethbar of a spin-0 field has spin -1")
        return np.stack([-np.sqrt(ell * (ell + 1.0)) * alm[0], np.zeros_like(alm[0])])
    if lower:
        if spin < 2:
            raise ValueError("ethbar of a spin-1 field has spin 0")
        f = -np.sqrt(np.maximum((ell + spin) * (ell - spin + 1.0), 0.0))
    else:
        f = np.sqrt(np.maximum((ell - spin) * (ell + spin + 1.0), 0.0))
    return alm * f[None, :]


def lensed_forward(lmax: int, spin: int, theta0, phi0, phi_lm, lmax_phi: int, x) -> np.ndarray:
    """d = A(phi) x: deflect the points (Eq. "deflect", pointing) and synthesise x there."""
    th, ph, chi = deflected_points(theta0, phi0, phi_lm, lmax_phi)
    return synthesis(lmax, lmax, spin, th, ph, x, chi if spin else None)


def deflection_vjp(spin: int, alpha_theta, alpha_phi, g, p, a_up, b_down=None):
    """dL/dalpha (complex, theta + i phi) per point from the formula above."""
    at, ap = _f64(alpha_theta), _f64(alpha_phi)
    a = np.hypot(at, ap)
    safe = np.where(a > 0, a, 1.0)
    ah = np.where(a > 0, (at + 1j * ap) / safe, 1.0 + 0j)
    k = np.where(a > 0, np.sin(a) / safe, 1.0)
    c = np.where(a > 0, 2.0 * np.sin(0.5 * a) ** 2 / safe, 0.0)
    A = a_up[0] + 1j * a_up[1]
    if spin == 0:
        gc = _f64(g).reshape(-1) + 0j
        B = np.conj(A)
        P = _f64(p).reshape(-1) + 0j
    else:
        gc = g[0] + 1j * g[1]
        B = b_down[0] + 1j * b_down[1]
        P = p[0] + 1j * p[1]
    Y = -0.5 * (np.conj(gc) * A + gc * np.conj(B))
    par = (np.conj(ah) * Y).real
    JY = par * ah + k * (Y - par * ah)
    K = -spin * c * (np.conj(gc) * P).imag
    return JY + K * 1j * ah


def phi_gradient(lmax: int, spin: int, theta0, phi0, phi_lm, lmax_phi: int, x, g) -> np.ndarray:
    """dL/dphi_LM (dL/dRe + i dL/dIm) for L = sum_i g_i . (A(phi) x)_i."""
    theta0, phi0 = _f64(theta0), _f64(phi0)
    ellp = _ell(lmax_phi)
    gphi = _c128(phi_lm) * np.sqrt(ellp * (ellp + 1.0))
    alpha = synthesis(lmax_phi, lmax_phi, 1, theta0, phi0, np.stack([gphi, np.zeros_like(gphi)]))
    th, ph, chi = pointing(theta0, phi0, alpha[0], alpha[1])
    x = _c128(x).reshape(1 if spin == 0 else 2, -1)
    p = synthesis(lmax, lmax, spin, th, ph, x, chi if spin else None)
    a_up = synthesis(lmax, lmax, spin + 1, th, ph, eth_coeffs(lmax, spin, x), chi)
    b_down = None
    if spin >= 2:
        b_down = synthesis(lmax, lmax, spin - 1, th, ph, eth_coeffs(lmax, spin, x, lower=True), chi)
    g = _f64(g).reshape(p.shape)
    da = deflection_vjp(spin, alpha[0], alpha[1], g, p, a_up, b_down)
    adj = adjoint(lmax_phi, lmax_phi, 1, theta0, phi0, np.stack([da.real, da.imag]))
    return np.sqrt(ellp * (ellp + 1.0)) * _mweight(lmax_phi) * adj[0]


# ---------------------------------------------------------------- App. B
def magnification(theta, phi, phi_lm, lmax_phi: int) -> np.ndarray:
    """Magnification determinant |A| = |d^2 n'/d^2 n| of the remapping (App. B):
    (sin a / a)((1 - kappa)^2 - |gamma|^2) + (cos a - sin a / a)(1 - kappa - cos 2b gamma_1 - sin 2b gamma_2)
    with kappa = ethbar(1alpha)/2 (spin-0 synthesis of l(l+1)/2 phi_lm), gamma = eth(1alpha)/2
    (spin-2 synthesis of G = sqrt((l-1)l(l+1)(l+2))/2 phi_lm, C = 0), omega = 0 for a gradient
    deflection, a = |alpha| and b the angle of alpha from e_theta towards e_phi."""
    theta, phi = _f64(theta), _f64(phi)
    L = lmax_phi
    ell = _ell(L)
    p = _c128(phi_lm)
    kap = synthesis(L, L, 0, theta, phi, 0.5 * ell * (ell + 1.0) * p)[0]
    gam = synthesis(L, L, 2, theta, phi,
                    np.stack([0.5 * np.sqrt(np.maximum((ell - 1) * ell * (ell + 1) * (ell + 2), 0.0)) * p,
                              np.zeros_like(p)]))
    al = synthesis(L, L, 1, theta, phi, np.stack([np.sqrt(ell * (ell + 1.0)) * p, np.zeros_like(p)]))
    a = np.hypot(al[0], al[1])
    safe = np.where(a > 0, a, 1.0)
    sa = np.where(a > 0, np.sin(a) / safe, 1.0)
    ct, st = np.where(a > 0, al[0] / safe, 1.0), np.where(a > 0, al[1] / safe, 0.0)
    c2b, s2b = ct * ct - st * st, 2 * ct * st
    cma = np.where(a > 0, np.cos(a) - sa, 0.0)
    return sa * ((1 - kap) ** 2 - (gam[0] ** 2 + gam[1] ** 2)) + cma * (1 - kap - c2b * gam[0] - s2b * gam[1])
