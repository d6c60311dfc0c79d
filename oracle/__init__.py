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


def slambda(lmax: int, m: int, spin: int, theta: float) -> np.ndarray:
    """spin lambda_{l,m}(theta) for l = 0..lmax, so that sY_lm = slambda * e^{i m phi}."""
    out = np.zeros(lmax + 1)
    rc = _load().oracle_slambda(lmax, m, spin, float(theta), _ptr(out))
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


def synthesis(lmax: int, mmax: int, spin: int, theta, phi, alm, chi=None) -> np.ndarray:
    """Forward lensing operator by direct summation.

    alm: [ncomp, nalm] complex (spin 0: [1, nalm] or [nalm]); returns [ncomp, npts]
    (spin 0: T; spin s: Q, U).
    """
    theta, phi = _f64(theta), _f64(phi)
    chi = None if chi is None else _f64(chi)
    ncomp = 1 if spin == 0 else 2
    alm = _c128(alm).reshape(ncomp, -1)
    if alm.shape[1] != nalm(lmax, mmax):
        raise ValueError("alm has the wrong size")
    out = np.zeros((ncomp, theta.size))
    rc = _load().oracle_synthesis(lmax, mmax, spin, theta.size, _ptr(theta), _ptr(phi), _ptr(chi),
                                  _ptr(alm), _ptr(out))
    if rc:
        raise ValueError("oracle_synthesis: bad arguments")
    return out


def adjoint(lmax: int, mmax: int, spin: int, theta, phi, m, chi=None) -> np.ndarray:
    """Adjoint lensing operator by direct summation; returns [ncomp, nalm] complex."""
    theta, phi = _f64(theta), _f64(phi)
    chi = None if chi is None else _f64(chi)
    ncomp = 1 if spin == 0 else 2
    m = _f64(m).reshape(ncomp, -1)
    if m.shape[1] != theta.size:
        raise ValueError("map has the wrong size")
    out = np.zeros((ncomp, nalm(lmax, mmax)), dtype=np.complex128)
    rc = _load().oracle_adjoint(lmax, mmax, spin, theta.size, _ptr(theta), _ptr(phi), _ptr(chi),
                                _ptr(m), _ptr(out))
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
