"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the transform itself: it draws harmonic
coefficients from power spectra, lays out HEALPix ring centres and, for the
largest cases, displaces them by an independent random offset.  Both the CUDA
path and the CPU oracle receive exactly these arrays.

Recipes (stand-ins for the paper's simulations, which are not public data):

* CMB spectrum  C_l = (l+10)^-2 exp(-(l/l_d)^2), with the damping scale l_d
  per workload (100, 1500, 3750).
* Lensing potential spectrum C_L^phiphi proportional to (L+1)^-4, monopole and
  dipole zero, rescaled so that the rms deflection
  sum_L (2L+1)/(4 pi) L(L+1) C_L^phiphi equals (2.5 arcmin)^2.
* a_lm draws: m = 0 real N(0, C_l); m > 0 complex with variance C_l/2 per part;
  entries with l < |spin| are zero.  Generator: numpy PCG64 with the given seed.
* HEALPix ring centres (Gorski et al. 2005), ring order, 12 Nside^2 points.
"""
from __future__ import annotations

import math

import numpy as np

ARCMIN = math.pi / (180.0 * 60.0)


def nalm(lmax: int, mmax: int | None = None) -> int:
    mmax = lmax if mmax is None else mmax
    return (mmax + 1) * (2 * lmax + 2 - mmax) // 2


def alm_l_of_index(lmax: int, mmax: int | None = None) -> np.ndarray:
    """l of every entry in the layout index(l, m) = m(2 lmax + 1 - m)/2 + l."""
    mmax = lmax if mmax is None else mmax
    return np.concatenate([np.arange(m, lmax + 1) for m in range(mmax + 1)])


def alm_m_of_index(lmax: int, mmax: int | None = None) -> np.ndarray:
    mmax = lmax if mmax is None else mmax
    return np.concatenate([np.full(lmax + 1 - m, m) for m in range(mmax + 1)])


def cmb_cl(lmax: int, l_damp: float) -> np.ndarray:
    ell = np.arange(lmax + 1, dtype=np.float64)
    return (ell + 10.0) ** -2 * np.exp(-(ell / l_damp) ** 2)


def phi_cl(lmax: int, rms_arcmin: float = 2.5) -> np.ndarray:
    ell = np.arange(lmax + 1, dtype=np.float64)
    cl = (ell + 1.0) ** -4
    cl[:2] = 0.0
    rms2 = np.sum((2 * ell + 1) / (4 * math.pi) * ell * (ell + 1) * cl)
    return cl * (rms_arcmin * ARCMIN) ** 2 / rms2


def draw_alm(cl: np.ndarray, lmax: int, seed: int, mmax: int | None = None, spin: int = 0) -> np.ndarray:
    """One realisation of a_lm (complex128, healpy-style triangular layout)."""
    mmax = lmax if mmax is None else mmax
    rng = np.random.Generator(np.random.PCG64(seed))
    ell = alm_l_of_index(lmax, mmax)
    em = alm_m_of_index(lmax, mmax)
    re = rng.standard_normal(ell.size)
    im = rng.standard_normal(ell.size)
    sd = np.sqrt(cl[ell])
    a = np.where(em == 0, sd * re, sd * np.sqrt(0.5) * (re + 1j * im)).astype(np.complex128)
    a[ell < abs(spin)] = 0.0
    return a


def healpix_centres(nside: int):
    """Ring centres (theta, phi) of a HEALPix grid in ring order (12 nside^2 points)."""
    n = nside
    thetas, phis = [], []
    for i in range(1, 4 * n):
        if i < n:  # north polar cap
            th = 2.0 * math.asin(i / (math.sqrt(6.0) * n))
            npix = 4 * i
            ph = (math.pi / (2.0 * i)) * (np.arange(1, npix + 1) - 0.5)
        elif i <= 3 * n:  # equatorial belt
            z = 4.0 / 3.0 - 2.0 * i / (3.0 * n)
            th = math.acos(z)
            npix = 4 * n
            s = (i - n + 1) % 2
            ph = (math.pi / (2.0 * n)) * (np.arange(1, npix + 1) - 0.5 * s)
        else:  # south polar cap
            ii = 4 * n - i
            th = math.pi - 2.0 * math.asin(ii / (math.sqrt(6.0) * n))
            npix = 4 * ii
            ph = (math.pi / (2.0 * ii)) * (np.arange(1, npix + 1) - 0.5)
        thetas.append(np.full(npix, th))
        phis.append(ph)
    return np.concatenate(thetas), np.concatenate(phis)


def displaced_points(theta, phi, rms_arcmin: float, seed: int, chi_scale: float = 1.0):
    """Independent random displacements with the lensing rms, and a spin phase.

    Used where a gradient-field deflection would need a transform of its own
    (largest sizes): the point density and locality match the lensed HEALPix
    geometry.  chi is drawn as chi_scale * N(0, 1) * alpha/rad * cot(theta),
    the first-order size of the lensing phase, clipped to (-pi, pi].
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    sig = rms_arcmin * ARCMIN / math.sqrt(2.0)
    dth = rng.standard_normal(theta.size) * sig
    dph = rng.standard_normal(theta.size) * sig
    th2 = theta + dth
    ph2 = phi + dph / np.maximum(np.sin(theta), 1e-3)
    over = th2 > math.pi
    under = th2 < 0.0
    th2 = np.where(over, 2.0 * math.pi - th2, th2)
    th2 = np.where(under, -th2, th2)
    ph2 = np.where(over | under, ph2 + math.pi, ph2)
    ph2 = np.mod(ph2, 2.0 * math.pi)
    cot = np.cos(theta) / np.maximum(np.sin(theta), 1e-3)
    chi = np.clip(chi_scale * rng.standard_normal(theta.size) * sig * cot, -math.pi, math.pi)
    return th2, ph2, chi


def random_points(n: int, seed: int):
    """Uniform points on the sphere (theta, phi) and a uniform phase chi."""
    rng = np.random.Generator(np.random.PCG64(seed))
    z = rng.uniform(-1.0, 1.0, n)
    return np.arccos(z), rng.uniform(0.0, 2.0 * math.pi, n), rng.uniform(-math.pi, math.pi, n)


def gauss_legendre_grid(nrings: int, nphi: int):
    """Gauss-Legendre rings x equispaced longitudes (theta, phi, weights)."""
    x, w = np.polynomial.legendre.leggauss(nrings)
    th = np.arccos(x)
    ph = 2.0 * math.pi * np.arange(nphi) / nphi
    T, P = np.meshgrid(th, ph, indexing="ij")
    W = np.repeat(w[:, None] * (2.0 * math.pi / nphi), nphi, axis=1)
    return T.ravel(), P.ravel(), W.ravel()
