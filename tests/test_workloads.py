"""Seeded input generators (paper_2304_10431_gb300.workloads): the HEALPix ring
layout, the lensing-potential normalisation, the a_lm draws and the point
displacements have the properties their recipes state."""
import math

import numpy as np

from paper_2304_10431_gb300 import workloads as W


def test_healpix_nside1_closed_form():
    th, ph = W.healpix_centres(1)
    assert th.size == 12
    z = np.cos(th)
    # HEALPix base pixels: rings at z = 2/3, 0, -2/3, four pixels each
    assert np.allclose(np.sort(z), np.repeat([-2.0 / 3.0, 0.0, 2.0 / 3.0], 4), atol=1e-15)
    # Gorski et al.: phi = pi/(2 nside) (j - s/2), j = 1 .. 4 nside (the last can be 2 pi)
    assert np.all((ph > 0) & (ph <= 2 * math.pi))
    assert np.allclose(np.sort(ph[4:8]), np.pi / 2 * np.arange(1, 5))


def test_healpix_equal_area_rings():
    n = 16
    th, ph = W.healpix_centres(n)
    assert th.size == 12 * n * n
    assert np.all(np.diff(th) >= -1e-15)  # ring order, north to south
    assert abs(np.mean(np.cos(th))) < 1e-12  # symmetric about the equator
    # equal areas: the fraction of points above a ring matches the area above it
    z = np.cos(th)
    for z0 in (0.9, 0.5, 0.0, -0.5):
        frac = np.mean(z > z0)
        assert abs(frac - (1 - z0) / 2) < 4.0 / (12 * n)


def test_phi_spectrum_normalisation():
    L = 200
    cl = W.phi_cl(L, 2.5)
    ell = np.arange(L + 1)
    assert cl[0] == 0.0 and cl[1] == 0.0 and np.all(cl[2:] > 0)
    rms2 = np.sum((2 * ell + 1) / (4 * math.pi) * ell * (ell + 1) * cl)
    assert abs(math.sqrt(rms2) - 2.5 * W.ARCMIN) < 1e-15


def test_draw_alm_structure_and_variance():
    L = 300
    cl = W.cmb_cl(L, 200.0)
    a = W.draw_alm(cl, L, 5, spin=2)
    ell, em = W.alm_l_of_index(L), W.alm_m_of_index(L)
    assert a.size == W.nalm(L) == ell.size == em.size
    assert np.all(a[em == 0].imag == 0) and np.all(a[ell < 2] == 0)
    # |a_lm|^2 / C_l has mean 1 (m = 0: chi^2_1, m > 0: chi^2_2 / 2)
    sel = ell >= 2
    r = np.abs(a[sel]) ** 2 / cl[ell[sel]]
    assert abs(np.mean(r) - 1.0) < 0.03
    assert np.array_equal(a, W.draw_alm(cl, L, 5, spin=2))


def test_displacements_have_the_lensing_rms():
    th0, ph0 = W.healpix_centres(64)
    th, ph, chi = W.displaced_points(th0, ph0, 2.5, seed=7)
    dth = th - th0
    dph = np.angle(np.exp(1j * (ph - ph0)))
    keep = (th0 > 0.05) & (th0 < math.pi - 0.05)  # away from the reflections at the poles
    rms = math.sqrt(np.mean(dth[keep] ** 2 + (np.sin(th0[keep]) * dph[keep]) ** 2))
    assert abs(rms / (2.5 * W.ARCMIN) - 1.0) < 0.02
    assert np.all((th >= 0) & (th <= math.pi)) and np.all((ph >= 0) & (ph < 2 * math.pi))
    assert np.all(np.abs(chi) <= math.pi)
    th2, ph2, chi2 = W.displaced_points(th0, ph0, 2.5, seed=7)
    assert np.array_equal(th, th2) and np.array_equal(chi, chi2)


def test_gauss_legendre_grid_weights():
    th, ph, w = W.gauss_legendre_grid(33, 70)
    assert th.size == ph.size == w.size == 33 * 70
    assert abs(w.sum() - 4 * math.pi) < 1e-12
    # exact for cos^2 theta (degree 2 in z): integral over the sphere is 4 pi / 3
    assert abs(np.sum(w * np.cos(th) ** 2) - 4 * math.pi / 3) < 1e-12
