"""Lensed harmonic coefficients (Sect. 4) and inverse lensing (App. B).

LensedAlm remaps the unlensed field onto a Gauss-Legendre grid with the lensing
synthesis and applies a backward SHT (the adjoint at the grid points with the
quadrature weights); its adjoint is the forward SHT followed by the adjoint
remapping; inverse() applies the adjoint to the lensed map times the
magnification |A|.  The oracle side builds its own grid with numpy's
Gauss-Legendre rule and evaluates every sum directly.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2304_10431_gb300 import LensedAlm, gl_grid
from paper_2304_10431_gb300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0") if torch.cuda.is_available() else None


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def np_grid(nrings, nphi):
    x, w = np.polynomial.legendre.leggauss(nrings)
    order = np.argsort(-x)  # theta ascending
    th = np.repeat(np.arccos(x[order]), nphi)
    ph = np.tile(2 * math.pi * np.arange(nphi) / nphi, nrings)
    wt = np.repeat(w[order] * 2 * math.pi / nphi, nphi)
    return th, ph, wt


def _phi(L, seed, rms):
    phi = W.draw_alm(W.phi_cl(L), L, seed)
    ell = W.alm_l_of_index(L).astype(float)
    w = np.where(W.alm_m_of_index(L) > 0, 2.0, 1.0)
    return phi * rms / np.sqrt(np.sum(w * ell * (ell + 1) * np.abs(phi) ** 2) / (4 * math.pi))


def _x(L, spin, seed):
    nc = 1 if spin == 0 else 2
    return np.stack([W.draw_alm(W.cmb_cl(L, 0.7 * L), L, seed + k, spin=spin) for k in range(nc)])


def test_gl_grid_matches_numpy():
    th, ph, w = (t.cpu().numpy() for t in gl_grid(37, 80, device=DEV))
    th2, ph2, w2 = np_grid(37, 80)
    assert np.max(np.abs(th - th2)) < 1e-14 and np.max(np.abs(ph - ph2)) < 1e-14
    assert np.max(np.abs(w - w2)) < 1e-15 and abs(w.sum() - 4 * math.pi) < 1e-12


@pytest.mark.parametrize("spin", [0, 2])
def test_zero_deflection_returns_the_input(spin):
    L = 48
    la = LensedAlm(L, L, spin=spin, epsilon=1e-12, precision="fp64", device=DEV)
    la.set_phi(torch.zeros(la.model.defl.nalm, dtype=torch.complex128, device=DEV))
    x = _x(L, spin, 10)
    got = la.forward(torch.as_tensor(x, device=DEV)).cpu().numpy()
    assert rel(got, x) <= 1e-11
    la.close()


@pytest.mark.parametrize("spin", [0, 2])
def test_lensed_alm_and_adjoint_vs_oracle(spin):
    Lu, Ll, nr, nphi = 40, 32, 49, 98
    la = LensedAlm(Lu, Ll, spin=spin, lmax_phi=Lu, nrings=nr, nphi=nphi, epsilon=1e-12, precision="fp64",
                   device=DEV)
    phi = _phi(Lu, 5, 0.01)
    la.set_phi(torch.as_tensor(phi, device=DEV))
    x = _x(Lu, spin, 20)
    got = la.forward(torch.as_tensor(x, device=DEV)).cpu().numpy()
    th, ph, wt = np_grid(nr, nphi)
    t2, p2, chi = O.deflected_points(th, ph, phi, Lu)
    m = O.synthesis(Lu, Lu, spin, t2, p2, x, chi if spin else None)
    ref = O.adjoint(Ll, Ll, spin, th, ph, m * wt[None, :])
    assert rel(got, ref) <= 1e-10
    # adjoint: forward SHT onto the grid, weights, adjoint remapping
    y = _x(Ll, spin, 30)
    gota = la.adjoint(torch.as_tensor(y, device=DEV)).cpu().numpy()
    g = O.synthesis(Ll, Ll, spin, th, ph, y)
    refa = O.adjoint(Lu, Lu, spin, t2, p2, g * wt[None, :], chi if spin else None)
    assert rel(gota, refa) <= 1e-10
    la.close()


def test_adjoint_identity():
    """<D x, y> = <x, D^+ y> with the real-field a_lm product (FP64)."""
    Lu, Ll = 40, 32
    la = LensedAlm(Lu, Ll, spin=2, epsilon=1e-12, precision="fp64", device=DEV)
    la.set_phi(torch.as_tensor(_phi(Lu, 6, 0.02), device=DEV))
    x = torch.as_tensor(_x(Lu, 2, 40), device=DEV)
    y = torch.as_tensor(_x(Ll, 2, 50), device=DEV)

    def dot(a, b, L):
        w = torch.as_tensor(np.where(W.alm_m_of_index(L) > 0, 2.0, 1.0), device=DEV)
        return float(torch.sum(w * (a.real * b.real + a.imag * b.imag)))

    lhs, rhs = dot(la.forward(x), y, Ll), dot(x, la.adjoint(y), Lu)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    la.close()


@pytest.mark.parametrize("spin", [0, 2])
def test_inverse_lensing(spin):
    """App. B: the adjoint of the lensed map times |A| gives back the unlensed
    coefficients (to the accuracy of the grid's quadrature in the deflected
    coordinates), and equals the oracle's evaluation of the same sum."""
    L, nr = 32, 96
    la = LensedAlm(L, L, spin=spin, nrings=nr, nphi=2 * nr, epsilon=1e-12, precision="fp64", device=DEV)
    phi = _phi(L, 7, 0.005)
    la.set_phi(torch.as_tensor(phi, device=DEV))
    x = _x(L, spin, 60)
    d = la.model.forward(torch.as_tensor(x, device=DEV))
    got = la.inverse(d).cpu().numpy()
    assert rel(got, x) <= 1e-4
    th, ph, wt = np_grid(nr, 2 * nr)
    t2, p2, chi = O.deflected_points(th, ph, phi, L)
    det = O.magnification(th, ph, phi, L)
    ref = O.adjoint(L, L, spin, t2, p2, d.cpu().numpy() * (wt * det)[None, :], chi if spin else None)
    assert rel(got, ref) <= 1e-10
    la.close()
