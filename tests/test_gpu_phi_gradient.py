"""Gradients of d = A(phi) x with respect to x and to the lensing potential phi.

The deflection (Eq. "deflect"), the pointing and the lensed synthesis run on the
GPU (LensingModel); lens_phi_gradient assembles dL/dphi from spin-raised and
-lowered syntheses at the deflected points.  Checked against
  * the oracle's phi gradient (its chain rule is pinned by finite differences of
    the oracle's forward model in tests/test_oracle_pins.py), at lmax 64;
  * central finite differences of the GPU forward model itself, for the loss
    0.5 ||A(phi) x - d||^2 of the differentiable-lensing workload, along 32
    random directions in phi and in x (FP64 plans);
  * the FP64 gradient, for an FP32 model at lmax 2048 / Nside 1024 (the
    differentiable-lensing workload's size).
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2304_10431_gb300 import LensingModel, lensed
from paper_2304_10431_gb300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0") if torch.cuda.is_available() else None


def _phi(L, seed, rms):
    phi = W.draw_alm(W.phi_cl(L), L, seed)
    ell = W.alm_l_of_index(L).astype(float)
    w = np.where(W.alm_m_of_index(L) > 0, 2.0, 1.0)
    return phi * rms / np.sqrt(np.sum(w * ell * (ell + 1) * np.abs(phi) ** 2) / (4 * math.pi))


def _deflection_rms(phi, L):
    ell = W.alm_l_of_index(L).astype(float)
    w = np.where(W.alm_m_of_index(L) > 0, 2.0, 1.0)
    return float(np.sqrt(np.sum(w * ell * (ell + 1) * np.abs(phi) ** 2) / (4 * math.pi)))


def _x(L, spin, seed, l_damp):
    nc = 1 if spin == 0 else 2
    return np.stack([W.draw_alm(W.cmb_cl(L, l_damp), L, seed + k, spin=spin) for k in range(nc)])


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("spin", [0, 2])
def test_phi_gradient_vs_oracle(spin):
    L = 64
    th0, ph0 = W.healpix_centres(16)
    phi = _phi(L, 9, 0.05)
    x = _x(L, spin, 30, 50.0)
    g = np.random.default_rng(1).standard_normal((x.shape[0], th0.size))
    model = LensingModel(L, th0, ph0, spin=spin, epsilon=1e-12, precision="fp64", device=DEV)
    model.set_phi(torch.as_tensor(phi, device=DEV))
    xt = torch.as_tensor(x, device=DEV)
    gt = torch.as_tensor(g, device=DEV)
    got = model.grad_phi(xt, gt).cpu().numpy()
    ref = O.phi_gradient(L, spin, th0, ph0, phi, L, x, g)
    assert rel(got, ref) <= 1e-9
    # passing the forward map instead of recomputing it gives the same result
    got2 = model.grad_phi(xt, gt, model.forward(xt)).cpu().numpy()
    assert rel(got2, ref) <= 1e-9
    model.close()


def test_quadratic_loss_finite_differences_32_directions():
    """0.5 ||A(phi) x - d||^2, spin 2, FP64: autograd gradients in x and phi
    against central differences (Richardson) of the GPU forward model."""
    L, spin = 48, 2
    th0, ph0 = W.healpix_centres(16)
    model = LensingModel(L, th0, ph0, spin=spin, epsilon=1e-12, precision="fp64", device=DEV)
    phi0 = torch.as_tensor(_phi(L, 4, 0.02), device=DEV)
    x0 = torch.as_tensor(_x(L, spin, 60, 40.0), device=DEV)
    data = torch.as_tensor(np.random.default_rng(2).standard_normal((2, th0.size)), device=DEV)

    def loss_value(x, p):
        model.set_phi(p)
        return 0.5 * float(torch.sum((model.forward(x) - data) ** 2))

    x = x0.clone().requires_grad_(True)
    p = phi0.clone().requires_grad_(True)
    loss = 0.5 * torch.sum((lensed(model, x, p) - data) ** 2)
    loss.backward()
    gx, gp = x.grad.detach(), p.grad.detach()
    rng = np.random.default_rng(77)
    worst = 0.0
    for k in range(32):
        dp = rng.standard_normal(phi0.numel()) + 1j * rng.standard_normal(phi0.numel())
        dp = torch.as_tensor(dp * (1e-4 / _deflection_rms(dp, L)), device=DEV)  # 1e-4 rad rms deflection change
        t = 1.0
        f1 = (loss_value(x0, phi0 + t * dp) - loss_value(x0, phi0 - t * dp)) / (2 * t)
        f2 = (loss_value(x0, phi0 + 0.5 * t * dp) - loss_value(x0, phi0 - 0.5 * t * dp)) / t
        fd = (4 * f2 - f1) / 3
        an = float(torch.sum(gp.real * dp.real + gp.imag * dp.imag))
        worst = max(worst, abs(an - fd) / abs(fd))
    print("worst relative FD mismatch over 32 directions: %.2e" % worst)
    assert worst <= 1e-6, worst
    for k in range(4):  # the loss is quadratic in x: central differences are exact up to rounding
        dx = torch.as_tensor(rng.standard_normal(x0.shape) + 1j * rng.standard_normal(x0.shape), device=DEV)
        fd = (loss_value(x0 + dx, phi0) - loss_value(x0 - dx, phi0)) / 2
        an = float(torch.sum(gx.real * dx.real + gx.imag * dx.imag))
        assert abs(an - fd) <= 1e-9 * abs(fd)
    model.close()


def test_fp32_gradients_at_workload_size():
    """lmax 2048, Nside 1024 (12.6M points), spin 2, 2.5' rms deflection: FP32 model
    gradients in x and phi against the FP64 model's."""
    L, spin, nside = 2048, 2, 1024
    th0, ph0 = W.healpix_centres(nside)
    cl = W.phi_cl(L)
    phi = torch.as_tensor(W.draw_alm(cl, L, 2000), device=DEV)
    x = _x(L, spin, 1000, 1500.0)
    g = np.random.default_rng(3).standard_normal((2, th0.size))
    res = {}
    for prec, eps in (("fp32", 1e-5), ("fp64", 1e-10)):
        model = LensingModel(L, th0, ph0, spin=spin, epsilon=eps, precision=prec, device=DEV)
        model.set_phi(phi)
        cdt = torch.complex64 if prec == "fp32" else torch.complex128
        rdt = torch.float32 if prec == "fp32" else torch.float64
        xt = torch.as_tensor(x, dtype=cdt, device=DEV)
        gt = torch.as_tensor(g, dtype=rdt, device=DEV)
        res[prec] = (model.grad_x(gt).cpu().numpy(), model.grad_phi(xt, gt).cpu().numpy())
        model.close()
        torch.cuda.empty_cache()
    assert rel(res["fp32"][0], res["fp64"][0]) <= 1e-4
    assert rel(res["fp32"][1], res["fp64"][1]) <= 1e-4
