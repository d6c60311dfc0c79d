"""Reverse-mode differentiation through the transform pair.

synthesis(plan, a) and adjoint(plan, x) are torch.autograd functions whose
backward passes are lens_synthesis_vjp / lens_adjoint_vjp, i.e. the exact
adjoint of Sect. 2 with the real-field order weight (m > 0 coefficients
appear for +m and -m in the forward).  Checked three ways:
  * directional derivatives: for the linear maps, <grad, delta> must equal the
    change of the loss along delta computed by the forward transform itself;
  * against the oracle: the gradient of sum(g * synthesis(a)) is w_m times the
    oracle's adjoint of g (w_0 = 1, w_m = 2);
  * a quadratic loss against central finite differences.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2304_10431_gb300 import LensPlan, adjoint, synthesis
from paper_2304_10431_gb300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0") if torch.cuda.is_available() else None
L = 40


def _setup(spin, n=3000, seed=11):
    th, ph, chi = W.random_points(n, seed)
    plan = LensPlan(L, th, ph, chi if spin else None, spin=spin, epsilon=1e-12, precision="fp64", device=DEV)
    return plan, th, ph, chi


def _rand_alm(plan, seed):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((plan.ncomp, plan.nalm)) + 1j * rng.standard_normal((plan.ncomp, plan.nalm))
    return torch.as_tensor(a, dtype=torch.complex128, device=DEV)


def _rand_map(plan, seed):
    rng = np.random.default_rng(seed)
    return torch.as_tensor(rng.standard_normal((plan.ncomp, plan.npoints)), dtype=torch.float64, device=DEV)


def _re_dot(u, v):  # real inner product of complex tensors: sum Re(conj(u) v)
    return float(torch.sum(u.real * v.real + u.imag * v.imag))


def _m_weight(plan):
    m = W.alm_m_of_index(plan.lmax, plan.mmax)
    return np.where(m > 0, 2.0, 1.0)


@pytest.mark.parametrize("spin", [0, 2])
def test_synthesis_gradient_directional_and_oracle(spin):
    plan, th, ph, chi = _setup(spin)
    a = _rand_alm(plan, 1).requires_grad_(True)
    g = _rand_map(plan, 2)
    loss = torch.sum(g * synthesis(plan, a))
    loss.backward()
    grad = a.grad.detach()
    for k in range(3):
        d = _rand_alm(plan, 10 + k)  # includes imaginary parts at m = 0, which must get zero gradient
        dl = float(torch.sum(g * plan.synthesis(d)))
        assert abs(_re_dot(grad, d) - dl) <= 1e-12 * max(1.0, abs(dl))
    ref = O.adjoint(L, L, spin, th, ph, g.cpu().numpy(), chi if spin else None) * _m_weight(plan)[None, :]
    got = grad.cpu().numpy()
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)
    m0 = W.alm_m_of_index(L, L) == 0
    assert np.all(got[:, m0].imag == 0)
    plan.close()


@pytest.mark.parametrize("spin", [0, 2])
def test_adjoint_gradient_directional(spin):
    plan, *_ = _setup(spin)
    x = _rand_map(plan, 3).requires_grad_(True)
    h = _rand_alm(plan, 4)
    out = adjoint(plan, x)
    loss = torch.sum(h.real * out.real + h.imag * out.imag)
    loss.backward()
    for k in range(3):
        d = _rand_map(plan, 20 + k)
        dl = _re_dot(h, plan.adjoint(d))
        assert abs(float(torch.sum(x.grad * d)) - dl) <= 1e-12 * max(1.0, abs(dl))
    plan.close()


def test_quadratic_loss_finite_differences():
    plan, *_ = _setup(2, n=2000, seed=5)
    data = _rand_map(plan, 6)
    a0 = _rand_alm(plan, 7)
    a = a0.clone().requires_grad_(True)
    loss = torch.sum((synthesis(plan, a) - data) ** 2)
    loss.backward()
    d = _rand_alm(plan, 8)
    t = 1e-4

    def f(z):
        return float(torch.sum((plan.synthesis(z) - data) ** 2))

    fd = (f(a0 + t * d) - f(a0 - t * d)) / (2 * t)
    assert abs(_re_dot(a.grad, d) - fd) <= 1e-8 * abs(fd)
    plan.close()
