"""Host check of the polynomial kernel weights FP32 plans evaluate (no GPU).

The NUFFT steps (Sect. 3) weight tap a of a point by the ES kernel
phi(x) = exp(beta (sqrt(1 - x^2) - 1)) for |x| < 1, x = (frac - a) 2 / W, with
frac = u - ceil(u - W/2) in (W/2 - 1, W/2].  ``lens_kernel_poly`` returns the
per-tap polynomials in t = 2 frac - (W - 1) that FP32 plans use instead; here they
are evaluated by Horner's rule in FP32 and compared with phi written out in FP64.
"""
import ctypes

import numpy as np
import pytest

from paper_2304_10431_gb300 import _native


def es_kernel(x, beta):
    q = 1.0 - x * x
    return np.where(q > 0, np.exp(beta * (np.sqrt(np.maximum(q, 0.0)) - 1.0)), 0.0)


def kernel_poly(lib, W, beta):
    out = np.zeros(W * (W + 2), dtype=np.float32)
    assert lib.lens_kernel_poly(W, beta, out.ctypes.data) == 0
    return out.reshape(W, W + 2)


def horner_f32(c, t):
    acc = np.full(t.shape, c[-1], dtype=np.float32)
    for k in range(len(c) - 2, -1, -1):  # one rounding per step, as a fused multiply-add
        acc = (acc.astype(np.float64) * t.astype(np.float64) + np.float64(c[k])).astype(np.float32)
    return acc


@pytest.mark.parametrize("sigma", [1.25, 1.5, 2.0])
@pytest.mark.parametrize("W", [4, 6, 8, 11, 16])
def test_polynomial_weights_follow_the_es_kernel(W, sigma):
    lib = _native.load()
    beta = np.pi * W * (1.0 - 0.5 / sigma)
    c = kernel_poly(lib, W, beta)
    assert np.abs(c).max() < 1.5  # well-conditioned monomial form on [-1, 1]
    frac = (W / 2 - 1) + (np.arange(4000) + 0.5) / 4000  # inside (W/2 - 1, W/2]
    t = (2 * frac - (W - 1)).astype(np.float32)
    err = 0.0
    for a in range(W):
        exact = es_kernel((frac - a) * 2.0 / W, beta)
        err = max(err, np.abs(horner_f32(c[a], t) - exact).max())
    # the interpolant's own error stays below the kernel's step exp(-beta) at |x| = 1;
    # FP32 evaluation adds ~1e-7
    assert err < max(1.5 * np.exp(-beta), 1.5e-7), (W, sigma, err)


def test_polynomial_weights_taps_are_mirror_images():
    # phi is even: tap a at t equals tap W - 1 - a at -t
    lib = _native.load()
    W, beta = 8, np.pi * 8 * (1 - 0.5 / 1.5)
    c = kernel_poly(lib, W, beta)
    sign = (-1.0) ** np.arange(W + 2)
    np.testing.assert_allclose(c[::-1] * sign, c, atol=2e-7)


def test_polynomial_weights_argument_checks():
    lib = _native.load()
    out = np.zeros(18 * 16, dtype=np.float32)
    assert lib.lens_kernel_poly(3, 10.0, out.ctypes.data) == 1
    assert lib.lens_kernel_poly(17, 10.0, out.ctypes.data) == 1
    assert lib.lens_kernel_poly(8, 0.0, out.ctypes.data) == 1
    assert lib.lens_kernel_poly(8, 10.0, ctypes.c_void_p()) == 1


def horner_f64(c, t):
    acc = np.full(t.shape, np.float64(c[-1]))
    for k in range(len(c) - 2, -1, -1):
        acc = acc * t + np.float64(c[k])
    return acc


@pytest.mark.parametrize("W", list(range(4, 17)))
def test_default_beta_is_accepted(W):
    # plan creation refuses an explicit FP32 beta whose polynomials miss phi by more than
    # 4 max(e^-beta, 1e-7); the default beta = pi W (1 - 1/(2 sigma)) meets that bound with
    # a factor 2 to spare for every oversampling factor the cost model picks (1.2 .. 2.5)
    lib = _native.load()
    t = -1.0 + (np.arange(256) + 0.5) / 128.0
    for sigma in np.linspace(1.2, 2.5, 14):
        beta = np.pi * W * (1.0 - 0.5 / sigma)
        c = kernel_poly(lib, W, beta)
        err = max(np.abs(horner_f64(c[a], t) - es_kernel((0.5 * t + 0.5 * (W - 1) - a) * 2.0 / W, beta)).max()
                  for a in range(W))
        assert err < 0.5 * 4.0 * max(np.exp(-beta), 1e-7), (W, sigma, err)


def test_fp32_plan_refuses_a_beta_the_polynomials_cannot_follow():
    # the check runs before any device work, so it needs no GPU
    lib = _native.load()
    h = ctypes.c_void_p()
    prm = _native.PlanParams(1.5, 4, 16.0, 0, 0, 0, 0, 0, 0, 0, 0, 0)  # sigma, W, beta
    st = lib.lens_plan_create_ex(ctypes.byref(h), 64, 64, 0, 0, None, None, None, 1e-2, 0, 0, None,
                                 ctypes.byref(prm))
    assert st == 1
    assert b"polynomial kernel weights" in lib.lens_last_error_message()
