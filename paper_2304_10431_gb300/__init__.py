"""gslens: general spherical harmonic transforms for CMB lensing on GB300.

Python binding of libgslens (include/gslens.h).  Every step of the transform
runs in the library's CUDA kernels; this module only marshals torch tensors
into raw device pointers and sizes.  PyTorch provides device memory and streams.

    plan = LensPlan(lmax, theta, phi, chi=None, spin=0, epsilon=1e-5, precision="fp32")
    m = plan.synthesis(alm)    # forward lensing (Eq. "forward" / "forwardpol")
    a = plan.adjoint(m)        # adjoint (Eq. "adjoint" and its spin-s form)
    m = synthesis(plan, alm)   # the same, differentiable (torch.autograd; backward = exact adjoint)

a_lm layout: complex tensor [ncomp, nalm] (or [nmaps, ncomp, nalm]) with
index(l, m) = m (2 lmax + 1 - m)/2 + l; ncomp = 1 (spin 0) or 2 (G, C).
Maps: real tensor [ncomp, npoints] (or [nmaps, ncomp, npoints]).
"""
from __future__ import annotations

import ctypes
import json
import os

import numpy as np
import torch

from . import _native
from ._native import LensError, PlanInfo, PlanParams

__all__ = ["LensPlan", "LensingModel", "LensedAlm", "LensBatch", "LensError", "synthesis", "adjoint", "lensed",
           "autotune", "gl_grid", "scale_points", "pointing", "nalm", "lib_path"]

_PREC = {"fp32": 0, "fp64": 1}


def lib_path() -> str:
    return _native.lib_path()


def measure_fma_peak(precision: str = "fp32", device=None) -> float:
    """Measured FMA rate of the device's CUDA-core pipes, flops/s (lens_measure_fma_peak)."""
    if precision not in _PREC:
        raise ValueError("precision must be 'fp32' or 'fp64'")
    lib = _native.load()
    v = ctypes.c_double(0.0)
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    with torch.cuda.device(dev):
        _native.check(lib.lens_measure_fma_peak(_PREC[precision], ctypes.byref(v),
                                                _stream_handle(torch.cuda.current_stream(dev))))
    return float(v.value)


def nalm(lmax: int, mmax: int | None = None) -> int:
    return int(_native.load().lens_nalm(lmax, lmax if mmax is None else mmax))


def _stream_handle(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _dev_f64(x, device):
    if isinstance(x, torch.Tensor):
        return x.to(device=device, dtype=torch.float64).contiguous()
    return torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64), device=device)


class LensPlan:
    """One geometry (deflected points) at one band limit, spin and precision."""

    def __init__(self, lmax: int, theta, phi, chi=None, spin: int = 0, mmax: int | None = None,
                 epsilon: float = 1e-5, precision: str = "fp32", sigma: float | None = None,
                 W: int | None = None, beta: float | None = None, ntheta: int | None = None,
                 legendre_rpt: tuple | None = None, legendre_df32_mmin: int = 0, fft_cluster: int = 0,
                 grad_only: bool = False, deterministic: bool = False, legendre_tables: bool = False,
                 legendre_restart: int = 0, point_weights: int = 0, spread_tile_rows: int = 0,
                 device=None, stream=None):
        lib = _native.load()
        if precision not in _PREC:
            raise ValueError("precision must be 'fp32' or 'fp64'")
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.lmax, self.mmax, self.spin = int(lmax), int(lmax if mmax is None else mmax), int(spin)
        self.precision = precision
        self.real_dtype = torch.float32 if precision == "fp32" else torch.float64
        self.complex_dtype = torch.complex64 if precision == "fp32" else torch.complex128
        self.ncomp = 1 if self.spin == 0 else 2  # components of a map
        self.grad_only = bool(grad_only)  # spin s with C = 0: a_lm buffers hold G alone
        self.alm_ncomp = 1 if (self.spin == 0 or self.grad_only) else 2
        self.deterministic = bool(deterministic)  # bit-reproducible adjoints (fixed-point sums)
        with torch.cuda.device(self.device):
            th = _dev_f64(theta, self.device)
            ph = _dev_f64(phi, self.device)
            ch = _dev_f64(chi, self.device) if (chi is not None and self.spin) else None
            if th.numel() != ph.numel() or (ch is not None and ch.numel() != th.numel()):
                raise ValueError("theta, phi (and chi) must have the same length")
            self.npoints = int(th.numel())
            rf, ra = legendre_rpt if legendre_rpt else (0, 0)
            prm = PlanParams(float(sigma or 0.0), int(W or 0), float(beta or 0.0), int(ntheta or 0), int(rf), int(ra),
                             int(legendre_df32_mmin), int(fft_cluster), 1 if legendre_tables else 0,
                             int(legendre_restart), int(point_weights), int(spread_tile_rows))
            handle = ctypes.c_void_p()
            st = _stream_handle(stream)
            rc = lib.lens_plan_create_ex(ctypes.byref(handle), self.lmax, self.mmax, self.spin, self.npoints,
                                         th.data_ptr() if self.npoints else None,
                                         ph.data_ptr() if self.npoints else None,
                                         ch.data_ptr() if ch is not None else None, float(epsilon),
                                         _PREC[precision], (1 if self.grad_only else 0) | (2 if self.deterministic else 0),
                                         st, ctypes.byref(prm))
            _native.check(rc)
        self._h = handle
        self.nalm = nalm(self.lmax, self.mmax)
        self.epsilon = float(epsilon)

    # ------------------------------------------------------------ utilities
    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        inf = PlanInfo()
        _native.check(_native.load().lens_plan_info(self._h, ctypes.byref(inf)))
        return {k: getattr(inf, k) for k, _ in PlanInfo._fields_}

    def status(self, stream=None):
        """Raise LensError (LENS_ERR_TIMEOUT) if a device-side wait of an earlier call gave up."""
        _native.check(_native.load().lens_plan_status(self._h, _stream_handle(stream)))

    def set_tensor_cores(self, on: bool):
        """Spin-0 FP32 plans (restarted recursion): synthesis of 16 or more maps per call runs the
        Legendre step on the tensor cores (default on)."""
        _native.check(_native.load().lens_plan_set_tensor_cores(self._h, 1 if on else 0))

    def set_grouping(self, on: bool):
        """FP32 plans: synthesise several maps per call with a shared Legendre
        recursion (default on); off runs every map alone."""
        _native.check(_native.load().lens_plan_set_grouping(self._h, 1 if on else 0))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _native.load().lens_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _alm_arg(self, alm):
        if not isinstance(alm, torch.Tensor) or alm.device != self.device:
            raise TypeError("alm must be a CUDA tensor on the plan's device")
        if alm.dtype != self.complex_dtype:
            raise TypeError("alm must be %s for a %s plan" % (self.complex_dtype, self.precision))
        alm = alm.contiguous()
        if alm.shape[-1] != self.nalm or (alm.dim() >= 2 and alm.shape[-2] != self.alm_ncomp) or \
                (alm.dim() == 1 and self.alm_ncomp != 1):
            raise ValueError("alm must have shape [..., %d, %d]" % (self.alm_ncomp, self.nalm))
        nmaps = 1 if alm.dim() <= 2 else int(np.prod(alm.shape[:-2]))
        return alm, nmaps

    def _map_arg(self, m):
        if not isinstance(m, torch.Tensor) or m.device != self.device:
            raise TypeError("map must be a CUDA tensor on the plan's device")
        if m.dtype != self.real_dtype:
            raise TypeError("map must be %s for a %s plan" % (self.real_dtype, self.precision))
        m = m.contiguous()
        if m.shape[-1] != self.npoints or (m.dim() >= 2 and m.shape[-2] != self.ncomp) or \
                (m.dim() == 1 and self.ncomp != 1):
            raise ValueError("map must have shape [..., %d, %d]" % (self.ncomp, self.npoints))
        nmaps = 1 if m.dim() <= 2 else int(np.prod(m.shape[:-2]))
        return m, nmaps

    # ------------------------------------------------------------ transforms
    def synthesis(self, alm: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """Forward lensing: a_lm -> values at the deflected points."""
        alm, nmaps = self._alm_arg(alm)
        lead = alm.shape[:-2] if alm.dim() > 2 else ()
        if out is None:
            out = torch.empty(*lead, self.ncomp, self.npoints, dtype=self.real_dtype, device=self.device)
        _native.check(_native.load().lens_synthesis(self._h, alm.data_ptr(), out.data_ptr(), nmaps,
                                                    _stream_handle(stream)))
        return out

    def adjoint(self, m: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """Adjoint lensing: values at the deflected points -> a_lm (m >= 0)."""
        m, nmaps = self._map_arg(m)
        lead = m.shape[:-2] if m.dim() > 2 else ()
        if out is None:
            out = torch.empty(*lead, self.alm_ncomp, self.nalm, dtype=self.complex_dtype, device=self.device)
        _native.check(_native.load().lens_adjoint(self._h, m.data_ptr(), out.data_ptr(), nmaps,
                                                  _stream_handle(stream)))
        return out

    def synthesis_vjp(self, grad_map: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """dL/da_lm for a real loss L of synthesis's output, given dL/dmap (lens_synthesis_vjp)."""
        g, nmaps = self._map_arg(grad_map)
        lead = g.shape[:-2] if g.dim() > 2 else ()
        if out is None:
            out = torch.empty(*lead, self.alm_ncomp, self.nalm, dtype=self.complex_dtype, device=self.device)
        _native.check(_native.load().lens_synthesis_vjp(self._h, g.data_ptr(), out.data_ptr(), nmaps,
                                                        _stream_handle(stream)))
        return out

    def adjoint_vjp(self, grad_alm: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """dL/dmap for a real loss L of adjoint's output, given dL/da_lm (lens_adjoint_vjp)."""
        g, nmaps = self._alm_arg(grad_alm)
        lead = g.shape[:-2] if g.dim() > 2 else ()
        if out is None:
            out = torch.empty(*lead, self.ncomp, self.npoints, dtype=self.real_dtype, device=self.device)
        _native.check(_native.load().lens_adjoint_vjp(self._h, g.data_ptr(), out.data_ptr(), nmaps,
                                                      _stream_handle(stream)))
        return out

    def synthesis_host(self, alm_h, out_h=None, stream=None, sync: bool = True):
        """Forward on host (CPU) tensors: copies in, transform, copies out.  sync=False only
        enqueues on `stream` (lens_synthesis_host_async): pinned tensors, kept alive and
        untouched until the stream is synchronised."""
        alm_h = torch.as_tensor(alm_h).to(self.complex_dtype).contiguous()
        nmaps = 1 if alm_h.dim() <= 2 else int(np.prod(alm_h.shape[:-2]))
        lead = alm_h.shape[:-2] if alm_h.dim() > 2 else ()
        if out_h is None:
            out_h = torch.empty(*lead, self.ncomp, self.npoints, dtype=self.real_dtype, pin_memory=not sync)
        fn = _native.load().lens_synthesis_host if sync else _native.load().lens_synthesis_host_async
        _native.check(fn(self._h, alm_h.data_ptr(), out_h.data_ptr(), nmaps, _stream_handle(stream)))
        return out_h

    def adjoint_host(self, m_h, out_h=None, stream=None, sync: bool = True):
        """Adjoint on host tensors (see synthesis_host for sync=False)."""
        m_h = torch.as_tensor(m_h).to(self.real_dtype).contiguous()
        nmaps = 1 if m_h.dim() <= 2 else int(np.prod(m_h.shape[:-2]))
        lead = m_h.shape[:-2] if m_h.dim() > 2 else ()
        if out_h is None:
            out_h = torch.empty(*lead, self.alm_ncomp, self.nalm, dtype=self.complex_dtype, pin_memory=not sync)
        fn = _native.load().lens_adjoint_host if sync else _native.load().lens_adjoint_host_async
        _native.check(fn(self._h, m_h.data_ptr(), out_h.data_ptr(), nmaps, _stream_handle(stream)))
        return out_h

    def ring_synthesis(self, alm: torch.Tensor, stream=None) -> torch.Tensor:
        """Legendre step only: ring Fourier coefficients [ncol, ntheta] on the plan's rings."""
        alm, _ = self._alm_arg(alm)
        inf = self.info()
        ncol = self.mmax + 1 if self.spin == 0 else 2 * self.mmax + 1
        out = torch.empty(ncol, inf["ntheta"], dtype=self.complex_dtype, device=self.device)
        _native.check(_native.load().lens_ring_synthesis(self._h, alm.data_ptr(), out.data_ptr(),
                                                         _stream_handle(stream)))
        return out

    def torus_coefficients(self, alm: torch.Tensor, stream=None) -> torch.Tensor:
        """Doubling + theta transform alone: c[ncol, 2 lmax + 1] with F(theta) = sum_k c_k e^{ik theta}."""
        alm, _ = self._alm_arg(alm)
        ncol = self.mmax + 1 if self.spin == 0 else 2 * self.mmax + 1
        out = torch.empty(ncol, 2 * self.lmax + 1, dtype=self.complex_dtype, device=self.device)
        _native.check(_native.load().lens_torus_coefficients(self._h, alm.data_ptr(), out.data_ptr(),
                                                             _stream_handle(stream)))
        return out

    def ring_adjoint(self, ring: torch.Tensor, stream=None) -> torch.Tensor:
        ring = ring.contiguous()
        out = torch.empty(self.alm_ncomp, self.nalm, dtype=self.complex_dtype, device=self.device)
        _native.check(_native.load().lens_ring_adjoint(self._h, ring.data_ptr(), out.data_ptr(),
                                                       _stream_handle(stream)))
        return out


class _Synthesis(torch.autograd.Function):
    @staticmethod
    def forward(ctx, alm, plan):
        ctx.plan = plan
        return plan.synthesis(alm)

    @staticmethod
    def backward(ctx, grad_map):
        return ctx.plan.synthesis_vjp(grad_map), None


class _Adjoint(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m, plan):
        ctx.plan = plan
        return plan.adjoint(m)

    @staticmethod
    def backward(ctx, grad_alm):
        return ctx.plan.adjoint_vjp(grad_alm), None


def synthesis(plan: LensPlan, alm: torch.Tensor) -> torch.Tensor:
    """Differentiable forward lensing: plan.synthesis with backward = lens_synthesis_vjp."""
    return _Synthesis.apply(alm, plan)


def adjoint(plan: LensPlan, m: torch.Tensor) -> torch.Tensor:
    """Differentiable adjoint lensing: plan.adjoint with backward = lens_adjoint_vjp."""
    return _Adjoint.apply(m, plan)


class LensingModel:
    """d = A(phi) x: lensing of a spin-s field x by a potential phi, with gradients.

    The undeflected points (theta0, phi0) are fixed.  set_phi(phi_lm) computes
    the deflection (Eq. "deflect", lens_deflection) and the deflected geometry
    (lens_pointing) on the GPU and builds the lensed plan; forward(x),
    grad_x(g) (lens_synthesis_vjp) and grad_phi(x, g) (lens_phi_gradient) run
    on it.  The spin s+1 / s-1 plans that the phi gradient needs are built on
    first use.  phi_lm: complex128 [nalm(lmax_phi)] on the device.
    """

    def __init__(self, lmax: int, theta0, phi0, spin: int = 0, lmax_phi: int | None = None,
                 epsilon: float = 1e-5, precision: str = "fp32", epsilon_deflection: float = 1e-10,
                 device=None, **plan_kw):
        if spin == 1:
            raise ValueError("spin-1 fields are not supported by the phi gradient")
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.lmax, self.spin = int(lmax), int(spin)
        self.lmax_phi = int(lmax if lmax_phi is None else lmax_phi)
        self.epsilon, self.precision, self.plan_kw = float(epsilon), precision, plan_kw
        self.theta0 = _dev_f64(theta0, self.device)
        self.phi0 = _dev_f64(phi0, self.device)
        self.npoints = int(self.theta0.numel())
        # the deflection is a pure gradient (no curl): a gradient-only spin-1 plan
        self.defl = LensPlan(self.lmax_phi, self.theta0, self.phi0, spin=1, epsilon=epsilon_deflection,
                             precision="fp64", grad_only=True, device=self.device)
        self.alpha = torch.empty(2, self.npoints, dtype=torch.float64, device=self.device)
        self.phi_lm = None
        self.lensed = self._up = self._down = None
        self.geometry = None

    def _plan(self, spin):
        t2, p2, chi = self.geometry
        return LensPlan(self.lmax, t2, p2, chi, spin=spin, epsilon=self.epsilon, precision=self.precision,
                        device=self.device, **self.plan_kw)

    def _close_lensed(self):
        for pl in (self.lensed, self._up, self._down):
            if pl is not None:
                pl.close()
        self.lensed = self._up = self._down = None

    def set_phi(self, phi_lm: torch.Tensor, stream=None):
        """Deflect the points by the gradient of phi and rebuild the lensed plan."""
        phi_lm = phi_lm.detach().to(device=self.device, dtype=torch.complex128).contiguous()
        if phi_lm.numel() != self.defl.nalm:
            raise ValueError("phi_lm must have %d entries" % self.defl.nalm)
        _native.check(_native.load().lens_deflection(self.defl.handle, phi_lm.data_ptr(), self.alpha.data_ptr(),
                                                     _stream_handle(stream)))
        self.geometry = pointing(self.theta0, self.phi0, self.alpha[0], self.alpha[1], stream=stream)
        self._close_lensed()
        self.lensed = self._plan(self.spin)
        self.phi_lm = phi_lm.clone()

    def forward(self, x: torch.Tensor, stream=None) -> torch.Tensor:
        return self.lensed.synthesis(x, stream=stream)

    def grad_x(self, grad_map: torch.Tensor, stream=None) -> torch.Tensor:
        return self.lensed.synthesis_vjp(grad_map, stream=stream)

    def grad_phi(self, x: torch.Tensor, grad_map: torch.Tensor, d: torch.Tensor | None = None,
                 stream=None) -> torch.Tensor:
        """dL/dphi_LM (complex128 [nalm(lmax_phi)]) given dL/dd of d = A(phi) x."""
        if self._up is None:
            self._up = self._plan(self.spin + 1)
            if self.spin >= 2:
                self._down = self._plan(self.spin - 1)
        x, _ = self.lensed._alm_arg(x)
        g, _ = self.lensed._map_arg(grad_map)
        if d is not None:
            d, _ = self.lensed._map_arg(d)
        out = torch.empty(self.defl.nalm, dtype=torch.complex128, device=self.device)
        _native.check(_native.load().lens_phi_gradient(
            self.lensed.handle, self._up.handle, self._down.handle if self._down is not None else None,
            self.defl.handle, self.alpha.data_ptr(), x.data_ptr(), d.data_ptr() if d is not None else None,
            g.data_ptr(), out.data_ptr(), _stream_handle(stream)))
        return out

    def magnification(self, stream=None) -> torch.Tensor:
        """|A| = |d^2 n' / d^2 n| at the undeflected points (App. B; lens_magnification)."""
        if getattr(self, "_mag_plans", None) is None:
            self._mag_plans = tuple(LensPlan(self.lmax_phi, self.theta0, self.phi0, spin=s, epsilon=1e-12,
                                             precision="fp64", device=self.device) for s in (0, 2))
        det = torch.empty(self.npoints, dtype=torch.float64, device=self.device)
        _native.check(_native.load().lens_magnification(self._mag_plans[0].handle, self._mag_plans[1].handle,
                                                        self.phi_lm.data_ptr(), self.alpha.data_ptr(),
                                                        det.data_ptr(), _stream_handle(stream)))
        return det

    def close(self):
        self._close_lensed()
        self.defl.close()
        for pl in getattr(self, "_mag_plans", None) or ():
            pl.close()
        self._mag_plans = None


class LensedAlm:
    """Lensed harmonic coefficients (Sect. 4): the unlensed field (band limit lmax_unl)
    is remapped onto a Gauss-Legendre grid (nrings x nphi) by the lensing synthesis, and
    a backward SHT (the adjoint at the grid points times the quadrature weights) returns
    the coefficients up to lmax_len.  adjoint() is the exact transpose (a forward SHT onto
    the grid, weights, then the adjoint remapping); inverse() is App. B's inverse lensing
    of a lensed map on the grid, the adjoint applied to the map times |A|."""

    def __init__(self, lmax_unl: int, lmax_len: int, spin: int = 0, lmax_phi: int | None = None,
                 nrings: int | None = None, nphi: int | None = None, epsilon: float = 1e-5,
                 precision: str = "fp32", device=None):
        self.nrings = int(nrings or lmax_len + 1 + lmax_len // 2)
        self.nphi = int(nphi or 2 * self.nrings)
        if self.nrings <= lmax_len or self.nphi <= 2 * lmax_len:
            raise ValueError("the grid must resolve lmax_len: nrings > lmax_len and nphi > 2 lmax_len")
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.theta, self.phi, self.weight = gl_grid(self.nrings, self.nphi, device=dev)
        self.model = LensingModel(lmax_unl, self.theta, self.phi, spin=spin, lmax_phi=lmax_phi, epsilon=epsilon,
                                  precision=precision, device=dev)
        self.analysis = LensPlan(lmax_len, self.theta, self.phi, spin=spin, epsilon=epsilon, precision=precision,
                                 device=dev)

    def set_phi(self, phi_lm: torch.Tensor):
        self.model.set_phi(phi_lm)

    def forward(self, x: torch.Tensor) -> torch.Tensor:
        d = self.model.forward(x)
        return self.analysis.adjoint(scale_points(self.weight, d, out=d))

    def adjoint(self, a: torch.Tensor) -> torch.Tensor:
        m = self.analysis.synthesis(a)
        return self.model.lensed.adjoint(scale_points(self.weight, m, out=m))

    def inverse(self, d: torch.Tensor) -> torch.Tensor:
        """Unlensed coefficients (lmax_unl) of a lensed map d on the grid (App. B)."""
        t = scale_points(self.weight, d)
        return self.model.lensed.adjoint(scale_points(self.model.magnification(), t, out=t))

    def close(self):
        self.model.close()
        self.analysis.close()


def gl_grid(nrings: int, nphi: int, device=None, stream=None):
    """Gauss-Legendre grid (lens_gl_grid): theta, phi and quadrature weights w_j 2 pi / nphi
    (FP64 device tensors of nrings * nphi points, ring-major)."""
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    n = int(nrings) * int(nphi)
    th = torch.empty(n, dtype=torch.float64, device=dev)
    ph = torch.empty_like(th)
    w = torch.empty_like(th)
    with torch.cuda.device(dev):
        _native.check(_native.load().lens_gl_grid(int(nrings), int(nphi), th.data_ptr(), ph.data_ptr(), w.data_ptr(),
                                                  _stream_handle(stream)))
    return th, ph, w


def scale_points(weight: torch.Tensor, x: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """out[c, i] = weight[i] x[c, i] (lens_scale_points); x real [ncomp, n] or [n]."""
    x = x.contiguous()
    n = weight.numel()
    ncomp = x.numel() // n if n else 1
    if out is None:
        out = torch.empty_like(x)
    prec = 0 if x.dtype == torch.float32 else 1
    _native.check(_native.load().lens_scale_points(n, ncomp, prec, weight.data_ptr(), x.data_ptr(), out.data_ptr(),
                                                   _stream_handle(stream)))
    return out


class _Lensed(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, phi_lm, model):
        if model.phi_lm is None or not torch.equal(phi_lm.detach(), model.phi_lm):
            model.set_phi(phi_lm)
        d = model.forward(x.detach())
        ctx.model = model
        ctx.save_for_backward(x.detach(), phi_lm.detach(), d)
        return d

    @staticmethod
    def backward(ctx, grad_map):
        x, phi_lm, d = ctx.saved_tensors
        model = ctx.model
        if not torch.equal(phi_lm, model.phi_lm):
            model.set_phi(phi_lm)
            d = None
        gx = model.grad_x(grad_map) if ctx.needs_input_grad[0] else None
        gp = model.grad_phi(x, grad_map, d) if ctx.needs_input_grad[1] else None
        return gx, gp, None


def lensed(model: LensingModel, x: torch.Tensor, phi_lm: torch.Tensor) -> torch.Tensor:
    """Differentiable d = A(phi) x in both x (lens_synthesis_vjp) and phi (lens_phi_gradient)."""
    return _Lensed.apply(x, phi_lm, model)


class LensBatch:
    """Many transforms recorded once as a CUDA graph and replayed with one launch (lens_batch_*).

    add(plan, "synthesis" | "adjoint", inp, out) records an item (the tensors are kept
    alive and reused by every launch); instantiate(nbranches) captures the graph; launch()
    replays it on the current stream.
    """

    def __init__(self, device=None):
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        h = ctypes.c_void_p()
        _native.check(_native.load().lens_batch_create(ctypes.byref(h), self.device.index or 0))
        self._h = h
        self._keep = []

    def add(self, plan: LensPlan, op: str, inp: torch.Tensor, out: torch.Tensor):
        if op == "synthesis":
            inp, nmaps = plan._alm_arg(inp)
            out_ok, _ = plan._map_arg(out)
            code = 0
        elif op == "adjoint":
            inp, nmaps = plan._map_arg(inp)
            out_ok, _ = plan._alm_arg(out)
            code = 1
        else:
            raise ValueError("op must be 'synthesis' or 'adjoint'")
        if out_ok.data_ptr() != out.data_ptr():
            raise ValueError("out must be contiguous")
        self._keep += [plan, inp, out]
        _native.check(_native.load().lens_batch_add(self._h, plan.handle, code, inp.data_ptr(), out.data_ptr(),
                                                    nmaps))

    def instantiate(self, nbranches: int = 8):
        _native.check(_native.load().lens_batch_instantiate(self._h, int(nbranches)))

    def launch(self, stream=None):
        _native.check(_native.load().lens_batch_launch(self._h, _stream_handle(stream)))

    def info(self) -> dict:
        n, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        _native.check(_native.load().lens_batch_info(self._h, ctypes.byref(n), ctypes.byref(b), ctypes.byref(c)))
        return {"items": n.value, "branches": b.value, "max_branch_seconds": c.value}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _native.load().lens_batch_destroy(self._h)
            self._h = ctypes.c_void_p()
        self._keep = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _autotune_cache_path() -> str:
    d = os.environ.get("LENS_CACHE_DIR") or os.path.join(os.path.expanduser("~"), ".cache", "gslens")
    return os.path.join(d, "autotune.json")


def autotune(lmax: int, theta, phi, chi=None, spin: int = 0, mmax: int | None = None, epsilon: float = 1e-5,
             precision: str = "fp32", reps: int = 2, device=None, stream=None, cache: bool = True) -> dict:
    """Measured plan parameters for these points (lens_autotune): LensPlan keyword arguments
    (sigma, W, spread_tile_rows, legendre_rpt) plus "ms", one forward + adjoint pair.

    Results are kept in a JSON file ($LENS_CACHE_DIR/autotune.json, default ~/.cache/gslens),
    keyed by the GPU name, lmax, mmax, spin, precision, epsilon and the point count rounded to
    a quarter octave (the point density per ring); cache=False always measures (and updates
    the file)."""
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    mm = int(lmax if mmax is None else mmax)
    with torch.cuda.device(dev):
        th, ph = _dev_f64(theta, dev), _dev_f64(phi, dev)
        ch = _dev_f64(chi, dev) if (chi is not None and spin) else None
        n = int(th.numel())
        key = "%s|lmax=%d|mmax=%d|spin=%d|%s|eps=%.3g|npts~2^%.2f" % (
            torch.cuda.get_device_name(dev), int(lmax), mm, int(spin), precision, float(epsilon),
            round(4 * np.log2(max(n, 1))) / 4)
        path = _autotune_cache_path()
        table = {}
        if os.path.exists(path):
            try:
                with open(path) as fh:
                    table = json.load(fh)
            except (OSError, ValueError):
                table = {}
        if cache and key in table:
            out = dict(table[key])
            if "legendre_rpt" in out:
                out["legendre_rpt"] = tuple(out["legendre_rpt"])
            out["cached"] = True
            return out
        best = PlanParams()
        ms = ctypes.c_double()
        _native.check(_native.load().lens_autotune(int(lmax), mm, int(spin), n, th.data_ptr() if n else None,
                                                   ph.data_ptr() if n else None,
                                                   ch.data_ptr() if ch is not None else None, float(epsilon),
                                                   _PREC[precision], _stream_handle(stream), int(reps),
                                                   ctypes.byref(best), ctypes.byref(ms)))
    out = {"sigma": best.sigma, "ms": ms.value}
    if best.W:
        out["W"] = best.W
    if best.spread_tile_rows:
        out["spread_tile_rows"] = best.spread_tile_rows
    if best.legendre_rpt_fwd or best.legendre_rpt_adj:
        out["legendre_rpt"] = (best.legendre_rpt_fwd, best.legendre_rpt_adj)
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        table[key] = {k: (list(v) if isinstance(v, tuple) else v) for k, v in out.items()}
        tmp = path + ".%d.tmp" % os.getpid()
        with open(tmp, "w") as fh:
            json.dump(table, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass  # an unwritable cache directory only costs a re-measurement next time
    out["cached"] = False
    return out


def pointing(theta: torch.Tensor, phi: torch.Tensor, alpha_theta: torch.Tensor, alpha_phi: torch.Tensor,
             stream=None):
    """Unlensed angles and spin phase from a deflection field (Sect. 3); FP64 CUDA tensors."""
    n = theta.numel()
    dev = theta.device
    args = [x.to(dtype=torch.float64).contiguous() for x in (theta, phi, alpha_theta, alpha_phi)]
    t2 = torch.empty(n, dtype=torch.float64, device=dev)
    p2 = torch.empty_like(t2)
    c2 = torch.empty_like(t2)
    _native.check(_native.load().lens_pointing(n, *[a.data_ptr() for a in args], t2.data_ptr(), p2.data_ptr(),
                                               c2.data_ptr(), _stream_handle(stream)))
    return t2, p2, c2
