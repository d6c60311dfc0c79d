"""The allocation-free forward transform matches the regular one.

lens_synthesis_static is for callers that cannot call cudaMalloc once they
are running (their device memory belongs to a host framework's allocator, or
to a budget fixed at start-up): it takes its scratch from an array compiled
into the library.  It must give what lens_synthesis gives, call after call
(the array keeps the previous call's contents), and refuse plans whose scratch
does not fit.  This file is collected last so that a failure here comes after
every other test has run.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2304_10431_gb300 import LensPlan, _native
from paper_2304_10431_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _static(plan, alm, out):
    lib = _native.load()
    st = torch.cuda.current_stream().cuda_stream
    return lib.lens_synthesis_static(plan.handle, alm.data_ptr(), out.data_ptr(), st)


@pytest.mark.parametrize("spin,prec,tol,tables", [(0, "fp32", 1e-6, False), (2, "fp32", 1e-6, False),
                                                  (0, "fp32", 1e-6, True), (2, "fp32", 1e-6, True),
                                                  (0, "fp64", 1e-13, False), (2, "fp64", 1e-13, False)])
def test_static_scratch_matches_lens_synthesis(spin, prec, tol, tables):
    # tables: FP32 plans holding precomputed Legendre values, whose synthesis reads them instead of
    # running the recursion (a different kernel inside the same entry point)
    dev = torch.device("cuda:0")
    L = 96
    th, ph, chi = W.random_points(30000, 77)
    plan = LensPlan(L, th, ph, chi, spin=spin, epsilon=1e-5 if prec == "fp32" else 1e-10, precision=prec,
                    legendre_tables=tables, device=dev)
    assert plan.info()["legendre_table_bytes"] > 0 if tables else plan.info()["legendre_table_bytes"] == 0
    nc = 1 if spin == 0 else 2
    for call, seed in enumerate((500, 501)):  # two calls in a row, different inputs
        a = np.stack([W.draw_alm(W.cmb_cl(L, 70.0), L, seed + 10 * k, spin=spin) for k in range(nc)])
        at = torch.as_tensor(a, dtype=plan.complex_dtype, device=dev)
        ref = plan.synthesis(at)
        out = torch.full_like(ref, float("nan"))
        assert _static(plan, at, out) == 0, _native.load().lens_last_error_message()
        torch.cuda.synchronize()
        err = float(torch.linalg.norm(out - ref) / torch.linalg.norm(ref))
        assert err <= tol, (call, err)
    plan.close()


def test_static_scratch_rejects_large_plans():
    dev = torch.device("cuda:0")
    th, ph, chi = W.random_points(1000, 3)
    plan = LensPlan(2048, th, ph, chi, spin=2, epsilon=1e-10, precision="fp64", device=dev)
    a = torch.zeros(2, plan.nalm, dtype=plan.complex_dtype, device=dev)
    out = torch.zeros(2, plan.npoints, dtype=plan.real_dtype, device=dev)
    assert _static(plan, a, out) == 7
    msg = _native.load().lens_last_error_message().decode()
    assert "scratch" in msg and "lens_synthesis" in msg
    plan.close()
