#!/usr/bin/env python
"""Benchmark: lensed points/sec of the general-SHT lensing pair on GB300.

Workload (headline): lmax 4096, HEALPix Nside 2048 (50,331,648 points)
deflected along the gradient of a lensing potential (phi lmax 4096,
C_L^phiphi ~ (L+1)^-4 rescaled to 2.5 arcmin rms), CMB a_lm drawn from
C_l = (l+10)^-2 exp(-(l/2990)^2).  One step = the whole hot path on that
geometry: spin-0 T synthesis + adjoint, spin-2 E/B -> Q/U synthesis + adjoint.
value = points / step time (FP32 plans, epsilon 1e-5, Legendre functions by the
restarted FP32 recursion); the same step with plan-time Legendre tables
("tables"), the FP64 plans (epsilon 1e-10, "fp64") and the lmax 5120 workload
of the paper's Fig. 2 ("lmax5120") are measured in the same run.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gslens|reference]

Deflected coordinates are computed on the GPU with the library itself (spin-1
synthesis of sqrt(L(L+1)) phi_LM at the HEALPix centres, then the pointing
kernel) and, like plan creation, are outside the timed region, as in the
paper's benchmarks.  --impl reference times the FP64 CPU oracle on a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

HBM_PEAK_FALLBACK = 6800.0
FP32_LANES_PER_SM = 128
NUM_SMS = 152

STAGES = ["legendre_synthesis", "theta_fwd", "phi_fwd", "interp", "spread", "phi_adj", "theta_adj",
          "legendre_adjoint"]
KERNEL_FILES = {"legendre_synthesis": "legendre.cu", "legendre_adjoint": "legendre.cu", "theta_fwd": "torus.cu",
                "theta_adj": "torus.cu", "phi_fwd": "torus.cu", "phi_adj": "torus.cu", "interp": "nufft.cu",
                "spread": "nufft.cu"}
# DRAM bytes per launch from one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum),
# keyed by (slot name, sha1 of the kernel's source file at capture time).  A changed
# source makes the entry stale and the bench reports traffic null.
NCU_TRAFFIC = {
    # df32-recursion adjoint, spin 2, lmax 4096 (capture of the kernel alone on a small point set)
    ("legendre_adjoint/spin2/fp32", "d846cc9777e2"): 741691904,
    # table adjoint: lmax 2048 capture (12.756 GB for 11.977 GB of table + a_lm + ring bytes, ratio 1.065)
    # scaled to lmax 4096's 92.75 GB of table + a_lm + ring bytes
    ("legendre_adjoint_tables/spin2/fp32", "4df24e5ff172"): 98778851588,
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gslens", choices=["gslens", "reference"])
    ap.add_argument("--lmax", type=int, default=4096)
    ap.add_argument("--nside", type=int, default=2048)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--sigma", type=float, default=None,
                    help="force the NUFFT oversampling factor of the FP32 plans (small profiling cases)")
    ap.add_argument("--no-tables-compare", action="store_true",
                    help="skip the extra measurement of the FP32 step with Legendre-table plans")
    ap.add_argument("--tables", action="store_true",
                    help="headline FP32 plans read plan-time Legendre tables instead of running the recursion")
    ap.add_argument("--no-lmax5120", action="store_true",
                    help="skip the lmax 5120 workload (paper's Fig. 2 configuration)")
    ap.add_argument("--tc-maps", default="32,64",
                    help="batched T synthesis with the tensor-core Legendre step: comma list of map counts "
                         "('' to skip)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-seconds", type=float, default=150.0,
                    help="oracle time budget of the whole --impl reference run")
    ap.add_argument("--scan", default=None,
                    help="N_side x lmax scan (the paper's Fig. 4): comma list of NSIDE:LMAX pairs; prints one JSON "
                         "line per pair and precision instead of the benchmark line")
    ap.add_argument("--scan-eps", default="fp32:1e-5,fp64:1e-13")
    return ap.parse_args()


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": HBM_PEAK_FALLBACK, "sm_max_mhz": 2070.0}, "fallback"


def src_hash(fname):
    with open(os.path.join(ROOT, "paper_2304_10431_gb300", "csrc", fname), "rb") as f:
        return hashlib.sha1(f.read()).hexdigest()[:12]


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), "gslens_clocks_%d.csv" % os.getpid())

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ workload
def alm_inputs(lmax):
    from paper_2304_10431_gb300 import workloads as W
    ld = 0.73 * lmax
    cl = W.cmb_cl(lmax, ld)
    aT = W.draw_alm(cl, lmax, 1000)[None]
    aEB = np.stack([W.draw_alm(cl, lmax, 1001, spin=2), W.draw_alm(cl, lmax, 1002, spin=2)])
    return aT, aEB, ld


def workload_arrays(lmax, nside):
    from paper_2304_10431_gb300 import workloads as W
    th0, ph0 = W.healpix_centres(nside)
    phi_lm = W.draw_alm(W.phi_cl(lmax), lmax, 2000)
    aT, aEB, ld = alm_inputs(lmax)
    return th0, ph0, phi_lm, aT, aEB, ld


def deflect_on_gpu(th0, ph0, phi_lm, lmax, dev):
    """Lensed geometry with the library: Eq. "deflect" (spin-1 synthesis) + pointing."""
    import torch
    from paper_2304_10431_gb300 import LensPlan, pointing
    from paper_2304_10431_gb300 import workloads as W
    ell = W.alm_l_of_index(lmax)
    g = np.stack([phi_lm * np.sqrt(ell * (ell + 1.0)), np.zeros_like(phi_lm)])
    t0 = torch.as_tensor(th0, device=dev)
    p0 = torch.as_tensor(ph0, device=dev)
    plan = LensPlan(lmax, t0, p0, spin=1, epsilon=1e-10, precision="fp64", device=dev)
    alpha = plan.synthesis(torch.as_tensor(g, dtype=torch.complex128, device=dev))
    plan.close()
    th, ph, chi = pointing(t0, p0, alpha[0], alpha[1])
    del alpha
    return th, ph, chi


def legendre_triples(lmax, spin, nnorth):
    """Dense (ring pair, l, m) triple count of one Legendre step."""
    tot = 0
    for m in range(lmax + 1):
        l0 = max(m, spin)
        tot += max(lmax - l0 + 1, 0)
    return tot * nnorth


def stage_units(info, npts, spin, prec):
    """Algorithmic work per launch of each stage: flops for the Legendre recursion (8 per spin-0
    triple, 24 per spin-s triple, non-negligible triples as the plan counted them, else the dense
    count), bytes otherwise; a plan with Legendre tables streams table + coefficients + ring
    coefficients."""
    esz = 8 if prec == "fp32" else 16  # complex element
    rsz = esz // 2
    L, nt, ncol = info["lmax"], info["ntheta"], (2 * info["mmax"] + 1 if spin else info["mmax"] + 1)
    R, N2 = info["rows_kept"], info["n2"]
    gsz = rsz * (2 if spin else 1)
    nnorth = (nt + 1) // 2
    triples = info.get("legendre_triples") or legendre_triples(L, spin, nnorth)
    leg_flops = 8 * (3 if spin else 1) * triples
    ring_b = ncol * nt * esz
    x_b = R * ncol * esz
    grid_b = R * N2 * gsz
    pt_b = npts * (4 + esz + 4 + (esz if spin else 0) + rsz * (2 if spin else 1))
    nalm = (info["mmax"] + 1) * (2 * L + 2 - info["mmax"]) // 2
    alm_b = info["alm_ncomp"] * esz * nalm
    tab_b = info.get("legendre_table_bytes", 0)
    leg = ("hbm", tab_b + alm_b + ring_b, "GB/s") if tab_b else ("alu", leg_flops, "TFLOP/s")
    return {
        "legendre_synthesis": leg,
        "legendre_adjoint": leg,
        "theta_fwd": ("hbm", ring_b + x_b, "GB/s"),
        "theta_adj": ("hbm", ring_b + x_b, "GB/s"),
        "phi_fwd": ("hbm", x_b + grid_b, "GB/s"),
        "phi_adj": ("hbm", x_b + grid_b, "GB/s"),
        "interp": ("hbm", grid_b + pt_b, "GB/s"),
        "spread": ("hbm", 2 * grid_b + pt_b, "GB/s"),
    }


def fp64_arithmetic(info):
    """What the FP64 plan's steps compute in (the Legendre part depends on epsilon)."""
    if info["legendre_restart"]:
        leg = ("double-float (pairs of FP32) Legendre recursion and sums for every order, restarted from "
               "FP64-recursion values every 16 / 64 / %d degrees (low / middle / other orders)"
               % info["legendre_restart"])
    else:
        leg = ("FP64 Legendre recursion for orders m < %d, double-float (pairs of FP32) above"
               % info["legendre_df32_mmin"])
    taps = ("double-float interpolation and spreading taps (64-bit integer spreading tiles)"
            if info["epsilon"] >= 5e-11 and info["point_weight_bytes"] else "FP64 interpolation and spreading taps")
    return leg + "; FP64 FFTs and kernel weights; " + taps


def kernel_launches(info, prec):
    """Kernels one synthesis + one adjoint launch on a (non-deterministic) plan: synthesis = coefficient
    preparation (twice for the restarted FP32 recursion: plain and monic coefficients), Legendre, theta,
    phi, interpolation; adjoint = the map's largest |value| (fixed-point spreading tiles: FP32 plans at
    epsilon >= 1e-5, FP64 plans), spreading, phi, theta, Legendre; FP64 plans with FP64 low orders split
    each Legendre step into two launches (memsets not counted)."""
    leg = 2 if (prec == "fp64" and 0 < info["legendre_df32_mmin"] <= info["mmax"]) else 1
    prep = 2 if (prec == "fp32" and info["legendre_restart"] and not info["legendre_table_bytes"]) else 1
    det = bool(info["flags"] & 2)
    maxabs = 1 if (not det and (prec == "fp64" or info["epsilon"] >= 1e-5)) else 0
    return (prep + 3 + leg) + (maxabs + 3 + leg)


# ------------------------------------------------------------------ ranks
# One process per GPU (torchrun); the transform does not shard, so ranks are
# independent replicas: they meet only at the barriers around the timed region
# and in the max over ranks of each time.
def rank_env():
    """(world, rank, local rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(value, world, device):
    """Largest `value` over the ranks (the slowest replica's time)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, units_per_rank, ms):
    """Units all ranks processed per second, from the slowest rank's time per step."""
    return world * units_per_rank / (ms * 1e-3)


# ------------------------------------------------------------------ GPU arm
def analyze(prof_ms, cnt, steps, units, slot0, peaks, prec):
    """Stage rows of one profiled timed region (slots slot0 .. slot0 + 15: spin 0 then spin s) and the
    roofline of its dominant kernel.  ALU work is divided by the measured FP32 FMA rate (the FP64
    plans' Legendre kernels run their orders m >= m_df in double-float on the FP32 pipes; their
    native-FP64 orders are a small share), bytes by the measured copy bandwidth."""
    rows = []
    for slot in range(slot0, slot0 + 16):
        if cnt[slot] == 0:
            continue
        sp = (slot - slot0) // 8
        name = STAGES[slot % 8]
        avg = prof_ms[slot] / cnt[slot]
        bound, work, unit = units[sp][name]
        rows.append((prof_ms[slot] / steps, name, sp, avg, bound, work, unit, int(cnt[slot])))
    rows.sort(reverse=True)
    _, name, sp, avg, bound, work, unit, _ = rows[0]
    if bound == "alu":
        peak, achieved, note = peaks["fp32_tflops"], work / (avg * 1e-3) / 1e12, peaks["fp32_note"]
    else:
        peak, achieved, note = peaks["hbm_gbs"], work / (avg * 1e-3) / 1e9, peaks["hbm_note"]
    roof = {"bound": bound, "achieved": round(achieved, 3), "peak": round(peak, 1), "unit": unit,
            "frac": round(achieved / peak, 4), "traffic": None,
            "kernel": "%s (spin %d, %s)" % (name, 2 if sp else 0, prec), "avg_launch_ms": round(avg, 4),
            "peak_source": note, "slot": (name, sp)}
    stages = [{"stage": r[1], "spin": 2 if r[2] else 0, "ms_per_step": round(r[0], 4),
               "avg_launch_ms": round(r[3], 4), "bound": r[4],
               "achieved": round(r[5] / (r[3] * 1e-3) / (1e12 if r[4] == "alu" else 1e9), 2),
               "unit": r[6], "frac": round(r[5] / (r[3] * 1e-3) / (1e12 * peaks["fp32_tflops"] if r[4] == "alu"
                                                                    else 1e9 * peaks["hbm_gbs"]), 4)}
              for r in rows]
    t_roof = 1e3 * sum(r[5] / (peaks["fp32_tflops"] * 1e12 if r[4] == "alu" else peaks["hbm_gbs"] * 1e9) * r[7] / steps
                       for r in rows)
    return stages, roof, t_roof


def run_gpu(args):
    import torch
    import torch.distributed as dist
    from paper_2304_10431_gb300 import LensPlan, _native, lib_path, measure_fma_peak

    world, rank, local = rank_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    lib = _native.load()
    mp, peak_src = load_peaks()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # FMA rates of the CUDA-core pipes, measured here (the Legendre recursion's roofline denominator)
    clk = ClockSampler(local)
    clk.start()
    time.sleep(0.5)  # the sampler's first lines
    fma32 = max(measure_fma_peak("fp32") for _ in range(3))
    fma64 = max(measure_fma_peak("fp64") for _ in range(2))
    fma_clocks = clk.stop()
    peaks = {"hbm_gbs": float(mp.get("hbm_gbs", HBM_PEAK_FALLBACK)),
             "hbm_note": "HBM copy bandwidth (MEASURED_PEAKS.json, %s)" % peak_src,
             "fp32_tflops": fma32 / 1e12,
             "fp32_note": "FP32 FMA rate measured by lens_measure_fma_peak in this run (fma chains on every SM)"}
    measured_peaks = {"fp32_fma_tflops": round(fma32 / 1e12, 2), "fp64_fma_tflops": round(fma64 / 1e12, 3),
                      "clocks": fma_clocks, "hbm_gbs": peaks["hbm_gbs"], "hbm_source": peak_src}

    lmax, nside = args.lmax, args.nside
    th0, ph0, phi_lm, aT, aEB, ld = workload_arrays(lmax, nside)
    npts = th0.size
    th, ph, chi = deflect_on_gpu(th0, ph0, phi_lm, lmax, dev)

    def make(prec, eps, tables=False, L=None, geom=None, alms=None):
        L = L or lmax
        gth, gph, gchi = geom or (th, ph, chi)
        at, aeb = alms or (aT, aEB)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sg = args.sigma if prec == "fp32" else None
        pT = LensPlan(L, gth, gph, spin=0, epsilon=eps, precision=prec, legendre_tables=tables, sigma=sg, device=dev)
        pP = LensPlan(L, gth, gph, gchi, spin=2, epsilon=eps, precision=prec, legendre_tables=tables, sigma=sg,
                      device=dev)
        torch.cuda.synchronize()
        make.plan_s = time.perf_counter() - t0
        ct = pT.complex_dtype
        a_T = torch.as_tensor(at, dtype=ct, device=dev)
        a_P = torch.as_tensor(aeb, dtype=ct, device=dev)
        mT = pT.synthesis(a_T)
        mP = pP.synthesis(a_P)
        bufs = dict(a_T=a_T, a_P=a_P, m_T=mT, m_P=mP, o_mT=torch.empty_like(mT), o_mP=torch.empty_like(mP),
                    o_aT=torch.empty_like(a_T), o_aP=torch.empty_like(a_P))
        return pT, pP, bufs

    def step(pT, pP, b):
        pT.synthesis(b["a_T"], out=b["o_mT"])
        pT.adjoint(b["m_T"], out=b["o_aT"])
        pP.synthesis(b["a_P"], out=b["o_mP"])
        pP.adjoint(b["m_P"], out=b["o_aP"])

    stream = torch.cuda.current_stream()

    def timed(pT, pP, b, steps, warmup, profile, nvtx_name):
        for _ in range(warmup):
            step(pT, pP, b)
        barrier()
        lib.lens_profile_reset()
        if profile:
            lib.lens_profile_enable(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push(nvtx_name)
        e0.record(stream)
        for _ in range(steps):
            step(pT, pP, b)
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        lib.lens_profile_enable(0)
        return max_over_ranks(e0.elapsed_time(e1) / steps, world, dev)

    def profile_read():
        pm = np.zeros(32)
        cn = np.zeros(32, dtype=np.int64)
        lib.lens_profile_read(pm.ctypes.data, cn.ctypes.data, 32)
        return pm, cn

    def per_transform(pT, pP, b, reps=3, n=None):
        out = {}
        for name, fn in (("T_synthesis", lambda: pT.synthesis(b["a_T"], out=b["o_mT"])),
                         ("T_adjoint", lambda: pT.adjoint(b["m_T"], out=b["o_aT"])),
                         ("EB_synthesis", lambda: pP.synthesis(b["a_P"], out=b["o_mP"])),
                         ("EB_adjoint", lambda: pP.adjoint(b["m_P"], out=b["o_aP"]))):
            fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            out[name] = round((n or npts) / (e0.elapsed_time(e1) / reps * 1e-3), 1)
        return out

    def leg_mode(info):
        if info["legendre_table_bytes"]:
            return {"mode": "tables", "bytes": info["legendre_table_bytes"]}
        if info["legendre_restart"]:
            return {"mode": "restarted FP32 recursion" if info["prec"] == 0 else "restarted double-float recursion",
                    "restart_every": info["legendre_restart"], "restart_bytes": info["restart_bytes"],
                    "triples": info["legendre_triples"]}
        return {"mode": "double-float recursion" if info["prec"] == 0 else "FP64 + double-float recursion",
                "df32_from_m": info["legendre_df32_mmin"]}

    # ---------------- FP32 headline: restarted FP32 Legendre recursion (--tables: plan-time tables)
    tables = bool(args.tables)
    pT, pP, b = make("fp32", 1e-5, tables)
    plan_s = make.plan_s
    info_T, info_P = pT.info(), pP.info()
    clk = ClockSampler(local)
    clk.start()
    ms = timed(pT, pP, b, args.steps, max(args.warmup, 3), profile=True, nvtx_name="timed_fp32")
    clocks = clk.stop()
    pm, cn = profile_read()
    pt = per_transform(pT, pP, b)
    units = {0: stage_units(info_T, npts, 0, "fp32"), 1: stage_units(info_P, npts, 2, "fp32")}
    stages, roofline, t_roof = analyze(pm, cn, args.steps, units, 0, peaks, "fp32")
    name, sp = roofline.pop("slot")
    key = ("%s%s/spin%d/fp32" % (name, "_tables" if tables else "", 2 if sp else 0), src_hash(KERNEL_FILES[name]))
    roofline["traffic"] = NCU_TRAFFIC.get(key)
    step_roofline = {"t_roof_ms": round(t_roof, 3), "t_measured_ms": round(ms, 3), "frac": round(t_roof / ms, 4),
                     "rule": "sum over stages of work / peak of the stage's bound (HBM bytes at %.1f GB/s, %s; "
                             "FP32 FMA flops at the measured %.1f TFLOP/s)" % (peaks["hbm_gbs"], peak_src,
                                                                               peaks["fp32_tflops"])}
    gpu_launches = (kernel_launches(info_T, "fp32") + kernel_launches(info_P, "fp32")) * args.steps

    # ---------------- e2e through the host-buffer entry points (pinned memory)
    e2e = None
    if not args.no_e2e:
        import torch as _t
        hT = b["a_T"].cpu().pin_memory()
        hP = b["a_P"].cpu().pin_memory()
        hmT = b["m_T"].cpu().pin_memory()
        hmP = b["m_P"].cpu().pin_memory()
        o_mT, o_mP = _t.empty_like(hmT).pin_memory(), _t.empty_like(hmP).pin_memory()
        o_aT, o_aP = _t.empty_like(hT).pin_memory(), _t.empty_like(hP).pin_memory()

        # T on one stream and E/B on another (lens_*_host_async): each field's copies overlap
        # the other's kernels; the step ends when both streams have finished
        s1, s2 = _t.cuda.Stream(), _t.cuda.Stream()

        def hstep():
            pT.synthesis_host(hT, o_mT, stream=s1, sync=False)
            pT.adjoint_host(hmT, o_aT, stream=s1, sync=False)
            pP.synthesis_host(hP, o_mP, stream=s2, sync=False)
            pP.adjoint_host(hmP, o_aP, stream=s2, sync=False)
            s1.synchronize()
            s2.synchronize()

        for _ in range(max(args.warmup, 3)):
            hstep()
        barrier()
        # wall time of every step (each host call returns after its stream finished);
        # the median over the steps, max over ranks, is the reported figure
        times = []
        for _ in range(max(args.steps, 10)):
            t0 = time.perf_counter()
            hstep()
            barrier()
            times.append((time.perf_counter() - t0) * 1e3)
        ems = max_over_ranks(float(np.median(times)), world, dev)
        h2d = sum(x.numel() * x.element_size() for x in (hT, hP, hmT, hmP))
        e2e = {"value": round(whole_job_rate(world, npts, ems), 1), "unit": "lensed points/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(h2d), "ms_per_step": round(ems, 3),
               "statistic": "median of %d steps" % len(times), "ms_mean": round(float(np.mean(times)), 3),
               "api": "lens_synthesis_host_async / lens_adjoint_host_async, T and E/B on two streams",
               "ms_min": round(float(np.min(times)), 3), "ms_max": round(float(np.max(times)), 3),
               "ms_all": [round(t, 2) for t in times]}
    del b
    pP.close()
    torch.cuda.empty_cache()

    # ---------------- many T maps of the same geometry: Legendre step on the tensor cores
    tc = None
    if args.tc_maps and not tables:
        tc = {"what": "synthesis of nm spin-0 maps in one lens_synthesis call (T plan of the headline); the "
                      "Legendre step runs on the tensor cores (tcgen05 kind::tf32, hi/lo split: 3 MMAs per term), "
                      "32 maps per launch; the Fourier stages and interpolation per map",
              "peak_tf32_tflops": round(mp.get("bf16_tflops", 1900.0) * 1.1 / 2.25, 1),
              "peak_source": "measured bf16 burst (MEASURED_PEAKS.json) x nominal TF32/BF16 ratio 1.1/2.25",
              "legs": []}
        rng = np.random.default_rng(7)
        for nm in [int(v) for v in args.tc_maps.split(",") if v]:
            a = torch.zeros(nm, 1, pT.nalm, dtype=pT.complex_dtype, device=dev)
            a.real.normal_()
            a.imag.normal_()
            out = torch.empty(nm, 1, npts, dtype=torch.float32, device=dev)
            res = {"maps": nm}
            for on in (True, False):
                pT.set_tensor_cores(on)
                pT.synthesis(a, out=out)
                barrier()
                lib.lens_profile_reset()
                lib.lens_profile_enable(1)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.nvtx.range_push("timed_tc" if on else "timed_tc_off")
                e0.record(stream)
                pT.synthesis(a, out=out)
                e1.record(stream)
                torch.cuda.synchronize()
                torch.cuda.nvtx.range_pop()
                lib.lens_profile_enable(0)
                tpm, tcn = profile_read()
                call_ms = e0.elapsed_time(e1)
                key = "tensor_cores" if on else "cuda_cores"
                res[key] = {"synthesis_points_per_s": round(nm * npts / (call_ms * 1e-3), 1),
                            "call_ms": round(call_ms, 3), "legendre_ms": round(tpm[0], 3),
                            "legendre_ms_per_map": round(tpm[0] / nm, 4), "legendre_launches": int(tcn[0])}
                if on:
                    alg = 4.0 * nm * info_T["legendre_triples"]  # complex coefficient x real value per triple
                    res[key]["legendre_alg_tflops"] = round(alg / (tpm[0] * 1e-3) / 1e12, 2)
                    res[key]["tensor_tflops_split"] = round(3 * alg / (tpm[0] * 1e-3) / 1e12, 2)
                    res[key]["tensor_frac"] = round(3 * alg / (tpm[0] * 1e-3) / 1e12 / tc["peak_tf32_tflops"], 4)
            pT.set_tensor_cores(True)
            tc["legs"].append(res)
            del a, out
        pT.status()
    pT.close()
    torch.cuda.empty_cache()

    # ---------------- the same FP32 step with plan-time Legendre tables (when they fit)
    alt = None
    if not args.no_tables_compare:
        try:
            rT, rP, rb = make("fp32", 1e-5, not tables)
            alt_plan_s = make.plan_s
            kr = args.steps
            msr = timed(rT, rP, rb, kr, 3, profile=True, nvtx_name="timed_fp32_alt")
            apm, acn = profile_read()
            ui = {0: stage_units(rT.info(), npts, 0, "fp32"), 1: stage_units(rP.info(), npts, 2, "fp32")}
            ast, aroof, at_roof = analyze(apm, acn, kr, ui, 0, peaks, "fp32")
            aroof.pop("slot")
            alt = {"value": round(whole_job_rate(world, npts, msr), 1), "unit": "lensed points/s",
                   "ms_per_step": round(msr, 3), "steps": kr, "legendre": leg_mode(rT.info()) | {"EB": leg_mode(rP.info())},
                   "plan_creation_s": round(alt_plan_s, 3), "roofline": aroof, "stages": ast,
                   "step_roofline": {"t_roof_ms": round(at_roof, 3), "frac": round(at_roof / msr, 4)},
                   "what": "same step, FP32 plans %s" % ("running the restarted FP32 recursion" if tables else
                                                         "reading plan-time Legendre tables")}
            del rb
            rT.close(); rP.close()
        except _native.LensError as err:  # LENS_ERR_NOMEM: the tables (138 GB at lmax 4096) did not fit
            alt = {"unavailable": str(err)}
        torch.cuda.empty_cache()

    # ---------------- FP64 plans (epsilon 1e-10), same geometry
    fp64 = None
    if not args.no_fp64:
        qT, qP, c = make("fp64", 1e-10)
        k64 = max(1, min(args.steps, 3))
        ms64 = timed(qT, qP, c, k64, 1, profile=True, nvtx_name="timed_fp64")
        p64, c64 = profile_read()
        u64 = {0: stage_units(qT.info(), npts, 0, "fp64"), 1: stage_units(qP.info(), npts, 2, "fp64")}
        st64, roof64, tr64 = analyze(p64, c64, k64, u64, 16, peaks, "fp64")
        roof64.pop("slot")
        fp64 = {"value": round(whole_job_rate(world, npts, ms64), 1), "unit": "lensed points/s", "epsilon": 1e-10,
                "ms_per_step": round(ms64, 3), "steps": k64, "per_transform": per_transform(qT, qP, c, reps=1),
                "arithmetic": fp64_arithmetic(qT.info()),
                "plan": {k: qT.info()[k] for k in ("n1", "W", "sigma")} | {"W_spin2": qP.info()["W"]},
                "roofline": roof64, "stages": st64,
                "step_roofline": {"t_roof_ms": round(tr64, 3), "frac": round(tr64 / ms64, 4)}}
        del c
        qT.close(); qP.close()
        torch.cuda.empty_cache()

    # ---------------- lmax 5120 (Fig. 2 configuration: lmax_unl 5120 on the same Nside 2048 points)
    l5120 = None
    if not args.no_lmax5120 and lmax == 4096:
        from paper_2304_10431_gb300 import workloads as W
        L5 = 5120
        phi5 = W.draw_alm(W.phi_cl(4096), 4096, 2000)
        th5, ph5, chi5 = deflect_on_gpu(th0, ph0, phi5, 4096, dev)
        cl5 = W.cmb_cl(L5, 3750.0)
        a5 = (W.draw_alm(cl5, L5, 1000)[None],
              np.stack([W.draw_alm(cl5, L5, 1001, spin=2), W.draw_alm(cl5, L5, 1002, spin=2)]))
        l5120 = {"workload": "T + E/B, lmax_unl 5120, l_damp 3750, phi lmax 4096, HEALPix Nside %d (%d points)"
                             % (nside, npts), "legs": []}
        for prec, eps in (("fp32", 1e-4), ("fp64", 1e-6), ("fp64", 1e-10), ("fp64", 1e-12)):
            qT, qP, c = make(prec, eps, False, L=L5, geom=(th5, ph5, chi5), alms=a5)
            ps = make.plan_s
            k5 = 2 if prec == "fp32" else 1
            ms5 = timed(qT, qP, c, k5, 1, profile=True, nvtx_name="timed_l5120")
            p5, c5 = profile_read()
            u5 = {0: stage_units(qT.info(), npts, 0, prec), 1: stage_units(qP.info(), npts, 2, prec)}
            st5, roof5, tr5 = analyze(p5, c5, k5, u5, 0 if prec == "fp32" else 16, peaks, prec)
            roof5.pop("slot")
            l5120["legs"].append({"precision": prec, "epsilon": eps, "value": round(whole_job_rate(world, npts, ms5), 1),
                                  "unit": "lensed points/s", "ms_per_step": round(ms5, 3), "steps": k5,
                                  "per_transform": per_transform(qT, qP, c, reps=1),
                                  "legendre": leg_mode(qT.info()), "W": qT.info()["W"],
                                  "sigma": round(qT.info()["sigma"], 3), "plan_creation_s": round(ps, 2),
                                  "roofline": roof5, "stages": st5[:6]})
            del c
            qT.close(); qP.close()
            torch.cuda.empty_cache()
        del th5, ph5, chi5

    result = {
        "metric": "lensed points/sec (synthesis and adjoint), lmax 4096, eps 1e-5 FP32 vs 1e-10 FP64",
        "value": round(whole_job_rate(world, npts, ms), 1),
        "unit": "lensed points/s",
        "n_gpus": world, "steps": args.steps, "warmup": max(args.warmup, 3),
        "ms_per_step": round(ms, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (Legendre values from plan-time tables)" if tables else
                 "f32 (FP32 Legendre recursion restarted from FP64-derived values)",
        "data": "synthetic: seeded CMB/phi a_lm, HEALPix centres lensed on the GPU",
        "config": {"workload": "T + E/B lensing, lmax 4096, HEALPix Nside %d (%d points), phi lmax %d, "
                               "2.5 arcmin rms deflection, l_damp %.0f" % (nside, npts, lmax, ld),
                   "lmax": lmax, "nside": nside, "points": npts, "epsilon": 1e-5,
                   "step": "T synthesis + T adjoint + E/B synthesis + E/B adjoint",
                   "plan_T": {k: info_T[k] for k in ("ntheta", "n1", "n2", "W", "sigma", "beta")},
                   "plan_EB": {k: info_P[k] for k in ("ntheta", "n1", "n2", "W", "sigma", "beta")},
                   "l2": "per-step inputs 0.8 GB > 129 MB L2 (no flush)",
                   "legendre": {"T": leg_mode(info_T), "EB": leg_mode(info_P), "plan_creation_s": round(plan_s, 3)},
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "per_transform": pt,
        "roofline": roofline,
        "stages": stages,
        "step_roofline": step_roofline,
        "measured_peaks": measured_peaks,
        "gpu_launches": gpu_launches,
        "library": os.path.relpath(lib_path(), ROOT),
        "clocks": clocks,
        "e2e": e2e,
        "tables" if not tables else "recursion": alt,
        "tensor_cores": tc,
        "fp64": fp64,
        "lmax5120": l5120,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(lmax, nside, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ------------------------------------------------------------------ CPU oracle
def oracle_sample(lmax, nside, k, seed=0):
    """k points of the same lensed geometry, spread over rings near both poles and the equator."""
    import oracle as O
    from paper_2304_10431_gb300 import workloads as W
    rng = np.random.default_rng(seed)
    n = 12 * nside * nside
    idx = np.sort(np.concatenate([rng.integers(0, n // 50, k // 4), rng.integers(n - n // 50, n, k // 4),
                                  rng.integers(n // 2 - n // 20, n // 2 + n // 20, k - 2 * (k // 4))]))
    th0, ph0 = W.healpix_centres(nside)
    th0, ph0 = th0[idx], ph0[idx]
    phi_lm = W.draw_alm(W.phi_cl(lmax), lmax, 2000)
    th, ph, chi = O.deflected_points(th0, ph0, phi_lm, lmax)
    return th, ph, chi


def oracle_step(lmax, th, ph, chi, aT, aEB):
    import oracle as O
    mT = O.synthesis(lmax, lmax, 0, th, ph, aT)
    O.adjoint(lmax, lmax, 0, th, ph, mT)
    mP = O.synthesis(lmax, lmax, 2, th, ph, aEB, chi)
    O.adjoint(lmax, lmax, 2, th, ph, mP, chi)


def cpu_baseline(lmax, nside, seconds, steps=1, warmup=0, return_times=False):
    import oracle as O
    aT, aEB, _ = alm_inputs(lmax)
    # calibrate on 8 points, then size the sample to ~`seconds` per step
    th, ph, chi = oracle_sample(lmax, nside, 8, seed=1)
    t0 = time.perf_counter()
    oracle_step(lmax, th, ph, chi, aT, aEB)
    per_pt = (time.perf_counter() - t0) / 8
    k = int(max(8, min(4096, seconds / per_pt)))
    th, ph, chi = oracle_sample(lmax, nside, k, seed=2)
    for _ in range(warmup):
        oracle_step(lmax, th, ph, chi, aT, aEB)
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        oracle_step(lmax, th, ph, chi, aT, aEB)
        times.append(time.perf_counter() - t0)
    t = sum(times) / len(times)
    res = {"value": round(k / t, 3), "unit": "lensed points/s", "cores": O.num_threads(), "kind": "oracle",
           "sample": "%d lensed HEALPix points (Nside %d, near both poles and the equator), lmax %d, "
                     "T + E/B synthesis and adjoint by direct FP64 summation" % (k, nside, lmax),
           "seconds_per_step": round(t, 3)}
    return (res, t) if return_times else res


def run_reference(args):
    _, rank, _ = rank_env()
    if rank != 0:  # under torchrun only rank 0 times the oracle; the others exit without work
        return
    steps, warmup = args.steps, max(args.warmup, 0)
    per_step = max(min(2.0, args.ref_seconds), args.ref_seconds / max(steps + warmup, 1))
    cb, t = cpu_baseline(args.lmax, args.nside, per_step, steps=steps, warmup=warmup, return_times=True)
    out = {"metric": "lensed points/sec (synthesis and adjoint), lmax 4096, eps 1e-5 FP32 vs 1e-10 FP64",
           "value": cb["value"], "unit": "lensed points/s", "n_gpus": args.gpus, "steps": steps,
           "warmup": warmup, "ms_per_step": round(t * 1e3, 3), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic: seeded CMB/phi a_lm, lensed HEALPix sample",
           "config": {"workload": "T + E/B lensing, lmax %d, HEALPix Nside %d sample" % (args.lmax, args.nside),
                      "lmax": args.lmax, "nside": args.nside},
           "impl": "reference", "cpu_baseline": cb,
           "e2e": {"value": cb["value"], "unit": "lensed points/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_scan(args):
    """Forward + adjoint time of one spin-0 and one spin-2 map per (N_side, lmax) pair, on
    HEALPix centres displaced by 2.5 arcmin (the paper's Fig. 4 grid, one GPU)."""
    import torch
    from paper_2304_10431_gb300 import LensPlan
    from paper_2304_10431_gb300 import workloads as Wk
    dev = torch.device("cuda:0")
    precs = [(q.split(":")[0], float(q.split(":")[1])) for q in args.scan_eps.split(",")]
    for pair in args.scan.split(","):
        nside, lmax = (int(v) for v in pair.split(":"))
        th0, ph0 = Wk.healpix_centres(nside)
        th, ph, chi = Wk.displaced_points(th0, ph0, 2.5, seed=nside)
        for prec, eps in precs:
            row = {"scan": "nside x lmax", "nside": nside, "lmax": lmax, "npoints": int(th.size),
                   "precision": prec, "epsilon": eps}
            try:
                for spin in (0, 2):
                    plan = LensPlan(lmax, th, ph, chi if spin else None, spin=spin, epsilon=eps, precision=prec,
                                    device=dev)
                    nc = plan.ncomp
                    a = torch.zeros(nc, plan.nalm, dtype=plan.complex_dtype, device=dev)
                    a.real.normal_()
                    m = plan.synthesis(a)
                    plan.adjoint(m, out=a)  # warm-up
                    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
                    torch.cuda.synchronize()
                    ev[0].record()
                    plan.synthesis(a, out=m)
                    ev[1].record()
                    plan.adjoint(m, out=a)
                    ev[2].record()
                    torch.cuda.synchronize()
                    inf = plan.info()
                    row["spin%d" % spin] = {"synthesis_s": round(ev[0].elapsed_time(ev[1]) * 1e-3, 4),
                                            "adjoint_s": round(ev[1].elapsed_time(ev[2]) * 1e-3, 4),
                                            "W": inf["W"], "sigma": round(inf["sigma"], 3),
                                            "plan_GB": round((inf["plan_bytes"] + inf["workspace_bytes"]) / 1e9, 2)}
                    plan.close()
                    del a, m
                    torch.cuda.empty_cache()
            except Exception as exc:  # a configuration outside this build's limits
                row["error"] = str(exc)
            print(json.dumps(row), flush=True)


def main():
    args = parse()
    if args.scan:
        run_scan(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
