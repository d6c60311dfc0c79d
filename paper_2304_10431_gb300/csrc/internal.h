// Internal plan layout and kernel-launcher declarations of libgslens.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/gslens.h"

namespace gsl {

constexpr int kMaxFftStages = 24;
constexpr int kScaleBits = 60;       // exponent step of the scaled Legendre recursion
constexpr int kLegBlock = 8;         // degrees per unrolled block of the Legendre kernels
constexpr int kTileR = 32, kTileC = 32;  // default grid tile of the point sort (rows x columns)
constexpr int kMaxW = 16;                 // largest kernel support

// FP32 plans: the weight of kernel tap a (0 <= a < W) as a polynomial of degree W + 1 in
// t = 2 frac - (W - 1), t in [-1, 1] (frac = u - ceil(u - W/2) in (W/2 - 1, W/2]);
// c[a (W + 2) + k] multiplies t^k.  Passed to the NUFFT kernels by value.
struct KerPoly {
    float c[kMaxW * (kMaxW + 2)];
};

// One FFT length: radix sequence (DIT stage order), twiddles e^{-2 pi i t/n}
// and the digit-reversal table (input element i is stored at position perm[i]).
struct FftDesc {
    int n = 0;
    int nst = 0;
    int radix[kMaxFftStages] = {0};
    const void *tw = nullptr;   // float2[n] or double2[n]
    const int *perm = nullptr;  // int[n]
};

// Per-ring tables of the equiangular grid, north half (theta <= pi/2).
struct RingTab {
    const double *x = nullptr;        // cos(theta_j)
    const float2 *xdf = nullptr;      // cos(theta_j) as a df32 pair
    const double *lsin2 = nullptr;    // log2 sin(theta_j / 2)  (-inf at the pole)
    const double *lcos2 = nullptr;    // log2 cos(theta_j / 2)
    const float *y1 = nullptr;        // 1 - cos(theta_j) = 2 sin^2(theta_j / 2), FP32
};

// Restart values of the FP32 Legendre recursion (FP32 plans, see legendre.cu):
// entry base[m] + (k - 1) nnorth + ring holds the recursion state before the
// k-th restart of order m (every K degrees) as the pair v (float2, spin s:
// float4 for +s then -s) scaled by 2^(-60 E) and its exponent E (e: short,
// spin s short2; kCkZero marks a state that is identically zero).  Rings
// below jb (a multiple of 128: no warp straddles it) run Reinsch's form of the
// recursion.
// kstart[m][g]: the restart at which the 32 rings g*32 .. g*32+31 of order m
// begin (every degree before it is below 2^-40 on all of them; 0 = from the
// start value).
constexpr int kCkZero = -30000;
struct CkTab {
    const void *v = nullptr;
    const void *e = nullptr;
    const int64_t *base = nullptr;
    const short *kstart = nullptr;
    const unsigned char *klog = nullptr;  // per-order log2 of the restart interval (nullptr: K for all)
    const float2 *cs = nullptr;           // FP32 plans: (c_l, 1/c_l) per alm index (monic scale, PolSM)
    int ngrp = 0;
    int K = 0, jb = 0;
};

// Restart interval of order m
__host__ __device__ __forceinline__ int ck_interval(const CkTab &ck, int m)
{
#ifdef __CUDA_ARCH__
    return ck.klog ? 1 << __ldg(ck.klog + m) : ck.K;
#else
    return ck.klog ? 1 << ck.klog[m] : ck.K;
#endif
}

// Restarts of an order whose block loop starts at degree lf (= max(m, s) + 1):
// the degrees lf + K k, k >= 1, at which a full block of kLegBlock degrees
// still runs.
__host__ __device__ __forceinline__ int ck_count(int lmax, int lf, int K)
{
    const int n = lmax + 1 - kLegBlock - lf;
    return (K > 0 && n >= K) ? n / K : 0;
}

struct Plan {
    // problem
    int lmax = 0, mmax = 0, spin = 0, prec = LENS_FP32;
    int64_t npts = 0;
    double eps = 0;
    int device = 0;
    cudaStream_t stream = nullptr;

    // geometry of the equiangular grid and the torus
    int ntheta = 0;   // rings incl. poles
    int nnorth = 0;   // rings with theta <= pi/2 (ring pairs)
    int M = 0;        // 2 ntheta - 2
    int N1 = 0, N2 = 0;
    int W = 0;
    double beta = 0, sigma = 0;
    KerPoly kpoly{};      // FP32 plans: polynomial kernel weights (fitted at plan creation)
    int r_lo = 0, R = 0;  // kept torus rows r in [r_lo, r_lo + R)
    int pitch = 0;        // grid row stride (elements)
    int cl_theta = 1, cl_phi = 1;  // CTAs per FFT vector (2: a cluster sharing the vector)
    int ncol = 0;         // m columns: mmax+1 (spin 0) or 2 mmax + 1
    int64_t nalm = 0;

    // Legendre launch shapes (forward, adjoint): rings per thread, warps per
    // CTA, CTAs per m.  FP64 plans may run orders m >= m_df with a df32
    // recursion and df32 accumulation (shapes leg_fd, leg_ad); FP32 plans run
    // every order in df32 (m_df = 0).
    struct LegShape { int rpt = 0, warps = 0, chunks = 0; };
    LegShape leg_f, leg_a, leg_fd, leg_ad;
    LegShape leg_fb[2];  // FP32 forward sharing the recursion among 2 / 4 maps
    int m_df = 0;
    // FP32 plans: restarted FP32 recursion (rst) with its step table rec_s
    // (float4 per alm index) and restart values ck (ck_bytes); otherwise the
    // df32 recursion of rec_a.  FP64 plans: rst selects the restarted df32
    // recursion (PolDDR), with a restart interval per order (ck_klog, on the
    // host; ck.klog on the device).
    bool rst = false;
    void *rec_s = nullptr;
    CkTab ck;
    size_t ck_bytes = 0;
    std::vector<unsigned char> ck_klog;
    int64_t leg_triples = 0;  // non-negligible (ring pair, l, m) triples (restarted plans)
    // tensor-core batched synthesis (spin-0 restarted plans, 16 or more maps per call):
    // ring coefficients of up to 64 maps, prepared coefficient tiles, chunk offsets per m
    bool tc_on = true;
    void *tc_ring = nullptr, *tc_coef = nullptr;
    int64_t *tc_cbase = nullptr;

    // tables (device)
    // monic-form recursion coefficients per alm index: alpha and (spin s) tau,
    // as df32 (FP32 plans: float2 alpha, or for spin s float4 (alpha, tau) in
    // rec_a) or double (FP64 plans: rec_a, rec_t); FP64 plans with m_df <= mmax
    // also hold the df32 table in rec_a_df (rec_t_df unused).  scale: c_l
    // (double, per alm index).
    void *rec_a = nullptr, *rec_t = nullptr;
    void *rec_a_df = nullptr, *rec_t_df = nullptr;
    double *scale = nullptr;
    void *coef = nullptr;     // workspace: forward coefficients c_l a_lm of one call
    void *coef_m = nullptr;   // workspace, restarted FP32 plans: c_l a_lm for the monic plain-form warps
                              // ([ncomp][nalm], float2 / double2 / df32 float4)
    // FP32 plans, several maps per call: ring coefficients and prepared
    // coefficients of up to 4 maps, allocated on the first such call
    void *ring_batch = nullptr, *coef_batch = nullptr;
    bool group_maps = true;  // false: every map runs alone (lens_plan_set_grouping)
    bool grad = false;       // gradient-only spin s plan (C = 0): a_lm holds G alone
    // deterministic plans (LENS_DETERMINISTIC): fixed-point accumulation
    bool det = false;
    void *fx_grid = nullptr;                  // FP32 plans: int64 spreading grid [R][pitch][ncomp]
    void *fx_alm = nullptr;                   // FP32 plans: int64 adjoint a_lm sums [alm_ncomp][nalm][2]
    double *fx_scale = nullptr;               // [0] spreading unit, [1 + m] adjoint Legendre unit of order m
    unsigned long long *fx_maxbits = nullptr; // max |map value| of a call (bits of a double)
    uint32_t *fx_kmax = nullptr;              // most points any grid cell receives
    // FP32 plans at epsilon >= 1e-5 (not deterministic): spreading tiles in 32-bit fixed point,
    // per tile the most of its points covering one cell (plan time) and the map's largest
    // |value| of a call (bits of a double)
    unsigned short *tile_kmax = nullptr;
    unsigned long long *maxbits = nullptr;
    // Legendre tables (FP32 plans, lens_plan_params.legendre_tables): values of
    // the monic functions per (m, l, ring group), see legendre.cu
    bool tab = false;
    float *tab_v = nullptr;          // entries: float (spin 0) / float2 (+s, -s)
    int64_t *tab_rowbase = nullptr;  // [nalm] row offset - first ring, in entries
    int *tab_jlo = nullptr;          // [nalm] first ring of the row (nnp: empty)
    int *tab_lstart = nullptr;       // [mmax+1][ng] first degree of each ring group
    int tab_nnp = 0, tab_ng = 0;
    int tab_fchunks = 0, tab_fthreads = 0, tab_achunks = 0, tab_athreads = 0;  // launch shapes
    size_t tab_bytes = 0;
    int alm_ncomp() const { return spin && !grad ? 2 : 1; }
    double *lognorm = nullptr;  // per m: log2 of the start-value normalisation
    RingTab rings;
    void *w1 = nullptr;       // [2 lmax + 1]  1/psihat(2 pi k / N1), k = -lmax..lmax
    void *w2 = nullptr;       // [ncol]        1/(M psihat(2 pi m / N2))
    FftDesc fM, fN1, fN2;

    // points, sorted by grid tile
    uint32_t *cell = nullptr;  // row * pitch + col of the first tap
    void *frac = nullptr;      // float2 / double2 (u - i0, v - j0)
    int32_t *perm = nullptr;   // sorted -> user index
    uint32_t *tile_start = nullptr;  // [ntiles + 1] first sorted point of each 32 x 32 grid tile
    int ntile_c = 0, ntiles = 0;     // tiles per grid row band, total tiles
    int tile_r = kTileR;             // rows of a tile (16, 32 or 64; 32 columns)
    void *phase = nullptr;     // float2 / double2 e^{i s chi}, spin != 0 only
    double *wts = nullptr;     // FP64 plans: [npts][2W] kernel weights (theta taps, then phi taps)
    bool wts_dd = false;       // weights as double-float pairs; double-float interpolation and
                               // spreading taps (FP64 plans with epsilon >= 5e-11)

    // per-call workspace
    void *ring = nullptr;      // [ncol][ntheta] complex
    void *X = nullptr;         // [R][ncol] complex
    void *grid = nullptr;      // [R][pitch] real (spin 0) or complex
    unsigned *flags = nullptr; // device status flags

    // device staging for the host-buffer entry points (allocated on first use)
    void *stage_in = nullptr, *stage_out = nullptr;

    size_t plan_bytes = 0, work_bytes = 0;
    void *allocs[128];
    int nallocs = 0;
};

Plan::LegShape legendre_shape(const Plan &p, bool adjoint, bool dd, int rpt, int nm = 1);

// launchers (return cudaError_t of the launch)
cudaError_t launch_rec_tables(Plan &p);
// restarted FP32 recursion: step table, then restart values from the FP64
// monic recursion (a64, t64: temporary FP64 alpha / tau tables of the plan)
cudaError_t launch_rec_tables_s(Plan &p);
cudaError_t launch_ck_build(Plan &p, double *a64, double *t64, void *v_out, void *e_out, int *lt, short *kstart);
cudaError_t launch_ck_build64(Plan &p, void *v_out, void *e_out, int *lt, short *kstart);
// Legendre tables: shape, first-entry degrees, rows, values (plan creation)
cudaError_t tab_shape(Plan &p);
// bounded-wait self-test kernel (one warp, an mbarrier that never completes)
cudaError_t launch_wait_selftest(unsigned *status, long long limit, cudaStream_t st);
cudaError_t launch_tab_first(const Plan &p, int *first);
cudaError_t launch_tab_rows(const Plan &p, const int *first, int *lstart, int *jlo, int64_t *rowlen);
cudaError_t launch_tab_fill(const Plan &p);
// wpos multiplies the orders m > 0 (1 for the transforms themselves; the
// gradient entry points use 1/2 forward and 2 adjoint)
cudaError_t launch_legendre_fwd(const Plan &p, const void *alm, void *ring, cudaStream_t st, double wpos = 1.0);
cudaError_t launch_legendre_adj(const Plan &p, const void *ring, void *alm, cudaStream_t st, double wpos = 1.0);
// FP32 plans: Legendre synthesis of nm = 2 or 4 maps (a_lm consecutive) sharing
// one recursion; ring and coef hold nm maps' ring / prepared coefficients
cudaError_t launch_legendre_fwd_batch(const Plan &p, const void *alm, void *ring, void *coef, int nm, cudaStream_t st,
                                      double wpos);
// Tensor-core Legendre synthesis of nm <= nb maps (nb = 16, 32 or 64; spin-0 FP32
// plans with the restarted recursion): prepares the coefficient tiles of the
// call in coefB (tc_coef_floats(nb, total chunks) floats, chunk offsets per m
// in cbase) and writes nm maps' ring coefficients (map stride ncol ntheta).
int64_t tc_chunks(int lmax, int m);
size_t tc_coef_floats(int nb, int64_t chunks);
cudaError_t launch_legendre_fwd_tc(const Plan &p, const void *alm, int nm, void *ring, void *coefB,
                                   const int64_t *cbase, int nb, cudaStream_t st);
cudaError_t launch_theta_fwd(const Plan &p, const void *ring, void *X, cudaStream_t st);
cudaError_t launch_theta_adj(const Plan &p, const void *X, void *ring, cudaStream_t st);
cudaError_t launch_phi_fwd(const Plan &p, const void *X, void *grid, cudaStream_t st);
cudaError_t launch_phi_adj(const Plan &p, const void *grid, void *X, cudaStream_t st);
cudaError_t launch_interp(const Plan &p, const void *grid, void *map, cudaStream_t st);
cudaError_t launch_spread(const Plan &p, const void *map, void *grid, cudaStream_t st);
cudaError_t launch_prep_points(Plan &p, const double *theta, const double *phi, const double *chi,
                               cudaStream_t st, std::string &err);
cudaError_t launch_pointing(int64_t n, const double *theta, const double *phi, const double *ath,
                            const double *aph, double *theta_out, double *phi_out, double *chi_out,
                            cudaStream_t st);

// One map through the whole forward (Legendre synthesis .. interpolation) or
// adjoint chain on stream st, with the order weight wpos (1 for the
// transforms; 2 / 0.5 for the gradient entry points).  Returns a lens_status
// and records failures.
int run_forward(const Plan &p, const void *alm, void *map, cudaStream_t st, double wpos);
int run_adjoint(const Plan &p, const void *map, void *alm, cudaStream_t st, double wpos);

// Sets the stage-timer switch, returning its previous state (stream capture
// runs with the timers off).
bool profile_swap(bool on);

// Bytes of the per-call work buffers of one map's forward chain: ring
// coefficients [ncol][ntheta], torus rows [R][ncol] (complex) and the
// oversampled grid [R][pitch] (real for spin 0, complex for spin s).
struct ScratchSizes { size_t ring, X, grid; };
inline ScratchSizes plan_scratch_sizes(const Plan &p)
{
    const size_t esz = p.prec == LENS_FP32 ? 8 : 16;
    return {esz * (size_t)p.ncol * p.ntheta, esz * (size_t)p.R * p.ncol,
            (esz / 2) * (p.spin ? 2 : 1) * (size_t)p.R * p.pitch};
}

// Bytes of one map's a_lm / point values for a plan.
inline size_t plan_alm_bytes(const Plan &p) { return (size_t)p.nalm * p.alm_ncomp() * (p.prec == LENS_FP32 ? 8 : 16); }
inline size_t plan_map_bytes(const Plan &p) { return (size_t)p.npts * (p.spin ? 2 : 1) * (p.prec == LENS_FP32 ? 4 : 8); }

// Records a failing status and message in the calling thread's error state
// (lens_get_last_error / lens_last_error_message) and returns the status.
int record_failure(int status, const char *msg);

// shared-memory elements of a one-CTA FFT vector of n elements of esz bytes
// (FP32 vectors: one padding element after every 16, see fft.cuh)
inline constexpr size_t fft_smem_elems(size_t n, size_t esz) { return esz == 8 ? n + n / 16 + 1 : n; }
size_t theta_smem_bytes(const Plan &p);
// torus coefficients c_k (|k| <= lmax) of every m column from ring coefficients
cudaError_t launch_theta_coeffs(const Plan &p, const void *ring, void *out, cudaStream_t st);
size_t phi_smem_bytes(const Plan &p);

}  // namespace gsl
