// Non-uniform FFT steps (Sect. 3 "NUFFT": type 2 for the forward operator,
// type 1 for the adjoint) on the oversampled torus grid.
//
// Kernel: exponential of semicircle, psi(z) = exp(beta (sqrt(1 - (2z/W)^2) - 1))
// for |z| < W/2 (grid units), zero outside.  A point at grid coordinates
// (u, v) = (theta N1 / 2pi, phi N2 / 2pi) touches the W x W cells
// i0 + a, j0 + b with i0 = ceil(u - W/2), j0 = ceil(v - W/2), a, b < W:
//   type 2:  f = sum_ab psi(u - i0 - a) psi(v - j0 - b) g[i0 + a, j0 + b]
//   type 1:  g[i0 + a, j0 + b] += psi(u - i0 - a) psi(v - j0 - b) f
// The two use the same weights, so they are exact transposes.
//
// Points are prepared once per plan (Sect. 4: the geometry is reused): cell
// offset into the row-padded grid, fractional offsets (u - i0, v - j0) from
// FP64 coordinates, the spin phase e^{i s chi}, a permutation that sorts
// points by 32 x 32 grid tiles (of the first tap) so that neighbouring
// threads share grid rows, and the first sorted point of every tile.
// Interpolation runs one thread per sorted point and reads its W x W taps
// through L1: sorted neighbours share rows, so the tile stays cached (staging
// the tile and its halo in shared memory first measured 1.36x slower for
// spin 0 at lmax 4096).  Spreading in FP32 runs one CTA per tile: its points
// add their W x W taps into the tile and its halo, (32 + W - 1) x (32 + W - 1)
// cells held in shared memory, and the CTA then adds the non-zero cells into
// the grid with one global atomic each.  FP64
// plans spread with one global atomic per tap instead: the L2 adds doubles
// natively, while double additions into shared memory measured 1.9x (spin s)
// to 2.4x (spin 0) slower at lmax 4096.
//
// Deterministic plans (LENS_DETERMINISTIC) spread in 64-bit fixed point: every
// tap value is scaled by a power of two 2^k and rounded to an integer, and the
// shared-memory and global atomics add integers, exactly and so in any order.
// k is chosen per call so that no cell can exceed 2^62: a cell receives at
// most Kmax points (the largest point count of a tile and its left, upper and
// upper-left neighbours, whose taps are the only ones that reach it), each
// contributing |x| psi psi <= max |x|.  A conversion pass then writes the
// grid in the plan's precision.
#include <cuda_runtime.h>
#include <math.h>

#include <type_traits>

#include <cub/cub.cuh>

#include "common.cuh"
#include "internal.h"

namespace gsl {
namespace {

constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr double kPi = 3.141592653589793238462643383280;
constexpr int kSpreadThreads = 64;
// FP64 tiles hold 64-bit cells (31 KB at W = 13, seven CTAs per SM): 256 threads keep
// more warps in flight per tile
constexpr int kSpreadThreads64 = 256;
// FP64 double-float spreading tiles stage this many points at a time (offset + value pair)
constexpr int kDDBatch = 512;

// Grid coordinate u = t c with c = N / (2 pi) held as a double-double (c.x +
// c.y): the product's rounding error, ~1e-16 of u (up to N/2 ~ 10^4 cells),
// would otherwise move the point by about one ulp of theta, i.e. a relative
// error of ~lmax * 1e-16 in the interpolated field.  Returns the cell index
// ceil(u - W/2) and the offset u - index to full double precision.
__device__ __forceinline__ int grid_coord(double t, double2 c, double hw, double &frac)
{
    const double p = t * c.x;
    const double e = fma(t, c.x, -p) + t * c.y;
    const int i0 = (int)ceil((p + e) - hw);
    frac = (p - (double)i0) + e;  // p - i0 is exact: both lie within W of each other
    return i0;
}

__global__ void k_prep(const double *__restrict__ theta, const double *__restrict__ phi,
                       const double *__restrict__ chi, int64_t n, int N1, int N2, int W, int r_lo, int R, int pitch,
                       int spin, double2 c1, double2 c2, int tile_r, uint32_t *__restrict__ key,
                       int32_t *__restrict__ idx, uint32_t *__restrict__ cell_u, double2 *__restrict__ frac_u,
                       double2 *__restrict__ phase_u, unsigned *__restrict__ flags)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double th = theta[i], ph = phi[i];
    bool bad = !(isfinite(th) && isfinite(ph)) || th < 0.0 || th > kPi;
    if (bad) {
        atomicOr(flags, FLAG_DOMAIN);
        th = 0.0;
        ph = 0.0;
    }
    ph = fmod(ph, kTwoPi);
    if (ph < 0.0) ph += kTwoPi;
    if (ph >= kTwoPi) ph = 0.0;
    const double hw = 0.5 * W;
    double fu, fv;
    const int i0 = grid_coord(th, c1, hw, fu);
    int j0 = grid_coord(ph, c2, hw, fv);
    if (j0 < 0) j0 += N2;
    if (j0 >= N2) j0 -= N2;
    int row = i0 - r_lo;
    if (row < 0 || row > R - W) {  // cannot happen for theta in [0, pi]; guard the table
        atomicOr(flags, FLAG_OOB);
        row = row < 0 ? 0 : R - W;
    }
    cell_u[i] = (uint32_t)row * (uint32_t)pitch + (uint32_t)j0;
    frac_u[i] = make_double2(fu, fv);
    const int ntc = (N2 + kTileC - 1) / kTileC;
    key[i] = (uint32_t)(row / tile_r) * (uint32_t)ntc + (uint32_t)(j0 / kTileC);
    idx[i] = (int32_t)i;
    if (spin) {
        const double c = chi ? chi[i] : 0.0;
        double sn, cs;
        sincos(spin * c, &sn, &cs);
        phase_u[i] = make_double2(cs, sn);
    }
}

__global__ void k_gather_points(const int32_t *__restrict__ perm, int64_t n, const uint32_t *__restrict__ cell_u,
                                const double2 *__restrict__ frac_u, const double2 *__restrict__ phase_u, int prec,
                                int spin, uint32_t *__restrict__ cell, void *__restrict__ frac,
                                void *__restrict__ phase)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int32_t i = perm[p];
    cell[p] = cell_u[i];
    const double2 f = frac_u[i];
    if (prec == LENS_FP32) ((float2 *)frac)[p] = make_float2((float)f.x, (float)f.y);
    else ((double2 *)frac)[p] = f;
    if (spin) {
        const double2 ph = phase_u[i];
        if (prec == LENS_FP32) ((float2 *)phase)[p] = make_float2((float)ph.x, (float)ph.y);
        else ((double2 *)phase)[p] = ph;
    }
}

// start[t] = first sorted point whose tile key is >= t, t = 0..ntiles (the
// ranges (key[p-1], key[p]] partition 0..ntiles, so each entry is written once)
__global__ void k_tile_bounds(const uint32_t *__restrict__ skey, int64_t n, int ntiles, uint32_t *__restrict__ start)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p > n) return;
    const int64_t lo = p == 0 ? -1 : (int64_t)skey[p - 1];
    const int64_t hi = p == n ? (int64_t)ntiles : (int64_t)skey[p];
    for (int64_t t = lo + 1; t <= hi; ++t) start[t] = (uint32_t)p;
}

// the ES kernel of tap offset z (FP64 plans)
template <typename T> __device__ __forceinline__ T es_kernel(T z, T twoW, T beta)
{
    const T t = z * twoW;
    const T q = T(1) - t * t;
    return q > T(0) ? exp(beta * (sqrt(q) - T(1))) : T(0);
}

// FP32 plans: the kernel weight of tap a by Horner's rule in t = 2 frac - (W - 1) from the plan's
// polynomial coefficients (W + 1 fused multiply-adds; interpolation and spreading read the same
// coefficients, so the pair stay exact transposes of each other)
template <int W> __device__ __forceinline__ float ker_poly(const KerPoly &kp, int a, float t)
{
    float acc = kp.c[a * (W + 2) + W + 1];
#pragma unroll
    for (int k = W; k >= 0; --k) acc = fmaf(acc, t, kp.c[a * (W + 2) + k]);
    return acc;
}

// fixed-point term: v 2^k (exact, 2^k a power of two) rounded to an integer
__device__ __forceinline__ unsigned long long to_fx(float v, float sc) { return (unsigned long long)__float2ll_rn(v * sc); }
__device__ __forceinline__ unsigned long long to_fx(double v, double sc)
{
    return (unsigned long long)__double2ll_rn(v * sc);
}

// FP64 plans' 2W kernel weights of every (sorted) point, computed once, evaluated in FP64 and kept as
// doubles or (dd, plans with epsilon >= 5e-11) as double-float pairs (8 bytes
// each either way): the latter plans compute the interpolation and spreading
// taps in double-float arithmetic on the FP32 pipe, GB300's FP64 pipe running
// at 1/60 of it.
__global__ void k_weights(const double2 *__restrict__ frac, int64_t n, int W, double beta, double *__restrict__ wts,
                          int dd)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const double2 f = frac[p];
    const double twoW = 2.0 / W;
    double *wd = wts + p * 2 * W;
    float2 *w = reinterpret_cast<float2 *>(wd);
    for (int a = 0; a < W; ++a) {
        const double x = es_kernel<double>(f.x - a, twoW, beta), y = es_kernel<double>(f.y - a, twoW, beta);
        if (dd) {
            const df32 xs = df_split(x), ys = df_split(y);
            w[a] = make_float2(xs.h, xs.l);
            w[W + a] = make_float2(ys.h, ys.l);
        } else {
            wd[a] = x;
            wd[W + a] = y;
        }
    }
}

__device__ __forceinline__ df32 ld_df(const float2 *p)
{
    const float2 v = __ldg(p);
    return {v.x, v.y};
}

// PRE: 0 evaluate the kernel, 1 read the double weights, 2 the double-float pairs
template <typename T, int W, int PRE>
__device__ __forceinline__ void tap_weights(T (&wa)[W], T (&wb)[W], const cplx<T> &f, const double *wts, int64_t p,
                                            T beta, const KerPoly &kp)
{
    if (PRE == 1) {
        const double *w = wts + p * 2 * W;
#pragma unroll
        for (int a = 0; a < W; ++a) {
            wa[a] = (T)__ldg(w + a);
            wb[a] = (T)__ldg(w + W + a);
        }
    } else if (PRE == 2) {
        const float2 *w = reinterpret_cast<const float2 *>(wts) + p * 2 * W;
#pragma unroll
        for (int a = 0; a < W; ++a) {
            wa[a] = (T)df_value(ld_df(w + a));
            wb[a] = (T)df_value(ld_df(w + W + a));
        }
    } else if constexpr (std::is_same<T, float>::value) {
        const float tx = fmaf(2.f, f.x, -(float)(W - 1)), ty = fmaf(2.f, f.y, -(float)(W - 1));
#pragma unroll
        for (int a = 0; a < W; ++a) {
            wa[a] = ker_poly<W>(kp, a, tx);
            wb[a] = ker_poly<W>(kp, a, ty);
        }
    } else {
        const T twoW = T(2) / T(W);
#pragma unroll
        for (int a = 0; a < W; ++a) {
            wa[a] = es_kernel<T>(f.x - T(a), twoW, beta);
            wb[a] = es_kernel<T>(f.y - T(a), twoW, beta);
        }
    }
}

template <typename T, int W, bool SPIN, int PRE>
__global__ void __launch_bounds__(256) k_interp(const void *__restrict__ grid, const uint32_t *__restrict__ cell,
                                                const cplx<T> *__restrict__ frac, const int32_t *__restrict__ perm,
                                                const cplx<T> *__restrict__ phase, const double *__restrict__ wts,
                                                T *__restrict__ map, int64_t n, int pitch, T beta,
                                                const __grid_constant__ KerPoly kp)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const uint32_t c0 = cell[p];
    T wa[W], wb[W];
    tap_weights<T, W, PRE>(wa, wb, PRE ? cplx<T>{} : frac[p], wts, p, beta, kp);
    const int32_t dst = perm[p];
    if (!SPIN) {
        const T *g = (const T *)grid + c0;
        T acc = T(0);
#pragma unroll
        for (int a = 0; a < W; ++a) {
            T r = T(0);
#pragma unroll
            for (int b = 0; b < W; ++b) r += wb[b] * __ldg(g + (int64_t)a * pitch + b);
            acc += wa[a] * r;
        }
        map[dst] = acc;
    } else {
        const cplx<T> *g = (const cplx<T> *)grid + c0;
        T ax = T(0), ay = T(0);
#pragma unroll
        for (int a = 0; a < W; ++a) {
            T rx = T(0), ry = T(0);
#pragma unroll
            for (int b = 0; b < W; ++b) {
                const cplx<T> v = __ldg(g + (int64_t)a * pitch + b);
                rx += wb[b] * v.x;
                ry += wb[b] * v.y;
            }
            ax += wa[a] * rx;
            ay += wa[a] * ry;
        }
        const cplx<T> ph = phase[p];
        map[dst] = ax * ph.x - ay * ph.y;
        map[n + dst] = ax * ph.y + ay * ph.x;
    }
}

// FP64 plans with point weights: the same sums in double-float arithmetic on
// the FP32 pipe.  The grid holds double-float pairs (k_phi_fwd writes them
// for these plans: float2 per real, spin s float4 (re h, re l, im h, im l));
// each row sum adds the exact products of the high words with two-sum and
// the products' error terms and cross terms in the low word, then the rows
// are combined the same way; ~2^-46 relative per term.
template <int W, bool SPIN>
__global__ void __launch_bounds__(256) k_interp_dd(const void *__restrict__ grid, const uint32_t *__restrict__ cell,
                                                   const int32_t *__restrict__ perm, const double2 *__restrict__ phase,
                                                   const double *__restrict__ wts, double *__restrict__ map,
                                                   int64_t n, int pitch)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const uint32_t c0 = cell[p];
    const float2 *w = reinterpret_cast<const float2 *>(wts) + p * 2 * W;
    df32 wb[W];
#pragma unroll
    for (int b = 0; b < W; ++b) wb[b] = ld_df(w + W + b);
    const int32_t dst = perm[p];
    if (!SPIN) {
        const float2 *g = reinterpret_cast<const float2 *>(grid) + c0;
        df32 acc = {0.f, 0.f};
#pragma unroll
        for (int a = 0; a < W; ++a) {
            df32 r = {0.f, 0.f};
#pragma unroll
            for (int b = 0; b < W; ++b) df_acc(r, df_mul(wb[b], ld_df(g + (int64_t)a * pitch + b)));
            df_acc(acc, df_mul(ld_df(w + a), df_renorm(r)));
        }
        map[dst] = df_value(acc);
    } else {
        const float4 *g = reinterpret_cast<const float4 *>(grid) + c0;
        df32 ax = {0.f, 0.f}, ay = {0.f, 0.f};
#pragma unroll
        for (int a = 0; a < W; ++a) {
            df32 rx = {0.f, 0.f}, ry = {0.f, 0.f};
#pragma unroll
            for (int b = 0; b < W; ++b) {
                const float4 v = __ldg(g + (int64_t)a * pitch + b);
                df_acc(rx, df_mul(wb[b], df32{v.x, v.y}));
                df_acc(ry, df_mul(wb[b], df32{v.z, v.w}));
            }
            const df32 wa = ld_df(w + a);
            df_acc(ax, df_mul(wa, df_renorm(rx)));
            df_acc(ay, df_mul(wa, df_renorm(ry)));
        }
        const double2 ph = phase[p];
        const double x = df_value(ax), y = df_value(ay);
        map[dst] = x * ph.x - y * ph.y;
        map[n + dst] = x * ph.y + y * ph.x;
    }
}

// one thread per sorted point, one global atomic per tap (FP64 plans); FX:
// fixed-point integers into the same grid memory (scale *fxs)
template <typename T, bool FX> struct Acc {
    using type = T;
};
template <typename T> struct Acc<T, true> {
    using type = unsigned long long;
};
template <typename T, bool FX>
__device__ __forceinline__ void acc_add(typename Acc<T, FX>::type *dst, T v, T sc)
{
    if constexpr (FX) atomicAdd(dst, to_fx(v, sc));
    else atomicAdd(dst, v);
}

template <typename T, int W, bool SPIN, int PRE, bool FX>
__global__ void __launch_bounds__(256) k_spread_direct(void *__restrict__ grid, const uint32_t *__restrict__ cell,
                                                       const cplx<T> *__restrict__ frac,
                                                       const int32_t *__restrict__ perm,
                                                       const cplx<T> *__restrict__ phase,
                                                       const double *__restrict__ wts, const T *__restrict__ map,
                                                       int64_t n, int pitch, T beta, const double *__restrict__ fxs,
                                                       const __grid_constant__ KerPoly kp)
{
    using G = typename Acc<T, FX>::type;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const T sc = FX ? (T)fxs[0] : T(1);
    const uint32_t c0 = cell[p];
    T wa[W], wb[W];
    tap_weights<T, W, PRE>(wa, wb, PRE ? cplx<T>{} : frac[p], wts, p, beta, kp);
    const int32_t src = perm[p];
    if (!SPIN) {
        const T x = map[src];
        G *g = (G *)grid + c0;
#pragma unroll
        for (int a = 0; a < W; ++a) {
            const T xa = wa[a] * x;
#pragma unroll
            for (int b = 0; b < W; ++b) acc_add<T, FX>(g + (int64_t)a * pitch + b, xa * wb[b], sc);
        }
    } else {
        // e^{-i s chi} (Q + i U)
        const cplx<T> ph = phase[p];
        const T q = map[src], u = map[n + src];
        const T zx = ph.x * q + ph.y * u, zy = ph.x * u - ph.y * q;
        G *g = (G *)grid + 2 * (int64_t)c0;
#pragma unroll
        for (int a = 0; a < W; ++a) {
            const T xa = wa[a] * zx, ya = wa[a] * zy;
#pragma unroll
            for (int b = 0; b < W; ++b) {
                G *q2 = g + 2 * ((int64_t)a * pitch + b);
                acc_add<T, FX>(q2, xa * wb[b], sc);
                acc_add<T, FX>(q2 + 1, ya * wb[b], sc);
            }
        }
    }
}

// FX: fixed-point integers in shared memory and in the grid (scale *fxs).
// IT (integer tiles; FP32 plans at epsilon >= 1e-5 and FP64 plans, not FX):
// the tile accumulates in fixed point in shared memory, 32-bit integers for
// FP32 plans (integer atomics there run ~3x the rate of float atomics) and
// 64-bit for FP64 plans (no FP64 atomics in the inner loop), in units of 1/u
// with u = 2^k per tile, k the largest integer with kmax_t max|x| u <= 2^30
// (FP64: 2^62): kmax_t (plan time) is the most of the tile's points whose
// W x W windows cover one cell and max|x| (per call) the map's largest |value|
// (|Q| + |U| for spin s), taps |psi| <= 1, so no cell sum can overflow.  Every
// term is rounded once (to 2^-k; FP64: relative 2^-62 of the tile's bound);
// the flush converts back for one global atomic per non-zero cell.  A map
// with a non-finite value makes the whole tile NaN.
template <typename T, bool FX, bool IT> struct SAcc { using type = typename Acc<T, FX>::type; };
template <> struct SAcc<float, false, true> { using type = int; };
template <> struct SAcc<double, false, true> { using type = long long; };
__device__ __forceinline__ int tile_int(float v) { return __float2int_rn(v); }
// A double-float term (p, e) with |p| < 2^53 as a 64-bit integer (nearest) without
// 64-bit conversions (those run at GB300's FP64 rate): p = p1 + p2 with p1 a multiple
// of 2^31 (|p1| / 2^31 < 2^22, read off the bits of p1 / 2^31 + 1.5 * 2^23) and
// |p2| <= 2^30 exact, then p2 and e by 32-bit conversions
__device__ __forceinline__ long long dd_tile_int(df32 t)
{
    const float big = 0x1.8p54f;  // 1.5 * 2^54: t.h + big rounds t.h to a multiple of 2^31
    const float p1 = __fsub_rn(__fadd_rn(t.h, big), big);
    const int i1 = __float_as_int(__fmaf_rn(p1, 0x1p-31f, 12582912.0f)) - 0x4B400000;
    const float p2 = __fsub_rn(t.h, p1);
    return ((long long)i1 << 31) + (long long)__float2int_rn(p2) + (long long)__float2int_rn(t.l);
}
__device__ __forceinline__ long long tile_int(double v) { return __double2ll_rn(v); }
__device__ __forceinline__ void tile_add(int *dst, int v) { atomicAdd(dst, v); }
__device__ __forceinline__ void tile_add(long long *dst, long long v)
{
    atomicAdd(reinterpret_cast<unsigned long long *>(dst), (unsigned long long)v);  // two's complement sum
}

template <typename T, int W, bool SPIN, int PRE, bool FX, bool IT = false>
__global__ void __launch_bounds__(sizeof(T) == 8 ? kSpreadThreads64 : kSpreadThreads) k_spread(void *__restrict__ grid, const uint32_t *__restrict__ cell,
                                                           const cplx<T> *__restrict__ frac,
                                                           const int32_t *__restrict__ perm,
                                                           const cplx<T> *__restrict__ phase,
                                                           const double *__restrict__ wts, const T *__restrict__ map,
                                                           int64_t n, int pitch, int R, int ntc,
                                                           const uint32_t *__restrict__ tile_start, T beta,
                                                           const double *__restrict__ fxs,
                                                           int tile_r, const unsigned short *__restrict__ tile_kmax,
                                                           const unsigned long long *__restrict__ maxbits,
                                                           const __grid_constant__ KerPoly kp)
{
    static_assert(!(IT && FX), "fixed-point tiles or fixed-point grid");
    using G = typename SAcc<T, FX, IT>::type;
    constexpr bool DD = std::is_same<T, double>::value && IT && PRE == 2;  // double-float taps
    constexpr int TC = kTileC + W - 1, NC = SPIN ? 2 : 1;
    const int TR = tile_r + W - 1;  // tile rows (16, 32 or 64) plus the kernel halo
    extern __shared__ __align__(16) unsigned char spread_smem[];
    G *buf = reinterpret_cast<G *>(spread_smem);  // TR x TC cells x NC planes
    const int t = blockIdx.x;
    const uint32_t p0 = tile_start[t], p1 = tile_start[t + 1];
    if (p0 == p1) return;
    T sc = FX ? (T)fxs[0] : T(1);
    bool bad = false;  // IT: non-finite map value
    if constexpr (IT) {
        constexpr int kBits = sizeof(T) == 4 ? 30 : DD ? 53 : 62;  // tile sums of |terms| below 2^kBits
        const double bound = (double)tile_kmax[t] * __longlong_as_double((long long)*maxbits);
        if (!(bound < 1e300)) bad = true;  // infinity or NaN in the map
        else if (bound > 0.0) sc = (T)ldexp(1.0, kBits - (ilogb(bound) + 1));  // bound < 2^(ilogb+1)
    }
    for (int i = threadIdx.x; i < TR * TC * NC; i += blockDim.x) buf[i] = G(0);
    __syncthreads();
    const int r0 = (t / ntc) * tile_r, c0 = (t % ntc) * kTileC;
    if constexpr (DD && SPIN) {
        // FP64 plans with point weights, spin s: work items (point, kernel row) instead of points, so
        // that the threads of a tile finish together (a tile holds 2-3 points per thread, and
        // one point per thread more meant a wait at the barrier) and the unrolled body is one
        // row of W taps.  Per batch of points: each point's value times the unit (exact) as a
        // double-float pair and its cell offset in shared memory; then the items.  Each tap is
        // the double-float product of the row value and the weight pair (~2^-46 relative),
        // rounded to an integer by dd_tile_int (tile sums of |terms| below 2^53).
        int *soff = reinterpret_cast<int *>(buf + ((TR * TC * NC + 1) & ~1));  // 16-byte aligned
        float4 *sval = reinterpret_cast<float4 *>(soff + kDDBatch);
        for (uint32_t pb = p0; pb < (bad ? p0 : p1); pb += kDDBatch) {
            const int nb = (int)min((uint32_t)kDDBatch, p1 - pb);
            for (int q = threadIdx.x; q < nb; q += blockDim.x) {
                const uint32_t p = pb + q;
                const uint32_t c = cell[p];
                const int lr = (int)(c / (uint32_t)pitch) - r0, lc = (int)(c % (uint32_t)pitch) - c0;
                const bool mine = (unsigned)lr < (unsigned)tile_r && (unsigned)lc < (unsigned)kTileC;
                soff[q] = mine ? lr * TC + lc : -1;
                if (!mine) continue;
                const int32_t src = perm[p];
                const cplx<T> ph = phase[p];
                const T qv = map[src], u = map[n + src];
                const df32 zx = df_split((ph.x * qv + ph.y * u) * sc), zy = df_split((ph.x * u - ph.y * qv) * sc);
                sval[q] = make_float4(zx.h, zx.l, zy.h, zy.l);
            }
            __syncthreads();
            for (int it = threadIdx.x; it < nb * W; it += blockDim.x) {
                const int q = it / W, a = it - q * W;
                const int off = soff[q];
                if (off < 0) continue;
                const float2 *w = reinterpret_cast<const float2 *>(wts) + (int64_t)(pb + q) * 2 * W;
                const df32 wa = ld_df(w + a);
                const float4 v = sval[q];
                G *row = buf + off + a * TC;
                const df32 xa = df_renorm(df_mul(wa, df32{v.x, v.y})), ya = df_renorm(df_mul(wa, df32{v.z, v.w}));
#pragma unroll
                for (int b = 0; b < W; ++b) {
                    const df32 wb = ld_df(w + W + b);
                    tile_add(row + b, dd_tile_int(df_mul(xa, wb)));
                    tile_add(row + b + TR * TC, dd_tile_int(df_mul(ya, wb)));
                }
            }
            __syncthreads();  // the batch's staging is rewritten next
        }
    }
    for (uint32_t p = p0 + threadIdx.x; p < ((bad || (DD && SPIN)) ? p0 : p1); p += blockDim.x) {
        const uint32_t c = cell[p];
        const int lr = (int)(c / (uint32_t)pitch) - r0, lc = (int)(c % (uint32_t)pitch) - c0;
        if ((unsigned)lr >= (unsigned)tile_r || (unsigned)lc >= (unsigned)kTileC) continue;  // not this tile's
        const int32_t src = perm[p];
        // spin s: two planes (real parts, then imaginary parts), so that the lanes'
        // atomics of one plane spread over all 32 banks
        G *b0 = buf + (lr * TC + lc);
        if constexpr (DD && !SPIN) {
            // FP64 plans with point weights, spin 0: the value (times the unit, exact) as a
            // double-float pair, each tap the double-float product with the pair of weights
            // (~2^-46 relative), rounded to an integer by dd_tile_int (tile sums of |terms|
            // below 2^53)
            const float2 *w = reinterpret_cast<const float2 *>(wts) + (int64_t)p * 2 * W;
            df32 wb[W];
#pragma unroll
            for (int b = 0; b < W; ++b) wb[b] = ld_df(w + W + b);
            const df32 x = df_split(map[src] * sc);
#pragma unroll
            for (int a = 0; a < W; ++a) {
                const df32 xa = df_renorm(df_mul(ld_df(w + a), x));
#pragma unroll
                for (int b = 0; b < W; ++b) tile_add(b0 + a * TC + b, dd_tile_int(df_mul(xa, wb[b])));
            }
            continue;
        }
        T wa[W], wb[W];
        tap_weights<T, W, PRE>(wa, wb, PRE ? cplx<T>{} : frac[p], wts, p, beta, kp);
        // IT: the power-of-two unit sc is applied to the point's value first (exact)
        if (!SPIN) {
            const T x = IT ? map[src] * sc : map[src];
#pragma unroll
            for (int a = 0; a < W; ++a) {
                const T xa = wa[a] * x;
#pragma unroll
                for (int b = 0; b < W; ++b) {
                    if constexpr (IT) tile_add(b0 + a * TC + b, tile_int(xa * wb[b]));
                    else acc_add<T, FX>(b0 + a * TC + b, xa * wb[b], sc);
                }
            }
        } else {
            // e^{-i s chi} (Q + i U)
            const cplx<T> ph = phase[p];
            const T q = map[src], u = map[n + src];
            T zx = ph.x * q + ph.y * u, zy = ph.x * u - ph.y * q;
            if constexpr (IT) { zx *= sc; zy *= sc; }
#pragma unroll
            for (int a = 0; a < W; ++a) {
                const T xa = wa[a] * zx, ya = wa[a] * zy;
#pragma unroll
                for (int b = 0; b < W; ++b) {
                    G *q2 = b0 + (a * TC + b);
                    if constexpr (IT) {
                        tile_add(q2, tile_int(xa * wb[b]));
                        tile_add(q2 + TR * TC, tile_int(ya * wb[b]));
                    } else {
                        acc_add<T, FX>(q2, xa * wb[b], sc);
                        acc_add<T, FX>(q2 + TR * TC, ya * wb[b], sc);
                    }
                }
            }
        }
    }
    __syncthreads();
    if constexpr (IT) {
        T *g = (T *)grid;
        const T inv = bad ? T(NAN) : T(1) / sc;
        for (int i = threadIdx.x; i < TR * TC; i += blockDim.x) {
            const int gr = r0 + i / TC, gc = c0 + i % TC;
            if (gr >= R || gc >= pitch) continue;
            const int64_t o = (int64_t)gr * pitch + gc;
            if (!SPIN) {
                const G v = buf[i];
                if (v != 0 || bad) atomicAdd(g + o, (T)v * inv);
            } else {
                const G vx = buf[i], vy = buf[TR * TC + i];
                if (vx != 0 || bad) atomicAdd(g + 2 * o, (T)vx * inv);
                if (vy != 0 || bad) atomicAdd(g + 2 * o + 1, (T)vy * inv);
            }
        }
    } else {
        G *g = (G *)grid;
        for (int i = threadIdx.x; i < TR * TC; i += blockDim.x) {
            const int gr = r0 + i / TC, gc = c0 + i % TC;
            if (gr >= R || gc >= pitch) continue;
            const int64_t o = (int64_t)gr * pitch + gc;
            if (!SPIN) {
                const G v = buf[i];
                if (v != G(0)) atomicAdd(g + o, v);
            } else {
                const G vx = buf[i], vy = buf[TR * TC + i];
                if (vx != G(0)) atomicAdd(g + 2 * o, vx);
                if (vy != G(0)) atomicAdd(g + 2 * o + 1, vy);
            }
        }
    }
}

// Plan time (integer-tile plans): kmax_t of every tile, the most of the tile's points
// whose W x W windows (from their first-tap cell) cover a single cell: counts
// h per first-tap cell of the tile, then window sums over W rows and W columns
// for every cell of the tile and its halo.
template <int W>
__global__ void __launch_bounds__(256) k_tile_window_kmax(const uint32_t *__restrict__ cell, int pitch, int ntc,
                                                         int tile_r, const uint32_t *__restrict__ tile_start,
                                                         unsigned short *__restrict__ out)
{
    constexpr int TC = kTileC + W - 1;
    const int TR = tile_r + W - 1;
    extern __shared__ int kmax_smem[];
    int *h = kmax_smem;                    // [tile_r][32] points per first-tap cell (lr, lc)
    int *v = kmax_smem + tile_r * kTileC;  // [TR][32]: v[r][c] = sum over a < W of h[r - a][c]
    __shared__ int best;
    const int t = blockIdx.x;
    const uint32_t p0 = tile_start[t], p1 = tile_start[t + 1];
    for (int i = threadIdx.x; i < tile_r * kTileC; i += blockDim.x) h[i] = 0;
    if (threadIdx.x == 0) best = 0;
    __syncthreads();
    const int r0 = (t / ntc) * tile_r, c0 = (t % ntc) * kTileC;
    for (uint32_t p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
        const uint32_t c = cell[p];
        const int lr = (int)(c / (uint32_t)pitch) - r0, lc = (int)(c % (uint32_t)pitch) - c0;
        if ((unsigned)lr < (unsigned)tile_r && (unsigned)lc < (unsigned)kTileC) atomicAdd(&h[lr * kTileC + lc], 1);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < TR * kTileC; i += blockDim.x) {
        const int r = i / kTileC, c = i % kTileC;
        int sum = 0;
        for (int a = 0; a < W; ++a)
            if (r - a >= 0 && r - a < tile_r) sum += h[(r - a) * kTileC + c];
        v[i] = sum;
    }
    __syncthreads();
    int mx = 0;
    for (int i = threadIdx.x; i < TR * TC; i += blockDim.x) {
        const int r = i / TC, c = i % TC;
        int sum = 0;
        for (int b = 0; b < W; ++b)
            if (c - b >= 0 && c - b < kTileC) sum += v[r * kTileC + c - b];
        mx = max(mx, sum);
    }
    atomicMax(&best, mx);
    __syncthreads();
    if (threadIdx.x == 0) out[t] = (unsigned short)min(best, 65535);
}

// ---------------------------------------------- fixed point (deterministic plans)
// Largest |x| (spin 0) or |Q| + |U| (spin s) of a map, as the bits of a
// non-negative double, which order like unsigned integers (a NaN input gives
// NaN bits, above those of infinity).
template <typename T, bool SPIN>
__global__ void k_fx_maxabs(const T *__restrict__ map, int64_t n, unsigned long long *__restrict__ out)
{
    double a = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = SPIN ? fabs((double)map[i]) + fabs((double)map[n + i]) : fabs((double)map[i]);
        a = (v > a || v != v) ? v : a;
    }
    unsigned long long b = (unsigned long long)__double_as_longlong(a);
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, b, off);
        b = o > b ? o : b;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(out, b);
}

// unit[0] = 2^k with k the largest integer (up to 122) such that
// Kmax max|x| 2^k <= 2^62; NaN when the bound is not finite
__global__ void k_fx_grid_unit(const unsigned long long *__restrict__ maxbits, const uint32_t *__restrict__ kmax,
                               double *__restrict__ unit)
{
    unit[0] = fx_unit((double)*kmax * __longlong_as_double((long long)*maxbits));
}

// grid[i] = fx[i] / unit in the plan's precision (fx and grid may coincide)
template <typename T>
__global__ void k_fx_to_grid(const unsigned long long *fx, T *grid, int64_t n, const double *__restrict__ unit)
{
    const double inv = 1.0 / unit[0];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        grid[i] = fx_value<T>((long long)fx[i], inv);
}

// Kmax: the most points any cell can receive (a tile's count plus those of
// its left, upper and upper-left neighbours); start as k_tile_bounds writes it
__global__ void k_tile_kmax(const uint32_t *__restrict__ start, int ntr, int ntc, uint32_t *__restrict__ kmax)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntr * ntc) return;
    const int tr = t / ntc, tc = t % ntc;
    auto cnt = [&](int r, int c) -> uint32_t {
        if (r < 0 || c < 0) return 0u;
        const int u = r * ntc + c;
        return start[u + 1] - start[u];
    };
    atomicMax(kmax, cnt(tr, tc) + cnt(tr, tc - 1) + cnt(tr - 1, tc) + cnt(tr - 1, tc - 1));
}

template <typename T, bool SPIN, int W>
cudaError_t interp_w(const Plan &p, const void *grid, void *map, cudaStream_t st)
{
    const int thr = 256;
    const int64_t blocks = (p.npts + thr - 1) / thr;
    if (blocks == 0) return cudaSuccess;
    const auto run = [&](auto kern) {
        kern<<<(unsigned)blocks, thr, 0, st>>>(grid, p.cell, (const cplx<T> *)p.frac, p.perm, (const cplx<T> *)p.phase,
                                               p.wts, (T *)map, p.npts, p.pitch, (T)p.beta, p.kpoly);
        return cudaGetLastError();
    };
    if constexpr (std::is_same<T, double>::value) {
        if (p.wts && p.wts_dd) {  // double-float taps on the double-float grid k_phi_fwd wrote
            k_interp_dd<W, SPIN><<<(unsigned)blocks, thr, 0, st>>>(grid, p.cell, p.perm, (const double2 *)p.phase,
                                                                   p.wts, (double *)map, p.npts, p.pitch);
            return cudaGetLastError();
        }
        if (p.wts) return run(k_interp<T, W, SPIN, 1>);
    }
    return run(k_interp<T, W, SPIN, 0>);
}

template <typename T, bool SPIN, int W>
cudaError_t spread_w(const Plan &p, const void *map, void *grid, cudaStream_t st)
{
    if (p.npts == 0) return cudaSuccess;
    const double *fxs = p.fx_scale;
    const size_t cells = (size_t)(p.tile_r + W - 1) * (kTileC + W - 1) * (SPIN ? 2 : 1);
    const auto run = [&](auto kern, size_t esz) {
        const size_t sm = cells * esz;
        cudaError_t e2 = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e2 != cudaSuccess) return e2;
        kern<<<(unsigned)p.ntiles, sizeof(T) == 8 ? kSpreadThreads64 : kSpreadThreads, sm, st>>>(
            grid, p.cell, (const cplx<T> *)p.frac, p.perm, (const cplx<T> *)p.phase, p.wts, (const T *)map, p.npts,
            p.pitch, p.R, p.ntile_c, p.tile_start, (T)p.beta, fxs, p.tile_r, p.tile_kmax, p.maxbits, p.kpoly);
        return cudaGetLastError();
    };
    if constexpr (std::is_same<T, double>::value) {
        if (!p.det && p.tile_kmax) {  // 64-bit integer tiles (double-float taps with double-float weights)
            if (p.wts && p.wts_dd && SPIN) {  // plus the staged points: int offset and float4 value each
                const size_t extra = (size_t)kDDBatch * (sizeof(int) + sizeof(float4));
                const auto kern = k_spread<T, W, SPIN, 2, false, true>;
                const size_t sm = ((cells + 1) & ~(size_t)1) * 8 + extra;
                cudaError_t e2 = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
                if (e2 != cudaSuccess) return e2;
                kern<<<(unsigned)p.ntiles, kSpreadThreads64, sm, st>>>(
                    grid, p.cell, (const cplx<T> *)p.frac, p.perm, (const cplx<T> *)p.phase, p.wts, (const T *)map,
                    p.npts, p.pitch, p.R, p.ntile_c, p.tile_start, (T)p.beta, fxs, p.tile_r, p.tile_kmax, p.maxbits,
                    p.kpoly);
                return cudaGetLastError();
            }
            if (p.wts && p.wts_dd) return run(k_spread<T, W, SPIN, 2, false, true>, 8);
            if (p.wts) return run(k_spread<T, W, SPIN, 1, false, true>, 8);
            return run(k_spread<T, W, SPIN, 0, false, true>, 8);
        }
        const unsigned blocks = (unsigned)((p.npts + 255) / 256);
        const cplx<T> *fr = (const cplx<T> *)p.frac, *ph = (const cplx<T> *)p.phase;
        const auto direct = [&](auto kern) {
            kern<<<blocks, 256, 0, st>>>(grid, p.cell, fr, p.perm, ph, p.wts, (const T *)map, p.npts, p.pitch,
                                         (T)p.beta, fxs, p.kpoly);
            return cudaGetLastError();
        };
        if (p.det) {
            if (p.wts) return p.wts_dd ? direct(k_spread_direct<T, W, SPIN, 2, true>)
                                       : direct(k_spread_direct<T, W, SPIN, 1, true>);
            return direct(k_spread_direct<T, W, SPIN, 0, true>);
        }
        if (p.wts) return p.wts_dd ? direct(k_spread_direct<T, W, SPIN, 2, false>)
                                   : direct(k_spread_direct<T, W, SPIN, 1, false>);
        return direct(k_spread_direct<T, W, SPIN, 0, false>);
    } else {
        if (p.det) return run(k_spread<T, W, SPIN, 0, true>, 8);
        if (p.tile_kmax) return run(k_spread<T, W, SPIN, 0, false, true>, 4);
        return run(k_spread<T, W, SPIN, 0, false>, sizeof(T));
    }
    return cudaGetLastError();
}

template <typename T, bool SPIN>
cudaError_t interp_dispatch(const Plan &p, const void *grid, void *map, cudaStream_t st)
{
    switch (p.W) {
    case 4: return interp_w<T, SPIN, 4>(p, grid, map, st);
    case 5: return interp_w<T, SPIN, 5>(p, grid, map, st);
    case 6: return interp_w<T, SPIN, 6>(p, grid, map, st);
    case 7: return interp_w<T, SPIN, 7>(p, grid, map, st);
    case 8: return interp_w<T, SPIN, 8>(p, grid, map, st);
    case 9: return interp_w<T, SPIN, 9>(p, grid, map, st);
    case 10: return interp_w<T, SPIN, 10>(p, grid, map, st);
    case 11: return interp_w<T, SPIN, 11>(p, grid, map, st);
    case 12: return interp_w<T, SPIN, 12>(p, grid, map, st);
    case 13: return interp_w<T, SPIN, 13>(p, grid, map, st);
    case 14: return interp_w<T, SPIN, 14>(p, grid, map, st);
    case 15: return interp_w<T, SPIN, 15>(p, grid, map, st);
    case 16: return interp_w<T, SPIN, 16>(p, grid, map, st);
    default: return cudaErrorInvalidValue;
    }
}

template <typename T, bool SPIN>
cudaError_t spread_dispatch(const Plan &p, const void *map, void *grid, cudaStream_t st)
{
    switch (p.W) {
    case 4: return spread_w<T, SPIN, 4>(p, map, grid, st);
    case 5: return spread_w<T, SPIN, 5>(p, map, grid, st);
    case 6: return spread_w<T, SPIN, 6>(p, map, grid, st);
    case 7: return spread_w<T, SPIN, 7>(p, map, grid, st);
    case 8: return spread_w<T, SPIN, 8>(p, map, grid, st);
    case 9: return spread_w<T, SPIN, 9>(p, map, grid, st);
    case 10: return spread_w<T, SPIN, 10>(p, map, grid, st);
    case 11: return spread_w<T, SPIN, 11>(p, map, grid, st);
    case 12: return spread_w<T, SPIN, 12>(p, map, grid, st);
    case 13: return spread_w<T, SPIN, 13>(p, map, grid, st);
    case 14: return spread_w<T, SPIN, 14>(p, map, grid, st);
    case 15: return spread_w<T, SPIN, 15>(p, map, grid, st);
    case 16: return spread_w<T, SPIN, 16>(p, map, grid, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_interp(const Plan &p, const void *grid, void *map, cudaStream_t st)
{
    if (p.prec == LENS_FP32)
        return p.spin ? interp_dispatch<float, true>(p, grid, map, st) : interp_dispatch<float, false>(p, grid, map, st);
    return p.spin ? interp_dispatch<double, true>(p, grid, map, st) : interp_dispatch<double, false>(p, grid, map, st);
}

cudaError_t launch_spread(const Plan &p, const void *map, void *grid, cudaStream_t st)
{
    const size_t eb = (p.prec == LENS_FP32 ? 4 : 8) * (p.spin ? 2 : 1);
    const size_t ncell = (size_t)p.R * p.pitch * (p.spin ? 2 : 1);
    cudaError_t e = cudaMemsetAsync(grid, 0, eb * (size_t)p.R * p.pitch, st);
    if (e != cudaSuccess) return e;
    const bool f32 = p.prec == LENS_FP32;
    if (!p.det) {
        if (p.tile_kmax) {  // fixed-point tiles: the map's largest |value| first
            if ((e = cudaMemsetAsync(p.maxbits, 0, sizeof(unsigned long long), st)) != cudaSuccess) return e;
            if (p.npts > 0) {
                const unsigned mb = (unsigned)std::min<int64_t>((p.npts + 255) / 256, 152 * 8);
                if (f32) {
                    if (p.spin) k_fx_maxabs<float, true><<<mb, 256, 0, st>>>((const float *)map, p.npts, p.maxbits);
                    else k_fx_maxabs<float, false><<<mb, 256, 0, st>>>((const float *)map, p.npts, p.maxbits);
                } else {
                    if (p.spin) k_fx_maxabs<double, true><<<mb, 256, 0, st>>>((const double *)map, p.npts, p.maxbits);
                    else k_fx_maxabs<double, false><<<mb, 256, 0, st>>>((const double *)map, p.npts, p.maxbits);
                }
                if ((e = cudaGetLastError()) != cudaSuccess) return e;
            }
        }
        if (f32)
            return p.spin ? spread_dispatch<float, true>(p, map, grid, st)
                          : spread_dispatch<float, false>(p, map, grid, st);
        return p.spin ? spread_dispatch<double, true>(p, map, grid, st)
                      : spread_dispatch<double, false>(p, map, grid, st);
    }
    // fixed point: FP32 plans accumulate in their own int64 grid, FP64 plans in place
    void *fxg = f32 ? p.fx_grid : grid;
    if (f32 && (e = cudaMemsetAsync(fxg, 0, 8 * ncell, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(p.fx_maxbits, 0, sizeof(unsigned long long), st)) != cudaSuccess) return e;
    const unsigned mb = (unsigned)std::min<int64_t>((p.npts + 255) / 256, 152 * 8);
    if (p.npts > 0) {
        if (f32) {
            if (p.spin) k_fx_maxabs<float, true><<<mb, 256, 0, st>>>((const float *)map, p.npts, p.fx_maxbits);
            else k_fx_maxabs<float, false><<<mb, 256, 0, st>>>((const float *)map, p.npts, p.fx_maxbits);
        } else {
            if (p.spin) k_fx_maxabs<double, true><<<mb, 256, 0, st>>>((const double *)map, p.npts, p.fx_maxbits);
            else k_fx_maxabs<double, false><<<mb, 256, 0, st>>>((const double *)map, p.npts, p.fx_maxbits);
        }
    }
    k_fx_grid_unit<<<1, 1, 0, st>>>(p.fx_maxbits, p.fx_kmax, p.fx_scale);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (f32)
        e = p.spin ? spread_dispatch<float, true>(p, map, fxg, st) : spread_dispatch<float, false>(p, map, fxg, st);
    else
        e = p.spin ? spread_dispatch<double, true>(p, map, fxg, st) : spread_dispatch<double, false>(p, map, fxg, st);
    if (e != cudaSuccess) return e;
    const unsigned cb = (unsigned)std::min<size_t>((ncell + 255) / 256, 152 * 16);
    if (f32) k_fx_to_grid<float><<<cb, 256, 0, st>>>((const unsigned long long *)fxg, (float *)grid, ncell, p.fx_scale);
    else k_fx_to_grid<double><<<cb, 256, 0, st>>>((const unsigned long long *)fxg, (double *)grid, ncell, p.fx_scale);
    return cudaGetLastError();
}

// Point preparation: validate, compute cells/offsets/phases in user order,
// radix-sort by tile key, gather into sorted order.  Temporary buffers are
// released before returning; the stream is synchronised once.
cudaError_t launch_prep_points(Plan &p, const double *theta, const double *phi, const double *chi,
                               cudaStream_t st, std::string &err)
{
    const int64_t n = p.npts;
    if (n == 0) return cudaSuccess;
    if (n > (int64_t)0x7fffffff) { err = "npoints above 2^31 - 1"; return cudaErrorInvalidValue; }
    uint32_t *key = nullptr, *key2 = nullptr, *cell_u = nullptr;
    int32_t *idx = nullptr;
    double2 *frac_u = nullptr, *phase_u = nullptr;
    void *tmp = nullptr;
    size_t tmp_bytes = 0;
    cudaError_t e = cudaSuccess;
    auto cleanup = [&]() {
        cudaFree(key); cudaFree(key2); cudaFree(cell_u); cudaFree(idx);
        cudaFree(frac_u); cudaFree(phase_u); cudaFree(tmp);
    };
#define GSL_TRY(x) do { e = (x); if (e != cudaSuccess) { cleanup(); return e; } } while (0)
    GSL_TRY(cudaMalloc(&key, n * sizeof(uint32_t)));
    GSL_TRY(cudaMalloc(&key2, n * sizeof(uint32_t)));
    GSL_TRY(cudaMalloc(&idx, n * sizeof(int32_t)));
    GSL_TRY(cudaMalloc(&cell_u, n * sizeof(uint32_t)));
    GSL_TRY(cudaMalloc(&frac_u, n * sizeof(double2)));
    if (p.spin) GSL_TRY(cudaMalloc(&phase_u, n * sizeof(double2)));
    GSL_TRY(cudaMemsetAsync(p.flags, 0, sizeof(unsigned), st));
    const int thr = 256;
    const unsigned blocks = (unsigned)((n + thr - 1) / thr);
    // N / (2 pi) as double-doubles: quotient of N by 2 pi = T_HI + T_LO, refined once
    auto scale_of = [](int N) {
        const double th = 6.283185307179586232, tl = 2.4492935982947064e-16;
        const double q1 = N / th;
        const double p = q1 * th, pe = fma(q1, th, -p);
        const double r = (((double)N - p) - pe) - q1 * tl;
        const double q2 = r / th;
        const double hi = q1 + q2;
        return make_double2(hi, q2 - (hi - q1));
    };
    k_prep<<<blocks, thr, 0, st>>>(theta, phi, chi, n, p.N1, p.N2, p.W, p.r_lo, p.R, p.pitch, p.spin, scale_of(p.N1),
                                   scale_of(p.N2), p.tile_r, key, idx, cell_u, frac_u, phase_u, p.flags);
    GSL_TRY(cudaGetLastError());
    const int ntc = (p.N2 + kTileC - 1) / kTileC;
    const uint64_t nkeys = (uint64_t)((p.R + p.tile_r - 1) / p.tile_r) * ntc;
    int bits = 1;
    while (bits < 32 && (1ull << bits) < nkeys) ++bits;
    GSL_TRY(cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, key, key2, idx, p.perm, (int)n, 0, bits, st));
    GSL_TRY(cudaMalloc(&tmp, tmp_bytes));
    GSL_TRY(cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, key, key2, idx, p.perm, (int)n, 0, bits, st));
    k_gather_points<<<blocks, thr, 0, st>>>(p.perm, n, cell_u, frac_u, phase_u, p.prec, p.spin, p.cell, p.frac,
                                            p.phase);
    GSL_TRY(cudaGetLastError());
    if (nkeys != (uint64_t)p.ntiles) { cleanup(); err = "internal: tile count mismatch"; return cudaErrorInvalidValue; }
    k_tile_bounds<<<(unsigned)((n + 1 + thr - 1) / thr), thr, 0, st>>>(key2, n, p.ntiles, p.tile_start);
    GSL_TRY(cudaGetLastError());
    if (p.det) {
        GSL_TRY(cudaMemsetAsync(p.fx_kmax, 0, sizeof(uint32_t), st));
        k_tile_kmax<<<(unsigned)((p.ntiles + thr - 1) / thr), thr, 0, st>>>(p.tile_start, p.ntiles / ntc, ntc, p.fx_kmax);
        GSL_TRY(cudaGetLastError());
    }
    if (p.tile_kmax) {  // fixed-point spreading tiles: kmax_t per tile
        const size_t sm = sizeof(int) * (size_t)kTileC * (2 * p.tile_r + p.W - 1);
        const auto run = [&](auto kern) {
            kern<<<(unsigned)p.ntiles, 256, sm, st>>>(p.cell, p.pitch, ntc, p.tile_r, p.tile_start, p.tile_kmax);
        };
        switch (p.W) {
        case 4: run(k_tile_window_kmax<4>); break;
        case 5: run(k_tile_window_kmax<5>); break;
        case 6: run(k_tile_window_kmax<6>); break;
        case 7: run(k_tile_window_kmax<7>); break;
        case 8: run(k_tile_window_kmax<8>); break;
        case 9: run(k_tile_window_kmax<9>); break;
        case 10: run(k_tile_window_kmax<10>); break;
        case 11: run(k_tile_window_kmax<11>); break;
        case 12: run(k_tile_window_kmax<12>); break;
        case 13: run(k_tile_window_kmax<13>); break;
        case 14: run(k_tile_window_kmax<14>); break;
        case 15: run(k_tile_window_kmax<15>); break;
        default: run(k_tile_window_kmax<16>); break;
        }
        GSL_TRY(cudaGetLastError());
    }
    if (p.wts) {
        k_weights<<<blocks, thr, 0, st>>>((const double2 *)p.frac, n, p.W, p.beta, p.wts, p.wts_dd ? 1 : 0);
        GSL_TRY(cudaGetLastError());
    }
    unsigned hflags = 0;
    GSL_TRY(cudaMemcpyAsync(&hflags, p.flags, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    GSL_TRY(cudaStreamSynchronize(st));
#undef GSL_TRY
    cleanup();
    if (hflags & FLAG_DOMAIN) { err = "a coordinate is not finite or theta is outside [0, pi]"; return cudaErrorInvalidValue; }
    if (hflags & FLAG_OOB) { err = "internal: a point fell outside the kept rows"; return cudaErrorInvalidValue; }
    return cudaSuccess;
}

}  // namespace gsl
