// Legendre recursion building blocks shared by the Legendre kernels
// (legendre.cu) and the tensor-core batched synthesis (legendre_tc.cu):
// arithmetic policies, start values and the per-thread ring state.  See
// legendre.cu for the recursion itself (monic and normalised forms, scaling).
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "common.cuh"
#include "internal.h"

namespace gsl {
namespace {

constexpr float kBigF = 0x1p60f;
constexpr float kSmallF = 0x1p-60f;
constexpr double kBigD = 0x1p60;
constexpr double kSmallD = 0x1p-60;
constexpr int kSkipE = -4;  // below 2^-180 before a block; 8 steps grow by at most 2^68
constexpr int kBlk = kLegBlock;

__device__ __forceinline__ int64_t alm_base(int lmax, int m) { return (int64_t)m * (2 * lmax + 1 - m) / 2; }

__device__ __forceinline__ df32 df_add_u(df32 a, df32 b) { return df_sub_u(a, {-b.h, -b.l}); }
__device__ __forceinline__ df32 df_norm(df32 a)  // two-sum: exact for any ordering of |h|, |l|
{
    const float h = __fadd_rn(a.h, a.l);
    const float bb = __fsub_rn(h, a.h);
    return {h, __fadd_rn(__fsub_rn(a.h, __fsub_rn(h, bb)), __fsub_rn(a.l, bb))};
}

// ------------------------------------------------------------ policies
// A recursion state holds two consecutive degrees in w[0], w[1]; which word is
// the newest alternates.  E is the power-of-2^60 scale shared by both words.
//
// Accumulation interface: V is the value handed from the recursion to the
// sums, K a real coefficient component (prepared a_lm or ring input), A a
// real accumulator; fma(acc, k, v) is acc += k v, fms(acc, k, v) acc -= k v.
struct PolDF {  // df32 recursion, FP32 accumulation (FP32 plans)
    static constexpr bool kRestart = false;  // no restart values (see PolS, PolDDR)
    static constexpr bool kMonic = true;     // values carry the monic scale c_l (scale table)
    static constexpr bool kScaleF = false;   // c_l from the FP32 (c_l, 1/c_l) table instead (PolSM)
    using R = float;
    using C = float2;
    using X = df32;
    using Tab = float2;   // alpha (hi, lo)
    using TTab = float2;  // tau (hi, lo)
    using V = float;
    using K = float;
    using A = float;
    struct St { df32 w[2]; int E; };
    static __device__ __forceinline__ X load(const Tab *tab, int l)
    {
        const float2 c = __ldg(tab + l);
        return {c.x, c.y};
    }
    static __device__ __forceinline__ X load_t(const TTab *tab, int l) { return load(tab, l); }
    // spin s: alpha and tau interleaved, float4 (alpha_hi, alpha_lo, tau_hi, tau_lo)
    using TabAT = float4;
    static __device__ __forceinline__ void load_at(const TabAT *tab, const TTab *, int l, X &al, X &t)
    {
        const float4 c = __ldg(tab + l);
        al = {c.x, c.y};
        t = {c.z, c.w};
    }
    static __device__ __forceinline__ X ring_x(const RingTab &rt, int j)
    {
        const float2 v = __ldg(rt.xdf + j);
        return {v.x, v.y};
    }
    static __device__ __forceinline__ X mul(X a, X b) { return df_mul(a, b); }
    static __device__ __forceinline__ X add(X a, X b) { return df_add_u(a, b); }
    static __device__ __forceinline__ X sub(X a, X b) { return df_sub_u(a, b); }
    // alpha x +- tau: Fast2Sum on the high words (exact when |alpha x| >= |tau|,
    // i.e. everywhere except on rings within ~m / l^2 of the equator, where the
    // step coefficient then carries an FP32-size error: negligible for the
    // FP32 plans' 2e-6 floor), plus the low words.
    static __device__ __forceinline__ X addx(X a, X t)
    {
        const float s = __fadd_rn(a.h, t.h);
        const float e = __fsub_rn(t.h, __fsub_rn(s, a.h));
        return {s, __fadd_rn(e, __fadd_rn(a.l, t.l))};
    }
    static __device__ __forceinline__ X subx(X a, X t)
    {
        const float s = __fsub_rn(a.h, t.h);
        const float e = __fsub_rn(__fsub_rn(a.h, s), t.h);
        return {s, __fadd_rn(e, __fsub_rn(a.l, t.l))};
    }
    // new = y q - p, written over p
    static __device__ __forceinline__ void step(df32 &p, const df32 &q, X y) { p = df_sub_u(df_mul(y, q), p); }
    // The words are not renormalised after every step (the low word carries
    // the compensation of the high-word recursion), so a value is h + l.
    static __device__ __forceinline__ V val(const df32 &a) { return __fadd_rn(a.h, a.l); }
    static __device__ __forceinline__ void renorm(St &s)
    {
        s.w[0] = df_norm(s.w[0]);
        s.w[1] = df_norm(s.w[1]);
    }
    static __device__ __forceinline__ void rescale(St &s, int newest)
    {
        if (s.E < 0 && fabsf(s.w[newest].h) > kBigF) {
            s.w[0] = df_scale_pow2(s.w[0], kSmallF);
            s.w[1] = df_scale_pow2(s.w[1], kSmallF);
            s.E += 1;
        }
    }
    static __device__ __forceinline__ float fac(int E) { return E == 0 ? 1.0f : (E == -1 ? kSmallF : 0.0f); }
    // start value 2^L2 * sign as mantissa * 2^(60 E), in w[1]; w[0] = 0
    static __device__ __forceinline__ void start(St &s, double L2, int sign, bool zero)
    {
        s.w[0] = {0.f, 0.f};
        if (zero) { s.w[1] = {0.f, 0.f}; s.E = -1000; return; }
        const double e = floor(L2 * (1.0 / kScaleBits));
        const double fr = L2 - e * kScaleBits;  // [0, 60)
        const double ip = floor(fr);
        const float m = ldexpf(exp2f((float)(fr - ip)), (int)ip);
        s.w[1] = {sign < 0 ? -m : m, 0.f};
        s.E = (int)e;
    }
    static __device__ __forceinline__ void zero(St &s) { s.w[0] = {0.f, 0.f}; s.w[1] = s.w[0]; s.E = 0; }
    // accumulation
    static __device__ __forceinline__ V vscale(V v, float f) { return v * f; }
    static __device__ __forceinline__ V vsign(V v, float sg) { return v * sg; }
    static __device__ __forceinline__ void fma(A &acc, K k, V v) { acc = __fmaf_rn(k, v, acc); }
    static __device__ __forceinline__ void fms(A &acc, K k, V v) { acc = __fmaf_rn(-k, v, acc); }
    static __device__ __forceinline__ void fma2(A &acc, K k1, V v1, K k2, V v2)
    {
        acc = __fmaf_rn(k2, v2, __fmaf_rn(k1, v1, acc));
    }
    static __device__ __forceinline__ void fma2m(A &acc, K k1, V v1, K k2, V v2)
    {
        acc = __fmaf_rn(-k2, v2, __fmaf_rn(k1, v1, acc));
    }
    static __device__ __forceinline__ A azero() { return 0.f; }
    static __device__ __forceinline__ K kadd(K a, K b) { return a + b; }
    static __device__ __forceinline__ K ksub(K a, K b) { return a - b; }
    static __device__ __forceinline__ K ksign(K a, float sg) { return a * sg; }
    static __device__ __forceinline__ void arenorm(A &) {}
    static __device__ __forceinline__ R aout(A a) { return a; }
    static __device__ __forceinline__ A aadd(A a, A b) { return a + b; }
    static __device__ __forceinline__ A asub(A a, A b) { return a - b; }
    static __device__ __forceinline__ A ascale(A a, float f) { return a * f; }
    static __device__ __forceinline__ A shfl_xor(A v, int off) { return __shfl_xor_sync(0xffffffffu, v, off); }
    // *dst += c v (c the monic-form scale of the degree)
    static __device__ __forceinline__ void atomic_add(R *dst, A v, double c) { atomicAdd(dst, v * (float)c); }
    // deterministic plans: the same term in fixed point, units of 1 / unit (a power of two)
    static __device__ __forceinline__ void atomic_add_fx(unsigned long long *dst, A v, double c, double unit)
    {
        atomicAdd(dst, (unsigned long long)__float2ll_rn(v * (float)c * (float)unit));
    }
    // prepared coefficient (re, im) of entry idx, component comp
    static __device__ __forceinline__ void coef(const void *tab, int64_t nalm, int comp, int64_t idx, K &re, K &im)
    {
        const float2 v = __ldg((const float2 *)tab + comp * nalm + idx);
        re = v.x;
        im = v.y;
    }
    static __device__ __forceinline__ void ring_in(const C *ring, int64_t idx, K &re, K &im)
    {
        const float2 v = ring[idx];
        re = v.x;
        im = v.y;
    }
    static __device__ __forceinline__ C cout(A re, A im) { return make_float2(re, im); }
};

struct PolF64 {  // native FP64 (FP64 plans, low orders)
    static constexpr bool kRestart = false;
    static constexpr bool kMonic = true;
    static constexpr bool kScaleF = false;
    using R = double;
    using C = double2;
    using X = double;
    using Tab = double;   // alpha
    using TTab = double;  // tau
    using V = double;
    using K = double;
    using A = double;
    struct St { double w[2]; int E; };
    static __device__ __forceinline__ X load(const Tab *tab, int l) { return __ldg(tab + l); }
    static __device__ __forceinline__ X load_t(const TTab *tab, int l) { return __ldg(tab + l); }
    using TabAT = double;  // alpha; tau in its own table
    static __device__ __forceinline__ void load_at(const TabAT *tab, const TTab *tt, int l, X &al, X &t)
    {
        al = __ldg(tab + l);
        t = __ldg(tt + l);
    }
    static __device__ __forceinline__ X ring_x(const RingTab &rt, int j) { return __ldg(rt.x + j); }
    static __device__ __forceinline__ X mul(X a, X b) { return a * b; }
    static __device__ __forceinline__ X add(X a, X b) { return a + b; }
    static __device__ __forceinline__ X sub(X a, X b) { return a - b; }
    static __device__ __forceinline__ X addx(X a, X t) { return a + t; }
    static __device__ __forceinline__ X subx(X a, X t) { return a - t; }
    static __device__ __forceinline__ void step(double &p, const double &q, X y) { p = __fma_rn(y, q, -p); }
    static __device__ __forceinline__ V val(const double &a) { return a; }
    static __device__ __forceinline__ void renorm(St &) {}
    static __device__ __forceinline__ void rescale(St &s, int newest)
    {
        if (s.E < 0 && fabs(s.w[newest]) > kBigD) {
            s.w[0] *= kSmallD;
            s.w[1] *= kSmallD;
            s.E += 1;
        }
    }
    static __device__ __forceinline__ double fac(int E) { return E == 0 ? 1.0 : (E == -1 ? kSmallD : 0.0); }
    static __device__ __forceinline__ void start(St &s, double L2, int sign, bool zero)
    {
        s.w[0] = 0.0;
        if (zero) { s.w[1] = 0.0; s.E = -1000; return; }
        const double e = floor(L2 * (1.0 / kScaleBits));
        const double fr = L2 - e * kScaleBits;
        const double m = exp2(fr);
        s.w[1] = sign < 0 ? -m : m;
        s.E = (int)e;
    }
    static __device__ __forceinline__ void zero(St &s) { s.w[0] = 0.0; s.w[1] = 0.0; s.E = 0; }
    static __device__ __forceinline__ V vscale(V v, double f) { return v * f; }
    static __device__ __forceinline__ V vsign(V v, double sg) { return v * sg; }
    static __device__ __forceinline__ void fma(A &acc, K k, V v) { acc = __fma_rn(k, v, acc); }
    static __device__ __forceinline__ void fms(A &acc, K k, V v) { acc = __fma_rn(-k, v, acc); }
    static __device__ __forceinline__ void fma2(A &acc, K k1, V v1, K k2, V v2)
    {
        acc = __fma_rn(k2, v2, __fma_rn(k1, v1, acc));
    }
    static __device__ __forceinline__ void fma2m(A &acc, K k1, V v1, K k2, V v2)
    {
        acc = __fma_rn(-k2, v2, __fma_rn(k1, v1, acc));
    }
    static __device__ __forceinline__ A azero() { return 0.0; }
    static __device__ __forceinline__ K kadd(K a, K b) { return a + b; }
    static __device__ __forceinline__ K ksub(K a, K b) { return a - b; }
    static __device__ __forceinline__ K ksign(K a, double sg) { return a * sg; }
    static __device__ __forceinline__ void arenorm(A &) {}
    static __device__ __forceinline__ R aout(A a) { return a; }
    static __device__ __forceinline__ A aadd(A a, A b) { return a + b; }
    static __device__ __forceinline__ A asub(A a, A b) { return a - b; }
    static __device__ __forceinline__ A ascale(A a, double f) { return a * f; }
    static __device__ __forceinline__ A shfl_xor(A v, int off) { return __shfl_xor_sync(0xffffffffu, v, off); }
    static __device__ __forceinline__ void atomic_add(R *dst, A v, double c) { atomicAdd(dst, v * c); }
    static __device__ __forceinline__ void atomic_add_fx(unsigned long long *dst, A v, double c, double unit)
    {
        atomicAdd(dst, (unsigned long long)__double2ll_rn(v * c * unit));
    }
    static __device__ __forceinline__ void coef(const void *tab, int64_t nalm, int comp, int64_t idx, K &re, K &im)
    {
        const double2 v = __ldg((const double2 *)tab + comp * nalm + idx);
        re = v.x;
        im = v.y;
    }
    static __device__ __forceinline__ void ring_in(const C *ring, int64_t idx, K &re, K &im)
    {
        const double2 v = ring[idx];
        re = v.x;
        im = v.y;
    }
    static __device__ __forceinline__ C cout(A re, A im) { return make_double2(re, im); }
};

// FP64 plans, orders m >= m_df: the df32 recursion of PolDF with df32 sums and
// df32 prepared coefficients.
struct PolDD : PolDF {
    using R = double;
    using C = double2;
    using V = df32;
    using K = df32;
    using A = df32;
    static __device__ __forceinline__ V val(const df32 &a) { return a; }
    // FP64 plans: the step coefficients keep full double-float accuracy
    static __device__ __forceinline__ X addx(X a, X t) { return df_add_u(a, t); }
    static __device__ __forceinline__ X subx(X a, X t) { return df_sub_u(a, t); }
    // start mantissa to df32 accuracy (exp2 in FP64, split in two words)
    static __device__ __forceinline__ void start(St &s, double L2, int sign, bool zero)
    {
        s.w[0] = {0.f, 0.f};
        if (zero) { s.w[1] = {0.f, 0.f}; s.E = -1000; return; }
        const double e = floor(L2 * (1.0 / kScaleBits));
        const double fr = L2 - e * kScaleBits;
        const double m = exp2(fr);
        s.w[1] = df_split(sign < 0 ? -m : m);
        s.E = (int)e;
    }
    static __device__ __forceinline__ V vscale(V v, float f) { return df_scale_pow2(v, f); }
    static __device__ __forceinline__ V vsign(V v, float sg) { return df_scale_pow2(v, sg); }
    static __device__ __forceinline__ void fma(A &acc, K k, V v) { acc = df_add_u(acc, df_mul(k, v)); }
    static __device__ __forceinline__ void fms(A &acc, K k, V v) { acc = df_sub_u(acc, df_mul(k, v)); }
    static __device__ __forceinline__ void fma2(A &acc, K k1, V v1, K k2, V v2)
    {
        acc = df_add_u(acc, df_add_u(df_mul(k1, v1), df_mul(k2, v2)));
    }
    static __device__ __forceinline__ void fma2m(A &acc, K k1, V v1, K k2, V v2)
    {
        acc = df_add_u(acc, df_sub_u(df_mul(k1, v1), df_mul(k2, v2)));
    }
    static __device__ __forceinline__ A azero() { return {0.f, 0.f}; }
    static __device__ __forceinline__ K kadd(K a, K b) { return df_add_u(a, b); }
    static __device__ __forceinline__ K ksub(K a, K b) { return df_sub_u(a, b); }
    static __device__ __forceinline__ K ksign(K a, float sg) { return df_scale_pow2(a, sg); }
    static __device__ __forceinline__ void arenorm(A &a) { a = df_norm(a); }
    static __device__ __forceinline__ R aout(A a) { return (double)a.h + (double)a.l; }
    static __device__ __forceinline__ A aadd(A a, A b) { return df_add_u(a, b); }
    static __device__ __forceinline__ A asub(A a, A b) { return df_sub_u(a, b); }
    static __device__ __forceinline__ A ascale(A a, float f) { return df_scale_pow2(a, f); }
    static __device__ __forceinline__ A shfl_xor(A v, int off)
    {
        return {__shfl_xor_sync(0xffffffffu, v.h, off), __shfl_xor_sync(0xffffffffu, v.l, off)};
    }
    static __device__ __forceinline__ void atomic_add(R *dst, A v, double c) { atomicAdd(dst, aout(v) * c); }
    static __device__ __forceinline__ void atomic_add_fx(unsigned long long *dst, A v, double c, double unit)
    {
        atomicAdd(dst, (unsigned long long)__double2ll_rn(aout(v) * c * unit));
    }
    // table entry: float4 (re_h, re_l, im_h, im_l)
    static __device__ __forceinline__ void coef(const void *tab, int64_t nalm, int comp, int64_t idx, K &re, K &im)
    {
        const float4 v = __ldg((const float4 *)tab + comp * nalm + idx);
        re = {v.x, v.y};
        im = {v.z, v.w};
    }
    static __device__ __forceinline__ void ring_in(const C *ring, int64_t idx, K &re, K &im)
    {
        const double2 v = ring[idx];
        re = df_split(v.x);
        im = df_split(v.y);
    }
    static __device__ __forceinline__ C cout(A re, A im) { return make_double2(aout(re), aout(im)); }
};

// FP64 plans with restart values (epsilon >= 5e-11): PolDD's monic df32
// recursion and df32 sums for every order, its state reset every K degrees to
// the FP64 recursion's monic values split into df32 words (k_ck_build64), so
// that df32 rounding accumulates over at most K steps and no order needs the
// FP64 pipe; each warp starts at its first restart with a value above 2^-64.
struct PolDDR : PolDD {
    static constexpr bool kRestart = true;
};

// FP32 plans with restart values (the default for epsilon >= 1e-5): FP32
// recursion state in the normalised form
//   lambda_l = (A_l x + sigma AT_l) lambda_{l-1} - B_l lambda_{l-2},  AT_l = A_l T_l,
// reset every K degrees to FP32 values of lambda computed at plan creation by
// an FP64 recursion (k_ck_build), so that FP32 rounding accumulates over at
// most K steps instead of lmax.  Table entry per (m, l): float4
// (A_l, B_l, AT_l, K_l) with K_l = 1 + B_l - A_l - AT_l (the +s value;
// -s: K_l + 2 AT_l).  The values are lambda itself (no monic scale c_l).
// Two forms of the step, chosen per warp by ring (Rings<PolS> / Rings<PolR>):
//  * PolS, rings with x = cos theta below ~0.7: the plain step above.
//  * PolR, rings nearer the pole: Reinsch's form, state (lambda_l,
//    D_l = lambda_l - lambda_{l-1}) with
//      D_l = B_l D_{l-1} - d_l lambda_{l-1},  lambda_l = lambda_{l-1} + D_l,
//      d_l = 1 + B_l - A_l x - sigma AT_l = K_l + A_l (1 - x).
//    There the plain step coefficient is close to 2 and its FP32 rounding
//    (an absolute 1e-7) shifts the phase of the oscillation by ~1e-7 / theta
//    per degree; d_l is formed from 1 - x and the small K_l, so its rounding
//    is relative to d_l instead.
// Accumulation as PolDF (FP32).  Start values and the 2^(60 E) scaling as PolDF.
struct PolS : PolDF {
    static constexpr bool kRestart = true;
    static constexpr bool kMonic = false;  // lambda itself
    static constexpr bool kScaleF = false;
    using X = float;
    using Tab = float4;
    using TTab = float4;
    using TabAT = float4;
    struct St { float w[2]; int E; };
    static __device__ __forceinline__ void start(St &s, double L2, int sign, bool zero)
    {
        s.w[0] = 0.f;
        if (zero) { s.w[1] = 0.f; s.E = -1000; return; }
        const double e = floor(L2 * (1.0 / kScaleBits));
        const double fr = L2 - e * kScaleBits;  // [0, 60)
        const double ip = floor(fr);
        const float m = ldexpf(exp2f((float)(fr - ip)), (int)ip);
        s.w[1] = sign < 0 ? -m : m;
        s.E = (int)e;
    }
    static __device__ __forceinline__ void zero(St &s) { s.w[0] = 0.f; s.w[1] = 0.f; s.E = 0; }
    static __device__ __forceinline__ void rescale(St &s, int newest)
    {
        if (s.E < 0 && fabsf(s.w[newest]) > kBigF) {
            s.w[0] *= kSmallF;
            s.w[1] *= kSmallF;
            s.E += 1;
        }
    }
};
struct PolR : PolS {};
// PolSM: the plain-form rings (cos theta below ~0.7) in the monic form,
//   mu_l = (alpha_l x + sigma tau_l) mu_{l-1} - mu_{l-2},  mu_l = lambda_l / c_l,
// with (alpha, tau) the high words of the df32 table: per step and sign of the
// spin one multiplication fewer than PolS.  The restart values stay those of
// PolS (lambda), divided by c_l as they are loaded (FP32 table of (c_l, 1/c_l));
// the forward coefficients carry c_l (a second prepared set).  Used by the
// forward only (the adjoint measured slower with it).  Reinsch's form (PolR)
// keeps the normalised step: the monic alpha_l alternates between even and odd l.
struct PolSM : PolS {
    using Tab = float2;    // spin 0: (alpha_h, alpha_l) of the df32 table
    using TabAT = float4;  // spin s: (alpha_h, alpha_l, tau_h, tau_l)
    static constexpr bool kScaleF = true;
};

// Start value of sigma lambda_{l0,m} at ring j (north half), sigma = +-s.
//   m >= s:  (-1)^m sqrt((2m+1)/4pi C(2m, m+s)) c^(m-sigma) s^(m+sigma)
//   m <  s:  sigma>0: (-1)^m ..(2s+1).. c^(s-m) s^(s+m); sigma<0: (-1)^s .. c^(s+m) s^(s-m)
// with c = cos(theta/2), s = sin(theta/2); lognorm[m] = log2 sqrt(...).
template <class P>
__device__ __forceinline__ void start_value(typename P::St &st, int m, int s, int sigma, double lognorm,
                                            double lsin2, double lcos2)
{
    int a, b, sign;
    if (m >= s) { a = m - sigma; b = m + sigma; sign = (m & 1) ? -1 : 1; }
    else if (sigma > 0) { a = s - m; b = s + m; sign = (m & 1) ? -1 : 1; }
    else { a = s + m; b = s - m; sign = (s & 1) ? -1 : 1; }
    bool zero = false;
    double L2 = lognorm;
    if (a > 0) L2 = fma((double)a, lcos2, L2);
    if (b > 0) {
        if (isinf(lsin2)) zero = true;
        else L2 = fma((double)b, lsin2, L2);
    }
    P::start(st, L2, sign, zero);
}

// Per-thread state of RPT rings (spin s: a +s and a -s recursion per ring).
template <class P, int RPT, bool SPIN> struct Rings {
    typename P::X x[RPT];
    typename P::St sp[RPT], sm[RPT];

    __device__ __forceinline__ void init(const RingTab &rt, int rp0, int nnorth, int m, int s, double lnm)
    {
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            const int rp = rp0 + k;
            if (rp < nnorth) {
                x[k] = P::ring_x(rt, rp);
                const double ls = rt.lsin2[rp], lc = rt.lcos2[rp];
                start_value<P>(sp[k], m, s, s, lnm, ls, lc);
                if (SPIN) start_value<P>(sm[k], m, s, -s, lnm, ls, lc);
            } else {
                x[k] = typename P::X{};
                P::zero(sp[k]);
                P::zero(sm[k]);
            }
        }
    }
    // ring geometry only (PolDDR: the state comes from a restart)
    __device__ __forceinline__ void init_geom(const RingTab &rt, int rp0, int nnorth)
    {
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            x[k] = rp0 + k < nnorth ? P::ring_x(rt, rp0 + k) : typename P::X{};
            P::zero(sp[k]);
            P::zero(sm[k]);
        }
    }
    // PolDDR restart: df32 words (w0.h, w0.l, w1.h, w1.l) per sign of the spin
    // (spin s: +s then -s, two float4) and the exponent E (short / short2)
    __device__ __forceinline__ void restart(const CkTab &ck, int64_t row, int rp0, int nnorth)
    {
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            const int rp = rp0 + k;
            if (rp >= nnorth) continue;
            if (!SPIN) {
                const float4 v = __ldg((const float4 *)ck.v + row + rp);
                sp[k].w[0] = {v.x, v.y}; sp[k].w[1] = {v.z, v.w};
                sp[k].E = __ldg((const short *)ck.e + row + rp);
            } else {
                const float4 a = __ldg((const float4 *)ck.v + 2 * (row + rp));
                const float4 b = __ldg((const float4 *)ck.v + 2 * (row + rp) + 1);
                const short2 e = __ldg((const short2 *)ck.e + row + rp);
                sp[k].w[0] = {a.x, a.y}; sp[k].w[1] = {a.z, a.w}; sp[k].E = e.x;
                sm[k].w[0] = {b.x, b.y}; sm[k].w[1] = {b.z, b.w}; sm[k].E = e.y;
            }
        }
    }
    // Regime of the next block for the whole warp: 0 all states at scale 0,
    // 1 all states negligible (scale <= kSkipE), 2 mixed.  Renormalises the
    // df32 words first (once per block).
    __device__ __forceinline__ int regime()
    {
        bool all0 = true, allneg = true;
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            P::renorm(sp[k]);
            all0 = all0 && sp[k].E == 0;
            allneg = allneg && sp[k].E <= kSkipE;
            if (SPIN) {
                P::renorm(sm[k]);
                all0 = all0 && sm[k].E == 0;
                allneg = allneg && sm[k].E <= kSkipE;
            }
        }
        if (__all_sync(0xffffffffu, all0)) return 0;
        if (__all_sync(0xffffffffu, allneg)) return 1;
        return 2;
    }
    // One step to degree l; the newest value goes into word NW.
    template <int NW, bool CHECK>
    __device__ __forceinline__ void advance(const typename P::Tab *reca, const typename P::TTab *rect, int l)
    {
        if (!SPIN) {
            const typename P::X al = P::load(reca, l);
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                P::step(sp[k].w[NW], sp[k].w[1 - NW], P::mul(al, x[k]));
                if (CHECK) P::rescale(sp[k], NW);
            }
        } else {
            typename P::X al, t;
            P::load_at(reinterpret_cast<const typename P::TabAT *>(reca), rect, l, al, t);
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                const typename P::X ax = P::mul(al, x[k]);
                P::step(sp[k].w[NW], sp[k].w[1 - NW], P::addx(ax, t));
                P::step(sm[k].w[NW], sm[k].w[1 - NW], P::subx(ax, t));
                if (CHECK) { P::rescale(sp[k], NW); P::rescale(sm[k], NW); }
            }
        }
    }
    // Tail step: word 1 moves to word 0, the newest goes into word 1.
    __device__ __forceinline__ void advance_moved(const typename P::Tab *reca, const typename P::TTab *rect, int l)
    {
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            const auto a = sp[k].w[0];
            sp[k].w[0] = sp[k].w[1];
            sp[k].w[1] = a;
            if (SPIN) {
                const auto b = sm[k].w[0];
                sm[k].w[0] = sm[k].w[1];
                sm[k].w[1] = b;
            }
        }
        advance<1, true>(reca, rect, l);
    }
    template <int NW, bool SCALED> __device__ __forceinline__ typename P::V vplus(int k) const
    {
        typename P::V v = P::val(sp[k].w[NW]);
        if (SCALED) v = P::vscale(v, P::fac(sp[k].E));
        return v;
    }
    template <int NW, bool SCALED> __device__ __forceinline__ typename P::V vminus(int k) const
    {
        typename P::V v = P::val(sm[k].w[NW]);
        if (SCALED) v = P::vscale(v, P::fac(sm[k].E));
        return v;
    }
};

// Rings of the restarted FP32 recursion, plain form: word NW receives the
// newest value (as in the generic Rings), so at a block boundary w[1] holds
// lambda_{l-1} and w[0] lambda_{l-2}.
template <int RPT, bool SPIN> struct Rings<PolS, RPT, SPIN> {
    using P = PolS;
    float x[RPT];
    P::St sp[RPT], sm[RPT];

    // ring geometry only (the state comes from a restart)
    __device__ __forceinline__ void init_geom(const RingTab &rt, int rp0, int nnorth)
    {
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            x[k] = rp0 + k < nnorth ? __ldg(rt.xdf + rp0 + k).x : 0.f;
            P::zero(sp[k]);
            P::zero(sm[k]);
        }
    }
    __device__ __forceinline__ void init(const RingTab &rt, int rp0, int nnorth, int m, int s, double lnm)
    {
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            const int rp = rp0 + k;
            if (rp < nnorth) {
                x[k] = __ldg(rt.xdf + rp).x;
                const double ls = rt.lsin2[rp], lc = rt.lcos2[rp];
                start_value<P>(sp[k], m, s, s, lnm, ls, lc);
                if (SPIN) start_value<P>(sm[k], m, s, -s, lnm, ls, lc);
            } else {
                x[k] = 0.f;
                P::zero(sp[k]);
                P::zero(sm[k]);
            }
        }
    }
    __device__ __forceinline__ int regime() const
    {
        bool all0 = true, allneg = true;
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            all0 = all0 && sp[k].E == 0;
            allneg = allneg && sp[k].E <= kSkipE;
            if (SPIN) {
                all0 = all0 && sm[k].E == 0;
                allneg = allneg && sm[k].E <= kSkipE;
            }
        }
        if (__all_sync(0xffffffffu, all0)) return 0;
        if (__all_sync(0xffffffffu, allneg)) return 1;
        return 2;
    }
    template <int NW, bool CHECK>
    __device__ __forceinline__ void advance(const float4 *reca, const float4 *, int l)
    {
        advance_c<NW, CHECK>(__ldg(reca + l));
    }
    // one step with the step-table entry c = (A, B, AT, K) of the degree already loaded
    template <int NW, bool CHECK> __device__ __forceinline__ void advance_c(const float4 c)
    {
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            if (!SPIN) {
                sp[k].w[NW] = __fmaf_rn(c.x * x[k], sp[k].w[1 - NW], -(c.y * sp[k].w[NW]));
            } else {
                const float cp = __fmaf_rn(c.x, x[k], c.z), cm = __fmaf_rn(c.x, x[k], -c.z);
                sp[k].w[NW] = __fmaf_rn(cp, sp[k].w[1 - NW], -(c.y * sp[k].w[NW]));
                sm[k].w[NW] = __fmaf_rn(cm, sm[k].w[1 - NW], -(c.y * sm[k].w[NW]));
            }
            if (CHECK) {
                P::rescale(sp[k], NW);
                if (SPIN) P::rescale(sm[k], NW);
            }
        }
    }
    __device__ __forceinline__ void advance_moved(const float4 *reca, const float4 *rect, int l)
    {
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            const float a = sp[k].w[0];
            sp[k].w[0] = sp[k].w[1];
            sp[k].w[1] = a;
            if (SPIN) {
                const float b = sm[k].w[0];
                sm[k].w[0] = sm[k].w[1];
                sm[k].w[1] = b;
            }
        }
        advance<1, true>(reca, rect, l);
    }
    template <int NW, bool SCALED> __device__ __forceinline__ float vplus(int k) const
    {
        return SCALED ? sp[k].w[NW] * P::fac(sp[k].E) : sp[k].w[NW];
    }
    template <int NW, bool SCALED> __device__ __forceinline__ float vminus(int k) const
    {
        return SCALED ? sm[k].w[NW] * P::fac(sm[k].E) : sm[k].w[NW];
    }
    // restart: state (w[0], w[1]) and exponent E from the table
    __device__ __forceinline__ void restart(const CkTab &ck, int64_t row, int rp0, int nnorth)
    {
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            const int rp = rp0 + k;
            if (rp >= nnorth) continue;
            if (!SPIN) {
                const float2 v = __ldg((const float2 *)ck.v + row + rp);
                sp[k].w[0] = v.x; sp[k].w[1] = v.y; sp[k].E = __ldg((const short *)ck.e + row + rp);
            } else {
                const float4 v = __ldg((const float4 *)ck.v + row + rp);
                const short2 e = __ldg((const short2 *)ck.e + row + rp);
                sp[k].w[0] = v.x; sp[k].w[1] = v.y; sp[k].E = e.x;
                sm[k].w[0] = v.z; sm[k].w[1] = v.w; sm[k].E = e.y;
            }
        }
    }
};

// Rings of the restarted FP32 recursion in the monic plain form (PolSM):
// state, words and scaling as Rings<PolS>.
template <int RPT, bool SPIN> struct Rings<PolSM, RPT, SPIN> {
    using P = PolS;
    float x[RPT];
    P::St sp[RPT], sm[RPT];

    __device__ __forceinline__ void init_geom(const RingTab &rt, int rp0, int nnorth)
    {
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            x[k] = rp0 + k < nnorth ? __ldg(rt.xdf + rp0 + k).x : 0.f;
            P::zero(sp[k]);
            P::zero(sm[k]);
        }
    }
    // start values at l0 (c_{l0} = c_{l0+1} = 1: the monic and plain states agree there)
    __device__ __forceinline__ void init(const RingTab &rt, int rp0, int nnorth, int m, int s, double lnm)
    {
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            const int rp = rp0 + k;
            if (rp < nnorth) {
                x[k] = __ldg(rt.xdf + rp).x;
                const double ls = rt.lsin2[rp], lc = rt.lcos2[rp];
                start_value<P>(sp[k], m, s, s, lnm, ls, lc);
                if (SPIN) start_value<P>(sm[k], m, s, -s, lnm, ls, lc);
            } else {
                x[k] = 0.f;
                P::zero(sp[k]);
                P::zero(sm[k]);
            }
        }
    }
    __device__ __forceinline__ int regime() const
    {
        bool all0 = true, allneg = true;
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            all0 = all0 && sp[k].E == 0;
            allneg = allneg && sp[k].E <= kSkipE;
            if (SPIN) {
                all0 = all0 && sm[k].E == 0;
                allneg = allneg && sm[k].E <= kSkipE;
            }
        }
        if (__all_sync(0xffffffffu, all0)) return 0;
        if (__all_sync(0xffffffffu, allneg)) return 1;
        return 2;
    }
    template <int NW, bool CHECK>
    __device__ __forceinline__ void advance(const float2 *reca, const float4 *, int l)
    {
        if (!SPIN) advance_c<NW, CHECK>(__ldg(reca + l));
        else advance_c<NW, CHECK>(__ldg(reinterpret_cast<const float4 *>(reca) + l));
    }
    // one step with the degree's df32 table entry already loaded: spin 0 (alpha_h, alpha_l)
    template <int NW, bool CHECK> __device__ __forceinline__ void advance_c(const float2 c)
    {
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            sp[k].w[NW] = __fmaf_rn(c.x * x[k], sp[k].w[1 - NW], -sp[k].w[NW]);
            if (CHECK) P::rescale(sp[k], NW);
        }
    }
    // spin s (alpha_h, alpha_l, tau_h, tau_l)
    template <int NW, bool CHECK> __device__ __forceinline__ void advance_c(const float4 c)
    {
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            const float cp = __fmaf_rn(c.x, x[k], c.z), cm = __fmaf_rn(c.x, x[k], -c.z);
            sp[k].w[NW] = __fmaf_rn(cp, sp[k].w[1 - NW], -sp[k].w[NW]);
            if (SPIN) sm[k].w[NW] = __fmaf_rn(cm, sm[k].w[1 - NW], -sm[k].w[NW]);
            if (CHECK) {
                P::rescale(sp[k], NW);
                if (SPIN) P::rescale(sm[k], NW);
            }
        }
    }
    __device__ __forceinline__ void advance_moved(const float2 *reca, const float4 *rect, int l)
    {
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            const float a = sp[k].w[0];
            sp[k].w[0] = sp[k].w[1];
            sp[k].w[1] = a;
            if (SPIN) {
                const float b = sm[k].w[0];
                sm[k].w[0] = sm[k].w[1];
                sm[k].w[1] = b;
            }
        }
        advance<1, true>(reca, rect, l);
    }
    template <int NW, bool SCALED> __device__ __forceinline__ float vplus(int k) const
    {
        return SCALED ? sp[k].w[NW] * P::fac(sp[k].E) : sp[k].w[NW];
    }
    template <int NW, bool SCALED> __device__ __forceinline__ float vminus(int k) const
    {
        return SCALED ? sm[k].w[NW] * P::fac(sm[k].E) : sm[k].w[NW];
    }
    // restart before degree l: the table's (lambda_{l-2}, lambda_{l-1}) divided by
    // (c_{l-2}, c_{l-1}) (cs: the order's (c, 1/c) entries)
    __device__ __forceinline__ void restart_scaled(const CkTab &ck, int64_t row, int rp0, int nnorth,
                                                   const float2 *cs, int l)
    {
        const float i0 = __ldg(cs + l - 2).y, i1 = __ldg(cs + l - 1).y;
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            const int rp = rp0 + k;
            if (rp >= nnorth) continue;
            if (!SPIN) {
                const float2 v = __ldg((const float2 *)ck.v + row + rp);
                sp[k].w[0] = v.x * i0; sp[k].w[1] = v.y * i1; sp[k].E = __ldg((const short *)ck.e + row + rp);
            } else {
                const float4 v = __ldg((const float4 *)ck.v + row + rp);
                const short2 e = __ldg((const short2 *)ck.e + row + rp);
                sp[k].w[0] = v.x * i0; sp[k].w[1] = v.y * i1; sp[k].E = e.x;
                sm[k].w[0] = v.z * i0; sm[k].w[1] = v.w * i1; sm[k].E = e.y;
            }
        }
    }
};

// Rings of the restarted FP32 recursion, Reinsch's form (PolR): w[1] holds
// the value lambda_l, w[0] the difference D_l = lambda_l - lambda_{l-1};
// the word index NW of the interface is not used.
template <int RPT, bool SPIN> struct Rings<PolR, RPT, SPIN> {
    using P = PolS;
    float y1[RPT];  // 1 - cos theta
    P::St sp[RPT], sm[RPT];

    __device__ __forceinline__ void init_geom(const RingTab &rt, int rp0, int nnorth)
    {
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            y1[k] = rp0 + k < nnorth ? __ldg(rt.y1 + rp0 + k) : 0.f;
            P::zero(sp[k]);
            P::zero(sm[k]);
        }
    }
    __device__ __forceinline__ void init(const RingTab &rt, int rp0, int nnorth, int m, int s, double lnm)
    {
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            const int rp = rp0 + k;
            if (rp < nnorth) {
                y1[k] = __ldg(rt.y1 + rp);
                const double ls = rt.lsin2[rp], lc = rt.lcos2[rp];
                start_value<P>(sp[k], m, s, s, lnm, ls, lc);
                sp[k].w[0] = sp[k].w[1];  // D_{l0} = lambda_{l0} (lambda_{l0-1} = 0)
                if (SPIN) {
                    start_value<P>(sm[k], m, s, -s, lnm, ls, lc);
                    sm[k].w[0] = sm[k].w[1];
                }
            } else {
                y1[k] = 0.f;
                P::zero(sp[k]);
                P::zero(sm[k]);
            }
        }
    }
    __device__ __forceinline__ int regime() const
    {
        bool all0 = true, allneg = true;
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            all0 = all0 && sp[k].E == 0;
            allneg = allneg && sp[k].E <= kSkipE;
            if (SPIN) {
                all0 = all0 && sm[k].E == 0;
                allneg = allneg && sm[k].E <= kSkipE;
            }
        }
        if (__all_sync(0xffffffffu, all0)) return 0;
        if (__all_sync(0xffffffffu, allneg)) return 1;
        return 2;
    }
    template <int NW, bool CHECK>
    __device__ __forceinline__ void advance(const float4 *reca, const float4 *, int l)
    {
        advance_c<NW, CHECK>(__ldg(reca + l));
    }
    template <int NW, bool CHECK> __device__ __forceinline__ void advance_c(const float4 c)
    {
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            const float dp = __fmaf_rn(c.x, y1[k], c.w);
            sp[k].w[0] = __fmaf_rn(c.y, sp[k].w[0], -(dp * sp[k].w[1]));
            sp[k].w[1] = __fadd_rn(sp[k].w[1], sp[k].w[0]);
            if (SPIN) {
                const float dm = __fmaf_rn(c.x, y1[k], __fmaf_rn(2.f, c.z, c.w));
                sm[k].w[0] = __fmaf_rn(c.y, sm[k].w[0], -(dm * sm[k].w[1]));
                sm[k].w[1] = __fadd_rn(sm[k].w[1], sm[k].w[0]);
            }
            if (CHECK) {
                P::rescale(sp[k], 1);
                if (SPIN) P::rescale(sm[k], 1);
            }
        }
    }
    __device__ __forceinline__ void advance_moved(const float4 *reca, const float4 *rect, int l)
    {
        advance<1, true>(reca, rect, l);
    }
    template <int NW, bool SCALED> __device__ __forceinline__ float vplus(int k) const
    {
        return SCALED ? sp[k].w[1] * P::fac(sp[k].E) : sp[k].w[1];
    }
    template <int NW, bool SCALED> __device__ __forceinline__ float vminus(int k) const
    {
        return SCALED ? sm[k].w[1] * P::fac(sm[k].E) : sm[k].w[1];
    }
    // restart: state (w[0], w[1]) and exponent E from the table
    __device__ __forceinline__ void restart(const CkTab &ck, int64_t row, int rp0, int nnorth)
    {
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            const int rp = rp0 + k;
            if (rp >= nnorth) continue;
            if (!SPIN) {
                const float2 v = __ldg((const float2 *)ck.v + row + rp);
                sp[k].w[0] = v.x; sp[k].w[1] = v.y; sp[k].E = __ldg((const short *)ck.e + row + rp);
            } else {
                const float4 v = __ldg((const float4 *)ck.v + row + rp);
                const short2 e = __ldg((const short2 *)ck.e + row + rp);
                sp[k].w[0] = v.x; sp[k].w[1] = v.y; sp[k].E = e.x;
                sm[k].w[0] = v.z; sm[k].w[1] = v.w; sm[k].E = e.y;
            }
        }
    }
};

// First restart of the calling warp for order m: the smallest kstart over the
// 32-ring groups its 32 RPT rings cover (uniform over the warp).
template <int RPT> __device__ __forceinline__ int first_restart(const CkTab &ck, int m)
{
    const int lane = threadIdx.x & 31;
    const int g0 = (((blockIdx.x * blockDim.x + threadIdx.x) & ~31) * RPT) >> 5;
    int k = 0x7fff;
    if (lane < RPT && g0 + lane < ck.ngrp) k = __ldg(ck.kstart + (int64_t)m * ck.ngrp + g0 + lane);
    return __reduce_min_sync(0xffffffffu, k);
}

}  // namespace
}  // namespace gsl
