// Legendre step of the general SHT (Sect. 3 "synthesis" and "adjoint
// synthesis"), on the equiangular grid theta_j = j pi / (ntheta - 1).
//
// Forward (per m >= 0, per ring):
//   spin 0:  F_m(theta)     =  sum_l a_lm lambda_lm(theta)
//   spin s:  F_m(theta)     = -sum_l (G + iC)_lm            s lambda_lm(theta)
//            F_{-m}(theta)  = -(-1)^s sum_l (G* + iC*)_lm  (-s)lambda_lm(theta)
// Adjoint (transpose, Sect. 2 spin-s adjoint and G/C split):
//   spin 0:  a_lm = sum_j H_m(theta_j) lambda_lm(theta_j)
//   spin s:  U_l = sum_j H_m s lambda_lm, V_l = sum_j H_{-m} (-s)lambda_lm,
//            G = -(U + (-1)^s conj V)/2,  C = i (U - (-1)^s conj V)/2
//
// s lambda_lm follows Wigner's d^l_{m,-s}: closed form at l0 = max(m, s),
// then the three-term recursion
//   lambda_l = A_l (x + sigma T_l) lambda_{l-1} - B_l lambda_{l-2},
//   T_l = m s / ((l-1) l), sigma = +1 for +s, -1 for -s, x = cos theta.
// Values are carried as mantissa * 2^(60 E) so that sin^m theta cannot
// underflow; contributions with E <= -2 are below 2^-60 and dropped.
//
// Arithmetic (policies below): FP32 plans run the recursion in df32 (pairs of
// FP32 words) and accumulate in FP32; FP64 plans run either native FP64, or
// (orders m >= m_df) the df32 recursion with df32 accumulation.
//
// Mapping: one CTA per (m, ring chunk); each thread owns RPT adjacent north
// rings (theta <= pi/2) and obtains the mirrored south ring from
//   s lambda_lm(pi - theta) = (-1)^{l+m} (-s)lambda_lm(theta).
// The degree loop runs in fully unrolled blocks of 8 steps; the two words of
// each recursion state swap roles every step (no register moves).  Before
// every block a warp vote picks one of three regimes: every state at scale 0
// (no checks), every state at scale <= -4 (contributions below 2^-180 for
// the whole block: recursion only), or mixed.  Recursion coefficients are
// read with warp-uniform addresses (L1 broadcast).  The adjoint reduces over
// rings inside each warp (transpose-reduce over the 8 degrees of a block) and
// adds the warp's sums into a_lm with one atomic per lane.
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
constexpr int kBlk = 8;

__device__ __forceinline__ int64_t alm_base(int lmax, int m) { return (int64_t)m * (2 * lmax + 1 - m) / 2; }

__device__ __forceinline__ df32 df_add_u(df32 a, df32 b) { return df_sub_u(a, {-b.h, -b.l}); }
__device__ __forceinline__ df32 df_neg(df32 a) { return {-a.h, -a.l}; }
__device__ __forceinline__ df32 df_split(double v)
{
    const float h = (float)v;
    return {h, (float)(v - (double)h)};
}
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
// sums, K a real coefficient component (a_lm or ring input), A a real
// accumulator; fma(acc, k, v) is acc += k v.
struct PolDF {  // df32 recursion, FP32 accumulation (FP32 plans)
    using R = float;
    using C = float2;
    using X = df32;
    using Tab = float4;   // (A_hi, A_lo, B_hi, B_lo)
    using TTab = float2;  // (T_hi, T_lo)
    using V = float;
    using K = float;
    using A = float;
    static constexpr bool kPreCombined = false;
    struct St { df32 w[2]; int E; };
    struct Co { df32 A, B; };
    static __device__ __forceinline__ Co load(const Tab *tab, int l)
    {
        const float4 c = __ldg(tab + l);
        return {{c.x, c.y}, {c.z, c.w}};
    }
    static __device__ __forceinline__ X load_t(const TTab *tab, int l)
    {
        const float2 c = __ldg(tab + l);
        return {c.x, c.y};
    }
    static __device__ __forceinline__ X ring_x(const RingTab &rt, int j)
    {
        const float2 v = __ldg(rt.xdf + j);
        return {v.x, v.y};
    }
    static __device__ __forceinline__ X add(X a, X b) { return df_add_u(a, b); }
    static __device__ __forceinline__ X sub(X a, X b) { return df_sub_u(a, b); }
    // new = A (y q) - B p, written over p
    static __device__ __forceinline__ void comb(df32 &p, const df32 &q, X y, const Co &c)
    {
        const df32 t = df_mul(y, q);
        const df32 v = df_mul(c.A, t);
        const df32 w = df_mul(c.B, p);
        p = df_sub_u(v, w);
    }
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
    static __device__ __forceinline__ void fma(A &acc, K k, V v) { acc += k * v; }
    static __device__ __forceinline__ void fma2(A &acc, K k1, V v1, K k2, V v2) { acc += k1 * v1 + k2 * v2; }
    static __device__ __forceinline__ A azero() { return 0.f; }
    static __device__ __forceinline__ K kadd(K a, K b) { return a + b; }
    static __device__ __forceinline__ K ksub(K a, K b) { return a - b; }
    static __device__ __forceinline__ K ksign(K a, float sg) { return a * sg; }
    static __device__ __forceinline__ void arenorm(A &) {}
    static __device__ __forceinline__ R aout(A a) { return a; }
    static __device__ __forceinline__ A aadd(A a, A b) { return a + b; }
    static __device__ __forceinline__ A ascale(A a, float f) { return a * f; }
    static __device__ __forceinline__ A shfl_xor(A v, int off) { return __shfl_xor_sync(0xffffffffu, v, off); }
    static __device__ __forceinline__ void atomic_add(R *dst, A v) { atomicAdd(dst, v); }
    // a_lm coefficient (re, im) of entry idx, component comp (0: G or T, 1: C)
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
    using R = double;
    using C = double2;
    using X = double;
    using Tab = double2;  // (A, B)
    using TTab = double;  // T
    using V = double;
    using K = double;
    using A = double;
    static constexpr bool kPreCombined = false;
    struct St { double w[2]; int E; };
    struct Co { double A, B; };
    static __device__ __forceinline__ Co load(const Tab *tab, int l)
    {
        const double2 c = __ldg(tab + l);
        return {c.x, c.y};
    }
    static __device__ __forceinline__ X load_t(const TTab *tab, int l) { return __ldg(tab + l); }
    static __device__ __forceinline__ X ring_x(const RingTab &rt, int j) { return __ldg(rt.x + j); }
    static __device__ __forceinline__ X add(X a, X b) { return a + b; }
    static __device__ __forceinline__ X sub(X a, X b) { return a - b; }
    static __device__ __forceinline__ void comb(double &p, const double &q, X y, const Co &c)
    {
        p = c.A * (y * q) - c.B * p;
    }
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
    static __device__ __forceinline__ void fma(A &acc, K k, V v) { acc += k * v; }
    static __device__ __forceinline__ void fma2(A &acc, K k1, V v1, K k2, V v2) { acc += k1 * v1 + k2 * v2; }
    static __device__ __forceinline__ A azero() { return 0.0; }
    static __device__ __forceinline__ K kadd(K a, K b) { return a + b; }
    static __device__ __forceinline__ K ksub(K a, K b) { return a - b; }
    static __device__ __forceinline__ K ksign(K a, double sg) { return a * sg; }
    static __device__ __forceinline__ void arenorm(A &) {}
    static __device__ __forceinline__ R aout(A a) { return a; }
    static __device__ __forceinline__ A aadd(A a, A b) { return a + b; }
    static __device__ __forceinline__ A ascale(A a, double f) { return a * f; }
    static __device__ __forceinline__ A shfl_xor(A v, int off) { return __shfl_xor_sync(0xffffffffu, v, off); }
    static __device__ __forceinline__ void atomic_add(R *dst, A v) { atomicAdd(dst, v); }
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

// FP64 plans, orders m >= m_df: the df32 recursion of PolDF with df32 sums.
// Coefficients come from a df32 table prepared per call (k_coef_dd); for
// spin s it already holds a = G + iC and b = (-1)^s (conj G + i conj C).
struct PolDD : PolDF {
    using R = double;
    using C = double2;
    using V = df32;
    using K = df32;
    using A = df32;
    static constexpr bool kPreCombined = true;
    static __device__ __forceinline__ V val(const df32 &a) { return a; }
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
    static __device__ __forceinline__ void fma2(A &acc, K k1, V v1, K k2, V v2)
    {
        acc = df_add_u(acc, df_add_u(df_mul(k1, v1), df_mul(k2, v2)));
    }
    static __device__ __forceinline__ A azero() { return {0.f, 0.f}; }
    static __device__ __forceinline__ K kadd(K a, K b) { return df_add_u(a, b); }
    static __device__ __forceinline__ K ksub(K a, K b) { return df_sub_u(a, b); }
    static __device__ __forceinline__ K ksign(K a, float sg) { return df_scale_pow2(a, sg); }
    static __device__ __forceinline__ void arenorm(A &a) { a = df_norm(a); }
    static __device__ __forceinline__ R aout(A a) { return (double)a.h + (double)a.l; }
    static __device__ __forceinline__ A aadd(A a, A b) { return df_add_u(a, b); }
    static __device__ __forceinline__ A ascale(A a, float f) { return df_scale_pow2(a, f); }
    static __device__ __forceinline__ A shfl_xor(A v, int off)
    {
        return {__shfl_xor_sync(0xffffffffu, v.h, off), __shfl_xor_sync(0xffffffffu, v.l, off)};
    }
    static __device__ __forceinline__ void atomic_add(R *dst, A v) { atomicAdd(dst, aout(v)); }
    // table entry: float4 (re_h, re_l, im_h, im_l); comp selects a (0) or b (1) for spin s
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
    __device__ __forceinline__ void advance(const typename P::Tab *recm, const typename P::TTab *recc, int l)
    {
        const typename P::Co co = P::load(recm, l);
        if (!SPIN) {
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                P::comb(sp[k].w[NW], sp[k].w[1 - NW], x[k], co);
                if (CHECK) P::rescale(sp[k], NW);
            }
        } else {
            const typename P::X t = P::load_t(recc, l);
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                P::comb(sp[k].w[NW], sp[k].w[1 - NW], P::add(x[k], t), co);
                P::comb(sm[k].w[NW], sm[k].w[1 - NW], P::sub(x[k], t), co);
                if (CHECK) { P::rescale(sp[k], NW); P::rescale(sm[k], NW); }
            }
        }
    }
    // Tail step: word 1 moves to word 0, the newest goes into word 1.
    __device__ __forceinline__ void advance_moved(const typename P::Tab *recm, const typename P::TTab *recc, int l)
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
        advance<1, true>(recm, recc, l);
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

// ---------------------------------------------------------------- forward
template <class P, int RPT, bool SPIN> struct FwdAcc {
    using A = typename P::A;
    using K = typename P::K;
    using Sg = decltype(P::fac(0));
    // north/south accumulators of column +m (p) and -m (q), (re, im)
    A pnr[RPT], pni[RPT], psr[RPT], psi[RPT], qnr[RPT], qni[RPT], qsr[RPT], qsi[RPT];
    const void *tab;
    int64_t nalm, base;
    int m;
    Sg sgs;

    __device__ __forceinline__ void init(const void *tab_, int64_t nalm_, int64_t base_, int m_, int s)
    {
        tab = tab_;
        nalm = nalm_;
        base = base_;
        m = m_;
        sgs = (s & 1) ? Sg(-1) : Sg(1);
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            pnr[k] = P::azero(); pni[k] = pnr[k]; psr[k] = pnr[k]; psi[k] = pnr[k];
            qnr[k] = pnr[k]; qni[k] = pnr[k]; qsr[k] = pnr[k]; qsi[k] = pnr[k];
        }
    }
    __device__ __forceinline__ void renorm()
    {
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            P::arenorm(pnr[k]); P::arenorm(pni[k]); P::arenorm(psr[k]); P::arenorm(psi[k]);
            if (SPIN) { P::arenorm(qnr[k]); P::arenorm(qni[k]); P::arenorm(qsr[k]); P::arenorm(qsi[k]); }
        }
    }
    // contribution of degree l (value in word NW); sg = (-1)^{l+m}
    template <int NW, bool SCALED> __device__ __forceinline__ void add(const Rings<P, RPT, SPIN> &st, int l, Sg sg)
    {
        K gr, gi;
        P::coef(tab, nalm, 0, base + l, gr, gi);
        if (!SPIN) {
            if (m == 0) gi = K{};
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                const typename P::V v = st.template vplus<NW, SCALED>(k);
                const typename P::V vs = P::vsign(v, sg);
                P::fma(pnr[k], gr, v); P::fma(pni[k], gi, v);
                P::fma(psr[k], gr, vs); P::fma(psi[k], gi, vs);
            }
        } else {
            K ar, ai, br, bi;
            if (P::kPreCombined) {  // table holds a and b (m = 0 imaginary parts already dropped)
                ar = gr; ai = gi;
                P::coef(tab, nalm, 1, base + l, br, bi);
            } else {
                K cr, ci;
                P::coef(tab, nalm, 1, base + l, cr, ci);
                if (m == 0) { gi = K{}; ci = K{}; }
                // a = G + iC ; b = (-1)^s (conj G + i conj C)
                ar = P::ksub(gr, ci); ai = P::kadd(gi, cr);
                br = P::ksign(P::kadd(gr, ci), sgs); bi = P::ksign(P::ksub(cr, gi), sgs);
            }
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                const typename P::V vp = st.template vplus<NW, SCALED>(k), vm = st.template vminus<NW, SCALED>(k);
                const typename P::V vps = P::vsign(vp, sg), vms = P::vsign(vm, sg);
                P::fma(pnr[k], ar, vp); P::fma(pni[k], ai, vp);     // north, column +m
                P::fma(psr[k], ar, vms); P::fma(psi[k], ai, vms);   // south, column +m
                P::fma(qnr[k], br, vm); P::fma(qni[k], bi, vm);     // north, column -m
                P::fma(qsr[k], br, vps); P::fma(qsi[k], bi, vps);   // south, column -m
            }
        }
    }
};

template <class P, int RPT, bool SPIN, int REG>
__device__ __forceinline__ void fwd_block(Rings<P, RPT, SPIN> &st, FwdAcc<P, RPT, SPIN> &acc,
                                          const typename P::Tab *recm, const typename P::TTab *recc, int lb,
                                          decltype(P::fac(0)) s0)
{
#pragma unroll
    for (int j = 0; j < kBlk; ++j) {
        const int l = lb + j;
        const auto sg = (j & 1) ? -s0 : s0;
        if (j & 1) {
            st.template advance<1, REG != 0>(recm, recc, l);
            if (REG != 1) acc.template add<1, REG == 2>(st, l, sg);
        } else {
            st.template advance<0, REG != 0>(recm, recc, l);
            if (REG != 1) acc.template add<0, REG == 2>(st, l, sg);
        }
    }
}

template <class P, int RPT, bool SPIN>
__global__ void __launch_bounds__(512) k_leg_fwd(const void *__restrict__ coef, const void *__restrict__ rec_ab,
                                                 const void *__restrict__ rec_c, const double *__restrict__ lognorm,
                                                 RingTab rt, typename P::C *__restrict__ ring, int lmax, int mmax,
                                                 int spin, int ntheta, int nnorth, int64_t nalm, int m_begin)
{
    using Sg = decltype(P::fac(0));
    using Cx = typename P::C;
    const int m = m_begin + blockIdx.y;
    const int s = SPIN ? spin : 0;
    const int l0 = m > s ? m : s;
    if (l0 > lmax) return;
    const int64_t base = alm_base(lmax, m);
    const typename P::Tab *recm = (const typename P::Tab *)rec_ab + base;
    const typename P::TTab *recc = SPIN ? (const typename P::TTab *)rec_c + base : nullptr;
    const int rp0 = (blockIdx.x * blockDim.x + threadIdx.x) * RPT;

    Rings<P, RPT, SPIN> st;
    st.init(rt, rp0, nnorth, m, s, lognorm[m]);
    FwdAcc<P, RPT, SPIN> acc;
    acc.init(coef, nalm, base, m, s);

    acc.template add<1, true>(st, l0, ((l0 - m) & 1) ? Sg(-1) : Sg(1));  // l0 = s > m for m < s
    int l = l0 + 1;
    const Sg s0 = ((l - m) & 1) ? Sg(-1) : Sg(1);  // sign of the first degree of every block
    for (; l + kBlk <= lmax + 1; l += kBlk) {
        const int reg = st.regime();
        acc.renorm();
        if (reg == 0) fwd_block<P, RPT, SPIN, 0>(st, acc, recm, recc, l, s0);
        else if (reg == 1) fwd_block<P, RPT, SPIN, 1>(st, acc, recm, recc, l, s0);
        else fwd_block<P, RPT, SPIN, 2>(st, acc, recm, recc, l, s0);
    }
    for (; l <= lmax; ++l) {  // tail: general path
        st.advance_moved(recm, recc, l);
        acc.template add<1, true>(st, l, ((l - m) & 1) ? Sg(-1) : Sg(1));
    }

    // write: spin 0 column m; spin s columns mmax + m (P) and mmax - m (Q), with the minus sign
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        const int jn = rp0 + k;
        if (jn >= nnorth) continue;
        const int js = ntheta - 1 - jn;
        if (!SPIN) {
            Cx *col = ring + (int64_t)m * ntheta;
            col[jn] = P::cout(acc.pnr[k], acc.pni[k]);
            if (js != jn) col[js] = P::cout(acc.psr[k], acc.psi[k]);
        } else {
            Cx *colp = ring + (int64_t)(mmax + m) * ntheta;
            const Cx pn = P::cout(acc.pnr[k], acc.pni[k]), ps = P::cout(acc.psr[k], acc.psi[k]);
            colp[jn] = mkc(-pn.x, -pn.y);
            if (js != jn) colp[js] = mkc(-ps.x, -ps.y);
            if (m > 0) {
                Cx *colq = ring + (int64_t)(mmax - m) * ntheta;
                const Cx qn = P::cout(acc.qnr[k], acc.qni[k]), qs = P::cout(acc.qsr[k], acc.qsi[k]);
                colq[jn] = mkc(-qn.x, -qn.y);
                if (js != jn) colq[js] = mkc(-qs.x, -qs.y);
            }
        }
    }
}

// ---------------------------------------------------------------- adjoint
// Transpose-reduce of NV values per lane over the 32 lanes of a warp: after
// it, lane t holds the warp sum of value index (t >> (5 - log2 NV)).
template <class P, int NV> __device__ __forceinline__ typename P::A warp_transpose_reduce(typename P::A (&v)[NV])
{
    static_assert(NV == 1 || NV == 2 || NV == 4 || NV == 8 || NV == 16 || NV == 32, "NV power of two <= 32");
    const int lane = threadIdx.x & 31;
    int cnt = NV;
    int off = 16;
#pragma unroll
    for (int stage = 0; stage < 5; ++stage) {
        if (cnt > 1) {
            const int half = cnt >> 1;
            const bool upper = (lane & off) != 0;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                if (i < half) {
                    const typename P::A send = upper ? v[i] : v[i + half];
                    const typename P::A keep = upper ? v[i + half] : v[i];
                    v[i] = P::aadd(keep, P::shfl_xor(send, off));
                }
            }
            cnt = half;
        } else {
            v[0] = P::aadd(v[0], P::shfl_xor(v[0], off));
        }
        off >>= 1;
    }
    return v[0];
}

template <class P, int RPT, bool SPIN> struct AdjIn {
    using K = typename P::K;
    using A = typename P::A;
    // spin 0: (hn) = H_N + H_S (even l+m), (hs) = H_N - H_S (odd l+m)
    // spin s: hn/hs column +m north/south, gn/gs column -m
    K hnr[RPT], hni[RPT], hsr[RPT], hsi[RPT], gnr[RPT], gni[RPT], gsr[RPT], gsi[RPT];

    __device__ __forceinline__ void init(const typename P::C *ring, int rp0, int nnorth, int ntheta, int m, int mmax)
    {
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            const int rp = rp0 + k;
            hnr[k] = K{}; hni[k] = K{}; hsr[k] = K{}; hsi[k] = K{};
            gnr[k] = K{}; gni[k] = K{}; gsr[k] = K{}; gsi[k] = K{};
            if (rp < nnorth) {
                const int js = ntheta - 1 - rp;
                const int64_t colp = (int64_t)(SPIN ? mmax + m : m) * ntheta;
                P::ring_in(ring, colp + rp, hnr[k], hni[k]);
                if (js != rp) P::ring_in(ring, colp + js, hsr[k], hsi[k]);
                if (SPIN) {
                    const int64_t colq = (int64_t)(mmax - m) * ntheta;
                    P::ring_in(ring, colq + rp, gnr[k], gni[k]);
                    if (js != rp) P::ring_in(ring, colq + js, gsr[k], gsi[k]);
                } else {
                    const K ar = hnr[k], ai = hni[k], br = hsr[k], bi = hsi[k];
                    hnr[k] = P::kadd(ar, br); hni[k] = P::kadd(ai, bi);
                    hsr[k] = P::ksub(ar, br); hsi[k] = P::ksub(ai, bi);
                }
            }
        }
    }
    // partial sums of one degree (value in word NW) into part[0..NCOMP)
    template <int NW, bool SCALED>
    __device__ __forceinline__ void add(const Rings<P, RPT, SPIN> &st, bool odd, A *part) const
    {
        using Sg = decltype(P::fac(0));
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            const typename P::V vp = st.template vplus<NW, SCALED>(k);
            if (!SPIN) {
                const K hr = odd ? hsr[k] : hnr[k], hi = odd ? hsi[k] : hni[k];
                P::fma(part[0], hr, vp);
                P::fma(part[1], hi, vp);
            } else {
                const typename P::V vm = st.template vminus<NW, SCALED>(k);
                const Sg sg = odd ? Sg(-1) : Sg(1);
                const typename P::V vms = P::vsign(vm, sg), vps = P::vsign(vp, sg);
                // U += lam+ H_m(N) + sg lam- H_m(S) ; V += lam- H_-m(N) + sg lam+ H_-m(S)
                P::fma2(part[0], hnr[k], vp, hsr[k], vms);
                P::fma2(part[1], hni[k], vp, hsi[k], vms);
                P::fma2(part[2], gnr[k], vm, gsr[k], vps);
                P::fma2(part[3], gni[k], vm, gsi[k], vps);
            }
        }
    }
};

// Adds the warp sums of the degrees lb + i (value index i * NCOMP + c) into
// a_lm (spin 0) or G, C (spin s).
template <class P, bool SPIN, int NV>
__device__ __forceinline__ void flush(typename P::A (&part)[NV], typename P::R *out, int64_t base, int64_t nalm, int m,
                                      int lb, int lmax, decltype(P::fac(0)) sgs)
{
    using A = typename P::A;
    using Sg = decltype(P::fac(0));
    constexpr int NCOMP = SPIN ? 4 : 2;
    constexpr int SH = (NV == 32 ? 0 : NV == 16 ? 1 : NV == 8 ? 2 : NV == 4 ? 3 : NV == 2 ? 4 : 5);
    const int lane = threadIdx.x & 31;
    const A tot = warp_transpose_reduce<P, NV>(part);
    const int v = lane >> SH;
    const int i = v / NCOMP, c = v % NCOMP;
    const int l = lb + i;
    if (!SPIN) {
        if ((lane & ((1 << SH) - 1)) == 0 && l <= lmax && !(m == 0 && c == 1))
            P::atomic_add(out + 2 * (base + l) + c, tot);
    } else {
        // lanes hold U.re, U.im, V.re, V.im of degree l at c = 0..3; the G/C
        // split is linear, so each warp adds its share directly:
        //   G.re = -(U.re + sgs V.re)/2   G.im = -(U.im - sgs V.im)/2
        //   C.re = -(U.im + sgs V.im)/2   C.im =  (U.re - sgs V.re)/2
        const A other = P::shfl_xor(tot, 2 << SH);  // U <-> V of the same l
        if ((lane & ((1 << SH) - 1)) == 0 && l <= lmax) {
            A val;
            int64_t dst;
            const Sg h = Sg(0.5);
            if (c == 0) { val = P::ascale(P::aadd(tot, P::ascale(other, sgs)), -h); dst = 2 * (base + l); }
            else if (c == 1) { val = P::ascale(P::aadd(tot, P::ascale(other, -sgs)), -h); dst = 2 * (base + l) + 1; }
            else if (c == 2) { val = P::ascale(P::aadd(other, P::ascale(tot, -sgs)), h); dst = 2 * (nalm + base + l) + 1; }
            else { val = P::ascale(P::aadd(other, P::ascale(tot, sgs)), -h); dst = 2 * (nalm + base + l); }
            if (!(m == 0 && (c == 1 || c == 2))) P::atomic_add(out + dst, val);
        }
    }
}

template <class P, int RPT, bool SPIN, int REG>
__device__ __forceinline__ void adj_block(Rings<P, RPT, SPIN> &st, const AdjIn<P, RPT, SPIN> &in, typename P::A *part,
                                          const typename P::Tab *recm, const typename P::TTab *recc, int lb, bool odd0)
{
    constexpr int NCOMP = SPIN ? 4 : 2;
#pragma unroll
    for (int j = 0; j < kBlk; ++j) {
        const int l = lb + j;
        const bool odd = (j & 1) ? !odd0 : odd0;
        if (j & 1) {
            st.template advance<1, REG != 0>(recm, recc, l);
            if (REG != 1) in.template add<1, REG == 2>(st, odd, part + j * NCOMP);
        } else {
            st.template advance<0, REG != 0>(recm, recc, l);
            if (REG != 1) in.template add<0, REG == 2>(st, odd, part + j * NCOMP);
        }
    }
}

template <class P, int RPT, bool SPIN>
__global__ void __launch_bounds__(512) k_leg_adj(const typename P::C *__restrict__ ring, const void *__restrict__ rec_ab,
                                                 const void *__restrict__ rec_c, const double *__restrict__ lognorm,
                                                 RingTab rt, typename P::C *__restrict__ alm, int lmax, int mmax,
                                                 int spin, int ntheta, int nnorth, int64_t nalm, int m_begin)
{
    using A = typename P::A;
    using R = typename P::R;
    using Sg = decltype(P::fac(0));
    constexpr int NCOMP = SPIN ? 4 : 2;
    constexpr int NV = kBlk * NCOMP;
    const int m = m_begin + blockIdx.y;
    const int s = SPIN ? spin : 0;
    const int l0 = m > s ? m : s;
    if (l0 > lmax) return;
    const int64_t base = alm_base(lmax, m);
    const typename P::Tab *recm = (const typename P::Tab *)rec_ab + base;
    const typename P::TTab *recc = SPIN ? (const typename P::TTab *)rec_c + base : nullptr;
    const int rp0 = (blockIdx.x * blockDim.x + threadIdx.x) * RPT;
    const Sg sgs = (s & 1) ? Sg(-1) : Sg(1);
    R *out = reinterpret_cast<R *>(alm);

    Rings<P, RPT, SPIN> st;
    st.init(rt, rp0, nnorth, m, s, lognorm[m]);
    AdjIn<P, RPT, SPIN> in;
    in.init(ring, rp0, nnorth, ntheta, m, mmax);

    {  // degree l0 (the start value): one reduction of NCOMP values
        A p0[NCOMP];
#pragma unroll
        for (int c = 0; c < NCOMP; ++c) p0[c] = P::azero();
        in.template add<1, true>(st, ((l0 - m) & 1) != 0, p0);  // l0 = s > m for m < s
        flush<P, SPIN, NCOMP>(p0, out, base, nalm, m, l0, lmax, sgs);
    }
    int l = l0 + 1;
    const bool odd0 = ((l - m) & 1) != 0;
    A part[NV];
    for (; l + kBlk <= lmax + 1; l += kBlk) {
        const int reg = st.regime();
        if (reg == 1) {  // every contribution of this block is below 2^-180: recursion only
            adj_block<P, RPT, SPIN, 1>(st, in, part, recm, recc, l, odd0);
            continue;
        }
#pragma unroll
        for (int i = 0; i < NV; ++i) part[i] = P::azero();
        if (reg == 0) adj_block<P, RPT, SPIN, 0>(st, in, part, recm, recc, l, odd0);
        else adj_block<P, RPT, SPIN, 2>(st, in, part, recm, recc, l, odd0);
        flush<P, SPIN, NV>(part, out, base, nalm, m, l, lmax, sgs);
    }
    if (l <= lmax) {  // tail: fewer than kBlk degrees, general path
#pragma unroll
        for (int i = 0; i < NV; ++i) part[i] = P::azero();
#pragma unroll
        for (int j = 0; j < kBlk; ++j) {
            if (l + j <= lmax) {
                st.advance_moved(recm, recc, l + j);
                in.template add<1, true>(st, ((l + j - m) & 1) != 0, part + j * NCOMP);
            }
        }
        flush<P, SPIN, NV>(part, out, base, nalm, m, l, lmax, sgs);
    }
}

// ------------------------------------------------------- coefficient tables
// For the step (l-1 -> l), j = l - 1:
//   A = (j+1) sqrt((2j+3)(2j+1) / (((j+1)^2-m^2)((j+1)^2-s^2)))
//   B = (j+1)/j sqrt((2j+3)/(2j-1)) sqrt((j^2-m^2)(j^2-s^2) / (((j+1)^2-m^2)((j+1)^2-s^2)))
//   T = m s / (j (j+1))
// Written as df32 (ab_df, t_df) and/or FP64 (ab64, t64) tables.
__global__ void k_rec_tables(int lmax, int spin, void *ab_df, void *t_df, void *ab64, void *t64)
{
    const int m = blockIdx.x;
    const int s = spin;
    const int l0 = m > s ? m : s;
    const int64_t base = alm_base(lmax, m);
    for (int l = l0 + 1 + threadIdx.x; l <= lmax; l += blockDim.x) {
        const double j = l - 1, mm = m, ss = s;
        const double den = ((j + 1) * (j + 1) - mm * mm) * ((j + 1) * (j + 1) - ss * ss);
        const double A = (j + 1) * sqrt((2 * j + 3) * (2 * j + 1) / den);
        double B = 0.0, T = 0.0;
        if (j > 0) {
            B = (j + 1) / j * sqrt((2 * j + 3) / (2 * j - 1)) * sqrt((j * j - mm * mm) * (j * j - ss * ss) / den);
            T = mm * ss / (j * (j + 1));
        }
        if (ab_df) {
            const float ah = (float)A, bh = (float)B, th = (float)T;
            ((float4 *)ab_df)[base + l] = make_float4(ah, (float)(A - ah), bh, (float)(B - bh));
            if (t_df) ((float2 *)t_df)[base + l] = make_float2(th, (float)(T - th));
        }
        if (ab64) {
            ((double2 *)ab64)[base + l] = make_double2(A, B);
            if (t64) ((double *)t64)[base + l] = T;
        }
    }
}

// df32 coefficients for the PolDD forward: spin 0 the a_lm; spin s
// a = G + iC and b = (-1)^s (conj G + i conj C) (m = 0 imaginary parts of
// G and C dropped).  One entry per alm index, orders m >= m_begin.
__global__ void k_coef_dd(const double2 *__restrict__ alm, float4 *__restrict__ out, int lmax, int mmax, int spin,
                          int64_t nalm, int m_begin)
{
    const int m = m_begin + blockIdx.y;
    const int64_t base = alm_base(lmax, m);
    const double sgs = (spin & 1) ? -1.0 : 1.0;
    for (int l = m + blockIdx.x * blockDim.x + threadIdx.x; l <= lmax; l += gridDim.x * blockDim.x) {
        const int64_t i = base + l;
        double2 g = alm[i];
        if (m == 0) g.y = 0.0;
        if (!spin) {
            const float rh = (float)g.x, ih = (float)g.y;
            out[i] = make_float4(rh, (float)(g.x - rh), ih, (float)(g.y - ih));
        } else {
            double2 c = alm[nalm + i];
            if (m == 0) c.y = 0.0;
            const double ar = g.x - c.y, ai = g.y + c.x;
            const double br = sgs * (g.x + c.y), bi = sgs * (c.x - g.y);
            float h0 = (float)ar, h1 = (float)ai;
            out[i] = make_float4(h0, (float)(ar - h0), h1, (float)(ai - h1));
            h0 = (float)br;
            h1 = (float)bi;
            out[nalm + i] = make_float4(h0, (float)(br - h0), h1, (float)(bi - h1));
        }
    }
}

template <class P, int RPT, bool SPIN>
cudaError_t fwd_launch(const Plan &p, const Plan::LegShape &sh, const void *coef, const void *ab, const void *tc,
                       void *ring, int m_begin, int m_end, cudaStream_t st)
{
    if (m_end <= m_begin) return cudaSuccess;
    dim3 grid(sh.chunks, m_end - m_begin);
    dim3 block(sh.warps * 32);
    k_leg_fwd<P, RPT, SPIN><<<grid, block, 0, st>>>(coef, ab, tc, p.lognorm, p.rings, (typename P::C *)ring, p.lmax,
                                                    p.mmax, p.spin, p.ntheta, p.nnorth, p.nalm, m_begin);
    return cudaGetLastError();
}

template <class P, int RPT, bool SPIN>
cudaError_t adj_launch(const Plan &p, const Plan::LegShape &sh, const void *ring, const void *ab, const void *tc,
                       void *alm, int m_begin, int m_end, cudaStream_t st)
{
    if (m_end <= m_begin) return cudaSuccess;
    dim3 grid(sh.chunks, m_end - m_begin);
    dim3 block(sh.warps * 32);
    k_leg_adj<P, RPT, SPIN><<<grid, block, 0, st>>>((const typename P::C *)ring, ab, tc, p.lognorm, p.rings,
                                                    (typename P::C *)alm, p.lmax, p.mmax, p.spin, p.ntheta, p.nnorth,
                                                    p.nalm, m_begin);
    return cudaGetLastError();
}

template <class P, bool SPIN>
cudaError_t fwd_rpt(const Plan &p, const Plan::LegShape &sh, const void *coef, const void *ab, const void *tc,
                    void *ring, int m_begin, int m_end, cudaStream_t st)
{
    if (sh.rpt == 1) return fwd_launch<P, 1, SPIN>(p, sh, coef, ab, tc, ring, m_begin, m_end, st);
    return fwd_launch<P, 2, SPIN>(p, sh, coef, ab, tc, ring, m_begin, m_end, st);
}

template <class P, bool SPIN>
cudaError_t adj_rpt(const Plan &p, const Plan::LegShape &sh, const void *ring, const void *ab, const void *tc,
                    void *alm, int m_begin, int m_end, cudaStream_t st)
{
    if (sh.rpt == 1) return adj_launch<P, 1, SPIN>(p, sh, ring, ab, tc, alm, m_begin, m_end, st);
    return adj_launch<P, 2, SPIN>(p, sh, ring, ab, tc, alm, m_begin, m_end, st);
}

template <class P>
cudaError_t fwd_spin(const Plan &p, const Plan::LegShape &sh, const void *coef, const void *ab, const void *tc,
                     void *ring, int m_begin, int m_end, cudaStream_t st)
{
    return p.spin ? fwd_rpt<P, true>(p, sh, coef, ab, tc, ring, m_begin, m_end, st)
                  : fwd_rpt<P, false>(p, sh, coef, ab, tc, ring, m_begin, m_end, st);
}

template <class P>
cudaError_t adj_spin(const Plan &p, const Plan::LegShape &sh, const void *ring, const void *ab, const void *tc,
                     void *alm, int m_begin, int m_end, cudaStream_t st)
{
    return p.spin ? adj_rpt<P, true>(p, sh, ring, ab, tc, alm, m_begin, m_end, st)
                  : adj_rpt<P, false>(p, sh, ring, ab, tc, alm, m_begin, m_end, st);
}

// Kernel entry of one (arithmetic, spin, rings-per-thread, direction) variant.
template <class P> const void *kernel_of(bool spin, int rpt, bool adjoint)
{
    if (adjoint) {
        if (spin) return rpt == 1 ? (const void *)k_leg_adj<P, 1, true> : (const void *)k_leg_adj<P, 2, true>;
        return rpt == 1 ? (const void *)k_leg_adj<P, 1, false> : (const void *)k_leg_adj<P, 2, false>;
    }
    if (spin) return rpt == 1 ? (const void *)k_leg_fwd<P, 1, true> : (const void *)k_leg_fwd<P, 2, true>;
    return rpt == 1 ? (const void *)k_leg_fwd<P, 1, false> : (const void *)k_leg_fwd<P, 2, false>;
}

}  // namespace

// Launch shape of a Legendre kernel: among 4..16 warps per CTA, the one with
// the most resident warps per SM (registers decide how many CTAs fit), then
// the fewest idle ring slots.
Plan::LegShape legendre_shape(const Plan &p, bool adjoint, bool dd, int rpt)
{
    const void *fn = p.prec == LENS_FP32 ? kernel_of<PolDF>(p.spin != 0, rpt, adjoint)
                     : dd               ? kernel_of<PolDD>(p.spin != 0, rpt, adjoint)
                                        : kernel_of<PolF64>(p.spin != 0, rpt, adjoint);
    const int nw = (p.nnorth + 32 * rpt - 1) / (32 * rpt);
    Plan::LegShape best;
    long best_active = -1, best_slots = 0;
    for (int w = 4; w <= 16; ++w) {
        const int chunks = (nw + w - 1) / w;
        const int warps = (nw + chunks - 1) / chunks;
        int blocks = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fn, warps * 32, 0) != cudaSuccess) blocks = 1;
        const long active = (long)blocks * warps;
        const long slots = (long)chunks * warps;
        if (active > best_active || (active == best_active && slots < best_slots)) {
            best_active = active;
            best_slots = slots;
            best.rpt = rpt;
            best.warps = warps;
            best.chunks = chunks;
        }
    }
    return best;
}

cudaError_t launch_rec_tables(Plan &p)
{
    if (p.prec == LENS_FP32)
        k_rec_tables<<<p.mmax + 1, 256, 0, p.stream>>>(p.lmax, p.spin, p.rec_ab, p.spin ? p.rec_c : nullptr, nullptr,
                                                       nullptr);
    else
        k_rec_tables<<<p.mmax + 1, 256, 0, p.stream>>>(p.lmax, p.spin, p.rec_ab_df, p.spin ? p.rec_c_df : nullptr,
                                                       p.rec_ab, p.spin ? p.rec_c : nullptr);
    return cudaGetLastError();
}

// Rings per thread, from a sweep at lmax 4096 on GB300 (ms per launch):
//   FP32 spin 0: fwd 19.7 / 18.5 / 29.7 and adj 21.2 / 18.8 / 31.4 for RPT 1 / 2 / 4
//   FP32 spin 2: fwd 47.4 / 73.4 / 158 and adj 52.4 / 75.6 / 193
//   FP64 spin 0: fwd 246 / 252 / 295 and adj 258 / 236 / 262
//   FP64 spin 2: fwd 760 / 700 / 790 and adj 851 / 801 / 916
int legendre_rpt(int prec, int spin, bool adjoint)
{
    if (prec == LENS_FP32) return spin ? 1 : 2;
    return spin ? 2 : (adjoint ? 2 : 1);
}

// df32 part of FP64 plans: twice the accumulator words of the FP32 plans
int legendre_rpt_dd(int spin, bool adjoint) { return (spin || adjoint) ? 1 : 2; }

bool legendre_rpt_supported(int, int, bool, int rpt) { return rpt == 1 || rpt == 2; }

cudaError_t launch_legendre_fwd(const Plan &p, const void *alm, void *ring, cudaStream_t st)
{
    // entries with l < spin / columns without rings are never written by the
    // kernel: start from zero
    const size_t eb = p.prec == LENS_FP32 ? 8 : 16;
    cudaError_t e = cudaMemsetAsync(ring, 0, eb * (size_t)p.ncol * p.ntheta, st);
    if (e != cudaSuccess) return e;
    if (p.prec == LENS_FP32) return fwd_spin<PolDF>(p, p.leg_f, alm, p.rec_ab, p.rec_c, ring, 0, p.mmax + 1, st);
    if (p.m_df > 0 && (e = fwd_spin<PolF64>(p, p.leg_f, alm, p.rec_ab, p.rec_c, ring, 0, p.m_df, st)) != cudaSuccess)
        return e;
    if (p.m_df <= p.mmax) {
        dim3 g(4, p.mmax + 1 - p.m_df);
        k_coef_dd<<<g, 256, 0, st>>>((const double2 *)alm, (float4 *)p.coef_dd, p.lmax, p.mmax, p.spin, p.nalm, p.m_df);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        e = fwd_spin<PolDD>(p, p.leg_fd, p.coef_dd, p.rec_ab_df, p.rec_c_df, ring, p.m_df, p.mmax + 1, st);
    }
    return e;
}

cudaError_t launch_legendre_adj(const Plan &p, const void *ring, void *alm, cudaStream_t st)
{
    const size_t ebytes = (p.prec == LENS_FP32 ? 8 : 16) * (size_t)p.nalm * (p.spin ? 2 : 1);
    cudaError_t e = cudaMemsetAsync(alm, 0, ebytes, st);  // the kernels add warp sums atomically
    if (e != cudaSuccess) return e;
    if (p.prec == LENS_FP32) return adj_spin<PolDF>(p, p.leg_a, ring, p.rec_ab, p.rec_c, alm, 0, p.mmax + 1, st);
    if (p.m_df > 0 && (e = adj_spin<PolF64>(p, p.leg_a, ring, p.rec_ab, p.rec_c, alm, 0, p.m_df, st)) != cudaSuccess)
        return e;
    if (p.m_df <= p.mmax) e = adj_spin<PolDD>(p, p.leg_ad, ring, p.rec_ab_df, p.rec_c_df, alm, p.m_df, p.mmax + 1, st);
    return e;
}

}  // namespace gsl
