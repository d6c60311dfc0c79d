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
// Mapping: one CTA per (m, ring chunk); each thread owns RPT adjacent north
// rings (theta <= pi/2) and obtains the mirrored south ring from
//   s lambda_lm(pi - theta) = (-1)^{l+m} (-s)lambda_lm(theta).
// Work proceeds in blocks of l; a warp vote picks one of three regimes per
// block: every state at scale 0 (no checks), every state at scale <= -4
// (contributions below 2^-180 for the whole block: recursion only), or mixed.
// Recursion coefficients are read with warp-uniform addresses (L1 broadcast).
// The adjoint reduces over rings inside each warp (transpose-reduce over a
// block of l) and adds the warp's sums into a_lm with one atomic per lane.
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
constexpr int kSkipE = -4;  // below 2^-240 before the block, < 2^-180 after 8 steps of growth <= 2^8.5

__device__ __forceinline__ int64_t alm_base(int lmax, int m) { return (int64_t)m * (2 * lmax + 1 - m) / 2; }

// ------------------------------------------------------------ policies
struct PolDF {  // df32 recursion, FP32 accumulation
    using R = float;
    using C = float2;
    using X = df32;
    struct St { df32 cur, prev; int E; };
    struct Co { df32 A, B; };
    static __device__ __forceinline__ Co load(const void *tab, int64_t i)
    {
        float4 c = __ldg((const float4 *)tab + i);
        return {{c.x, c.y}, {c.z, c.w}};
    }
    static __device__ __forceinline__ X load_t(const void *tab, int64_t i)
    {
        float2 c = __ldg((const float2 *)tab + i);
        return {c.x, c.y};
    }
    static __device__ __forceinline__ X ring_x(const RingTab &rt, int j)
    {
        float2 v = __ldg(rt.xdf + j);
        return {v.x, v.y};
    }
    static __device__ __forceinline__ X add(X a, X b) { return df_sub_u(a, {-b.h, -b.l}); }
    static __device__ __forceinline__ X sub(X a, X b) { return df_sub_u(a, b); }
    static __device__ __forceinline__ void step(St &s, X y, const Co &c)
    {
        df32 t = df_mul(y, s.cur);
        df32 v = df_mul(c.A, t);
        df32 w = df_mul(c.B, s.prev);
        s.prev = s.cur;
        s.cur = df_sub_u(v, w);
    }
    // The state is not renormalised after every step (the low word carries
    // the compensation of the high-word recursion), so the value is h + l.
    static __device__ __forceinline__ R val(const St &s) { return __fadd_rn(s.cur.h, s.cur.l); }
    static __device__ __forceinline__ df32 norm(df32 a)  // two-sum: exact for any ordering of |h|, |l|
    {
        const float h = __fadd_rn(a.h, a.l);
        const float bb = __fsub_rn(h, a.h);
        return {h, __fadd_rn(__fsub_rn(a.h, __fsub_rn(h, bb)), __fsub_rn(a.l, bb))};
    }
    static __device__ __forceinline__ void renorm(St &s)
    {
        s.cur = norm(s.cur);
        s.prev = norm(s.prev);
    }
    static __device__ __forceinline__ void rescale(St &s)
    {
        if (s.E < 0 && fabsf(s.cur.h) > kBigF) {
            s.cur = df_scale_pow2(s.cur, kSmallF);
            s.prev = df_scale_pow2(s.prev, kSmallF);
            s.E += 1;
        }
    }
    static __device__ __forceinline__ R fac(int E) { return E == 0 ? 1.0f : (E == -1 ? kSmallF : 0.0f); }
    // start value 2^L2 * sign as mantissa * 2^(60 E)
    static __device__ __forceinline__ void start(St &s, double L2, int sign, bool zero)
    {
        s.prev = {0.f, 0.f};
        if (zero) { s.cur = {0.f, 0.f}; s.E = -1000; return; }
        double e = floor(L2 * (1.0 / kScaleBits));
        double fr = L2 - e * kScaleBits;  // [0, 60)
        double ip = floor(fr);
        float m = ldexpf(exp2f((float)(fr - ip)), (int)ip);
        s.cur = {sign < 0 ? -m : m, 0.f};
        s.E = (int)e;
    }
    static __device__ __forceinline__ void zero(St &s) { s.cur = {0.f, 0.f}; s.prev = s.cur; s.E = 0; }
};

struct PolF64 {  // native FP64
    using R = double;
    using C = double2;
    using X = double;
    struct St { double cur, prev; int E; };
    struct Co { double A, B; };
    static __device__ __forceinline__ Co load(const void *tab, int64_t i)
    {
        double2 c = __ldg((const double2 *)tab + i);
        return {c.x, c.y};
    }
    static __device__ __forceinline__ X load_t(const void *tab, int64_t i) { return __ldg((const double *)tab + i); }
    static __device__ __forceinline__ X ring_x(const RingTab &rt, int j) { return __ldg(rt.x + j); }
    static __device__ __forceinline__ X add(X a, X b) { return a + b; }
    static __device__ __forceinline__ X sub(X a, X b) { return a - b; }
    static __device__ __forceinline__ void step(St &s, X y, const Co &c)
    {
        double n = c.A * (y * s.cur) - c.B * s.prev;
        s.prev = s.cur;
        s.cur = n;
    }
    static __device__ __forceinline__ R val(const St &s) { return s.cur; }
    static __device__ __forceinline__ void renorm(St &) {}
    static __device__ __forceinline__ void rescale(St &s)
    {
        if (s.E < 0 && fabs(s.cur) > kBigD) {
            s.cur *= kSmallD;
            s.prev *= kSmallD;
            s.E += 1;
        }
    }
    static __device__ __forceinline__ R fac(int E) { return E == 0 ? 1.0 : (E == -1 ? kSmallD : 0.0); }
    static __device__ __forceinline__ void start(St &s, double L2, int sign, bool zero)
    {
        s.prev = 0.0;
        if (zero) { s.cur = 0.0; s.E = -1000; return; }
        double e = floor(L2 * (1.0 / kScaleBits));
        double fr = L2 - e * kScaleBits;
        double m = exp2(fr);
        s.cur = sign < 0 ? -m : m;
        s.E = (int)e;
    }
    static __device__ __forceinline__ void zero(St &s) { s.cur = 0.0; s.prev = 0.0; s.E = 0; }
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

// Regime of the next block of l for the whole warp: 0 all states at scale 0,
// 1 all states negligible (scale <= kSkipE), 2 mixed.
template <class P, int RPT, bool SPIN>
__device__ __forceinline__ int warp_regime(typename P::St (&sp)[RPT], typename P::St (&sm)[RPT])
{
#pragma unroll
    for (int k = 0; k < RPT; ++k) {  // keep the df32 low words small (once per block)
        P::renorm(sp[k]);
        if (SPIN) P::renorm(sm[k]);
    }
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

// One recursion step of all states owned by the thread to degree l.
template <class P, int RPT, bool SPIN, bool CHECK>
__device__ __forceinline__ void advance(typename P::St (&sp)[RPT], typename P::St (&sm)[RPT],
                                        const typename P::X (&x)[RPT], const void *rec_ab, const void *rec_c,
                                        int64_t idx)
{
    const typename P::Co co = P::load(rec_ab, idx);
    if (!SPIN) {
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            P::step(sp[k], x[k], co);
            if (CHECK) P::rescale(sp[k]);
        }
    } else {
        const typename P::X t = P::load_t(rec_c, idx);
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            P::step(sp[k], P::add(x[k], t), co);
            P::step(sm[k], P::sub(x[k], t), co);
            if (CHECK) { P::rescale(sp[k]); P::rescale(sm[k]); }
        }
    }
}

// ---------------------------------------------------------------- forward
template <class P, int RPT, bool SPIN>
__global__ void __launch_bounds__(512) k_leg_fwd(const typename P::C *__restrict__ alm, const void *__restrict__ rec_ab,
                                                 const void *__restrict__ rec_c, const double *__restrict__ lognorm,
                                                 RingTab rt, typename P::C *__restrict__ ring, int lmax, int mmax,
                                                 int spin, int ntheta, int nnorth, int64_t nalm)
{
    using R = typename P::R;
    using Cx = typename P::C;
    using St = typename P::St;
    using X = typename P::X;
    constexpr int BLK = 8;
    const int m = blockIdx.y;
    const int per_chunk = blockDim.x * RPT;
    const int64_t base = alm_base(lmax, m);
    const int s = SPIN ? spin : 0;
    const int l0 = m > s ? m : s;
    if (l0 > lmax) return;

    X x[RPT];
    St sp[RPT], sm[RPT];
    Cx pn[RPT], ps[RPT], qn[RPT], qs[RPT];
    const int rp0 = blockIdx.x * per_chunk + threadIdx.x * RPT;
    const double lnm = lognorm[m];
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        const int rp = rp0 + k;
        pn[k] = mkc(R(0), R(0)); ps[k] = pn[k]; qn[k] = pn[k]; qs[k] = pn[k];
        if (rp < nnorth) {
            x[k] = P::ring_x(rt, rp);
            const double ls = rt.lsin2[rp], lc = rt.lcos2[rp];
            start_value<P>(sp[k], m, s, s, lnm, ls, lc);
            if (SPIN) start_value<P>(sm[k], m, s, -s, lnm, ls, lc);
        } else {
            x[k] = X{};
            P::zero(sp[k]);
            P::zero(sm[k]);
        }
    }
    const Cx *aG = alm;
    const Cx *aC = alm + nalm;
    const R sgs = (s & 1) ? R(-1) : R(1);

    auto accumulate = [&](int l, bool scaled) {
        Cx g = __ldg(aG + base + l);
        if (m == 0) g.y = R(0);
        const R sg = ((l - m) & 1) ? R(-1) : R(1);
        if (!SPIN) {
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                R v = P::val(sp[k]);
                if (scaled) v *= P::fac(sp[k].E);
                const R vs = sg * v;
                pn[k].x += g.x * v; pn[k].y += g.y * v;
                ps[k].x += g.x * vs; ps[k].y += g.y * vs;
            }
        } else {
            Cx c = __ldg(aC + base + l);
            if (m == 0) c.y = R(0);
            // a = G + iC ; b = (-1)^s (conj G + i conj C)
            const Cx a = mkc(g.x - c.y, g.y + c.x);
            const Cx b = mkc(sgs * (g.x + c.y), sgs * (c.x - g.y));
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                R vp = P::val(sp[k]), vm = P::val(sm[k]);
                if (scaled) { vp *= P::fac(sp[k].E); vm *= P::fac(sm[k].E); }
                const R vps = sg * vp, vms = sg * vm;
                pn[k].x += a.x * vp; pn[k].y += a.y * vp;     // north, column +m
                ps[k].x += a.x * vms; ps[k].y += a.y * vms;   // south, column +m
                qn[k].x += b.x * vm; qn[k].y += b.y * vm;     // north, column -m
                qs[k].x += b.x * vps; qs[k].y += b.y * vps;   // south, column -m
            }
        }
    };

    accumulate(l0, true);
    for (int lb = l0 + 1; lb <= lmax; lb += BLK) {
        const int lend = min(lb + BLK, lmax + 1);
        const int regime = warp_regime<P, RPT, SPIN>(sp, sm);
        if (regime == 0) {
            for (int l = lb; l < lend; ++l) {
                advance<P, RPT, SPIN, false>(sp, sm, x, rec_ab, rec_c, base + l);
                accumulate(l, false);
            }
        } else if (regime == 1) {
            for (int l = lb; l < lend; ++l) advance<P, RPT, SPIN, true>(sp, sm, x, rec_ab, rec_c, base + l);
        } else {
            for (int l = lb; l < lend; ++l) {
                advance<P, RPT, SPIN, true>(sp, sm, x, rec_ab, rec_c, base + l);
                accumulate(l, true);
            }
        }
    }

    // write: spin 0 column m; spin s columns mmax + m (P) and mmax - m (Q), with the minus sign
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        const int jn = rp0 + k;
        if (jn >= nnorth) continue;
        const int js = ntheta - 1 - jn;
        if (!SPIN) {
            Cx *col = ring + (int64_t)m * ntheta;
            col[jn] = pn[k];
            if (js != jn) col[js] = ps[k];
        } else {
            Cx *colp = ring + (int64_t)(mmax + m) * ntheta;
            colp[jn] = mkc(-pn[k].x, -pn[k].y);
            if (js != jn) colp[js] = mkc(-ps[k].x, -ps[k].y);
            if (m > 0) {
                Cx *colq = ring + (int64_t)(mmax - m) * ntheta;
                colq[jn] = mkc(-qn[k].x, -qn[k].y);
                if (js != jn) colq[js] = mkc(-qs[k].x, -qs[k].y);
            }
        }
    }
}

// ---------------------------------------------------------------- adjoint
// Transpose-reduce of NV values per lane over the 32 lanes of a warp: after
// it, lane t holds the warp sum of value index (t >> (5 - log2 NV)).
template <int NV, typename R>
__device__ __forceinline__ R warp_transpose_reduce(R (&v)[NV])
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
                    R send = upper ? v[i] : v[i + half];
                    R keep = upper ? v[i + half] : v[i];
                    R got = __shfl_xor_sync(0xffffffffu, send, off);
                    v[i] = keep + got;
                }
            }
            cnt = half;
        } else {
            v[0] += __shfl_xor_sync(0xffffffffu, v[0], off);
        }
        off >>= 1;
    }
    return v[0];
}

template <class P, int RPT, bool SPIN, int LCH>
__global__ void __launch_bounds__(512) k_leg_adj(const typename P::C *__restrict__ ring, const void *__restrict__ rec_ab,
                                                 const void *__restrict__ rec_c, const double *__restrict__ lognorm,
                                                 RingTab rt, typename P::C *__restrict__ alm, int lmax, int mmax,
                                                 int spin, int ntheta, int nnorth, int64_t nalm)
{
    using R = typename P::R;
    using Cx = typename P::C;
    using St = typename P::St;
    using X = typename P::X;
    constexpr int NCOMP = SPIN ? 4 : 2;  // reals per l: spin 0 (re, im); spin s U, V
    constexpr int NV = LCH * NCOMP;
    constexpr int SH = (NV == 32 ? 0 : NV == 16 ? 1 : NV == 8 ? 2 : NV == 4 ? 3 : NV == 2 ? 4 : 5);

    const int m = blockIdx.y;
    const int lane = threadIdx.x & 31;
    const int per_chunk = blockDim.x * RPT;
    const int64_t base = alm_base(lmax, m);
    const int s = SPIN ? spin : 0;
    const int l0 = m > s ? m : s;
    if (l0 > lmax) return;
    const R sgs = (s & 1) ? R(-1) : R(1);

    X x[RPT];
    St sp[RPT], sm[RPT];
    // spin 0: hn/hs = ring values at north/south ring of column m.
    // spin s: hn/hs column +m, gn/gs column -m.
    Cx hn[RPT], hs[RPT], gn[RPT], gs[RPT];
    const int rp0 = blockIdx.x * per_chunk + threadIdx.x * RPT;
    const double lnm = lognorm[m];
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        const int rp = rp0 + k;
        hn[k] = mkc(R(0), R(0)); hs[k] = hn[k]; gn[k] = hn[k]; gs[k] = hn[k];
        if (rp < nnorth) {
            x[k] = P::ring_x(rt, rp);
            const double ls = rt.lsin2[rp], lc = rt.lcos2[rp];
            start_value<P>(sp[k], m, s, s, lnm, ls, lc);
            if (SPIN) start_value<P>(sm[k], m, s, -s, lnm, ls, lc);
            const int js = ntheta - 1 - rp;
            const Cx *colp = ring + (int64_t)(SPIN ? mmax + m : m) * ntheta;
            hn[k] = colp[rp];
            if (js != rp) hs[k] = colp[js];
            if (SPIN) {
                const Cx *colq = ring + (int64_t)(mmax - m) * ntheta;
                gn[k] = colq[rp];
                if (js != rp) gs[k] = colq[js];
            }
        } else {
            x[k] = X{};
            P::zero(sp[k]);
            P::zero(sm[k]);
        }
    }
    // spin 0: p = H_N + H_S (even l+m) and q = H_N - H_S (odd l+m)
    if (!SPIN) {
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            const Cx a = hn[k], b = hs[k];
            hn[k] = cadd(a, b);
            hs[k] = csub(a, b);
        }
    }

    for (int lc0 = l0; lc0 <= lmax; lc0 += LCH) {
        const int regime = warp_regime<P, RPT, SPIN>(sp, sm);
        const bool scaled = regime != 0;
        R part[NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) part[i] = R(0);
#pragma unroll
        for (int i = 0; i < LCH; ++i) {
            const int l = lc0 + i;
            if (l <= lmax) {
                if (l > l0) {
                    if (scaled) advance<P, RPT, SPIN, true>(sp, sm, x, rec_ab, rec_c, base + l);
                    else advance<P, RPT, SPIN, false>(sp, sm, x, rec_ab, rec_c, base + l);
                }
                if (regime != 1) {
                    const bool odd = ((l - m) & 1) != 0;
#pragma unroll
                    for (int k = 0; k < RPT; ++k) {
                        R vp = P::val(sp[k]);
                        if (scaled) vp *= P::fac(sp[k].E);
                        if (!SPIN) {
                            const Cx h = odd ? hs[k] : hn[k];
                            part[i * 2 + 0] += vp * h.x;
                            part[i * 2 + 1] += vp * h.y;
                        } else {
                            R vm = P::val(sm[k]);
                            if (scaled) vm *= P::fac(sm[k].E);
                            const R sg = odd ? R(-1) : R(1);
                            const R vms = sg * vm, vps = sg * vp;
                            // U += lam+ H_m(N) + sg lam- H_m(S) ; V += lam- H_-m(N) + sg lam+ H_-m(S)
                            part[i * 4 + 0] += vp * hn[k].x + vms * hs[k].x;
                            part[i * 4 + 1] += vp * hn[k].y + vms * hs[k].y;
                            part[i * 4 + 2] += vm * gn[k].x + vps * gs[k].x;
                            part[i * 4 + 3] += vm * gn[k].y + vps * gs[k].y;
                        }
                    }
                }
            }
        }
        if (regime == 1) continue;  // every contribution of this block is below 2^-180
        // warp reduction: lane t ends with value index t >> SH
        R tot = warp_transpose_reduce<NV, R>(part);
        const int v = lane >> SH;
        const int i = v / NCOMP, c = v % NCOMP;
        const int l = lc0 + i;
        R *out = reinterpret_cast<R *>(alm);
        if (!SPIN) {
            if ((lane & ((1 << SH) - 1)) == 0 && l <= lmax && !(m == 0 && c == 1))
                atomicAdd(out + 2 * (base + l) + c, tot);
        } else {
            // lanes hold U.re, U.im, V.re, V.im of degree l at c = 0..3; the
            // G/C split is linear, so each warp adds its share directly:
            //   G.re = -(U.re + sgs V.re)/2   G.im = -(U.im - sgs V.im)/2
            //   C.re = -(U.im + sgs V.im)/2   C.im =  (U.re - sgs V.re)/2
            const R other = __shfl_xor_sync(0xffffffffu, tot, 2 << SH);  // U <-> V of the same l
            if ((lane & ((1 << SH) - 1)) == 0 && l <= lmax) {
                R val;
                int64_t dst;
                if (c == 0) { val = R(-0.5) * (tot + sgs * other); dst = 2 * (base + l); }
                else if (c == 1) { val = R(-0.5) * (tot - sgs * other); dst = 2 * (base + l) + 1; }
                else if (c == 2) { val = R(0.5) * (other - sgs * tot); dst = 2 * (nalm + base + l) + 1; }
                else { val = R(-0.5) * (other + sgs * tot); dst = 2 * (nalm + base + l); }
                if (!(m == 0 && (c == 1 || c == 2))) atomicAdd(out + dst, val);
            }
        }
    }
}

// ------------------------------------------------------- coefficient tables
// For the step (l-1 -> l), j = l - 1:
//   A = (j+1) sqrt((2j+3)(2j+1) / (((j+1)^2-m^2)((j+1)^2-s^2)))
//   B = (j+1)/j sqrt((2j+3)/(2j-1)) sqrt((j^2-m^2)(j^2-s^2) / (((j+1)^2-m^2)((j+1)^2-s^2)))
//   T = m s / (j (j+1))
__global__ void k_rec_tables(int lmax, int spin, int prec, void *ab, void *tt)
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
        if (prec == LENS_FP32) {
            float ah = (float)A, bh = (float)B, th = (float)T;
            ((float4 *)ab)[base + l] = make_float4(ah, (float)(A - ah), bh, (float)(B - bh));
            if (tt) ((float2 *)tt)[base + l] = make_float2(th, (float)(T - th));
        } else {
            ((double2 *)ab)[base + l] = make_double2(A, B);
            if (tt) ((double *)tt)[base + l] = T;
        }
    }
}

template <class P, int RPT, bool SPIN>
cudaError_t fwd_launch(const Plan &p, const void *alm, void *ring, cudaStream_t st)
{
    dim3 grid(p.leg_chunks, p.mmax + 1);
    dim3 block(p.leg_warps * 32);
    k_leg_fwd<P, RPT, SPIN><<<grid, block, 0, st>>>((const typename P::C *)alm, p.rec_ab, p.rec_c, p.lognorm, p.rings,
                                                    (typename P::C *)ring, p.lmax, p.mmax, p.spin, p.ntheta,
                                                    p.nnorth, p.nalm);
    return cudaGetLastError();
}

template <class P, int RPT, bool SPIN, int LCH>
cudaError_t adj_launch(const Plan &p, const void *ring, void *alm, cudaStream_t st)
{
    dim3 grid(p.leg_chunks, p.mmax + 1);
    dim3 block(p.leg_warps * 32);
    const size_t ebytes = (p.prec == LENS_FP32 ? 8 : 16) * (size_t)p.nalm * (SPIN ? 2 : 1);
    cudaError_t e = cudaMemsetAsync(alm, 0, ebytes, st);
    if (e != cudaSuccess) return e;
    k_leg_adj<P, RPT, SPIN, LCH><<<grid, block, 0, st>>>((const typename P::C *)ring, p.rec_ab, p.rec_c, p.lognorm,
                                                         p.rings, (typename P::C *)alm, p.lmax, p.mmax, p.spin,
                                                         p.ntheta, p.nnorth, p.nalm);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_rec_tables(Plan &p)
{
    k_rec_tables<<<p.mmax + 1, 256, 0, p.stream>>>(p.lmax, p.spin, p.prec, p.rec_ab, p.spin ? p.rec_c : nullptr);
    return cudaGetLastError();
}

// Ring pairs per thread: RPT = 4 (df32) / 2 (fp64); spin s uses RPT 2 / 1.
int legendre_rpt(int prec, int spin) { return prec == LENS_FP32 ? (spin ? 2 : 4) : (spin ? 1 : 2); }

cudaError_t launch_legendre_fwd(const Plan &p, const void *alm, void *ring, cudaStream_t st)
{
    // entries with l < spin / columns without rings are never written by the
    // kernel: start from zero
    const size_t eb = p.prec == LENS_FP32 ? 8 : 16;
    cudaError_t e = cudaMemsetAsync(ring, 0, eb * (size_t)p.ncol * p.ntheta, st);
    if (e != cudaSuccess) return e;
    if (p.prec == LENS_FP32)
        return p.spin ? fwd_launch<PolDF, 2, true>(p, alm, ring, st) : fwd_launch<PolDF, 4, false>(p, alm, ring, st);
    return p.spin ? fwd_launch<PolF64, 1, true>(p, alm, ring, st) : fwd_launch<PolF64, 2, false>(p, alm, ring, st);
}

cudaError_t launch_legendre_adj(const Plan &p, const void *ring, void *alm, cudaStream_t st)
{
    if (p.prec == LENS_FP32)
        return p.spin ? adj_launch<PolDF, 2, true, 8>(p, ring, alm, st) : adj_launch<PolDF, 4, false, 16>(p, ring, alm, st);
    return p.spin ? adj_launch<PolF64, 1, true, 4>(p, ring, alm, st) : adj_launch<PolF64, 2, false, 8>(p, ring, alm, st);
}

}  // namespace gsl
