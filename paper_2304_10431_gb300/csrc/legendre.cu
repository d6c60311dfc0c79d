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

// ------------------------------------------------------------ policies
// A recursion state holds two consecutive degrees in w[0], w[1]; which word is
// the newest alternates.  E is the power-of-2^60 scale shared by both words.
struct PolDF {  // df32 recursion, FP32 accumulation
    using R = float;
    using C = float2;
    using X = df32;
    using Tab = float4;  // (A_hi, A_lo, B_hi, B_lo)
    using TTab = float2; // (T_hi, T_lo)
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
    static __device__ __forceinline__ X add(X a, X b) { return df_sub_u(a, {-b.h, -b.l}); }
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
    static __device__ __forceinline__ R val(const df32 &a) { return __fadd_rn(a.h, a.l); }
    static __device__ __forceinline__ df32 norm(df32 a)  // two-sum: exact for any ordering of |h|, |l|
    {
        const float h = __fadd_rn(a.h, a.l);
        const float bb = __fsub_rn(h, a.h);
        return {h, __fadd_rn(__fsub_rn(a.h, __fsub_rn(h, bb)), __fsub_rn(a.l, bb))};
    }
    static __device__ __forceinline__ void renorm(St &s)
    {
        s.w[0] = norm(s.w[0]);
        s.w[1] = norm(s.w[1]);
    }
    static __device__ __forceinline__ void rescale(St &s, int newest)
    {
        if (s.E < 0 && fabsf(s.w[newest].h) > kBigF) {
            s.w[0] = df_scale_pow2(s.w[0], kSmallF);
            s.w[1] = df_scale_pow2(s.w[1], kSmallF);
            s.E += 1;
        }
    }
    static __device__ __forceinline__ R fac(int E) { return E == 0 ? 1.0f : (E == -1 ? kSmallF : 0.0f); }
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
};

struct PolF64 {  // native FP64
    using R = double;
    using C = double2;
    using X = double;
    using Tab = double2;  // (A, B)
    using TTab = double;  // T
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
    static __device__ __forceinline__ R val(const double &a) { return a; }
    static __device__ __forceinline__ void renorm(St &) {}
    static __device__ __forceinline__ void rescale(St &s, int newest)
    {
        if (s.E < 0 && fabs(s.w[newest]) > kBigD) {
            s.w[0] *= kSmallD;
            s.w[1] *= kSmallD;
            s.E += 1;
        }
    }
    static __device__ __forceinline__ R fac(int E) { return E == 0 ? 1.0 : (E == -1 ? kSmallD : 0.0); }
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
    template <int NW, bool SCALED> __device__ __forceinline__ typename P::R vplus(int k) const
    {
        typename P::R v = P::val(sp[k].w[NW]);
        if (SCALED) v *= P::fac(sp[k].E);
        return v;
    }
    template <int NW, bool SCALED> __device__ __forceinline__ typename P::R vminus(int k) const
    {
        typename P::R v = P::val(sm[k].w[NW]);
        if (SCALED) v *= P::fac(sm[k].E);
        return v;
    }
};

// ---------------------------------------------------------------- forward
template <class P, int RPT, bool SPIN> struct FwdAcc {
    using R = typename P::R;
    using Cx = typename P::C;
    Cx pn[RPT], ps[RPT], qn[RPT], qs[RPT];
    const Cx *aG, *aC;
    int m;
    R sgs;

    __device__ __forceinline__ void init(const Cx *almm_g, const Cx *almm_c, int m_, int s)
    {
        aG = almm_g;
        aC = almm_c;
        m = m_;
        sgs = (s & 1) ? R(-1) : R(1);
#pragma unroll
        for (int k = 0; k < RPT; ++k) { pn[k] = mkc(R(0), R(0)); ps[k] = pn[k]; qn[k] = pn[k]; qs[k] = pn[k]; }
    }
    // contribution of degree l (value in word NW); sg = (-1)^{l+m}
    template <int NW, bool SCALED> __device__ __forceinline__ void add(const Rings<P, RPT, SPIN> &st, int l, R sg)
    {
        Cx g = __ldg(aG + l);
        if (m == 0) g.y = R(0);
        if (!SPIN) {
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                const R v = st.template vplus<NW, SCALED>(k);
                const R vs = sg * v;
                pn[k].x += g.x * v; pn[k].y += g.y * v;
                ps[k].x += g.x * vs; ps[k].y += g.y * vs;
            }
        } else {
            Cx c = __ldg(aC + l);
            if (m == 0) c.y = R(0);
            // a = G + iC ; b = (-1)^s (conj G + i conj C)
            const Cx a = mkc(g.x - c.y, g.y + c.x);
            const Cx b = mkc(sgs * (g.x + c.y), sgs * (c.x - g.y));
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                const R vp = st.template vplus<NW, SCALED>(k), vm = st.template vminus<NW, SCALED>(k);
                const R vps = sg * vp, vms = sg * vm;
                pn[k].x += a.x * vp; pn[k].y += a.y * vp;     // north, column +m
                ps[k].x += a.x * vms; ps[k].y += a.y * vms;   // south, column +m
                qn[k].x += b.x * vm; qn[k].y += b.y * vm;     // north, column -m
                qs[k].x += b.x * vps; qs[k].y += b.y * vps;   // south, column -m
            }
        }
    }
};

template <class P, int RPT, bool SPIN, int REG>
__device__ __forceinline__ void fwd_block(Rings<P, RPT, SPIN> &st, FwdAcc<P, RPT, SPIN> &acc,
                                          const typename P::Tab *recm, const typename P::TTab *recc, int lb,
                                          typename P::R s0)
{
#pragma unroll
    for (int j = 0; j < kBlk; ++j) {
        const int l = lb + j;
        const typename P::R sg = (j & 1) ? -s0 : s0;
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
__global__ void __launch_bounds__(512) k_leg_fwd(const typename P::C *__restrict__ alm, const void *__restrict__ rec_ab,
                                                 const void *__restrict__ rec_c, const double *__restrict__ lognorm,
                                                 RingTab rt, typename P::C *__restrict__ ring, int lmax, int mmax,
                                                 int spin, int ntheta, int nnorth, int64_t nalm)
{
    using R = typename P::R;
    using Cx = typename P::C;
    const int m = blockIdx.y;
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
    acc.init(alm + base, alm + nalm + base, m, s);

    acc.template add<1, true>(st, l0, ((l0 - m) & 1) ? R(-1) : R(1));  // l0 = s > m for m < s
    int l = l0 + 1;
    const R s0 = ((l - m) & 1) ? R(-1) : R(1);  // sign of the first degree of every block
    for (; l + kBlk <= lmax + 1; l += kBlk) {
        const int reg = st.regime();
        if (reg == 0) fwd_block<P, RPT, SPIN, 0>(st, acc, recm, recc, l, s0);
        else if (reg == 1) fwd_block<P, RPT, SPIN, 1>(st, acc, recm, recc, l, s0);
        else fwd_block<P, RPT, SPIN, 2>(st, acc, recm, recc, l, s0);
    }
    for (; l <= lmax; ++l) {  // tail: general path
        st.advance_moved(recm, recc, l);
        acc.template add<1, true>(st, l, ((l - m) & 1) ? R(-1) : R(1));
    }

    // write: spin 0 column m; spin s columns mmax + m (P) and mmax - m (Q), with the minus sign
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        const int jn = rp0 + k;
        if (jn >= nnorth) continue;
        const int js = ntheta - 1 - jn;
        if (!SPIN) {
            Cx *col = ring + (int64_t)m * ntheta;
            col[jn] = acc.pn[k];
            if (js != jn) col[js] = acc.ps[k];
        } else {
            Cx *colp = ring + (int64_t)(mmax + m) * ntheta;
            colp[jn] = mkc(-acc.pn[k].x, -acc.pn[k].y);
            if (js != jn) colp[js] = mkc(-acc.ps[k].x, -acc.ps[k].y);
            if (m > 0) {
                Cx *colq = ring + (int64_t)(mmax - m) * ntheta;
                colq[jn] = mkc(-acc.qn[k].x, -acc.qn[k].y);
                if (js != jn) colq[js] = mkc(-acc.qs[k].x, -acc.qs[k].y);
            }
        }
    }
}

// ---------------------------------------------------------------- adjoint
// Transpose-reduce of NV values per lane over the 32 lanes of a warp: after
// it, lane t holds the warp sum of value index (t >> (5 - log2 NV)).
template <int NV, typename R> __device__ __forceinline__ R warp_transpose_reduce(R (&v)[NV])
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

template <class P, int RPT, bool SPIN> struct AdjIn {
    using R = typename P::R;
    using Cx = typename P::C;
    // spin 0: hn = H_N + H_S (even l+m), hs = H_N - H_S (odd l+m)
    // spin s: hn/hs column +m north/south, gn/gs column -m
    Cx hn[RPT], hs[RPT], gn[RPT], gs[RPT];

    __device__ __forceinline__ void init(const Cx *ring, int rp0, int nnorth, int ntheta, int m, int mmax)
    {
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            const int rp = rp0 + k;
            hn[k] = mkc(R(0), R(0)); hs[k] = hn[k]; gn[k] = hn[k]; gs[k] = hn[k];
            if (rp < nnorth) {
                const int js = ntheta - 1 - rp;
                const Cx *colp = ring + (int64_t)(SPIN ? mmax + m : m) * ntheta;
                hn[k] = colp[rp];
                if (js != rp) hs[k] = colp[js];
                if (SPIN) {
                    const Cx *colq = ring + (int64_t)(mmax - m) * ntheta;
                    gn[k] = colq[rp];
                    if (js != rp) gs[k] = colq[js];
                } else {
                    const Cx a = hn[k], b = hs[k];
                    hn[k] = cadd(a, b);
                    hs[k] = csub(a, b);
                }
            }
        }
    }
    // partial sums of one degree (value in word NW) into part[0..NCOMP)
    template <int NW, bool SCALED>
    __device__ __forceinline__ void add(const Rings<P, RPT, SPIN> &st, bool odd, R *part) const
    {
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            const R vp = st.template vplus<NW, SCALED>(k);
            if (!SPIN) {
                const Cx h = odd ? hs[k] : hn[k];
                part[0] += vp * h.x;
                part[1] += vp * h.y;
            } else {
                const R vm = st.template vminus<NW, SCALED>(k);
                const R sg = odd ? R(-1) : R(1);
                const R vms = sg * vm, vps = sg * vp;
                // U += lam+ H_m(N) + sg lam- H_m(S) ; V += lam- H_-m(N) + sg lam+ H_-m(S)
                part[0] += vp * hn[k].x + vms * hs[k].x;
                part[1] += vp * hn[k].y + vms * hs[k].y;
                part[2] += vm * gn[k].x + vps * gs[k].x;
                part[3] += vm * gn[k].y + vps * gs[k].y;
            }
        }
    }
};

// Adds the warp sums of the degrees lb + i (value index i * NCOMP + c) into
// a_lm (spin 0) or G, C (spin s).
template <typename R, bool SPIN, int NV>
__device__ __forceinline__ void flush(R (&part)[NV], R *out, int64_t base, int64_t nalm, int m, int lb, int lmax,
                                      R sgs)
{
    constexpr int NCOMP = SPIN ? 4 : 2;
    constexpr int SH = (NV == 32 ? 0 : NV == 16 ? 1 : NV == 8 ? 2 : NV == 4 ? 3 : NV == 2 ? 4 : 5);
    const int lane = threadIdx.x & 31;
    const R tot = warp_transpose_reduce<NV, R>(part);
    const int v = lane >> SH;
    const int i = v / NCOMP, c = v % NCOMP;
    const int l = lb + i;
    if (!SPIN) {
        if ((lane & ((1 << SH) - 1)) == 0 && l <= lmax && !(m == 0 && c == 1))
            atomicAdd(out + 2 * (base + l) + c, tot);
    } else {
        // lanes hold U.re, U.im, V.re, V.im of degree l at c = 0..3; the G/C
        // split is linear, so each warp adds its share directly:
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

template <class P, int RPT, bool SPIN, int REG>
__device__ __forceinline__ void adj_block(Rings<P, RPT, SPIN> &st, const AdjIn<P, RPT, SPIN> &in,
                                          typename P::R *part, const typename P::Tab *recm,
                                          const typename P::TTab *recc, int lb, bool odd0)
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
                                                 int spin, int ntheta, int nnorth, int64_t nalm)
{
    using R = typename P::R;
    constexpr int NCOMP = SPIN ? 4 : 2;
    constexpr int NV = kBlk * NCOMP;
    const int m = blockIdx.y;
    const int s = SPIN ? spin : 0;
    const int l0 = m > s ? m : s;
    if (l0 > lmax) return;
    const int64_t base = alm_base(lmax, m);
    const typename P::Tab *recm = (const typename P::Tab *)rec_ab + base;
    const typename P::TTab *recc = SPIN ? (const typename P::TTab *)rec_c + base : nullptr;
    const int rp0 = (blockIdx.x * blockDim.x + threadIdx.x) * RPT;
    const R sgs = (s & 1) ? R(-1) : R(1);
    R *out = reinterpret_cast<R *>(alm);

    Rings<P, RPT, SPIN> st;
    st.init(rt, rp0, nnorth, m, s, lognorm[m]);
    AdjIn<P, RPT, SPIN> in;
    in.init(ring, rp0, nnorth, ntheta, m, mmax);

    {  // degree l0 (the start value): one reduction of NCOMP values
        R p0[NCOMP];
#pragma unroll
        for (int c = 0; c < NCOMP; ++c) p0[c] = R(0);
        in.template add<1, true>(st, ((l0 - m) & 1) != 0, p0);  // l0 = s > m for m < s
        flush<R, SPIN, NCOMP>(p0, out, base, nalm, m, l0, lmax, sgs);
    }
    int l = l0 + 1;
    const bool odd0 = ((l - m) & 1) != 0;
    R part[NV];
    for (; l + kBlk <= lmax + 1; l += kBlk) {
        const int reg = st.regime();
        if (reg == 1) {  // every contribution of this block is below 2^-180: recursion only
            adj_block<P, RPT, SPIN, 1>(st, in, part, recm, recc, l, odd0);
            continue;
        }
#pragma unroll
        for (int i = 0; i < NV; ++i) part[i] = R(0);
        if (reg == 0) adj_block<P, RPT, SPIN, 0>(st, in, part, recm, recc, l, odd0);
        else adj_block<P, RPT, SPIN, 2>(st, in, part, recm, recc, l, odd0);
        flush<R, SPIN, NV>(part, out, base, nalm, m, l, lmax, sgs);
    }
    if (l <= lmax) {  // tail: fewer than kBlk degrees, general path
#pragma unroll
        for (int i = 0; i < NV; ++i) part[i] = R(0);
#pragma unroll
        for (int j = 0; j < kBlk; ++j) {
            if (l + j <= lmax) {
                st.advance_moved(recm, recc, l + j);
                in.template add<1, true>(st, ((l + j - m) & 1) != 0, part + j * NCOMP);
            }
        }
        flush<R, SPIN, NV>(part, out, base, nalm, m, l, lmax, sgs);
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
    dim3 grid(p.leg_f.chunks, p.mmax + 1);
    dim3 block(p.leg_f.warps * 32);
    k_leg_fwd<P, RPT, SPIN><<<grid, block, 0, st>>>((const typename P::C *)alm, p.rec_ab, p.rec_c, p.lognorm, p.rings,
                                                    (typename P::C *)ring, p.lmax, p.mmax, p.spin, p.ntheta,
                                                    p.nnorth, p.nalm);
    return cudaGetLastError();
}

template <class P, int RPT, bool SPIN>
cudaError_t adj_launch(const Plan &p, const void *ring, void *alm, cudaStream_t st)
{
    dim3 grid(p.leg_a.chunks, p.mmax + 1);
    dim3 block(p.leg_a.warps * 32);
    const size_t ebytes = (p.prec == LENS_FP32 ? 8 : 16) * (size_t)p.nalm * (SPIN ? 2 : 1);
    cudaError_t e = cudaMemsetAsync(alm, 0, ebytes, st);
    if (e != cudaSuccess) return e;
    k_leg_adj<P, RPT, SPIN><<<grid, block, 0, st>>>((const typename P::C *)ring, p.rec_ab, p.rec_c, p.lognorm,
                                                    p.rings, (typename P::C *)alm, p.lmax, p.mmax, p.spin,
                                                    p.ntheta, p.nnorth, p.nalm);
    return cudaGetLastError();
}

template <class P, bool SPIN> cudaError_t fwd_rpt(const Plan &p, const void *alm, void *ring, cudaStream_t st)
{
    switch (p.leg_f.rpt) {
    case 1: return fwd_launch<P, 1, SPIN>(p, alm, ring, st);
    case 2: return fwd_launch<P, 2, SPIN>(p, alm, ring, st);
    default: return fwd_launch<P, 4, SPIN>(p, alm, ring, st);
    }
}

template <class P, bool SPIN> cudaError_t adj_rpt(const Plan &p, const void *ring, void *alm, cudaStream_t st)
{
    switch (p.leg_a.rpt) {
    case 1: return adj_launch<P, 1, SPIN>(p, ring, alm, st);
    case 2: return adj_launch<P, 2, SPIN>(p, ring, alm, st);
    default: return adj_launch<P, 4, SPIN>(p, ring, alm, st);
    }
}

}  // namespace

cudaError_t launch_rec_tables(Plan &p)
{
    k_rec_tables<<<p.mmax + 1, 256, 0, p.stream>>>(p.lmax, p.spin, p.prec, p.rec_ab, p.spin ? p.rec_c : nullptr);
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

bool legendre_rpt_supported(int, int, bool, int rpt) { return rpt == 1 || rpt == 2 || rpt == 4; }

cudaError_t launch_legendre_fwd(const Plan &p, const void *alm, void *ring, cudaStream_t st)
{
    // entries with l < spin / columns without rings are never written by the
    // kernel: start from zero
    const size_t eb = p.prec == LENS_FP32 ? 8 : 16;
    cudaError_t e = cudaMemsetAsync(ring, 0, eb * (size_t)p.ncol * p.ntheta, st);
    if (e != cudaSuccess) return e;
    if (p.prec == LENS_FP32)
        return p.spin ? fwd_rpt<PolDF, true>(p, alm, ring, st) : fwd_rpt<PolDF, false>(p, alm, ring, st);
    return p.spin ? fwd_rpt<PolF64, true>(p, alm, ring, st) : fwd_rpt<PolF64, false>(p, alm, ring, st);
}

cudaError_t launch_legendre_adj(const Plan &p, const void *ring, void *alm, cudaStream_t st)
{
    if (p.prec == LENS_FP32)
        return p.spin ? adj_rpt<PolDF, true>(p, ring, alm, st) : adj_rpt<PolDF, false>(p, ring, alm, st);
    return p.spin ? adj_rpt<PolF64, true>(p, ring, alm, st) : adj_rpt<PolF64, false>(p, ring, alm, st);
}

}  // namespace gsl
