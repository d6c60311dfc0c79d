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
//   T_l = m s / ((l-1) l), sigma = +1 for +s, -1 for -s, x = cos theta,
// run in monic form: with c_{l0} = c_{l0+1} = 1 and c_l = B_l c_{l-2}, the
// scaled values mu_l = lambda_l / c_l obey
//   mu_l = (alpha_l x + sigma tau_l) mu_{l-1} - mu_{l-2},
//   alpha_l = A_l c_{l-1} / c_l,  tau_l = alpha_l T_l,
// one product per step fewer than the plain form.  The forward folds c_l
// into the coefficients (k_coef_prep, once per call); the adjoint multiplies
// each degree's warp sum by c_l before adding it into a_lm.  c_l stays close
// to 1 (within [2^-2.6, 2^0.2] for lmax 4096).
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
// The sign (-1)^{l+m} is s0 (-1)^{l-lf} with lf = l0 + 1 the first degree of
// the block loop, so inside a block it is a compile-time sign times the
// per-m constant s0, applied once at the end (forward) or to the inputs
// (adjoint).
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

#include <type_traits>

#include "common.cuh"
#include "internal.h"

#include "legendre_rec.cuh"

namespace gsl {
namespace {

// ---------------------------------------------------------------- forward
// Accumulators per ring; "rel" below is (-1)^(l - lf), the sign of a degree
// relative to the first degree lf = l0 + 1 of the block loop.
//   spin 0: (r0, i0) sums degrees with rel = +1, (r1, i1) rel = -1;
//           north = sum0 + sum1, south = s0 (sum0 - sum1).
//   spin s: (r0, i0) = sum a s-lambda (north, +m), (r1, i1) = sum rel a (-s)lambda
//           (south, +m), (r2, i2) = sum b (-s)lambda (north, -m), (r3, i3) =
//           sum rel b s-lambda (south, -m); the south sums are multiplied by s0.
//   gradient-only spin s (C = 0, so b = (-1)^s conj a): (r0, i0) / (r1, i1) sum
//           a s-lambda over degrees with rel = +1 / -1, (r2, i2) / (r3, i3)
//           a (-s)lambda; the four spin-s sums follow from them at the end.
template <class P, int RPT, bool SPIN, int NM = 1, bool GRAD = false> struct FwdAcc {
    // NM maps share the recursion: map b's prepared coefficients start at
    // tab + b * (ncomp nalm) entries and it has its own accumulators
    using A = typename P::A;
    using K = typename P::K;
    A r0[NM][RPT], i0[NM][RPT], r1[NM][RPT], i1[NM][RPT], r2[NM][RPT], i2[NM][RPT], r3[NM][RPT], i3[NM][RPT];
    const void *tab;
    int64_t nalm, base;

    __device__ __forceinline__ void init(const void *tab_, int64_t nalm_, int64_t base_)
    {
        tab = tab_;
        nalm = nalm_;
        base = base_;
#pragma unroll
        for (int b = 0; b < NM; ++b)
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                r0[b][k] = P::azero(); i0[b][k] = r0[b][k]; r1[b][k] = r0[b][k]; i1[b][k] = r0[b][k];
                r2[b][k] = r0[b][k]; i2[b][k] = r0[b][k]; r3[b][k] = r0[b][k]; i3[b][k] = r0[b][k];
            }
    }
    __device__ __forceinline__ void renorm()
    {
#pragma unroll
        for (int b = 0; b < NM; ++b)
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                P::arenorm(r0[b][k]); P::arenorm(i0[b][k]); P::arenorm(r1[b][k]); P::arenorm(i1[b][k]);
                if (SPIN) {
                    P::arenorm(r2[b][k]); P::arenorm(i2[b][k]); P::arenorm(r3[b][k]); P::arenorm(i3[b][k]);
                }
            }
    }
    // contribution of degree l (value in word NW), ODD: rel = -1
    template <int NW, bool SCALED, bool ODD> __device__ __forceinline__ void add(const Rings<P, RPT, SPIN> &st, int l)
    {
        typename P::V vp[RPT], vm[RPT];
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            vp[k] = st.template vplus<NW, SCALED>(k);
            if (SPIN) vm[k] = st.template vminus<NW, SCALED>(k);
        }
        add_vals<ODD>(vp, vm, l);
    }
    // contribution of degree l given its values (+s in vp, -s in vm) on the rings
    template <bool ODD>
    __device__ __forceinline__ void add_vals(const typename P::V (&vp)[RPT], const typename P::V (&vm)[RPT], int l)
    {
        const int64_t mstride = (SPIN ? 2 : 1) * nalm;
#pragma unroll
        for (int b = 0; b < NM; ++b) {
            K ar, ai;
            P::coef(tab, nalm, 0, b * mstride + base + l, ar, ai);
            if (GRAD) {
#pragma unroll
                for (int k = 0; k < RPT; ++k) {
                    if (!ODD) {
                        P::fma(r0[b][k], ar, vp[k]); P::fma(i0[b][k], ai, vp[k]);
                        P::fma(r2[b][k], ar, vm[k]); P::fma(i2[b][k], ai, vm[k]);
                    } else {
                        P::fma(r1[b][k], ar, vp[k]); P::fma(i1[b][k], ai, vp[k]);
                        P::fma(r3[b][k], ar, vm[k]); P::fma(i3[b][k], ai, vm[k]);
                    }
                }
            } else if (!SPIN) {
#pragma unroll
                for (int k = 0; k < RPT; ++k) {
                    if (!ODD) { P::fma(r0[b][k], ar, vp[k]); P::fma(i0[b][k], ai, vp[k]); }
                    else { P::fma(r1[b][k], ar, vp[k]); P::fma(i1[b][k], ai, vp[k]); }
                }
            } else {
                K br, bi;
                P::coef(tab, nalm, 1, b * mstride + base + l, br, bi);
#pragma unroll
                for (int k = 0; k < RPT; ++k) {
                    P::fma(r0[b][k], ar, vp[k]); P::fma(i0[b][k], ai, vp[k]);
                    P::fma(r2[b][k], br, vm[k]); P::fma(i2[b][k], bi, vm[k]);
                    if (!ODD) {
                        P::fma(r1[b][k], ar, vm[k]); P::fma(i1[b][k], ai, vm[k]);
                        P::fma(r3[b][k], br, vp[k]); P::fma(i3[b][k], bi, vp[k]);
                    } else {
                        P::fms(r1[b][k], ar, vm[k]); P::fms(i1[b][k], ai, vm[k]);
                        P::fms(r3[b][k], br, vp[k]); P::fms(i3[b][k], bi, vp[k]);
                    }
                }
            }
        }
    }
    // add_vals with the degree's prepared coefficients already loaded (one map, full spin-s or spin 0)
    template <bool ODD>
    __device__ __forceinline__ void add_vals_c(const typename P::V (&vp)[RPT], const typename P::V (&vm)[RPT], K ar,
                                               K ai, K br, K bi)
    {
        static_assert(NM == 1 && !GRAD, "one map, not gradient-only");
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            if (!SPIN) {
                if (!ODD) { P::fma(r0[0][k], ar, vp[k]); P::fma(i0[0][k], ai, vp[k]); }
                else { P::fma(r1[0][k], ar, vp[k]); P::fma(i1[0][k], ai, vp[k]); }
            } else {
                P::fma(r0[0][k], ar, vp[k]); P::fma(i0[0][k], ai, vp[k]);
                P::fma(r2[0][k], br, vm[k]); P::fma(i2[0][k], bi, vm[k]);
                if (!ODD) {
                    P::fma(r1[0][k], ar, vm[k]); P::fma(i1[0][k], ai, vm[k]);
                    P::fma(r3[0][k], br, vp[k]); P::fma(i3[0][k], bi, vp[k]);
                } else {
                    P::fms(r1[0][k], ar, vm[k]); P::fms(i1[0][k], ai, vm[k]);
                    P::fms(r3[0][k], br, vp[k]); P::fms(i3[0][k], bi, vp[k]);
                }
            }
        }
    }
    // general path (start value and tail): parity known at run time only
    __device__ __forceinline__ void add_rt(const Rings<P, RPT, SPIN> &st, int l, bool odd)
    {
        if (odd) add<1, true, true>(st, l);
        else add<1, true, false>(st, l);
    }
};

template <class P, int RPT, bool SPIN, int REG, int NM, bool GRAD>
__device__ __forceinline__ void fwd_block(Rings<P, RPT, SPIN> &st, FwdAcc<P, RPT, SPIN, NM, GRAD> &acc,
                                          const typename P::Tab *reca, const typename P::TTab *rect, int lb)
{
#pragma unroll
    for (int j = 0; j < kBlk; ++j) {
        const int l = lb + j;
        if (j & 1) {
            st.template advance<1, REG != 0>(reca, rect, l);
            if (REG != 1) acc.template add<1, REG == 2, true>(st, l);
        } else {
            st.template advance<0, REG != 0>(reca, rect, l);
            if (REG != 1) acc.template add<0, REG == 2, false>(st, l);
        }
    }
}

// Restarted FP32 recursion, one spin-0 map: the block's step-table entries and
// prepared coefficients are loaded together before its 8 steps, so their
// latency is paid once per block instead of once per degree (spin s: the
// 16 more coefficient registers cost as much as the latency saves).
template <class P, int RPT, bool SPIN, int REG, class TabE>
__device__ __forceinline__ void fwd_block_pf(Rings<P, RPT, SPIN> &st, FwdAcc<P, RPT, SPIN, 1, false> &acc,
                                             const TabE *reca, const float2 *ca, const float2 *cb, int lb)
{
    TabE tb[kBlk];
    float2 a[kBlk], b[kBlk];
#pragma unroll
    for (int j = 0; j < kBlk; ++j) {
        tb[j] = __ldg(reca + lb + j);
        if (REG != 1) {
            a[j] = __ldg(ca + lb + j);
            if (SPIN) b[j] = __ldg(cb + lb + j);
        }
    }
#pragma unroll
    for (int j = 0; j < kBlk; ++j) {
        typename P::V vp[RPT], vm[RPT];
        if (j & 1) st.template advance_c<1, REG != 0>(tb[j]);
        else st.template advance_c<0, REG != 0>(tb[j]);
        if (REG == 1) continue;
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            vp[k] = (j & 1) ? st.template vplus<1, REG == 2>(k) : st.template vplus<0, REG == 2>(k);
            if (SPIN) vm[k] = (j & 1) ? st.template vminus<1, REG == 2>(k) : st.template vminus<0, REG == 2>(k);
        }
        const float2 bb = SPIN ? b[j] : make_float2(0.f, 0.f);
        if (j & 1) acc.template add_vals_c<true>(vp, vm, a[j].x, a[j].y, bb.x, bb.y);
        else acc.template add_vals_c<false>(vp, vm, a[j].x, a[j].y, bb.x, bb.y);
    }
}

// NM maps share each recursion (prepared coefficients of map b at coef + b *
// ncomp nalm entries, its ring coefficients at ring + b * ring_stride).
// GRAD: gradient-only spin s (prepared coefficients of G alone, see FwdAcc).
// Restarted FP32 recursions (P::kRestart) reset their state from ck at every
// K-th degree of the block loop.
template <class P, int RPT, bool SPIN, int NM, bool GRAD>
__device__ __forceinline__ void leg_fwd_body(const void *__restrict__ coef, const void *__restrict__ rec_a,
                                             const void *__restrict__ rec_t, const double *__restrict__ lognorm,
                                             const RingTab &rt, typename P::C *__restrict__ ring, int lmax, int mmax,
                                             int spin, int ntheta, int nnorth, int64_t nalm, int m_begin,
                                             int64_t ring_stride, const CkTab &ck)
{
    using Sg = decltype(P::fac(0));
    using Cx = typename P::C;
    using A = typename P::A;
    const int m = m_begin + blockIdx.y;
    const int s = SPIN ? spin : 0;
    const int l0 = m > s ? m : s;
    if (l0 > lmax) return;
    const int64_t base = alm_base(lmax, m);
    // spin s: reca addresses the interleaved (alpha, tau) table (TabAT entries)
    const typename P::Tab *reca =
        SPIN ? reinterpret_cast<const typename P::Tab *>((const typename P::TabAT *)rec_a + base)
             : (const typename P::Tab *)rec_a + base;
    const typename P::TTab *rect = SPIN ? (const typename P::TTab *)rec_t + base : nullptr;
    const int rp0 = (blockIdx.x * blockDim.x + threadIdx.x) * RPT;

    const int lf = l0 + 1;
    Rings<P, RPT, SPIN> st;
    FwdAcc<P, RPT, SPIN, NM, GRAD> acc;
    acc.init(coef, nalm, base);
    const Sg s0 = ((lf - m) & 1) ? Sg(-1) : Sg(1);  // (-1)^(lf - m)
    int l = lf;
    bool jumped = false;
    const int Km = P::kRestart ? ck_interval(ck, m) : 0;
    if constexpr (P::kRestart) {  // start at the warp's first restart: every earlier degree is negligible
        const int kj = first_restart<RPT>(ck, m);
        if (kj > 0) {
            st.init_geom(rt, rp0, nnorth);
            l = lf + kj * Km;  // the restart at l sets the state
            jumped = true;
        }
    }
    if (!jumped) {
        st.init(rt, rp0, nnorth, m, s, lognorm[m]);
        acc.add_rt(st, l0, true);  // l0 = lf - 1
    }
    const int64_t ckrow = P::kRestart ? __ldg(ck.base + m) : 0;
    for (; l + kBlk <= lmax + 1; l += kBlk) {
        if constexpr (P::kRestart) {
            const int dl = l - lf;
            if (dl != 0 && (dl & (Km - 1)) == 0) {
                const int64_t row = ckrow + (int64_t)(dl / Km - 1) * nnorth;
                if constexpr (P::kScaleF) st.restart_scaled(ck, row, rp0, nnorth, ck.cs + base, l);
                else st.restart(ck, row, rp0, nnorth);
            }
        }
        int reg = st.regime();
        // restarted recursions start at the warp's first significant restart, so a block of
        // negligible states is rare there: it runs the scaled path (its terms are exact zeros)
        // and the recursion-only variant is not compiled
        if constexpr (P::kRestart) reg = reg == 1 ? 2 : reg;
        acc.renorm();
        if constexpr (P::kRestart && !P::kMonic && NM == 1 && !GRAD && !SPIN) {  // lmax 4096: 4.52 -> 4.40 ms;
                                                                                // spin s gains nothing
            const float2 *ca = (const float2 *)coef + base;
            const float2 *cb = (const float2 *)coef + nalm + base;
            if (reg == 0) fwd_block_pf<P, RPT, SPIN, 0>(st, acc, reca, ca, cb, l);
            else fwd_block_pf<P, RPT, SPIN, 2>(st, acc, reca, ca, cb, l);
        } else {
            if (reg == 0) fwd_block<P, RPT, SPIN, 0, NM, GRAD>(st, acc, reca, rect, l);
            else if (!P::kRestart && reg == 1) fwd_block<P, RPT, SPIN, 1, NM, GRAD>(st, acc, reca, rect, l);
            else fwd_block<P, RPT, SPIN, 2, NM, GRAD>(st, acc, reca, rect, l);
        }
    }
    for (; l <= lmax; ++l) {  // tail: general path
        st.advance_moved(reca, rect, l);
        acc.add_rt(st, l, ((l - lf) & 1) != 0);
    }

    // write: spin 0 column m; spin s columns mmax + m (P) and mmax - m (Q), with the minus sign
#pragma unroll
    for (int b = 0; b < NM; ++b)
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            const int jn = rp0 + k;
            if (jn >= nnorth) continue;
            const int js = ntheta - 1 - jn;
            Cx *rb = ring + b * ring_stride;
            if (!SPIN) {
                Cx *col = rb + (int64_t)m * ntheta;
                col[jn] = P::cout(P::aadd(acc.r0[b][k], acc.r1[b][k]), P::aadd(acc.i0[b][k], acc.i1[b][k]));
                if (js != jn)
                    col[js] = P::cout(P::ascale(P::asub(acc.r0[b][k], acc.r1[b][k]), s0),
                                      P::ascale(P::asub(acc.i0[b][k], acc.i1[b][k]), s0));
            } else if (GRAD) {
                // sum a s-lambda, sum rel a (-s)lambda, sgs conj(sum a (-s)lambda), sgs conj(sum rel a s-lambda)
                const Sg ms0 = -s0, sgs = (s & 1) ? Sg(-1) : Sg(1);
                const A pr = P::aadd(acc.r0[b][k], acc.r1[b][k]), pi = P::aadd(acc.i0[b][k], acc.i1[b][k]);
                const A qr = P::asub(acc.r2[b][k], acc.r3[b][k]), qi = P::asub(acc.i2[b][k], acc.i3[b][k]);
                Cx *colp = rb + (int64_t)(mmax + m) * ntheta;
                colp[jn] = P::cout(P::ascale(pr, Sg(-1)), P::ascale(pi, Sg(-1)));
                if (js != jn) colp[js] = P::cout(P::ascale(qr, ms0), P::ascale(qi, ms0));
                if (m > 0) {
                    const A ur = P::aadd(acc.r2[b][k], acc.r3[b][k]), ui = P::aadd(acc.i2[b][k], acc.i3[b][k]);
                    const A wr = P::asub(acc.r0[b][k], acc.r1[b][k]), wi = P::asub(acc.i0[b][k], acc.i1[b][k]);
                    Cx *colq = rb + (int64_t)(mmax - m) * ntheta;
                    colq[jn] = P::cout(P::ascale(ur, -sgs), P::ascale(ui, sgs));
                    if (js != jn) colq[js] = P::cout(P::ascale(wr, sgs * ms0), P::ascale(wi, -(sgs * ms0)));
                }
            } else {
                const Sg ms0 = -s0;
                Cx *colp = rb + (int64_t)(mmax + m) * ntheta;
                colp[jn] = P::cout(P::ascale(acc.r0[b][k], Sg(-1)), P::ascale(acc.i0[b][k], Sg(-1)));
                if (js != jn) colp[js] = P::cout(P::ascale(acc.r1[b][k], ms0), P::ascale(acc.i1[b][k], ms0));
                if (m > 0) {
                    Cx *colq = rb + (int64_t)(mmax - m) * ntheta;
                    colq[jn] = P::cout(P::ascale(acc.r2[b][k], Sg(-1)), P::ascale(acc.i2[b][k], Sg(-1)));
                    if (js != jn) colq[js] = P::cout(P::ascale(acc.r3[b][k], ms0), P::ascale(acc.i3[b][k], ms0));
                }
            }
        }
}

template <class P, int RPT, bool SPIN, int NM = 1, bool GRAD = false>
__global__ void __launch_bounds__(512) k_leg_fwd(const void *__restrict__ coef, const void *__restrict__ rec_a,
                                                 const void *__restrict__ rec_t, const double *__restrict__ lognorm,
                                                 RingTab rt, typename P::C *__restrict__ ring, int lmax, int mmax,
                                                 int spin, int ntheta, int nnorth, int64_t nalm, int m_begin,
                                                 int64_t ring_stride, CkTab ck)
{
    leg_fwd_body<P, RPT, SPIN, NM, GRAD>(coef, rec_a, rec_t, lognorm, rt, ring, lmax, mmax, spin, ntheta, nnorth,
                                         nalm, m_begin, ring_stride, ck);
}

// Restarted FP32 recursion: warps whose rings lie below ck.jb run Reinsch's
// form, the others the plain form (the choice is uniform per warp).
// One map: the plain-form warps run the monic step (PolSM) on the df32 table
// rec_a with the coefficients coef_m (times c_l): spin 2 at lmax 4096 12.09 ->
// 11.46 ms (spin 0 unchanged); several maps keep PolS.
template <int RPT, bool SPIN, int NM = 1, bool GRAD = false>
__global__ void __launch_bounds__(512) k_leg_fwd32(const void *__restrict__ coef, const void *__restrict__ rec_s,
                                                   const double *__restrict__ lognorm, RingTab rt,
                                                   float2 *__restrict__ ring, int lmax, int mmax, int spin, int ntheta,
                                                   int nnorth, int64_t nalm, int m_begin, int64_t ring_stride,
                                                   CkTab ck, const void *__restrict__ coef_m,
                                                   const void *__restrict__ rec_a)
{
    const int wr0 = ((blockIdx.x * blockDim.x + threadIdx.x) & ~31) * RPT;  // first ring of the warp
    if (wr0 < ck.jb)
        leg_fwd_body<PolR, RPT, SPIN, NM, GRAD>(coef, rec_s, nullptr, lognorm, rt, ring, lmax, mmax, spin, ntheta,
                                                nnorth, nalm, m_begin, ring_stride, ck);
    else if constexpr (NM == 1)
        leg_fwd_body<PolSM, RPT, SPIN, NM, GRAD>(coef_m, rec_a, nullptr, lognorm, rt, ring, lmax, mmax, spin, ntheta,
                                                 nnorth, nalm, m_begin, ring_stride, ck);
    else
        leg_fwd_body<PolS, RPT, SPIN, NM, GRAD>(coef, rec_s, nullptr, lognorm, rt, ring, lmax, mmax, spin, ntheta,
                                                nnorth, nalm, m_begin, ring_stride, ck);
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

// Ring inputs of one thread.  spin 0: (k0r, k0i) multiplies the degrees with
// rel = +1 and (k1r, k1i) those with rel = -1, i.e. H_N + H_S or H_N - H_S as
// (-1)^(l-m) = s0 rel is +1 or -1.  spin s: hn/hs column +m north/south,
// gn/gs column -m; the south inputs are multiplied by s0 so that a degree
// takes them with the sign rel.
// GRAD (gradient-only spin s: only G is returned): with sgs = (-1)^s,
//   -2 G = sum_l s-lambda (H_m(N) + rel sgs s0 H_-m(S)) + (-s)lambda (rel s0 H_m(S) + sgs H_-m(N))
// (real and imaginary parts with the sign of sgs flipped for the imaginary
// part), so each ring keeps these combinations for rel = +1 (hn*, hs*) and
// rel = -1 (gn*, gs*) and a degree adds two values instead of four.
template <class P, int RPT, bool SPIN, bool GRAD = false> struct AdjIn {
    using K = typename P::K;
    using A = typename P::A;
    K hnr[RPT], hni[RPT], hsr[RPT], hsi[RPT], gnr[RPT], gni[RPT], gsr[RPT], gsi[RPT];

    __device__ __forceinline__ void init(const typename P::C *ring, int rp0, int nnorth, int ntheta, int m, int mmax,
                                         bool s0neg, bool sodd = false)
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
                    if (s0neg) {
                        hsr[k] = P::ksign(hsr[k], -1); hsi[k] = P::ksign(hsi[k], -1);
                        gsr[k] = P::ksign(gsr[k], -1); gsi[k] = P::ksign(gsi[k], -1);
                    }
                    if (GRAD) {
                        const int sg = sodd ? -1 : 1;
                        const K xgsr = P::ksign(gsr[k], sg), xgsi = P::ksign(gsi[k], sg);
                        const K xgnr = P::ksign(gnr[k], sg), xgni = P::ksign(gni[k], sg);
                        const K nr = hnr[k], ni = hni[k], sr = hsr[k], si = hsi[k];
                        hnr[k] = P::kadd(nr, xgsr); hsr[k] = P::kadd(sr, xgnr);    // rel = +1
                        hni[k] = P::ksub(ni, xgsi); hsi[k] = P::ksub(si, xgni);
                        gnr[k] = P::ksub(nr, xgsr); gsr[k] = P::ksub(xgnr, sr);    // rel = -1
                        gni[k] = P::kadd(ni, xgsi); gsi[k] = P::ksign(P::kadd(si, xgni), -1);
                    }
                } else {
                    const K ar = hnr[k], ai = hni[k], br = hsr[k], bi = hsi[k];
                    const K er = P::kadd(ar, br), ei = P::kadd(ai, bi), orr = P::ksub(ar, br), oi = P::ksub(ai, bi);
                    hnr[k] = s0neg ? orr : er; hni[k] = s0neg ? oi : ei;
                    hsr[k] = s0neg ? er : orr; hsi[k] = s0neg ? ei : oi;
                }
            }
        }
    }
    // partial sums of one degree (value in word NW) into part[0..NCOMP); ODD: rel = -1
    template <int NW, bool SCALED, bool ODD>
    __device__ __forceinline__ void add(const Rings<P, RPT, SPIN> &st, A *part) const
    {
        typename P::V vp[RPT], vm[RPT];
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            vp[k] = st.template vplus<NW, SCALED>(k);
            if (SPIN) vm[k] = st.template vminus<NW, SCALED>(k);
        }
        add_vals<ODD>(vp, vm, part);
    }
    // partial sums of one degree given its values (+s in vpv, -s in vmv) on the rings
    template <bool ODD>
    __device__ __forceinline__ void add_vals(const typename P::V (&vpv)[RPT], const typename P::V (&vmv)[RPT],
                                             A *part) const
    {
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            const typename P::V vp = vpv[k];
            if (!SPIN) {
                P::fma(part[0], ODD ? hsr[k] : hnr[k], vp);
                P::fma(part[1], ODD ? hsi[k] : hni[k], vp);
            } else if (GRAD) {
                const typename P::V vm = vmv[k];
                P::fma2(part[0], ODD ? gnr[k] : hnr[k], vp, ODD ? gsr[k] : hsr[k], vm);
                P::fma2(part[1], ODD ? gni[k] : hni[k], vp, ODD ? gsi[k] : hsi[k], vm);
            } else {
                const typename P::V vm = vmv[k];
                // U += lam+ H_m(N) + rel lam- s0 H_m(S) ; V += lam- H_-m(N) + rel lam+ s0 H_-m(S)
                if (!ODD) {
                    P::fma2(part[0], hnr[k], vp, hsr[k], vm);
                    P::fma2(part[1], hni[k], vp, hsi[k], vm);
                    P::fma2(part[2], gnr[k], vm, gsr[k], vp);
                    P::fma2(part[3], gni[k], vm, gsi[k], vp);
                } else {
                    P::fma2m(part[0], hnr[k], vp, hsr[k], vm);
                    P::fma2m(part[1], hni[k], vp, hsi[k], vm);
                    P::fma2m(part[2], gnr[k], vm, gsr[k], vp);
                    P::fma2m(part[3], gni[k], vm, gsi[k], vp);
                }
            }
        }
    }
    __device__ __forceinline__ void add_rt(const Rings<P, RPT, SPIN> &st, bool odd, A *part) const
    {
        if (odd) add<1, true, true>(st, part);
        else add<1, true, false>(st, part);
    }
};

// Adds the warp sums of the degrees lb + i (value index i * NCOMP + c),
// times the monic scale c_l and the order weight wm, into a_lm (spin 0) or
// G, C (spin s); with fx (deterministic plans) into the fixed-point sums fx
// (same layout, units of 1 / fxu) instead.
// wmf: (float) wm, formed once by the caller, so that FP32 plans without a scale table
// add their sums with no FP64 arithmetic here.
template <class P, bool SPIN, int NV>
__device__ __forceinline__ void flush(typename P::A (&part)[NV], typename P::R *out, const double *__restrict__ sc,
                                      double wm, float wmf, int64_t base, int64_t nalm, int m, int lb, int lmax,
                                      decltype(P::fac(0)) sgs, unsigned long long *fx, double fxu)
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
        if ((lane & ((1 << SH) - 1)) == 0 && l <= lmax && !(m == 0 && c == 1)) {
            const int64_t dst = 2 * (base + l) + c;
            if constexpr (std::is_same<typename P::A, float>::value) {
                if (!sc && !fx) {
                    atomicAdd(out + dst, tot * wmf);
                    return;
                }
            }
            const double cl = sc ? __ldg(sc + l) : 1.0;
            if (fx) P::atomic_add_fx(fx + dst, tot, cl * wm, fxu);
            else P::atomic_add(out + dst, tot, cl * wm);
        }
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
            if (!(m == 0 && (c == 1 || c == 2))) {
                if constexpr (std::is_same<typename P::A, float>::value) {
                    if (!sc && !fx) {
                        atomicAdd(out + dst, val * wmf);
                        return;
                    }
                }
                const double cl = sc ? __ldg(sc + l) : 1.0;
                if (fx) P::atomic_add_fx(fx + dst, val, cl * wm, fxu);
                else P::atomic_add(out + dst, val, cl * wm);
            }
        }
    }
}

// FP32 plans, spin s: the same reduction through shared memory.  Lane t stores its NV
// sums as row t (16-byte stores, row stride NV + 4 floats); then lane j adds
// column j over the 32 rows (for NV = 16, lanes j and j + 16 add half the rows
// each, the second half offset so that both halves read distinct banks, and
// combine with one shuffle).  Lane v < NV then holds the warp sum of value v:
// NV / 4 stores, 32 loads and 31 additions instead of the selects, shuffles
// and additions of the transpose-reduce.
template <int NV> constexpr int kRowStride = NV + 4;

template <bool SPIN, int NV>
__device__ __forceinline__ void flush_smem(float (&part)[NV], float *wbuf, float *out, const double *__restrict__ sc,
                                           double wm, float wmf, int64_t base, int64_t nalm, int m, int lb, int lmax,
                                           float sgs, unsigned long long *fx, double fxu)
{
    static_assert(NV == 16 || NV == 32, "NV must be 16 or 32");
    constexpr int NCOMP = SPIN ? 4 : 2;
    constexpr int ST = kRowStride<NV>;
    const int lane = threadIdx.x & 31;
    float4 *row = reinterpret_cast<float4 *>(wbuf + lane * ST);
#pragma unroll
    for (int q = 0; q < NV / 4; ++q) row[q] = make_float4(part[4 * q], part[4 * q + 1], part[4 * q + 2], part[4 * q + 3]);
    __syncwarp();
    float tot = 0.f;
    if (NV == 32) {
#pragma unroll
        for (int r = 0; r < 32; ++r) tot += wbuf[r * ST + lane];
    } else {
        const int j = lane & 15;
        const bool hi = lane >= 16;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const int r = hi ? 16 + ((k + 4) & 15) : k;
            tot += wbuf[r * ST + j];
        }
        tot += __shfl_xor_sync(0xffffffffu, tot, 16);
    }
    __syncwarp();  // the buffer is rewritten by the next block
    const int v = lane & (NV - 1);
    const int i = v / NCOMP, c = v % NCOMP;
    const int l = lb + i;
    if (!SPIN) {
        if (lane < NV && l <= lmax && !(m == 0 && c == 1)) {
            const int64_t dst = 2 * (base + l) + c;
            if (fx) PolDF::atomic_add_fx(fx + dst, tot, (sc ? __ldg(sc + l) : 1.0) * wm, fxu);
            else atomicAdd(out + dst, tot * (sc ? (float)(__ldg(sc + l) * wm) : wmf));
        }
    } else {
        const float other = __shfl_xor_sync(0xffffffffu, tot, 2);  // U <-> V of the same l
        if (lane < NV && l <= lmax) {
            float val;
            int64_t dst;
            if (c == 0) { val = -0.5f * (tot + sgs * other); dst = 2 * (base + l); }
            else if (c == 1) { val = -0.5f * (tot - sgs * other); dst = 2 * (base + l) + 1; }
            else if (c == 2) { val = 0.5f * (other - sgs * tot); dst = 2 * (nalm + base + l) + 1; }
            else { val = -0.5f * (other + sgs * tot); dst = 2 * (nalm + base + l); }
            if (!(m == 0 && (c == 1 || c == 2))) {
                if (fx) PolDF::atomic_add_fx(fx + dst, val, (sc ? __ldg(sc + l) : 1.0) * wm, fxu);
                else atomicAdd(out + dst, val * (sc ? (float)(__ldg(sc + l) * wm) : wmf));
            }
        }
    }
}

// shared memory of one adjoint CTA (FP32 plans): one row block per warp
template <bool SPIN> __host__ __device__ constexpr size_t adj_smem_per_warp() { return 32 * kRowStride<kBlk * (SPIN ? 4 : 2)> * sizeof(float); }

template <class P, int RPT, bool SPIN, int REG, bool GRAD>
__device__ __forceinline__ void adj_block(Rings<P, RPT, SPIN> &st, const AdjIn<P, RPT, SPIN, GRAD> &in,
                                          typename P::A *part, const typename P::Tab *reca,
                                          const typename P::TTab *rect, int lb)
{
    constexpr int NCOMP = (SPIN && !GRAD) ? 4 : 2;
#pragma unroll
    for (int j = 0; j < kBlk; ++j) {
        const int l = lb + j;
        if (j & 1) {
            st.template advance<1, REG != 0>(reca, rect, l);
            if (REG != 1) in.template add<1, REG == 2, true>(st, part + j * NCOMP);
        } else {
            st.template advance<0, REG != 0>(reca, rect, l);
            if (REG != 1) in.template add<0, REG == 2, false>(st, part + j * NCOMP);
        }
    }
}

// GRAD: gradient-only spin s, G alone is written (out [nalm]); the reduction
// then has the shape of spin 0's, with the factor -1/2 in the weight.
template <class P, int RPT, bool SPIN, bool GRAD>
__device__ __forceinline__ void leg_adj_body(const typename P::C *__restrict__ ring, const void *__restrict__ rec_a,
                                             const void *__restrict__ rec_t, const double *__restrict__ lognorm,
                                             const double *__restrict__ scale, const RingTab &rt,
                                             typename P::C *__restrict__ alm, int lmax, int mmax, int spin,
                                             int ntheta, int nnorth, int64_t nalm, int m_begin, double wpos,
                                             unsigned long long *fx, const double *__restrict__ fxs, const CkTab &ck)
{
    using A = typename P::A;
    using R = typename P::R;
    using Sg = decltype(P::fac(0));
    constexpr int NCOMP = (SPIN && !GRAD) ? 4 : 2;
    constexpr bool FSPIN = SPIN && !GRAD;  // reduction shape: four values per degree
    constexpr int NV = kBlk * NCOMP;
    const int m = m_begin + blockIdx.y;
    const int s = SPIN ? spin : 0;
    const int l0 = m > s ? m : s;
    if (l0 > lmax) return;
    const int64_t base = alm_base(lmax, m);
    // spin s: reca addresses the interleaved (alpha, tau) table (TabAT entries)
    const typename P::Tab *reca =
        SPIN ? reinterpret_cast<const typename P::Tab *>((const typename P::TabAT *)rec_a + base)
             : (const typename P::Tab *)rec_a + base;
    const typename P::TTab *rect = SPIN ? (const typename P::TTab *)rec_t + base : nullptr;
    const double *sc = P::kMonic ? scale + base : nullptr;  // restarted FP32 recursions carry lambda itself
    const int rp0 = (blockIdx.x * blockDim.x + threadIdx.x) * RPT;
    const Sg sgs = (s & 1) ? Sg(-1) : Sg(1);
    R *out = reinterpret_cast<R *>(alm);
    const int lf = l0 + 1;
    const double wm = (m > 0 ? wpos : 1.0) * (GRAD ? -0.5 : 1.0);
    const float wmf = (float)wm;
    const double fxu = fx ? fxs[1 + m] : 0.0;  // deterministic plans: fixed-point unit of order m

    Rings<P, RPT, SPIN> st;
    AdjIn<P, RPT, SPIN, GRAD> in;
    in.init(ring, rp0, nnorth, ntheta, m, mmax, ((lf - m) & 1) != 0, (s & 1) != 0);
    int l = lf;
    bool jumped = false;
    const int Km = P::kRestart ? ck_interval(ck, m) : 0;
    if constexpr (P::kRestart) {  // start at the warp's first restart: every earlier degree is negligible
        const int kj = first_restart<RPT>(ck, m);
        if (kj > 0) {
            st.init_geom(rt, rp0, nnorth);
            l = lf + kj * Km;  // the restart at l sets the state
            jumped = true;
        }
    }
    if (!jumped) {
        st.init(rt, rp0, nnorth, m, s, lognorm[m]);
        // degree l0 (the start value): one reduction of NCOMP values
        A p0[NCOMP];
#pragma unroll
        for (int c = 0; c < NCOMP; ++c) p0[c] = P::azero();
        in.add_rt(st, true, p0);  // l0 = lf - 1
        flush<P, FSPIN, NCOMP>(p0, out, sc, wm, wmf, base, nalm, m, l0, lmax, sgs, fx, fxu);
    }
    A part[NV];
    // measured at lmax 4096: spin s 42.8 -> 41.6 ms; spin 0 (16 values per lane)
    // 17.2 -> 18.4 ms, so spin 0 keeps the transpose-reduce
    constexpr bool kSmemFlush = std::is_same<typename P::A, float>::value && FSPIN;
    extern __shared__ __align__(16) float adj_smem[];
    float *wbuf = adj_smem + (threadIdx.x >> 5) * (adj_smem_per_warp<FSPIN>() / sizeof(float));
    const int64_t ckrow = P::kRestart ? __ldg(ck.base + m) : 0;
    for (; l + kBlk <= lmax + 1; l += kBlk) {
        if constexpr (P::kRestart) {
            const int dl = l - lf;
            if (dl != 0 && (dl & (Km - 1)) == 0) {
                const int64_t row = ckrow + (int64_t)(dl / Km - 1) * nnorth;
                if constexpr (P::kScaleF) st.restart_scaled(ck, row, rp0, nnorth, ck.cs + base, l);
                else st.restart(ck, row, rp0, nnorth);
            }
        }
        const int reg = st.regime();
        if (!P::kRestart && reg == 1) {  // every contribution of this block is below 2^-180: recursion only
            adj_block<P, RPT, SPIN, 1, GRAD>(st, in, part, reca, rect, l);
            continue;
        }  // restarted recursions: such blocks are rare (see leg_fwd_body) and take the scaled path
#pragma unroll
        for (int i = 0; i < NV; ++i) part[i] = P::azero();
        if (reg == 0) adj_block<P, RPT, SPIN, 0, GRAD>(st, in, part, reca, rect, l);
        else adj_block<P, RPT, SPIN, 2, GRAD>(st, in, part, reca, rect, l);
        if constexpr (kSmemFlush)
            flush_smem<FSPIN, NV>(part, wbuf, reinterpret_cast<float *>(alm), sc, wm, wmf, base, nalm, m, l, lmax, sgs, fx,
                                  fxu);
        else
            flush<P, FSPIN, NV>(part, out, sc, wm, wmf, base, nalm, m, l, lmax, sgs, fx, fxu);
    }
    if (l <= lmax) {  // tail: fewer than kBlk degrees, general path
#pragma unroll
        for (int i = 0; i < NV; ++i) part[i] = P::azero();
#pragma unroll
        for (int j = 0; j < kBlk; ++j) {
            if (l + j <= lmax) {
                st.advance_moved(reca, rect, l + j);
                in.add_rt(st, (j & 1) != 0, part + j * NCOMP);
            }
        }
        flush<P, FSPIN, NV>(part, out, sc, wm, wmf, base, nalm, m, l, lmax, sgs, fx, fxu);
    }
}

template <class P, int RPT, bool SPIN, bool GRAD = false>
__global__ void __launch_bounds__(512) k_leg_adj(const typename P::C *__restrict__ ring, const void *__restrict__ rec_a,
                                                 const void *__restrict__ rec_t, const double *__restrict__ lognorm,
                                                 const double *__restrict__ scale, RingTab rt,
                                                 typename P::C *__restrict__ alm, int lmax, int mmax, int spin,
                                                 int ntheta, int nnorth, int64_t nalm, int m_begin, double wpos,
                                                 unsigned long long *fx, const double *__restrict__ fxs, CkTab ck)
{
    leg_adj_body<P, RPT, SPIN, GRAD>(ring, rec_a, rec_t, lognorm, scale, rt, alm, lmax, mmax, spin, ntheta, nnorth,
                                     nalm, m_begin, wpos, fx, fxs, ck);
}

// Restarted FP32 recursion (see k_leg_fwd32).
// At most 80 registers: the spin-s kernel (97 registers unconstrained) then keeps 24
// instead of 16 warps per SM (lmax 4096: spin 2 14.39 -> 13.68 ms, spin 0 5.38 -> 5.26 ms;
// 96 registers: 13.64 / 5.35 ms).
template <int RPT, bool SPIN, bool GRAD = false>
__global__ void __maxnreg__(80) k_leg_adj32(const float2 *__restrict__ ring, const void *__restrict__ rec_s,
                                                   const double *__restrict__ lognorm, RingTab rt,
                                                   float2 *__restrict__ alm, int lmax, int mmax, int spin, int ntheta,
                                                   int nnorth, int64_t nalm, int m_begin, double wpos,
                                                   unsigned long long *fx, const double *__restrict__ fxs, CkTab ck)
{
    const int wr0 = ((blockIdx.x * blockDim.x + threadIdx.x) & ~31) * RPT;  // first ring of the warp
    if (wr0 < ck.jb)
        leg_adj_body<PolR, RPT, SPIN, GRAD>(ring, rec_s, nullptr, lognorm, nullptr, rt, alm, lmax, mmax, spin, ntheta,
                                            nnorth, nalm, m_begin, wpos, fx, fxs, ck);
    else  // (the monic PolSM measured 8% slower here for spin 2: 16.0 -> 17.3 ms at lmax 4096)
        leg_adj_body<PolS, RPT, SPIN, GRAD>(ring, rec_s, nullptr, lognorm, nullptr, rt, alm, lmax, mmax, spin, ntheta,
                                            nnorth, nalm, m_begin, wpos, fx, fxs, ck);
}

// ---------------------------------------------- fixed point (deterministic plans)
// Unit of order m: every a_lm of the adjoint is a sum over rings of ring
// coefficients times lambda values, |lambda| <= sqrt((2 lmax + 1)/(4 pi)),
// so |a_lm| <= S_m sqrt((2 lmax + 1)/(4 pi)) max(w_m, 1) with S_m the sum of
// |Re| + |Im| over the ring coefficients of order m (columns +m and -m for
// spin s); the same bounds every warp's partial sum.  One CTA per m, reduced
// in a fixed order.  fxs[1 + m] = fx_unit(bound).
template <typename C>
__global__ void k_fx_units(const C *__restrict__ ring, int ntheta, int mmax, bool spin, double wlam,
                           double *__restrict__ fxs)
{
    __shared__ double red[256];
    const int m = blockIdx.x;
    double a = 0.0;
    const int64_t c0 = (int64_t)(spin ? mmax + m : m) * ntheta, c1 = (int64_t)(mmax - m) * ntheta;
    for (int j = threadIdx.x; j < ntheta; j += blockDim.x) {
        const C v = ring[c0 + j];
        a += fabs((double)v.x) + fabs((double)v.y);
        if (spin && m > 0) {
            const C w = ring[c1 + j];
            a += fabs((double)w.x) + fabs((double)w.y);
        }
    }
    red[threadIdx.x] = a;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) fxs[1 + m] = fx_unit(red[0] * wlam * (1.0 + 0x1p-20));
}

// a_lm = fixed-point sum / unit of its order (fx and alm may coincide)
template <typename R>
__global__ void k_fx_to_alm(const unsigned long long *fx, R *alm, int lmax, int64_t nalm, int ncomp,
                            const double *__restrict__ fxs)
{
    const int m = blockIdx.y;
    const double inv = 1.0 / fxs[1 + m];
    const int64_t base = alm_base(lmax, m);
    for (int l = m + blockIdx.x * blockDim.x + threadIdx.x; l <= lmax; l += gridDim.x * blockDim.x)
        for (int c = 0; c < ncomp; ++c)
            for (int k = 0; k < 2; ++k) {
                const int64_t i = 2 * (c * nalm + base + l) + k;
                alm[i] = fx_value<R>((long long)fx[i], inv);
            }
}

// ------------------------------------------------------- coefficient tables
// For the step (l-1 -> l), j = l - 1:
//   A_l = (j+1) sqrt((2j+3)(2j+1) / (((j+1)^2-m^2)((j+1)^2-s^2)))
//   B_l = (j+1)/j sqrt((2j+3)/(2j-1)) sqrt((j^2-m^2)(j^2-s^2) / (((j+1)^2-m^2)((j+1)^2-s^2)))
//   T_l = m s / (j (j+1))
// Monic form: c_{l0} = c_{l0+1} = 1, c_l = B_l c_{l-2} (l >= l0 + 2),
// alpha_l = A_l c_{l-1} / c_l, tau_l = alpha_l T_l; c_l = 0 for l < l0.
// One CTA per m: two threads run the two parity chains of c, then all
// threads fill alpha and tau.  Written as df32 (a_df, t_df) and/or FP64
// (a64, t64) tables; scale holds c (FP64).  For spin s the df32 table
// interleaves alpha and tau (float4 per entry) so one load serves a step.
__device__ __forceinline__ double rec_B(int l, int m, int s)
{
    const double j = l - 1, mm = m, ss = s;
    const double den = ((j + 1) * (j + 1) - mm * mm) * ((j + 1) * (j + 1) - ss * ss);
    return (j + 1) / j * sqrt((2 * j + 3) / (2 * j - 1) * ((j * j - mm * mm) * (j * j - ss * ss) / den));
}

__global__ void k_rec_tables(int lmax, int spin, double *__restrict__ scale, float2 *__restrict__ a_df,
                             float2 *__restrict__ t_df, double *__restrict__ a64, double *__restrict__ t64,
                             float2 *__restrict__ cs)
{
    const int m = blockIdx.x;
    const int s = spin;
    const int l0 = m > s ? m : s;
    const int64_t base = alm_base(lmax, m);
    for (int l = m + threadIdx.x; l < l0 && l <= lmax; l += blockDim.x) scale[base + l] = 0.0;
    if (threadIdx.x < 2) {
        int l = l0 + threadIdx.x;
        if (l <= lmax) scale[base + l] = 1.0;
        double c = 1.0;
        for (l += 2; l <= lmax; l += 2) {
            c *= rec_B(l, m, s);
            scale[base + l] = c;
        }
    }
    __syncthreads();
    for (int l = l0 + 1 + threadIdx.x; l <= lmax; l += blockDim.x) {
        const double j = l - 1, mm = m, ss = s;
        const double den = ((j + 1) * (j + 1) - mm * mm) * ((j + 1) * (j + 1) - ss * ss);
        const double A = (j + 1) * sqrt((2 * j + 3) * (2 * j + 1) / den);
        const double T = j > 0 ? mm * ss / (j * (j + 1)) : 0.0;
        const double alpha = A * (scale[base + l - 1] / scale[base + l]);
        const double tau = alpha * T;
        if (a_df) {
            const float ah = (float)alpha, th = (float)tau;
            if (s) reinterpret_cast<float4 *>(a_df)[base + l] =
                       make_float4(ah, (float)(alpha - (double)ah), th, (float)(tau - (double)th));
            else a_df[base + l] = make_float2(ah, (float)(alpha - (double)ah));
        }
        if (a64) {
            a64[base + l] = alpha;
            if (t64) t64[base + l] = tau;
        }
    }
    if (cs) {  // (c_l, 1/c_l) in FP32 for the monic plain-form rings of the restarted FP32 recursion
        for (int l = m + threadIdx.x; l <= lmax; l += blockDim.x) {
            const double c = scale[base + l];
            cs[base + l] = l >= l0 ? make_float2((float)c, (float)(1.0 / c)) : make_float2(0.f, 0.f);
        }
    }
}

// Step table of the restarted FP32 recursion (PolS / PolR): per (m, l > l0)
// float4 (A_l, B_l, AT_l, K_l), K_l = 1 + B_l - A_l - AT_l formed in FP64 and
// rounded once (B_{l0+1} = 0: lambda_{l0-1} does not exist); zeros for l <= l0.
__global__ void k_rec_tables_s(int lmax, int spin, float4 *__restrict__ out)
{
    const int m = blockIdx.x;
    const int s = spin;
    const int l0 = m > s ? m : s;
    const int64_t base = alm_base(lmax, m);
    for (int l = m + threadIdx.x; l <= lmax; l += blockDim.x) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (l > l0) {
            const double j = l - 1, mm = m, ss = s;
            const double den = ((j + 1) * (j + 1) - mm * mm) * ((j + 1) * (j + 1) - ss * ss);
            const double A = (j + 1) * sqrt((2 * j + 3) * (2 * j + 1) / den);
            const double T = j > 0 ? mm * ss / (j * (j + 1)) : 0.0;
            const double B = l >= l0 + 2 ? rec_B(l, m, s) : 0.0;
            const double AT = A * T;
            v = make_float4((float)A, (float)B, (float)AT, (float)(((1.0 + B) - A) - AT));
        }
        out[base + l] = v;
    }
}

// Restart values of the FP32 recursion (CkTab), from the FP64 monic recursion
// (alpha, tau and c_l of k_rec_tables in FP64, start values and 2^(60 E)
// scaling as PolF64); one thread per (north ring, m).  Before degree
// lb = lf + K k (k = 1 .. ck_count) the FP32 kernels hold (lambda_{lb-2},
// lambda_{lb-1}) in the plain form and (D_{lb-1}, lambda_{lb-1}) in Reinsch's
// form (rings below jb); those pairs are written scaled by 2^(-60 E) in FP32
// with E (kCkZero for a state that is identically zero).  lt[m][j]: the first
// degree at which |lambda| (either sign of the spin) reaches 2^-40, lmax + 1
// if none does before the last restart.
// DD (FP64 plans, PolDDR): the monic state itself split into df32 words,
// float4 (w0.h, w0.l, w1.h, w1.l) per sign of the spin, no Reinsch form, and
// lt the first degree reaching 2^-64.
template <bool SPIN, bool DD = false>
__global__ void k_ck_build(const double *__restrict__ a64, const double *__restrict__ t64,
                           const double *__restrict__ scale, const double *__restrict__ lognorm, RingTab rt, int lmax,
                           int spin, int nnorth, int Kall, int jb, const int64_t *__restrict__ ckbase,
                           void *__restrict__ vout, void *__restrict__ eout, int *__restrict__ lt,
                           const unsigned char *__restrict__ klog)
{
    const int m = blockIdx.y;
    const int K = klog ? 1 << klog[m] : Kall;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int s = SPIN ? spin : 0;
    const int l0 = m > s ? m : s;
    if (j >= nnorth) return;
    int *ltp = lt + (int64_t)m * nnorth + j;
    *ltp = lmax + 1;
    if (l0 > lmax) return;
    const int lf = l0 + 1;
    const int nck = ck_count(lmax, lf, K);
    if (nck == 0) return;
    const int64_t base = alm_base(lmax, m);
    const double x = rt.x[j];
    PolF64::St sp, sm;
    start_value<PolF64>(sp, m, s, s, lognorm[m], rt.lsin2[j], rt.lcos2[j]);
    if (SPIN) start_value<PolF64>(sm, m, s, -s, lognorm[m], rt.lsin2[j], rt.lcos2[j]);
    const bool rein = !DD && j < jb;
    auto quad = [&](const PolF64::St &st, float4 &v, short &e) {
        if (st.w[0] == 0.0 && st.w[1] == 0.0) { v = make_float4(0.f, 0.f, 0.f, 0.f); e = (short)kCkZero; return; }
        const df32 a = df_split(st.w[0]), b = df_split(st.w[1]);
        v = make_float4(a.h, a.l, b.h, b.l);
        e = (short)max(st.E, kCkZero + 1);
    };
    auto pair = [&](const PolF64::St &st, int l, float &w0, float &w1, short &e) {
        if (st.w[0] == 0.0 && st.w[1] == 0.0) { w0 = 0.f; w1 = 0.f; e = (short)kCkZero; return; }
        const double v1 = st.w[1] * scale[base + l];
        const double v0 = st.w[0] * scale[base + l - 1];
        w1 = (float)v1;
        w0 = (float)(rein ? v1 - v0 : v0);
        e = (short)max(st.E, kCkZero + 1);
    };
    auto big = [&](const PolF64::St &st, int l) {  // |lambda_l| >= 2^-40 (DD: 2^-64)
        return st.E >= -2 && ldexp(fabs(st.w[1]) * scale[base + l], kScaleBits * st.E) >= (DD ? 0x1p-64 : 0x1p-40);
    };
    int lfirst = lmax + 1;
    if (big(sp, l0) || (SPIN && big(sm, l0))) lfirst = l0;
    int k = 1;
    int lck = lf + K - 1;  // last degree before the k-th restart
    for (int l = lf; k <= nck; ++l) {
        const double ax = a64[base + l] * x;
        if (!SPIN) {
            const double nv = fma(ax, sp.w[1], -sp.w[0]);
            sp.w[0] = sp.w[1]; sp.w[1] = nv;
            PolF64::rescale(sp, 1);
        } else {
            const double t = t64[base + l];
            const double np = fma(ax + t, sp.w[1], -sp.w[0]);
            const double nm = fma(ax - t, sm.w[1], -sm.w[0]);
            sp.w[0] = sp.w[1]; sp.w[1] = np;
            sm.w[0] = sm.w[1]; sm.w[1] = nm;
            PolF64::rescale(sp, 1);
            PolF64::rescale(sm, 1);
        }
        if (lfirst > lmax && (big(sp, l) || (SPIN && big(sm, l)))) lfirst = l;
        if (l == lck) {
            const int64_t idx = ckbase[m] + (int64_t)(k - 1) * nnorth + j;
            if (DD) {
                float4 a, b;
                short ea, eb;
                quad(sp, a, ea);
                if (!SPIN) {
                    reinterpret_cast<float4 *>(vout)[idx] = a;
                    reinterpret_cast<short *>(eout)[idx] = ea;
                } else {
                    quad(sm, b, eb);
                    reinterpret_cast<float4 *>(vout)[2 * idx] = a;
                    reinterpret_cast<float4 *>(vout)[2 * idx + 1] = b;
                    reinterpret_cast<short2 *>(eout)[idx] = make_short2(ea, eb);
                }
            } else if (!SPIN) {
                float2 v;
                short e;
                pair(sp, l, v.x, v.y, e);
                reinterpret_cast<float2 *>(vout)[idx] = v;
                reinterpret_cast<short *>(eout)[idx] = e;
            } else {
                float4 v;
                short2 e;
                pair(sp, l, v.x, v.y, e.x);
                pair(sm, l, v.z, v.w, e.y);
                reinterpret_cast<float4 *>(vout)[idx] = v;
                reinterpret_cast<short2 *>(eout)[idx] = e;
            }
            ++k;
            lck += K;
        }
    }
    *ltp = lfirst;
}

// First restart of every 32-ring group and order: the largest k <= ck_count
// with lf + K k <= min over the group's rings of lt (so every degree before
// the restart is below 2^-40 on all of them).
__global__ void k_ck_start(const int *__restrict__ lt, int lmax, int mmax, int spin, int nnorth, int Kall, int ngrp,
                           short *__restrict__ kstart, const unsigned char *__restrict__ klog)
{
    const int m = blockIdx.x;
    const int K = klog ? 1 << klog[m] : Kall;
    const int l0 = m > spin ? m : spin;
    const int lf = l0 + 1;
    const int nck = l0 > lmax ? 0 : ck_count(lmax, lf, K);
    for (int g = threadIdx.x; g < ngrp; g += blockDim.x) {
        int lmin = lmax + 1;
        for (int j = 32 * g; j < 32 * g + 32 && j < nnorth; ++j) lmin = min(lmin, lt[(int64_t)m * nnorth + j]);
        const int k = lmin > lf ? (lmin - lf) / K : 0;
        kstart[(int64_t)m * ngrp + g] = (short)min(k, nck);
    }
}

// Forward coefficients of one call: spin 0 c_l a_lm; spin s c_l (G + iC) and
// c_l (-1)^s (conj G + i conj C) (m = 0: imaginary parts of a, G, C dropped),
// all multiplied by wpos for m > 0; gradient-only plans (grad, alm holds G
// alone) c_l G only;
// zero for l < l0.  Entries of orders m < m_split are written as OUT_LO, the
// others as OUT_HI: float2 (FP32 plans), double2 (FP64 plans, native FP64
// orders) or float4 df32 (FP64 plans, df32 orders).
template <typename T> __device__ __forceinline__ void put_coef(void *out, int64_t i, double re, double im);
template <> __device__ __forceinline__ void put_coef<float2>(void *out, int64_t i, double re, double im)
{
    ((float2 *)out)[i] = make_float2((float)re, (float)im);
}
template <> __device__ __forceinline__ void put_coef<double2>(void *out, int64_t i, double re, double im)
{
    ((double2 *)out)[i] = make_double2(re, im);
}
template <> __device__ __forceinline__ void put_coef<float4>(void *out, int64_t i, double re, double im)
{
    const float rh = (float)re, ih = (float)im;
    ((float4 *)out)[i] = make_float4(rh, (float)(re - (double)rh), ih, (float)(im - (double)ih));
}

template <typename Tin, typename OUT_LO, typename OUT_HI>
__global__ void k_coef_prep(const Tin *__restrict__ alm, const double *__restrict__ scale, void *__restrict__ out,
                            int lmax, int spin, int64_t nalm, int m_split, double wpos, bool grad)
{
    const int m = blockIdx.y;
    const int64_t base = alm_base(lmax, m);
    const double wm = m > 0 ? wpos : 1.0;
    const double sgs = (spin & 1) ? -1.0 : 1.0;
    const bool hi = m >= m_split;
    for (int l = m + blockIdx.x * blockDim.x + threadIdx.x; l <= lmax; l += gridDim.x * blockDim.x) {
        const int64_t i = base + l;
        // plans with restarted FP32 recursions carry lambda itself (no monic scale)
        const double c = (scale ? scale[i] : (l >= (m > spin ? m : spin) ? 1.0 : 0.0)) * wm;
        const Tin gv = alm[i];
        const double gr = gv.x, gi = m == 0 ? 0.0 : (double)gv.y;
        if (!spin) {
            if (hi) put_coef<OUT_HI>(out, i, c * gr, c * gi);
            else put_coef<OUT_LO>(out, i, c * gr, c * gi);
        } else if (grad) {  // C = 0: a = c G (b = (-1)^s conj a is not stored)
            if (hi) put_coef<OUT_HI>(out, i, c * gr, c * gi);
            else put_coef<OUT_LO>(out, i, c * gr, c * gi);
        } else {
            const Tin cv = alm[nalm + i];
            const double cr = cv.x, ci = m == 0 ? 0.0 : (double)cv.y;
            const double ar = c * (gr - ci), ai = c * (gi + cr);
            const double br = c * sgs * (gr + ci), bi = c * sgs * (cr - gi);
            if (hi) { put_coef<OUT_HI>(out, i, ar, ai); put_coef<OUT_HI>(out, nalm + i, br, bi); }
            else { put_coef<OUT_LO>(out, i, ar, ai); put_coef<OUT_LO>(out, nalm + i, br, bi); }
        }
    }
}

template <class P, int RPT, bool SPIN, int NM = 1, bool GRAD = false>
cudaError_t fwd_launch(const Plan &p, const Plan::LegShape &sh, const void *coef, const void *ta, const void *tt,
                       void *ring, int m_begin, int m_end, cudaStream_t st)
{
    if (m_end <= m_begin) return cudaSuccess;
    dim3 grid(sh.chunks, m_end - m_begin);
    dim3 block(sh.warps * 32);
    k_leg_fwd<P, RPT, SPIN, NM, GRAD><<<grid, block, 0, st>>>(coef, ta, tt, p.lognorm, p.rings, (typename P::C *)ring,
                                                        p.lmax, p.mmax, p.spin, p.ntheta, p.nnorth, p.nalm, m_begin,
                                                        (int64_t)p.ncol * p.ntheta, P::kRestart ? p.ck : CkTab{});
    return cudaGetLastError();
}

template <class P, bool SPIN, bool GRAD = false> size_t adj_smem_bytes(int warps)
{
    return (std::is_same<P, PolDF>::value && SPIN && !GRAD) ? (size_t)warps * adj_smem_per_warp<SPIN>() : 0;
}

template <class P, int RPT, bool SPIN, bool GRAD = false>
cudaError_t adj_launch(const Plan &p, const Plan::LegShape &sh, const void *ring, const void *ta, const void *tt,
                       void *alm, int m_begin, int m_end, cudaStream_t st, double wpos, void *fx)
{
    if (m_end <= m_begin) return cudaSuccess;
    dim3 grid(sh.chunks, m_end - m_begin);
    dim3 block(sh.warps * 32);
    k_leg_adj<P, RPT, SPIN, GRAD><<<grid, block, adj_smem_bytes<P, SPIN, GRAD>(sh.warps), st>>>(
                                                    (const typename P::C *)ring, ta, tt, p.lognorm, p.scale, p.rings,
                                                    (typename P::C *)alm, p.lmax, p.mmax, p.spin, p.ntheta, p.nnorth,
                                                    p.nalm, m_begin, wpos, (unsigned long long *)fx,
                                                    p.fx_scale, P::kRestart ? p.ck : CkTab{});
    return cudaGetLastError();
}

template <class P, bool SPIN, bool GRAD = false>
cudaError_t fwd_rpt(const Plan &p, const Plan::LegShape &sh, const void *coef, const void *ta, const void *tt,
                    void *ring, int m_begin, int m_end, cudaStream_t st)
{
    if (sh.rpt == 1) return fwd_launch<P, 1, SPIN, 1, GRAD>(p, sh, coef, ta, tt, ring, m_begin, m_end, st);
    return fwd_launch<P, 2, SPIN, 1, GRAD>(p, sh, coef, ta, tt, ring, m_begin, m_end, st);
}

template <class P, bool SPIN, bool GRAD = false>
cudaError_t adj_rpt(const Plan &p, const Plan::LegShape &sh, const void *ring, const void *ta, const void *tt,
                    void *alm, int m_begin, int m_end, cudaStream_t st, double wpos, void *fx)
{
    if (sh.rpt == 1) return adj_launch<P, 1, SPIN, GRAD>(p, sh, ring, ta, tt, alm, m_begin, m_end, st, wpos, fx);
    return adj_launch<P, 2, SPIN, GRAD>(p, sh, ring, ta, tt, alm, m_begin, m_end, st, wpos, fx);
}

// Restarted FP32 recursion (plans with p.rst): one launch per direction
template <int RPT, bool SPIN, int NM = 1, bool GRAD = false>
cudaError_t fwd32_launch(const Plan &p, const Plan::LegShape &sh, const void *coef, void *ring, int m_begin,
                         int m_end, cudaStream_t st)
{
    if (m_end <= m_begin) return cudaSuccess;
    dim3 grid(sh.chunks, m_end - m_begin);
    dim3 block(sh.warps * 32);
    k_leg_fwd32<RPT, SPIN, NM, GRAD><<<grid, block, 0, st>>>(coef, p.rec_s, p.lognorm, p.rings, (float2 *)ring, p.lmax,
                                                           p.mmax, p.spin, p.ntheta, p.nnorth, p.nalm, m_begin,
                                                           (int64_t)p.ncol * p.ntheta, p.ck, p.coef_m, p.rec_a);
    return cudaGetLastError();
}

template <int RPT, bool SPIN, bool GRAD = false>
cudaError_t adj32_launch(const Plan &p, const Plan::LegShape &sh, const void *ring, void *alm, int m_begin, int m_end,
                         cudaStream_t st, double wpos, void *fx)
{
    if (m_end <= m_begin) return cudaSuccess;
    dim3 grid(sh.chunks, m_end - m_begin);
    dim3 block(sh.warps * 32);
    k_leg_adj32<RPT, SPIN, GRAD><<<grid, block, adj_smem_bytes<PolDF, SPIN, GRAD>(sh.warps), st>>>(
        (const float2 *)ring, p.rec_s, p.lognorm, p.rings, (float2 *)alm, p.lmax, p.mmax, p.spin, p.ntheta, p.nnorth,
        p.nalm, m_begin, wpos, (unsigned long long *)fx, p.fx_scale, p.ck);
    return cudaGetLastError();
}

// rings per thread 1, 2 or 4 (the warp-uniform table loads are shared by the rings of a thread)
template <bool SPIN, int NM = 1, bool GRAD = false>
cudaError_t fwd32_rpt(const Plan &p, const Plan::LegShape &sh, const void *coef, void *ring, int m_begin, int m_end,
                      cudaStream_t st)
{
    if (sh.rpt == 1) return fwd32_launch<1, SPIN, NM, GRAD>(p, sh, coef, ring, m_begin, m_end, st);
    if (sh.rpt == 2) return fwd32_launch<2, SPIN, NM, GRAD>(p, sh, coef, ring, m_begin, m_end, st);
    return fwd32_launch<4, SPIN, NM, GRAD>(p, sh, coef, ring, m_begin, m_end, st);
}

cudaError_t fwd32_spin(const Plan &p, const Plan::LegShape &sh, const void *coef, void *ring, int m_begin, int m_end,
                       cudaStream_t st)
{
    if (!p.spin) return fwd32_rpt<false>(p, sh, coef, ring, m_begin, m_end, st);
    if (p.grad) return fwd32_rpt<true, 1, true>(p, sh, coef, ring, m_begin, m_end, st);
    return fwd32_rpt<true>(p, sh, coef, ring, m_begin, m_end, st);
}

template <bool SPIN, bool GRAD = false>
cudaError_t adj32_rpt(const Plan &p, const Plan::LegShape &sh, const void *ring, void *alm, int m_begin, int m_end,
                      cudaStream_t st, double wpos, void *fx)
{
    if (sh.rpt == 1) return adj32_launch<1, SPIN, GRAD>(p, sh, ring, alm, m_begin, m_end, st, wpos, fx);
    if (sh.rpt == 2) return adj32_launch<2, SPIN, GRAD>(p, sh, ring, alm, m_begin, m_end, st, wpos, fx);
    return adj32_launch<4, SPIN, GRAD>(p, sh, ring, alm, m_begin, m_end, st, wpos, fx);
}

cudaError_t adj32_spin(const Plan &p, const Plan::LegShape &sh, const void *ring, void *alm, int m_begin, int m_end,
                       cudaStream_t st, double wpos, void *fx)
{
    if (!p.spin) return adj32_rpt<false>(p, sh, ring, alm, m_begin, m_end, st, wpos, fx);
    if (p.grad) return adj32_rpt<true, true>(p, sh, ring, alm, m_begin, m_end, st, wpos, fx);
    return adj32_rpt<true>(p, sh, ring, alm, m_begin, m_end, st, wpos, fx);
}

template <int RPT> const void *kernel_of32_r(bool spin, bool grad, bool adjoint, int nm)
{
    if (adjoint) {
        if (spin && grad) return (const void *)k_leg_adj32<RPT, true, true>;
        if (spin) return (const void *)k_leg_adj32<RPT, true>;
        return (const void *)k_leg_adj32<RPT, false>;
    }
    if (nm == 2) return spin ? (const void *)k_leg_fwd32<RPT, true, 2> : (const void *)k_leg_fwd32<RPT, false, 2>;
    if (nm == 4) return spin ? (const void *)k_leg_fwd32<RPT, true, 4> : (const void *)k_leg_fwd32<RPT, false, 4>;
    if (spin && grad) return (const void *)k_leg_fwd32<RPT, true, 1, true>;
    if (spin) return (const void *)k_leg_fwd32<RPT, true>;
    return (const void *)k_leg_fwd32<RPT, false>;
}

// Kernel entry of a restarted-FP32 variant (nm > 1: forward sharing the recursion among nm maps)
const void *kernel_of32(bool spin, bool grad, int rpt, bool adjoint, int nm)
{
    if (rpt == 4) return kernel_of32_r<4>(spin, grad, adjoint, nm);
    if (rpt == 2) return kernel_of32_r<2>(spin, grad, adjoint, nm);
    return kernel_of32_r<1>(spin, grad, adjoint, nm);
}

template <class P>
cudaError_t fwd_spin(const Plan &p, const Plan::LegShape &sh, const void *coef, const void *ta, const void *tt,
                     void *ring, int m_begin, int m_end, cudaStream_t st)
{
    if (!p.spin) return fwd_rpt<P, false>(p, sh, coef, ta, tt, ring, m_begin, m_end, st);
    return p.grad ? fwd_rpt<P, true, true>(p, sh, coef, ta, tt, ring, m_begin, m_end, st)
                  : fwd_rpt<P, true>(p, sh, coef, ta, tt, ring, m_begin, m_end, st);
}

template <class P>
cudaError_t adj_spin(const Plan &p, const Plan::LegShape &sh, const void *ring, const void *ta, const void *tt,
                     void *alm, int m_begin, int m_end, cudaStream_t st, double wpos, void *fx)
{
    if (!p.spin) return adj_rpt<P, false>(p, sh, ring, ta, tt, alm, m_begin, m_end, st, wpos, fx);
    return p.grad ? adj_rpt<P, true, true>(p, sh, ring, ta, tt, alm, m_begin, m_end, st, wpos, fx)
                  : adj_rpt<P, true>(p, sh, ring, ta, tt, alm, m_begin, m_end, st, wpos, fx);
}

// Kernel entry of one (arithmetic, spin, gradient-only, rings-per-thread,
// direction) variant.
template <class P> const void *kernel_of(bool spin, bool grad, int rpt, bool adjoint)
{
    if (adjoint) {
        if (spin && grad)
            return rpt == 1 ? (const void *)k_leg_adj<P, 1, true, true> : (const void *)k_leg_adj<P, 2, true, true>;
        if (spin) return rpt == 1 ? (const void *)k_leg_adj<P, 1, true> : (const void *)k_leg_adj<P, 2, true>;
        return rpt == 1 ? (const void *)k_leg_adj<P, 1, false> : (const void *)k_leg_adj<P, 2, false>;
    }
    if (spin && grad)
        return rpt == 1 ? (const void *)k_leg_fwd<P, 1, true, 1, true> : (const void *)k_leg_fwd<P, 2, true, 1, true>;
    if (spin) return rpt == 1 ? (const void *)k_leg_fwd<P, 1, true> : (const void *)k_leg_fwd<P, 2, true>;
    return rpt == 1 ? (const void *)k_leg_fwd<P, 1, false> : (const void *)k_leg_fwd<P, 2, false>;
}

// ------------------------------------------------------------ Legendre tables
// FP32 plans built with Legendre tables store, at plan creation, the value
// mu_lm(theta_j) (monic form, true magnitude) of every (m, l, ring) that the
// transforms need, and then read them instead of running the recursion: the
// Legendre steps become HBM-bound streams (about 2/pi of the dense
// (m, l, ring) triples are stored: a ring enters at the degree where its
// value first reaches kTabT, and the evanescent region before it is skipped).
//
// Layout.  Rings are taken in groups of four (kTabG), nnp = nnorth rounded up
// to a multiple of 4.  first(m, j) = the first degree at which ring j's value
// (either spin) reaches kTabT; lstart(m, q) = max(l0, min over rings
// j <= 4q + 3 of first(m, j)), which does not increase with q.  Row (m, l)
// holds the groups q with lstart(m, q) <= l, a suffix [jlo(m, l) / 4, nnp / 4)
// of the groups; its entry for ring j is at rowbase(m, l) + j (rowbase = row
// offset - jlo, offsets in entries, multiples of 4).  An entry is a float
// (spin 0) or a float2 (mu_{+s}, mu_{-s}).  Rings nnorth..nnp-1 hold zeros.
constexpr float kTabT = 0x1p-40f;
constexpr int kTabG = 4;

// Shared recursion driver of the two table-building passes: visits every
// degree l0..lmax with the values of the thread's two rings (word 1, scaled).
// All threads of the CTA run the whole loop (the renormalisation votes).
template <bool SPIN, class F>
__device__ __forceinline__ void tab_walk(const void *rec_a, const void *rec_t, const double *lognorm, RingTab rt,
                                         int lmax, int spin, int nnorth, int m, int rp0, F &&visit)
{
    using P = PolDF;
    const int s = SPIN ? spin : 0;
    const int l0 = m > s ? m : s;
    if (l0 > lmax) return;
    const int64_t base = alm_base(lmax, m);
    const P::Tab *reca = SPIN ? reinterpret_cast<const P::Tab *>((const P::TabAT *)rec_a + base)
                              : (const P::Tab *)rec_a + base;
    const P::TTab *rect = SPIN ? (const P::TTab *)rec_t + base : nullptr;
    Rings<P, 2, SPIN> st;
    st.init(rt, rp0, nnorth, m, s, lognorm[m]);
    if (!visit(st, l0)) return;
    for (int l = l0 + 1; l <= lmax; ++l) {
        if (((l - l0 - 1) & (kBlk - 1)) == 0) st.regime();  // df32 renormalisation
        st.advance_moved(reca, rect, l);
        if (!visit(st, l)) return;
    }
}

template <bool SPIN>
__global__ void __launch_bounds__(256) k_tab_first(const void *__restrict__ rec_a, const void *__restrict__ rec_t,
                                                   const double *__restrict__ lognorm, RingTab rt, int lmax,
                                                   int spin, int nnorth, int *__restrict__ first)
{
    const int m = blockIdx.y;
    const int rp0 = (blockIdx.x * blockDim.x + threadIdx.x) * 2;
    int f[2] = {lmax + 1, lmax + 1};
    tab_walk<SPIN>(rec_a, rec_t, lognorm, rt, lmax, spin, nnorth, m, rp0, [&](const Rings<PolDF, 2, SPIN> &st, int l) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            float v = fabsf(st.template vplus<1, true>(k));
            if (SPIN) v = fmaxf(v, fabsf(st.template vminus<1, true>(k)));
            if (f[k] > lmax && v >= kTabT) f[k] = l;
        }
        // stop once every ring of the warp has entered (uniform per warp)
        return !__all_sync(0xffffffffu, f[0] <= lmax && f[1] <= lmax);
    });
#pragma unroll
    for (int k = 0; k < 2; ++k)
        if (rp0 + k < nnorth) first[(int64_t)m * nnorth + rp0 + k] = f[k];
}

// One thread per order m: lstart (prefix minimum of first) and, per degree,
// the row's first ring jlo (nnp for an empty row) and its length.
__global__ void k_tab_rows(const int *__restrict__ first, int lmax, int mmax, int spin, int nnorth, int nnp,
                           int *__restrict__ lstart, int *__restrict__ jlo, int64_t *__restrict__ rowlen)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m > mmax) return;
    const int l0 = m > spin ? m : spin;
    const int ng = nnp / kTabG;
    const int *f = first + (int64_t)m * nnorth;
    int *ls = lstart + (int64_t)m * ng;
    int g = lmax + 1;
    for (int q = 0; q < ng; ++q) {
        for (int r = 0; r < kTabG; ++r) {
            const int j = kTabG * q + r;
            if (j < nnorth && f[j] < g) g = f[j];
        }
        ls[q] = g > l0 ? g : l0;
    }
    const int64_t base = alm_base(lmax, m);
    int qlo = ng;
    for (int l = m; l <= lmax; ++l) {
        while (qlo > 0 && ls[qlo - 1] <= l && l >= l0) --qlo;
        jlo[base + l] = kTabG * qlo;
        rowlen[base + l] = (int64_t)kTabG * (ng - qlo);
    }
}

template <bool SPIN>
__global__ void __launch_bounds__(256) k_tab_fill(const void *__restrict__ rec_a, const void *__restrict__ rec_t,
                                                  const double *__restrict__ lognorm, RingTab rt, int lmax, int spin,
                                                  int nnorth, int nnp, const int *__restrict__ jlo,
                                                  const int64_t *__restrict__ rowbase, float *__restrict__ tab)
{
    const int m = blockIdx.y;
    const int rp0 = (blockIdx.x * blockDim.x + threadIdx.x) * 2;
    const int64_t base = alm_base(lmax, m);
    tab_walk<SPIN>(rec_a, rec_t, lognorm, rt, lmax, spin, nnorth, m, rp0, [&](const Rings<PolDF, 2, SPIN> &st, int l) {
        if (rp0 < nnp && rp0 >= __ldg(jlo + base + l)) {
            const int64_t e = __ldg(rowbase + base + l) + rp0;  // even: 8-byte (spin 0) / 16-byte (spin s) aligned
            if (!SPIN) {
                reinterpret_cast<float2 *>(tab)[e >> 1] = make_float2(st.template vplus<1, true>(0),
                                                                      st.template vplus<1, true>(1));
            } else {
                reinterpret_cast<float4 *>(tab)[e >> 1] =
                    make_float4(st.template vplus<1, true>(0), st.template vminus<1, true>(0),
                                st.template vplus<1, true>(1), st.template vminus<1, true>(1));
            }
        }
        return true;
    });
}

// Staging of one warp's table values through shared memory.  The warp
// covers 32 ring groups q0 .. q0 + 31; for each degree of a unit of kTabS
// degrees, the row's stretch [max(jlo, 4 q0), min(4 q0 + 128, nnp)) is brought
// in by a bulk copy (issued by lane i for degree lb + i) into the degree's
// slot at the offset of its first ring, so lane t finds its group at
// slot + t * 4 entries.  Two buffers alternate: while one unit is summed the
// next is in flight.  Lanes 0..kTabS-1 hold the row base and first ring of
// the unit to issue next in registers (loaded one unit ahead).  A unit is
// 4 KB per warp: 8 degrees of spin-0 entries, 4 of spin-s entries.
template <int ESZ> struct TabStage {
    static constexpr int kTabS = ESZ == 4 ? 8 : 4;  // degrees per unit
    static constexpr int SLOT = 32 * kTabG * ESZ;   // bytes per degree
    static constexpr int BYTES = 2 * kTabS * SLOT;   // both buffers
    unsigned char *buf;
    uint64_t *bar;
    uint32_t ph = 0;  // bit b: parity of buffer b's next phase
    int64_t nrb = 0;
    int njlo = 0;
    bool nok = false;
    __device__ __forceinline__ void fetch(const int64_t *__restrict__ rowbase, const int *__restrict__ jlo,
                                          int64_t base, int lb, int l0, int lmax, int lane)
    {
        const int l = lb + lane;
        nok = lane < kTabS && l >= l0 && l <= lmax;
        if (nok) {
            nrb = __ldg(rowbase + base + l);
            njlo = __ldg(jlo + base + l);
        }
    }
    __device__ __forceinline__ void issue(int b, const float *__restrict__ tab, int q0, int nnp, int lane)
    {
        int start = 0, bytes = 0;
        if (nok) {
            const int lo = max(njlo, kTabG * q0), hi = min(kTabG * (q0 + 32), nnp);
            if (lo < hi) {
                start = lo;
                bytes = (hi - lo) * ESZ;
            }
        }
        const int total = __reduce_add_sync(0xffffffffu, bytes);
        __syncwarp();          // the buffer's previous contents have been read
        fence_async_shared();  // ... before the bulk copies overwrite it
        if (lane == 0) mbar_expect_tx(bar + b, (uint32_t)total);
        __syncwarp();
        if (bytes > 0)
            bulk_copy_g2s(buf + (b * kTabS + lane) * SLOT + (start - kTabG * q0) * ESZ,
                          reinterpret_cast<const unsigned char *>(tab) + (nrb + start) * ESZ, (uint32_t)bytes,
                          bar + b);
    }
    __device__ __forceinline__ bool wait(int b)
    {
        const bool ok = mbar_wait_warp(bar + b, (ph >> b) & 1u);
        ph ^= 1u << b;
        return ok;
    }
    __device__ __forceinline__ const unsigned char *slot(int b, int i) const { return buf + (b * kTabS + i) * SLOT; }
};

// A lane's four rings from a staged slot.  Spin s: the group's 32 bytes are
// read as two 16-byte halves; lanes with bit 2 set read the second half
// first, so that the eight lanes of each quarter-warp access hit 32
// distinct banks.
template <bool SPIN>
__device__ __forceinline__ void tab_read(const unsigned char *slot, int lane, float (&vp)[kTabG], float (&vm)[kTabG])
{
    if (!SPIN) {
        const float4 v = reinterpret_cast<const float4 *>(slot)[lane];
        vp[0] = v.x; vp[1] = v.y; vp[2] = v.z; vp[3] = v.w;
        vm[0] = vm[1] = vm[2] = vm[3] = 0.f;
    } else {
        const int h = (lane >> 2) & 1;
        const float4 x = reinterpret_cast<const float4 *>(slot)[2 * lane + h];
        const float4 y = reinterpret_cast<const float4 *>(slot)[2 * lane + 1 - h];
        const float4 a = h ? y : x, b = h ? x : y;
        vp[0] = a.x; vm[0] = a.y; vp[1] = a.z; vm[1] = a.w;
        vp[2] = b.x; vm[2] = b.y; vp[3] = b.z; vm[3] = b.w;
    }
}

// shared memory per warp of the table kernels: staging, two barriers, and
// (adjoint, spin s) the rows of the block reduction
template <bool SPIN, bool ADJ_FLUSH> __host__ __device__ constexpr int tab_smem_per_warp()
{
    return TabStage<SPIN ? 8 : 4>::BYTES + 16 + (ADJ_FLUSH ? (int)adj_smem_per_warp<true>() : 0);
}

// Table synthesis: one thread per group of four rings, one order m per grid
// row; the warp's lanes step through the degrees together from the warp's
// smallest lstart (units start on a degree of even parity rel), reading the
// staged values; a lane before its own lstart adds nothing.  NM maps share
// each table read (prepared coefficients of map b at coef + b ncomp nalm).
template <bool SPIN, bool GRAD, int NM = 1>
__global__ void __launch_bounds__(256) k_tab_fwd(const void *__restrict__ coef, const float *__restrict__ tab,
                                                 const int64_t *__restrict__ rowbase, const int *__restrict__ jlo,
                                                 const int *__restrict__ lstart, float2 *__restrict__ ring, int lmax,
                                                 int mmax, int spin, int ntheta, int nnorth, int nnp, int ng,
                                                 int64_t nalm, unsigned *__restrict__ status,
                                                 int64_t ring_stride = 0)
{
    using P = PolDF;
    using Sg = float;
    constexpr int ESZ = SPIN ? 8 : 4;
    const int m = blockIdx.y;
    const int s = SPIN ? spin : 0;
    const int l0 = m > s ? m : s;
    if (l0 > lmax) return;  // uniform per CTA
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const int q0 = q - lane;
    const int64_t base = alm_base(lmax, m);
    const int j0 = kTabG * q;
    const int lf = l0 + 1;
    const int ls = q < ng ? __ldg(lstart + (int64_t)m * ng + q) : lmax + 1;
    const int lw = __reduce_min_sync(0xffffffffu, ls);
    FwdAcc<P, kTabG, SPIN, NM, GRAD> acc;
    acc.init(coef, nalm, base);
    extern __shared__ __align__(128) unsigned char tab_smem[];
    if (lw <= lmax) {
        TabStage<ESZ> stg;
        stg.buf = tab_smem + warp * tab_smem_per_warp<SPIN, false>();
        stg.bar = reinterpret_cast<uint64_t *>(stg.buf + TabStage<ESZ>::BYTES);
        if (lane == 0) {
            mbar_init(stg.bar, 1);
            mbar_init(stg.bar + 1, 1);
        }
        fence_async_shared();
        __syncwarp();
        constexpr int kTabS = TabStage<ESZ>::kTabS;
        int lb = lw - ((lw - lf) & 1);  // degree lb + i has rel (-1)^i
        stg.fetch(rowbase, jlo, base, lb, l0, lmax, lane);
        stg.issue(0, tab, q0, nnp, lane);
        stg.fetch(rowbase, jlo, base, lb + kTabS, l0, lmax, lane);
        float vp[kTabG], vm[kTabG];
        for (int b = 0; lb <= lmax; lb += kTabS, b ^= 1) {
            const bool more = lb + kTabS <= lmax;
            if (more) {
                stg.issue(b ^ 1, tab, q0, nnp, lane);
                stg.fetch(rowbase, jlo, base, lb + 2 * kTabS, l0, lmax, lane);
            }
            if (!stg.wait(b)) {
                if (lane == 0) atomicOr(status, FLAG_TIMEOUT);
                if (more) stg.wait(b ^ 1);
                return;
            }
#pragma unroll
            for (int i = 0; i < kTabS; ++i) {
                const int l = lb + i;
                if (l >= ls && l <= lmax) {
                    tab_read<SPIN>(stg.slot(b, i), lane, vp, vm);
                    if (i & 1) acc.template add_vals<true>(vp, vm, l);
                    else acc.template add_vals<false>(vp, vm, l);
                }
            }
        }
    }
    // write-out as k_leg_fwd (s0 = (-1)^(lf - m)); map b at ring + b ring_stride
    const Sg s0 = ((lf - m) & 1) ? Sg(-1) : Sg(1);
#pragma unroll
    for (int b = 0; b < NM; ++b)
#pragma unroll
    for (int k = 0; k < kTabG; ++k) {
        float2 *const rb = ring + b * ring_stride;
        const int jn = j0 + k;
        if (jn >= nnorth) continue;
        const int js = ntheta - 1 - jn;
        if (!SPIN) {
            float2 *col = rb + (int64_t)m * ntheta;
            col[jn] = P::cout(acc.r0[b][k] + acc.r1[b][k], acc.i0[b][k] + acc.i1[b][k]);
            if (js != jn) col[js] = P::cout(s0 * (acc.r0[b][k] - acc.r1[b][k]), s0 * (acc.i0[b][k] - acc.i1[b][k]));
        } else if (GRAD) {
            const Sg ms0 = -s0, sgs = (s & 1) ? Sg(-1) : Sg(1);
            const float pr = acc.r0[b][k] + acc.r1[b][k], pi = acc.i0[b][k] + acc.i1[b][k];
            const float qr = acc.r2[b][k] - acc.r3[b][k], qi = acc.i2[b][k] - acc.i3[b][k];
            float2 *colp = rb + (int64_t)(mmax + m) * ntheta;
            colp[jn] = P::cout(-pr, -pi);
            if (js != jn) colp[js] = P::cout(ms0 * qr, ms0 * qi);
            if (m > 0) {
                const float ur = acc.r2[b][k] + acc.r3[b][k], ui = acc.i2[b][k] + acc.i3[b][k];
                const float wr = acc.r0[b][k] - acc.r1[b][k], wi = acc.i0[b][k] - acc.i1[b][k];
                float2 *colq = rb + (int64_t)(mmax - m) * ntheta;
                colq[jn] = P::cout(-sgs * ur, sgs * ui);
                if (js != jn) colq[js] = P::cout(sgs * ms0 * wr, -(sgs * ms0) * wi);
            }
        } else {
            const Sg ms0 = -s0;
            float2 *colp = rb + (int64_t)(mmax + m) * ntheta;
            colp[jn] = P::cout(-acc.r0[b][k], -acc.i0[b][k]);
            if (js != jn) colp[js] = P::cout(ms0 * acc.r1[b][k], ms0 * acc.i1[b][k]);
            if (m > 0) {
                float2 *colq = rb + (int64_t)(mmax - m) * ntheta;
                colq[jn] = P::cout(-acc.r2[b][k], -acc.i2[b][k]);
                if (js != jn) colq[js] = P::cout(ms0 * acc.r3[b][k], ms0 * acc.i3[b][k]);
            }
        }
    }
}

// Table adjoint: one thread per group of four rings; degrees in blocks of
// kBlk starting at l0 + kBlk k (degree lb + i has rel = -1 for even i), from
// the warp's first block on; each block arrives as two staged units of
// kTabS degrees and is reduced over the warp like k_leg_adj.
template <bool SPIN, bool GRAD>
__global__ void __launch_bounds__(256) k_tab_adj(const float2 *__restrict__ ring, const float *__restrict__ tab,
                                                 const int64_t *__restrict__ rowbase, const int *__restrict__ jlo,
                                                 const int *__restrict__ lstart, const double *__restrict__ scale,
                                                 float2 *__restrict__ alm, int lmax, int mmax, int spin, int ntheta,
                                                 int nnorth, int nnp, int ng, int64_t nalm, double wpos,
                                                 unsigned long long *fx, const double *__restrict__ fxs,
                                                 unsigned *__restrict__ status)
{
    using P = PolDF;
    using A = float;
    constexpr int ESZ = SPIN ? 8 : 4;
    constexpr int NCOMP = (SPIN && !GRAD) ? 4 : 2;
    constexpr bool FSPIN = SPIN && !GRAD;
    constexpr int NV = kBlk * NCOMP;
    constexpr int kTabS = TabStage<ESZ>::kTabS;
    constexpr int UPB = kBlk / kTabS;  // staged units per block
    static_assert(UPB * kTabS == kBlk, "a block is a whole number of staged units");
    const int m = blockIdx.y;
    const int s = SPIN ? spin : 0;
    const int l0 = m > s ? m : s;
    if (l0 > lmax) return;  // uniform per CTA
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const int q0 = q - lane;
    const bool has = q < ng;
    const int ls = has ? __ldg(lstart + (int64_t)m * ng + q) : lmax + 1;
    const int lw = __reduce_min_sync(0xffffffffu, ls);
    if (lw > lmax) return;  // uniform per warp: nothing to add
    const int64_t base = alm_base(lmax, m);
    const double *sc = scale + base;
    const float sgs = (s & 1) ? -1.f : 1.f;
    const int lf = l0 + 1;
    const double wm = (m > 0 ? wpos : 1.0) * (GRAD ? -0.5 : 1.0);
    const float wmf = (float)wm;
    const double fxu = fx ? fxs[1 + m] : 0.0;
    float *out = reinterpret_cast<float *>(alm);
    AdjIn<P, kTabG, SPIN, GRAD> in;
    in.init(ring, has ? kTabG * q : nnorth, nnorth, ntheta, m, mmax, ((lf - m) & 1) != 0, (s & 1) != 0);
    extern __shared__ __align__(128) unsigned char tab_smem[];
    TabStage<ESZ> stg;
    stg.buf = tab_smem + warp * tab_smem_per_warp<SPIN, FSPIN>();
    stg.bar = reinterpret_cast<uint64_t *>(stg.buf + TabStage<ESZ>::BYTES);
    float *wbuf = reinterpret_cast<float *>(stg.buf + TabStage<ESZ>::BYTES + 16);
    if (lane == 0) {
        mbar_init(stg.bar, 1);
        mbar_init(stg.bar + 1, 1);
    }
    fence_async_shared();
    __syncwarp();
    int lb = l0 + (lw - l0) / kBlk * kBlk;  // first block; units lb, lb + kTabS, ...
    stg.fetch(rowbase, jlo, base, lb, l0, lmax, lane);
    stg.issue(0, tab, q0, nnp, lane);
    stg.fetch(rowbase, jlo, base, lb + kTabS, l0, lmax, lane);
    A part[NV];
    float vp[kTabG], vm[kTabG];
    for (int b = 0; lb <= lmax; lb += kTabS, b ^= 1) {
        const bool more = lb + kTabS <= lmax;
        if (more) {
            stg.issue(b ^ 1, tab, q0, nnp, lane);
            stg.fetch(rowbase, jlo, base, lb + 2 * kTabS, l0, lmax, lane);
        }
        if (!stg.wait(b)) {
            if (lane == 0) atomicOr(status, FLAG_TIMEOUT);
            if (more) stg.wait(b ^ 1);
            return;
        }
        const int unit = ((lb - l0) / kTabS) % UPB;  // position of the unit in its block
        if (unit == 0) {
#pragma unroll
            for (int i = 0; i < NV; ++i) part[i] = 0.f;
        }
#pragma unroll
        for (int w = 0; w < UPB; ++w) {
            if (w != unit) continue;
#pragma unroll
            for (int u = 0; u < kTabS; ++u) {
                const int l = lb + u;
                if (l >= ls && l <= lmax) {
                    tab_read<SPIN>(stg.slot(b, u), lane, vp, vm);
                    // block index i = w kTabS + u: rel = -1 for even i
                    if (u & 1) in.template add_vals<false>(vp, vm, part + (w * kTabS + u) * NCOMP);
                    else in.template add_vals<true>(vp, vm, part + (w * kTabS + u) * NCOMP);
                }
            }
        }
        if (unit == UPB - 1 || !more) {
            const int blk = lb - unit * kTabS;
            if constexpr (FSPIN)
                flush_smem<FSPIN, NV>(part, wbuf, out, sc, wm, wmf, base, nalm, m, blk, lmax, sgs, fx, fxu);
            else
                flush<P, FSPIN, NV>(part, out, sc, wm, wmf, base, nalm, m, blk, lmax, sgs, fx, fxu);
        }
    }
}

// Self-test of the bounded wait: one warp arms an mbarrier for 16 bytes that
// no copy delivers, waits with a short limit, and reports the timeout the
// way the table kernels do (a status bit).  Nothing is in flight.
__global__ void k_wait_selftest(unsigned *status, long long limit)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    fence_async_shared();
    __syncwarp();
    if (threadIdx.x == 0) mbar_expect_tx(&bar, 16);
    __syncwarp();
    if (!mbar_wait_warp(&bar, 0, limit) && threadIdx.x == 0) atomicOr(status, FLAG_TIMEOUT);
}

// FP32 forward kernel sharing the recursion among nm = 2 or 4 maps
const void *kernel_of_batch(bool spin, int rpt, int nm)
{
    if (nm == 2) {
        if (spin) return rpt == 1 ? (const void *)k_leg_fwd<PolDF, 1, true, 2> : (const void *)k_leg_fwd<PolDF, 2, true, 2>;
        return rpt == 1 ? (const void *)k_leg_fwd<PolDF, 1, false, 2> : (const void *)k_leg_fwd<PolDF, 2, false, 2>;
    }
    if (spin) return rpt == 1 ? (const void *)k_leg_fwd<PolDF, 1, true, 4> : (const void *)k_leg_fwd<PolDF, 2, true, 4>;
    return rpt == 1 ? (const void *)k_leg_fwd<PolDF, 1, false, 4> : (const void *)k_leg_fwd<PolDF, 2, false, 4>;
}

}  // namespace

// Launch shape of a Legendre kernel: among 4..16 warps per CTA, the one with
// the most resident warps per SM (registers decide how many CTAs fit), then
// the fewest idle ring slots.  nm > 1: the FP32 forward kernel for nm maps.
Plan::LegShape legendre_shape(const Plan &p, bool adjoint, bool dd, int rpt, int nm)
{
    const void *fn = (p.rst && p.prec == LENS_FP32) ? kernel_of32(p.spin != 0, p.grad, rpt, adjoint, nm)
                     : (nm > 1)            ? kernel_of_batch(p.spin != 0, rpt, nm)
                     : p.prec == LENS_FP32 ? kernel_of<PolDF>(p.spin != 0, p.grad, rpt, adjoint)
                     : (dd && p.rst)       ? kernel_of<PolDDR>(p.spin != 0, p.grad, rpt, adjoint)
                     : dd                  ? kernel_of<PolDD>(p.spin != 0, p.grad, rpt, adjoint)
                                           : kernel_of<PolF64>(p.spin != 0, p.grad, rpt, adjoint);
    const int nw = (p.nnorth + 32 * rpt - 1) / (32 * rpt);
    Plan::LegShape best;
    long best_active = -1, best_slots = 0;
    for (int w = 4; w <= 16; ++w) {
        const int chunks = (nw + w - 1) / w;
        const int warps = (nw + chunks - 1) / chunks;
        int blocks = 0;
        const size_t smem = (adjoint && p.prec == LENS_FP32 && p.spin) ? (size_t)warps * adj_smem_per_warp<true>() : 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fn, warps * 32, smem) != cudaSuccess) blocks = 1;
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

cudaError_t launch_rec_tables_s(Plan &p)
{
    k_rec_tables_s<<<p.mmax + 1, 256, 0, p.stream>>>(p.lmax, p.spin, (float4 *)p.rec_s);
    return cudaGetLastError();
}

cudaError_t launch_ck_build(Plan &p, double *a64, double *t64, void *v_out, void *e_out, int *lt, short *kstart)
{
    // FP64 alpha / tau / c_l of the monic recursion (c_l rewritten with the same values)
    k_rec_tables<<<p.mmax + 1, 256, 0, p.stream>>>(p.lmax, p.spin, p.scale, nullptr, nullptr, a64,
                                                   p.spin ? t64 : nullptr, nullptr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const dim3 g((p.nnorth + 127) / 128, p.mmax + 1);
    if (p.spin)
        k_ck_build<true><<<g, 128, 0, p.stream>>>(a64, t64, p.scale, p.lognorm, p.rings, p.lmax, p.spin, p.nnorth,
                                                  p.ck.K, p.ck.jb, p.ck.base, v_out, e_out, lt, nullptr);
    else
        k_ck_build<false><<<g, 128, 0, p.stream>>>(a64, nullptr, p.scale, p.lognorm, p.rings, p.lmax, p.spin, p.nnorth,
                                                   p.ck.K, p.ck.jb, p.ck.base, v_out, e_out, lt, nullptr);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_ck_start<<<p.mmax + 1, 128, 0, p.stream>>>(lt, p.lmax, p.mmax, p.spin, p.nnorth, p.ck.K, p.ck.ngrp, kstart,
                                                 p.ck.klog);
    return cudaGetLastError();
}

// FP64 plans: restart values of PolDDR from the plan's FP64 recursion tables
cudaError_t launch_ck_build64(Plan &p, void *v_out, void *e_out, int *lt, short *kstart)
{
    const dim3 g((p.nnorth + 127) / 128, p.mmax + 1);
    if (p.spin)
        k_ck_build<true, true><<<g, 128, 0, p.stream>>>((const double *)p.rec_a, (const double *)p.rec_t, p.scale,
                                                        p.lognorm, p.rings, p.lmax, p.spin, p.nnorth, p.ck.K, 0,
                                                        p.ck.base, v_out, e_out, lt, p.ck.klog);
    else
        k_ck_build<false, true><<<g, 128, 0, p.stream>>>((const double *)p.rec_a, nullptr, p.scale, p.lognorm,
                                                         p.rings, p.lmax, p.spin, p.nnorth, p.ck.K, 0, p.ck.base,
                                                         v_out, e_out, lt, p.ck.klog);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_ck_start<<<p.mmax + 1, 128, 0, p.stream>>>(lt, p.lmax, p.mmax, p.spin, p.nnorth, p.ck.K, p.ck.ngrp, kstart,
                                                 p.ck.klog);
    return cudaGetLastError();
}

cudaError_t launch_rec_tables(Plan &p)
{
    if (p.prec == LENS_FP32)
        k_rec_tables<<<p.mmax + 1, 256, 0, p.stream>>>(p.lmax, p.spin, p.scale, (float2 *)p.rec_a, nullptr, nullptr,
                                                       nullptr, const_cast<float2 *>(p.ck.cs));
    else
        k_rec_tables<<<p.mmax + 1, 256, 0, p.stream>>>(p.lmax, p.spin, p.scale, (float2 *)p.rec_a_df, nullptr,
                                                       (double *)p.rec_a, p.spin ? (double *)p.rec_t : nullptr,
                                                       nullptr);
    return cudaGetLastError();
}

// Rings per thread, from a sweep at lmax 4096 on GB300 (ms per launch):
//   FP32 spin 0: fwd 19.7 / 18.5 / 29.7 and adj 21.2 / 18.8 / 31.4 for RPT 1 / 2 / 4
//   FP32 spin 2: fwd 47.4 / 73.4 / 158 and adj 52.4 / 75.6 / 193
//   FP64 spin 0: fwd 246 / 252 / 295 and adj 258 / 236 / 262
//   FP64 spin 2: fwd 760 / 700 / 790 and adj 851 / 801 / 916
// Restarted FP32 recursion (FP32 state, rst), lmax 4096 (ms per launch, fwd / adj):
//   spin 0: 6.9 / 8.7, 4.8 / 5.9, 4.5 / 5.7 for RPT 1 / 2 / 4
//   spin 2: 12.3 / 17.1, 14.0 / 15.9, 15.8 / 20.5
int legendre_rpt(int prec, int spin, bool adjoint, bool rst)
{
    if (prec == LENS_FP32 && rst) return spin ? (adjoint ? 2 : 1) : 4;
    if (prec == LENS_FP32) return spin ? 1 : 2;
    return spin ? 2 : (adjoint ? 2 : 1);
}

// df32 part of FP64 plans: twice the accumulator words of the FP32 plans.  Restarted
// double-float recursion at lmax 4096 (ms, RPT 1 / 2): spin 0 synthesis 20.4 / 19.2,
// adjoint 29.9 / 27.0; spin 2 synthesis 63.6 / 100.0, adjoint 100.9 / 124.1
int legendre_rpt_dd(int spin, bool) { return spin ? 1 : 2; }

bool legendre_rpt_supported(int prec, int, bool, int rpt, bool rst)
{
    return rpt == 1 || rpt == 2 || (rpt == 4 && prec == LENS_FP32 && rst);
}

cudaError_t launch_legendre_fwd(const Plan &p, const void *alm, void *ring, cudaStream_t st, double wpos)
{
    // entries with l < spin / columns without rings are never written by the
    // kernel: start from zero
    const size_t eb = p.prec == LENS_FP32 ? 8 : 16;
    cudaError_t e = cudaMemsetAsync(ring, 0, eb * (size_t)p.ncol * p.ntheta, st);
    if (e != cudaSuccess) return e;
    const dim3 g(4, p.mmax + 1);
    if (p.prec == LENS_FP32) {
        k_coef_prep<float2, float2, float2><<<g, 256, 0, st>>>((const float2 *)alm, p.rst ? nullptr : p.scale, p.coef,
                                                               p.lmax, p.spin, p.nalm, p.mmax + 1, wpos, p.grad);
        if (p.rst && !p.tab) {  // the monic plain-form warps' coefficients carry c_l
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            k_coef_prep<float2, float2, float2><<<g, 256, 0, st>>>((const float2 *)alm, p.scale, p.coef_m, p.lmax,
                                                                   p.spin, p.nalm, p.mmax + 1, wpos, p.grad);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (p.tab) {
            const dim3 tg(p.tab_fchunks, p.mmax + 1);
            const size_t smem = (size_t)(p.tab_fthreads / 32) *
                                (p.spin ? tab_smem_per_warp<true, false>() : tab_smem_per_warp<false, false>());
            const auto args = [&](auto kern) {
                kern<<<tg, p.tab_fthreads, smem, st>>>(p.coef, p.tab_v, p.tab_rowbase, p.tab_jlo, p.tab_lstart,
                                                       (float2 *)ring, p.lmax, p.mmax, p.spin, p.ntheta, p.nnorth,
                                                       p.tab_nnp, p.tab_ng, p.nalm, p.flags + 1, (int64_t)0);
            };
            if (!p.spin) args(k_tab_fwd<false, false>);
            else if (p.grad) args(k_tab_fwd<true, true>);
            else args(k_tab_fwd<true, false>);
            return cudaGetLastError();
        }
        if (p.rst) return fwd32_spin(p, p.leg_f, p.coef, ring, 0, p.mmax + 1, st);
        return fwd_spin<PolDF>(p, p.leg_f, p.coef, p.rec_a, p.rec_t, ring, 0, p.mmax + 1, st);
    }
    k_coef_prep<double2, double2, float4><<<g, 256, 0, st>>>((const double2 *)alm, p.scale, p.coef, p.lmax, p.spin,
                                                             p.nalm, p.m_df, wpos, p.grad);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = fwd_spin<PolF64>(p, p.leg_f, p.coef, p.rec_a, p.rec_t, ring, 0, p.m_df, st)) != cudaSuccess) return e;
    if (p.rst) return fwd_spin<PolDDR>(p, p.leg_fd, p.coef, p.rec_a_df, p.rec_t_df, ring, p.m_df, p.mmax + 1, st);
    return fwd_spin<PolDD>(p, p.leg_fd, p.coef, p.rec_a_df, p.rec_t_df, ring, p.m_df, p.mmax + 1, st);
}

cudaError_t launch_legendre_fwd_batch(const Plan &p, const void *alm, void *ring, void *coef, int nm, cudaStream_t st,
                                      double wpos)
{
    if (p.prec != LENS_FP32 || (nm != 2 && nm != 4)) return cudaErrorInvalidValue;
    const size_t ring_elems = (size_t)p.ncol * p.ntheta;
    cudaError_t e = cudaMemsetAsync(ring, 0, 8 * ring_elems * nm, st);
    if (e != cudaSuccess) return e;
    const int ncomp = p.spin ? 2 : 1;
    const dim3 g(4, p.mmax + 1);
    for (int b = 0; b < nm; ++b) {
        k_coef_prep<float2, float2, float2><<<g, 256, 0, st>>>((const float2 *)alm + (size_t)b * ncomp * p.nalm,
                                                               p.rst ? nullptr : p.scale,
                                                               (float2 *)coef + (size_t)b * ncomp * p.nalm,
                                                               p.lmax, p.spin, p.nalm, p.mmax + 1, wpos, false);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (p.tab) {  // one table read serves the nm maps
        const dim3 tg(p.tab_fchunks, p.mmax + 1);
        const size_t smem = (size_t)(p.tab_fthreads / 32) *
                            (p.spin ? tab_smem_per_warp<true, false>() : tab_smem_per_warp<false, false>());
        const int64_t rs = (int64_t)p.ncol * p.ntheta;
        const auto args = [&](auto kern) {
            kern<<<tg, p.tab_fthreads, smem, st>>>(coef, p.tab_v, p.tab_rowbase, p.tab_jlo, p.tab_lstart,
                                                   (float2 *)ring, p.lmax, p.mmax, p.spin, p.ntheta, p.nnorth,
                                                   p.tab_nnp, p.tab_ng, p.nalm, p.flags + 1, rs);
        };
        if (p.spin) {
            if (nm != 2) return cudaErrorInvalidValue;
            args(k_tab_fwd<true, false, 2>);
        } else if (nm == 2) {
            args(k_tab_fwd<false, false, 2>);
        } else {
            args(k_tab_fwd<false, false, 4>);
        }
        return cudaGetLastError();
    }
    const Plan::LegShape &sh = p.leg_fb[nm == 2 ? 0 : 1];
    if (p.rst) {
        if (p.spin)
            return nm == 2 ? fwd32_rpt<true, 2>(p, sh, coef, ring, 0, p.mmax + 1, st)
                           : fwd32_rpt<true, 4>(p, sh, coef, ring, 0, p.mmax + 1, st);
        return nm == 2 ? fwd32_rpt<false, 2>(p, sh, coef, ring, 0, p.mmax + 1, st)
                       : fwd32_rpt<false, 4>(p, sh, coef, ring, 0, p.mmax + 1, st);
    }
    if (p.spin) {
        if (sh.rpt == 1)
            return nm == 2 ? fwd_launch<PolDF, 1, true, 2>(p, sh, coef, p.rec_a, p.rec_t, ring, 0, p.mmax + 1, st)
                           : fwd_launch<PolDF, 1, true, 4>(p, sh, coef, p.rec_a, p.rec_t, ring, 0, p.mmax + 1, st);
        return nm == 2 ? fwd_launch<PolDF, 2, true, 2>(p, sh, coef, p.rec_a, p.rec_t, ring, 0, p.mmax + 1, st)
                       : fwd_launch<PolDF, 2, true, 4>(p, sh, coef, p.rec_a, p.rec_t, ring, 0, p.mmax + 1, st);
    }
    if (sh.rpt == 1)
        return nm == 2 ? fwd_launch<PolDF, 1, false, 2>(p, sh, coef, p.rec_a, p.rec_t, ring, 0, p.mmax + 1, st)
                       : fwd_launch<PolDF, 1, false, 4>(p, sh, coef, p.rec_a, p.rec_t, ring, 0, p.mmax + 1, st);
    return nm == 2 ? fwd_launch<PolDF, 2, false, 2>(p, sh, coef, p.rec_a, p.rec_t, ring, 0, p.mmax + 1, st)
                   : fwd_launch<PolDF, 2, false, 4>(p, sh, coef, p.rec_a, p.rec_t, ring, 0, p.mmax + 1, st);
}

cudaError_t launch_legendre_adj(const Plan &p, const void *ring, void *alm, cudaStream_t st, double wpos)
{
    const size_t ebytes = (p.prec == LENS_FP32 ? 8 : 16) * (size_t)p.nalm * p.alm_ncomp();
    cudaError_t e = cudaMemsetAsync(alm, 0, ebytes, st);  // the kernels add warp sums atomically
    if (e != cudaSuccess) return e;
    // deterministic plans: fixed-point sums (FP32 plans in their own buffer,
    // FP64 plans in alm itself), units per order from the ring inputs
    const bool f32 = p.prec == LENS_FP32;
    void *fx = nullptr;
    if (p.det) {
        fx = f32 ? p.fx_alm : alm;
        if (f32 && (e = cudaMemsetAsync(fx, 0, 16 * (size_t)p.nalm * p.alm_ncomp(), st)) != cudaSuccess) return e;
        const double lam = sqrt((2.0 * p.lmax + 1.0) / (4.0 * 3.14159265358979323846));
        const double wmax = (wpos > 1.0 ? wpos : 1.0) * lam;
        if (f32) k_fx_units<float2><<<p.mmax + 1, 256, 0, st>>>((const float2 *)ring, p.ntheta, p.mmax, p.spin != 0, wmax, p.fx_scale);
        else k_fx_units<double2><<<p.mmax + 1, 256, 0, st>>>((const double2 *)ring, p.ntheta, p.mmax, p.spin != 0, wmax, p.fx_scale);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (f32 && p.tab) {
        const dim3 tg(p.tab_achunks, p.mmax + 1);
        const size_t warps = (size_t)(p.tab_athreads / 32);
        const auto args = [&](auto kern, size_t smem) {
            kern<<<tg, p.tab_athreads, smem, st>>>((const float2 *)ring, p.tab_v, p.tab_rowbase, p.tab_jlo,
                                                   p.tab_lstart, p.scale, (float2 *)alm, p.lmax, p.mmax, p.spin,
                                                   p.ntheta, p.nnorth, p.tab_nnp, p.tab_ng, p.nalm, wpos,
                                                   (unsigned long long *)fx, p.fx_scale, p.flags + 1);
        };
        if (!p.spin) args(k_tab_adj<false, false>, warps * tab_smem_per_warp<false, false>());
        else if (p.grad) args(k_tab_adj<true, true>, warps * tab_smem_per_warp<true, false>());
        else args(k_tab_adj<true, false>, warps * tab_smem_per_warp<true, true>());
        e = cudaGetLastError();
    } else if (f32) {
        e = p.rst ? adj32_spin(p, p.leg_a, ring, alm, 0, p.mmax + 1, st, wpos, fx)
                  : adj_spin<PolDF>(p, p.leg_a, ring, p.rec_a, p.rec_t, alm, 0, p.mmax + 1, st, wpos, fx);
    } else {
        e = adj_spin<PolF64>(p, p.leg_a, ring, p.rec_a, p.rec_t, alm, 0, p.m_df, st, wpos, fx);
        if (e == cudaSuccess)
            e = p.rst ? adj_spin<PolDDR>(p, p.leg_ad, ring, p.rec_a_df, p.rec_t_df, alm, p.m_df, p.mmax + 1, st, wpos, fx)
                      : adj_spin<PolDD>(p, p.leg_ad, ring, p.rec_a_df, p.rec_t_df, alm, p.m_df, p.mmax + 1, st, wpos, fx);
    }
    if (e != cudaSuccess || !p.det) return e;
    const dim3 g(4, p.mmax + 1);
    const int nc = p.alm_ncomp();
    if (f32) k_fx_to_alm<float><<<g, 256, 0, st>>>((const unsigned long long *)fx, (float *)alm, p.lmax, p.nalm, nc, p.fx_scale);
    else k_fx_to_alm<double><<<g, 256, 0, st>>>((const unsigned long long *)fx, (double *)alm, p.lmax, p.nalm, nc, p.fx_scale);
    return cudaGetLastError();
}

cudaError_t launch_wait_selftest(unsigned *status, long long limit, cudaStream_t st)
{
    k_wait_selftest<<<1, 32, 0, st>>>(status, limit);
    return cudaGetLastError();
}

// ---- Legendre tables (plan creation)
// Launch shapes of the table kernels: warps of 32 ring groups, at most wmax
// warps per CTA (shared memory: 8 KB of staging per warp, plus the spin-s
// adjoint's reduction rows), as few idle warps as possible.
// Opts the kernels into the dynamic shared memory they need.
cudaError_t tab_shape(Plan &p)
{
    p.tab_nnp = (p.nnorth + kTabG - 1) / kTabG * kTabG;
    p.tab_ng = p.tab_nnp / kTabG;
    const int nw = (p.tab_ng + 31) / 32;
    auto shape = [&](int wmax, int &chunks, int &threads) {
        chunks = (nw + wmax - 1) / wmax;
        threads = 32 * ((nw + chunks - 1) / chunks);
    };
    const int fw = 8, aw = p.spin ? 4 : 8;  // the attributes below allow the largest shape
    shape(fw, p.tab_fchunks, p.tab_fthreads);
    shape(aw, p.tab_achunks, p.tab_athreads);
    cudaError_t e;
    if (p.spin) {
        if ((e = cudaFuncSetAttribute(k_tab_fwd<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      fw * tab_smem_per_warp<true, false>())) != cudaSuccess ||
            (e = cudaFuncSetAttribute(k_tab_fwd<true, false, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      fw * tab_smem_per_warp<true, false>())) != cudaSuccess ||
            (e = cudaFuncSetAttribute(k_tab_fwd<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      fw * tab_smem_per_warp<true, false>())) != cudaSuccess ||
            (e = cudaFuncSetAttribute(k_tab_adj<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      aw * tab_smem_per_warp<true, true>())) != cudaSuccess ||
            (e = cudaFuncSetAttribute(k_tab_adj<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      aw * tab_smem_per_warp<true, false>())) != cudaSuccess)
            return e;
    } else {
        if ((e = cudaFuncSetAttribute(k_tab_fwd<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      fw * tab_smem_per_warp<false, false>())) != cudaSuccess ||
            (e = cudaFuncSetAttribute(k_tab_fwd<false, false, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      fw * tab_smem_per_warp<false, false>())) != cudaSuccess ||
            (e = cudaFuncSetAttribute(k_tab_fwd<false, false, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      fw * tab_smem_per_warp<false, false>())) != cudaSuccess ||
            (e = cudaFuncSetAttribute(k_tab_adj<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      aw * tab_smem_per_warp<false, false>())) != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

cudaError_t launch_tab_first(const Plan &p, int *first)
{
    const dim3 g((p.tab_nnp + 511) / 512, p.mmax + 1);
    if (p.spin) k_tab_first<true><<<g, 256, 0, p.stream>>>(p.rec_a, p.rec_t, p.lognorm, p.rings, p.lmax, p.spin, p.nnorth, first);
    else k_tab_first<false><<<g, 256, 0, p.stream>>>(p.rec_a, p.rec_t, p.lognorm, p.rings, p.lmax, p.spin, p.nnorth, first);
    return cudaGetLastError();
}

cudaError_t launch_tab_rows(const Plan &p, const int *first, int *lstart, int *jlo, int64_t *rowlen)
{
    k_tab_rows<<<(p.mmax + 1 + 127) / 128, 128, 0, p.stream>>>(first, p.lmax, p.mmax, p.spin, p.nnorth, p.tab_nnp,
                                                              lstart, jlo, rowlen);
    return cudaGetLastError();
}

cudaError_t launch_tab_fill(const Plan &p)
{
    const dim3 g((p.tab_nnp + 511) / 512, p.mmax + 1);
    if (p.spin)
        k_tab_fill<true><<<g, 256, 0, p.stream>>>(p.rec_a, p.rec_t, p.lognorm, p.rings, p.lmax, p.spin, p.nnorth,
                                                  p.tab_nnp, p.tab_jlo, p.tab_rowbase, p.tab_v);
    else
        k_tab_fill<false><<<g, 256, 0, p.stream>>>(p.rec_a, p.rec_t, p.lognorm, p.rings, p.lmax, p.spin, p.nnorth,
                                                   p.tab_nnp, p.tab_jlo, p.tab_rowbase, p.tab_v);
    return cudaGetLastError();
}

}  // namespace gsl
