// Torus steps of the general SHT (Sect. 3 "doubling" and "FFT", and their
// adjoints "FFT" and "undoubling").
//
// Forward, per m column (theta kernel; two adjacent columns of opposite parity
// share each transform, see k_theta_fwd):
//   doubled ring sequence G_j, j in [0, M), M = 2 ntheta - 2:
//       G_j = F_m(theta_j) for j < ntheta,  G_{M-j} = (-1)^{m+s} F_m(theta_j)
//   (mirror theta -> 2 pi - theta, phi -> phi + pi; odd spins flip sign),
//   c_k = (1/M) sum_j G_j e^{-2 pi i jk/M} for |k| <= lmax (exact: band limit),
//   b_k = c_k / (psihat(2 pi k/N1) psihat(2 pi m/N2))   (kernel deconvolution),
//   zero padding to N1 and y_r = sum_k b_k e^{+2 pi i kr/N1} on the kept rows
//   r in [r_lo, r_lo + R) (theta in [0, pi] plus the kernel halo).
// Forward, per kept row (phi kernel):
//   g_r(c) = sum_m y_r(m) e^{+2 pi i mc/N2}, c in [0, N2), plus W-1 wrap columns.
//   Spin 0 rows are real (m < 0 by Hermitian symmetry); two rows share one
//   complex transform (row a in the real part, row b in the imaginary part).
// The ring data never visit phi space: the paper's per-ring phi FFT and the
// phi FFT of the 2D transform cancel because n_phi >= 2 lmax + 2.
//
// Adjoint: exact transposes in reverse order (fold the wrap columns, forward
// phi FFT, weights; forward theta FFT, weights, inverse length-M transform,
// fold j and M - j with (-1)^{m+s}).
#include <cuda_runtime.h>

#include "common.cuh"
#include "fft.cuh"
#include "internal.h"

namespace gsl {
namespace {

// a mod n for -n <= a < 2n (every use: a row r_lo + rr with -W <= r_lo and rr < R < N1,
// or an order m with |m| <= mmax < N2): one wrap instead of a division
__device__ __forceinline__ int pmod(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

template <typename C, int CL> __device__ __forceinline__ Buf<C, CL> make_buf(C *local, int chunk);
// theta transforms: FP32 single-CTA vectors use the padded layout
template <typename C, int CL> struct ThetaBuf {
    using type = Buf<C, CL>;
    static __device__ __forceinline__ type make(C *l, int chunk) { return make_buf<C, CL>(l, chunk); }
};
template <> struct ThetaBuf<float2, 1> {
    using type = PadBuf<float2>;
    static __device__ __forceinline__ type make(float2 *l, int) { return PadBuf<float2>(l); }
};
template <> __device__ __forceinline__ Buf<float2, 1> make_buf<float2, 1>(float2 *l, int) { return Buf<float2, 1>(l); }
template <> __device__ __forceinline__ Buf<double2, 1> make_buf<double2, 1>(double2 *l, int)
{
    return Buf<double2, 1>(l);
}
template <> __device__ __forceinline__ Buf<float2, 2> make_buf<float2, 2>(float2 *l, int ch)
{
    return Buf<float2, 2>(l, ch);
}
template <> __device__ __forceinline__ Buf<double2, 2> make_buf<double2, 2>(double2 *l, int ch)
{
    return Buf<double2, 2>(l, ch);
}
template <> __device__ __forceinline__ Buf<float2, 4> make_buf<float2, 4>(float2 *l, int ch)
{
    return Buf<float2, 4>(l, ch);
}
template <> __device__ __forceinline__ Buf<double2, 4> make_buf<double2, 4>(double2 *l, int ch)
{
    return Buf<double2, 4>(l, ch);
}

// Every kernel below is written for a team of CL CTAs sharing one vector
// (fft.cuh): CL = 1 is one CTA with the vector in its shared memory, CL = 2 or
// 4 a cluster of CTAs holding `chunk` elements each.  Cluster teams start
// with a cluster barrier (all CTAs resident before any remote access) and end
// with one (no CTA exits while a partner may still read its part).

// ----------------------------------------------------------------- theta fwd
// Columns c and c + 1 have opposite parities (-1)^(m+s), so one complex
// transform serves both: with G = G_a + i G_b (G_a the even, G_b the odd
// doubled column, the odd column's pole samples zero as its symmetry requires)
// Z = FFT(G) splits as Z_k = C_a(k) + i C_b(k), Z_-k = C_a(k) - i C_b(k), so
// C_c(k) = (Z_k + par_c Z_-k) / 2 and (Z_k + par_c Z_-k) / 2i; the weighted
// coefficients recombine as B_k = b_1(k) + i b_2(k), B_-k = par_1 b_1(k) +
// i par_2 b_2(k), and the rows of the inverse transform Y = y_1 + i y_2 split
// the same way, y_c(r) = (Y_r + par_c Y_-r) / 2 (resp. / 2i).  One length-M and
// one length-N1 transform per pair of columns instead of per column.
template <typename T> __device__ __forceinline__ cplx<T> pack_i(cplx<T> a, cplx<T> b)  // a + i b
{
    return mkc(a.x - b.y, a.y + b.x);
}
// (u + p v) / 2 and (u + q v) / 2i for q = -p: the parts of the two columns
template <typename T>
__device__ __forceinline__ void split_pair(cplx<T> u, cplx<T> v, T p1, cplx<T> &x1, cplx<T> &x2)
{
    const cplx<T> s = mkc(T(0.5) * (u.x + p1 * v.x), T(0.5) * (u.y + p1 * v.y));  // (u + p1 v) / 2
    const cplx<T> d = mkc(T(0.5) * (u.x - p1 * v.x), T(0.5) * (u.y - p1 * v.y));  // (u + p2 v) / 2, p2 = -p1
    x1 = s;
    x2 = mkc(d.y, -d.x);  // d / i
}

template <typename T, int CL, int OCC = 1>
__global__ void __launch_bounds__(512, OCC) k_theta_fwd(const cplx<T> *__restrict__ ring, cplx<T> *__restrict__ X,
                                                    FftDesc fM, FftDesc fN1, const T *__restrict__ w1,
                                                    const T *__restrict__ w2, int ntheta, int lmax, int mmax,
                                                    int spin, int ncol, int r_lo, int R, int chunk)
{
    using C = cplx<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Team<CL> tm;
    if (CL > 1) tm.sync();
    const auto buf = ThetaBuf<C, CL>::make(reinterpret_cast<C *>(smem_raw), chunk);
    const int c1 = 2 * tm.vec(), c2 = c1 + 1;
    const bool has2 = c2 < ncol;
    const int mc = spin == 0 ? c1 : c1 - mmax;
    const T p1 = ((mc + spin) & 1) ? T(-1) : T(1), p2 = -p1;
    const int M = fM.n, N1 = fN1.n, N = ntheta - 1;
    const int tid = tm.tid, nthr = tm.nthr;
    const C *F1 = ring + (int64_t)c1 * ntheta;
    const C *F2 = ring + (int64_t)c2 * ntheta;
    const C zero = mkc(T(0), T(0));

    for (int i = tid; i < M; i += nthr) {
        const int j = i < ntheta ? i : M - i;
        const bool pole = j == 0 || j == N;
        C a = F1[j], b = has2 ? F2[j] : zero;
        if (i >= ntheta) { a = cscale(a, p1); b = cscale(b, p2); }
        if (pole) { if (p1 < T(0)) a = zero; else b = zero; }
        buf[__ldg(fM.perm + i)] = pack_i<T>(a, b);
    }
    tm.sync();
    fft_smem<-1, T, CL>(buf, fM, tm);  // natural order: Z_k * M

    // split (k, -k), weight by w1(k) w2(m) per column, recombine at k and N1 - k; the
    // other positions become zero.  In one pass when the source range of the negative
    // frequencies [M - lmax, M) lies below their target [N1 - lmax, N1)
    const T wa = w2[c1], wb = has2 ? w2[c2] : T(0);
    auto pair_at = [&](int k, C zk, C zm, C &bk, C &bm) {
        C x1, x2;
        split_pair<T>(zk, zm, p1, x1, x2);
        const T wk = w1[k + lmax];
        x1 = cscale(x1, wk * wa);
        x2 = cscale(x2, wk * wb);
        bk = pack_i<T>(x1, x2);
        bm = pack_i<T>(cscale(x1, p1), cscale(x2, p2));
    };
    if (N1 - lmax >= M) {
        for (int k = tid; k <= lmax; k += nthr) {
            C bk, bm;
            pair_at(k, buf[k], buf[k == 0 ? 0 : M - k], bk, bm);
            buf[k] = bk;
            if (k > 0) buf[N1 - k] = bm;
        }
        tm.sync();
        for (int i = lmax + 1 + tid; i < N1 - lmax; i += nthr) buf[i] = zero;
    } else {
        // overlapping ranges: N1 - k is the source M - k' of k' = k - (N1 - M) <= k, so the
        // chunks run from k = 0 up
        for (int k0 = 0; k0 <= lmax; k0 += nthr) {
            const int k = k0 + tid;
            C bk = zero, bm = zero;
            if (k <= lmax) pair_at(k, buf[k], buf[k == 0 ? 0 : M - k], bk, bm);
            tm.sync();
            if (k <= lmax) {
                buf[k] = bk;
                if (k > 0) buf[N1 - k] = bm;
            }
            tm.sync();
        }
        for (int i = lmax + 1 + tid; i < N1 - lmax; i += nthr) buf[i] = zero;
    }
    tm.sync();
    fft_smem_dif<+1, T, CL>(buf, fN1, tm);  // Y_r at position perm_N1[r]

    for (int rr = tid; rr < R; rr += nthr) {
        const int r = pmod(r_lo + rr, N1);
        const int rm = r == 0 ? 0 : N1 - r;
        C y1, y2;
        split_pair<T>(buf[__ldg(fN1.perm + r)], buf[__ldg(fN1.perm + rm)], p1, y1, y2);
        X[(int64_t)rr * ncol + c1] = y1;
        if (has2) X[(int64_t)rr * ncol + c2] = y2;
    }
    if (CL > 1) tm.sync();
}

// Torus coefficients of one m column (diagnostic entry point): the doubled
// sequence and its length-M transform as in k_theta_fwd, written unscaled by
// the kernel deconvolution: out[c][k + lmax] = c_k = (1/M) sum_j G_j
// e^{-2 pi i jk/M}, |k| <= lmax, so that F_m(theta) = sum_k c_k e^{ik theta}
// for every theta (one CTA per column).
template <typename T>
__global__ void __launch_bounds__(512) k_theta_coeffs(const cplx<T> *__restrict__ ring, cplx<T> *__restrict__ out,
                                                       FftDesc fM, int ntheta, int lmax, int mmax, int spin)
{
    using C = cplx<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Team<1> tm;
    const auto buf = ThetaBuf<C, 1>::make(reinterpret_cast<C *>(smem_raw), 0);
    const int c = tm.vec();
    const int mc = spin == 0 ? c : c - mmax;
    const T par = ((mc + spin) & 1) ? T(-1) : T(1);
    const int M = fM.n;
    const C *F = ring + (int64_t)c * ntheta;
    for (int i = tm.tid; i < M; i += tm.nthr) buf[__ldg(fM.perm + i)] = i < ntheta ? F[i] : cscale(F[M - i], par);
    tm.sync();
    fft_smem<-1, T, 1>(buf, fM, tm);
    const T inv = T(1) / T(M);
    for (int k = -lmax + tm.tid; k <= lmax; k += tm.nthr)
        out[(int64_t)c * (2 * lmax + 1) + (k + lmax)] = cscale(buf[k < 0 ? M + k : k], inv);
}

// ----------------------------------------------------------------- theta adj
// Adjoint of the paired forward: the rows of each column are symmetrised first,
// h~_c(r) = h_c(r) + par_c h_c(-r) (the fold of the forward's doubling moved
// before the transforms, with which it commutes), packed h~_1 + i h~_2 and
// split after each transform as in the forward; the even column's pole rings
// take half of the symmetric result, the odd column's pole rings zero.
template <typename T, int CL, int OCC = 1>
__global__ void __launch_bounds__(512, OCC) k_theta_adj(const cplx<T> *__restrict__ X, cplx<T> *__restrict__ ring,
                                                    FftDesc fM, FftDesc fN1, const T *__restrict__ w1,
                                                    const T *__restrict__ w2, int ntheta, int lmax, int mmax,
                                                    int spin, int ncol, int r_lo, int R, int chunk)
{
    using C = cplx<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Team<CL> tm;
    if (CL > 1) tm.sync();
    const auto buf = ThetaBuf<C, CL>::make(reinterpret_cast<C *>(smem_raw), chunk);
    const int c1 = 2 * tm.vec(), c2 = c1 + 1;
    const bool has2 = c2 < ncol;
    const int mc = spin == 0 ? c1 : c1 - mmax;
    const T p1 = ((mc + spin) & 1) ? T(-1) : T(1), p2 = -p1;
    const int M = fM.n, N1 = fN1.n, N = ntheta - 1;
    const int tid = tm.tid, nthr = tm.nthr;
    const C zero = mkc(T(0), T(0));

    // row r of a column: X[rr] with rr = r - r_lo (mod N1) when rr < R, else zero
    auto row = [&](int r, int c) -> C {
        const int rr = pmod(r - r_lo, N1);
        return rr < R ? X[(int64_t)rr * ncol + c] : zero;
    };
    for (int r = tid; r <= N1 / 2; r += nthr) {
        const int rm = r == 0 ? 0 : N1 - r;
        const C a = row(r, c1), am = row(rm, c1);
        const C b = has2 ? row(r, c2) : zero, bm = has2 ? row(rm, c2) : zero;
        C h1 = cadd(a, cscale(am, p1)), h2 = cadd(b, cscale(bm, p2));
        if (rm == r) { h1 = cscale(a, T(1) + p1); h2 = cscale(b, T(1) + p2); }
        buf[__ldg(fN1.perm + r)] = pack_i<T>(h1, h2);
        if (rm != r) buf[__ldg(fN1.perm + rm)] = pack_i<T>(cscale(h1, p1), cscale(h2, p2));
    }
    tm.sync();
    fft_smem<-1, T, CL>(buf, fN1, tm);  // natural order

    // split (k, -k), weight, recombine at k and M - k (positions of the length-M
    // transform); in one pass when [N1 - lmax, N1) lies above [M - lmax, M)
    const T wa = w2[c1], wb = has2 ? w2[c2] : T(0);
    auto pair_at = [&](int k, C zk, C zm, C &bk, C &bm) {
        C x1, x2;
        split_pair<T>(zk, zm, p1, x1, x2);
        const T wk = w1[k + lmax];
        x1 = cscale(x1, wk * wa);
        x2 = cscale(x2, wk * wb);
        bk = pack_i<T>(x1, x2);
        bm = pack_i<T>(cscale(x1, p1), cscale(x2, p2));
    };
    if (N1 - lmax >= M) {
        for (int k = tid; k <= lmax; k += nthr) {
            C bk, bm;
            pair_at(k, buf[k], buf[k == 0 ? 0 : N1 - k], bk, bm);
            buf[k] = bk;
            if (k > 0) buf[M - k] = bm;
        }
        tm.sync();
        for (int i = lmax + 1 + tid; i < M - lmax; i += nthr) buf[i] = zero;
    } else {
        // overlapping ranges: M - k is the source N1 - k' of k' = k + N1 - M >= k, so the
        // chunks run from the highest k down
        for (int k0 = lmax; k0 >= 0; k0 -= nthr) {
            const int k = k0 - tid;
            C bk = zero, bm = zero;
            if (k >= 0) pair_at(k, buf[k], buf[k == 0 ? 0 : N1 - k], bk, bm);
            tm.sync();
            if (k >= 0) {
                buf[k] = bk;
                if (k > 0) buf[M - k] = bm;
            }
            tm.sync();
        }
        for (int i = lmax + 1 + tid; i < M - lmax; i += nthr) buf[i] = zero;
    }
    tm.sync();
    fft_smem_dif<+1, T, CL>(buf, fM, tm);  // V_j at position perm_M[j]

    C *F1 = ring + (int64_t)c1 * ntheta;
    C *F2 = ring + (int64_t)c2 * ntheta;
    for (int j = tid; j < ntheta; j += nthr) {
        const int jm = j == 0 ? 0 : M - j;
        C g1, g2;
        split_pair<T>(buf[__ldg(fM.perm + j)], buf[__ldg(fM.perm + jm)], p1, g1, g2);
        if (j == 0 || j == N) {  // pole rings: half of the symmetric sum (even), zero (odd)
            g1 = p1 > T(0) ? cscale(g1, T(0.5)) : zero;
            g2 = p2 > T(0) ? cscale(g2, T(0.5)) : zero;
        }
        F1[j] = g1;
        if (has2) F2[j] = g2;
    }
    if (CL > 1) tm.sync();
}

// ------------------------------------------------------------------- phi fwd
// spin 0: team = row pair (2b, 2b+1); spin s: team = one row.
template <typename T, bool SPIN, int CL, int OCC = 1>
__global__ void __launch_bounds__(512, OCC) k_phi_fwd(const cplx<T> *__restrict__ X, void *__restrict__ grid,
                                                 FftDesc fN2, int mmax, int ncol, int R, int pitch, int W, int chunk,
                                                 int dd)
{
    using C = cplx<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Team<CL> tm;
    if (CL > 1) tm.sync();
    const Buf<C, CL> buf = make_buf<C, CL>(reinterpret_cast<C *>(smem_raw), chunk);
    const int N2 = fN2.n;
    const int tid = tm.tid, nthr = tm.nthr;
    for (int i = tid; i < N2; i += nthr) buf[i] = mkc(T(0), T(0));
    tm.sync();
    if (!SPIN) {
        const int ra = 2 * tm.vec(), rb = ra + 1;
        const bool hb = rb < R;
        const C *xa = X + (int64_t)ra * ncol;
        const C *xb = X + (int64_t)rb * ncol;
        for (int m = tid; m <= mmax; m += nthr) {
            C a = xa[m];
            C b = hb ? xb[m] : mkc(T(0), T(0));
            if (m == 0) {
                buf[__ldg(fN2.perm + 0)] = mkc(a.x, b.x);
            } else {
                // Z_m = a + i b ; Z_{-m} = conj(a) + i conj(b)
                buf[__ldg(fN2.perm + m)] = mkc(a.x - b.y, a.y + b.x);
                buf[__ldg(fN2.perm + (N2 - m))] = mkc(a.x + b.y, b.x - a.y);
            }
        }
        tm.sync();
        fft_smem<+1, T, CL>(buf, fN2, tm);
        if (sizeof(T) == 8 && dd) {  // double-float pairs for k_interp_dd
            float2 *ga = (float2 *)grid + (int64_t)ra * pitch;
            float2 *gb = (float2 *)grid + (int64_t)rb * pitch;
            for (int c = tid; c < N2 + W - 1; c += nthr) {
                C v = buf[c < N2 ? c : c - N2];
                const df32 x = df_split((double)v.x), y = df_split((double)v.y);
                ga[c] = make_float2(x.h, x.l);
                if (hb) gb[c] = make_float2(y.h, y.l);
            }
        } else {
            T *ga = (T *)grid + (int64_t)ra * pitch;
            T *gb = (T *)grid + (int64_t)rb * pitch;
            for (int c = tid; c < N2 + W - 1; c += nthr) {
                C v = buf[c < N2 ? c : c - N2];
                ga[c] = v.x;
                if (hb) gb[c] = v.y;
            }
        }
    } else {
        const int r = tm.vec();
        const C *xr = X + (int64_t)r * ncol;
        for (int i = tid; i < ncol; i += nthr) {
            const int m = i - mmax;
            buf[__ldg(fN2.perm + pmod(m, N2))] = xr[i];
        }
        tm.sync();
        fft_smem<+1, T, CL>(buf, fN2, tm);
        if (sizeof(T) == 8 && dd) {
            float4 *gr = (float4 *)grid + (int64_t)r * pitch;
            for (int c = tid; c < N2 + W - 1; c += nthr) {
                const C v = buf[c < N2 ? c : c - N2];
                const df32 x = df_split((double)v.x), y = df_split((double)v.y);
                gr[c] = make_float4(x.h, x.l, y.h, y.l);
            }
        } else {
            C *gr = (C *)grid + (int64_t)r * pitch;
            for (int c = tid; c < N2 + W - 1; c += nthr) gr[c] = buf[c < N2 ? c : c - N2];
        }
    }
    if (CL > 1) tm.sync();
}

// ------------------------------------------------------------------- phi adj
template <typename T, bool SPIN, int CL, int OCC = 1>
__global__ void __launch_bounds__(512, OCC) k_phi_adj(const void *__restrict__ grid, cplx<T> *__restrict__ X,
                                                 FftDesc fN2, int mmax, int ncol, int R, int pitch, int W, int chunk)
{
    using C = cplx<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Team<CL> tm;
    if (CL > 1) tm.sync();
    const Buf<C, CL> buf = make_buf<C, CL>(reinterpret_cast<C *>(smem_raw), chunk);
    const int N2 = fN2.n;
    const int tid = tm.tid, nthr = tm.nthr;
    if (!SPIN) {
        const int ra = 2 * tm.vec(), rb = ra + 1;
        const bool hb = rb < R;
        const T *ga = (const T *)grid + (int64_t)ra * pitch;
        const T *gb = (const T *)grid + (int64_t)rb * pitch;
        for (int c = tid; c < N2; c += nthr) {
            T a = ga[c], b = hb ? gb[c] : T(0);
            if (c < W - 1) { a += ga[N2 + c]; if (hb) b += gb[N2 + c]; }
            buf[__ldg(fN2.perm + c)] = mkc(a, b);
        }
        tm.sync();
        fft_smem<-1, T, CL>(buf, fN2, tm);
        C *xa = X + (int64_t)ra * ncol;
        C *xb = X + (int64_t)rb * ncol;
        for (int m = tid; m <= mmax; m += nthr) {
            C z = buf[m], zc = buf[m == 0 ? 0 : N2 - m];
            // A_m = (z + conj zc)/2 ; B_m = (z - conj zc)/(2i)
            C A = mkc(T(0.5) * (z.x + zc.x), T(0.5) * (z.y - zc.y));
            C B = mkc(T(0.5) * (z.y + zc.y), T(-0.5) * (z.x - zc.x));
            xa[m] = A;
            if (hb) xb[m] = B;
        }
    } else {
        const int r = tm.vec();
        const C *gr = (const C *)grid + (int64_t)r * pitch;
        for (int c = tid; c < N2; c += nthr) {
            C v = gr[c];
            if (c < W - 1) v = cadd(v, gr[N2 + c]);
            buf[__ldg(fN2.perm + c)] = v;
        }
        tm.sync();
        fft_smem<-1, T, CL>(buf, fN2, tm);
        C *xr = X + (int64_t)r * ncol;
        for (int i = tid; i < ncol; i += nthr) {
            const int m = i - mmax;
            xr[i] = buf[pmod(m, N2)];
        }
    }
    if (CL > 1) tm.sync();
}

}  // namespace

// Per-CTA shared memory: the vector's elements divided over the team.
size_t theta_smem_bytes(const Plan &p)
{
    const size_t n = (size_t)(p.N1 > p.M ? p.N1 : p.M), esz = p.prec == LENS_FP32 ? 8 : 16;
    if (p.cl_theta == 1) return fft_smem_elems(n, esz) * esz;
    return (n + p.cl_theta - 1) / p.cl_theta * esz;
}
size_t phi_smem_bytes(const Plan &p)
{
    return ((size_t)p.N2 + p.cl_phi - 1) / p.cl_phi * (p.prec == LENS_FP32 ? 8 : 16);
}

namespace {

constexpr int kThetaThreads = 512;
int phi_threads(const Plan &p) { return p.prec == LENS_FP32 ? 512 : 256; }
// Two 512-thread CTAs per SM need at most 64 registers per thread and half the
// SM's shared memory each; FP32 single-CTA vectors that fit then run the
// variant compiled for two CTAs per SM (measured at lmax 4096, sigma 1.5:
// theta 0.82 -> 0.68 ms, phi 0.35 -> 0.29 ms spin 0; at sigma 2.26, where one
// vector takes 148 KB, the cap only adds spills).
constexpr size_t kTwoCtaSmem = 113 * 1024;

// Launches nvec teams of cl CTAs (a cluster of two when cl = 2).
template <class... KArgs, class... Args>
cudaError_t launch_team(void (*kern)(KArgs...), int cl, int nvec, int threads, size_t smem, cudaStream_t st,
                        Args... args)
{
    cudaError_t e = cudaFuncSetAttribute((const void *)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess || nvec == 0) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)nvec * (unsigned)cl);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = cl > 1 ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

template <typename T>
cudaError_t theta_fwd_t(const Plan &p, const void *ring, void *X, cudaStream_t st)
{
    using C = cplx<T>;
    const size_t sm = theta_smem_bytes(p);
    const int chunk = (int)(sm / sizeof(C));
    auto args = [&](auto kern) {
        return launch_team(kern, p.cl_theta, (p.ncol + 1) / 2, kThetaThreads, sm, st, (const C *)ring, (C *)X, p.fM, p.fN1,
                           (const T *)p.w1, (const T *)p.w2, p.ntheta, p.lmax, p.mmax, p.spin, p.ncol, p.r_lo, p.R,
                           chunk);
    };
    if constexpr (sizeof(T) == 4)
        if (p.cl_theta == 1 && sm <= kTwoCtaSmem) return args(k_theta_fwd<T, 1, 2>);
    return p.cl_theta == 4 ? args(k_theta_fwd<T, 4>) : p.cl_theta == 2 ? args(k_theta_fwd<T, 2>) : args(k_theta_fwd<T, 1>);
}

template <typename T>
cudaError_t theta_adj_t(const Plan &p, const void *X, void *ring, cudaStream_t st)
{
    using C = cplx<T>;
    const size_t sm = theta_smem_bytes(p);
    const int chunk = (int)(sm / sizeof(C));
    auto args = [&](auto kern) {
        return launch_team(kern, p.cl_theta, (p.ncol + 1) / 2, kThetaThreads, sm, st, (const C *)X, (C *)ring, p.fM, p.fN1,
                           (const T *)p.w1, (const T *)p.w2, p.ntheta, p.lmax, p.mmax, p.spin, p.ncol, p.r_lo, p.R,
                           chunk);
    };
    if constexpr (sizeof(T) == 4)
        if (p.cl_theta == 1 && sm <= kTwoCtaSmem) return args(k_theta_adj<T, 1, 2>);
    return p.cl_theta == 4 ? args(k_theta_adj<T, 4>) : p.cl_theta == 2 ? args(k_theta_adj<T, 2>) : args(k_theta_adj<T, 1>);
}

template <typename T, bool SPIN>
cudaError_t phi_fwd_t(const Plan &p, const void *X, void *grid, cudaStream_t st)
{
    using C = cplx<T>;
    const size_t sm = phi_smem_bytes(p);
    const int chunk = (int)(sm / sizeof(C));
    const int nvec = SPIN ? p.R : (p.R + 1) / 2;
    auto args = [&](auto kern) {
        // FP64 plans with point weights interpolate in double-float: the grid as double-float pairs
        return launch_team(kern, p.cl_phi, nvec, phi_threads(p), sm, st, (const C *)X, grid, p.fN2, p.mmax, p.ncol,
                           p.R, p.pitch, p.W, chunk, (sizeof(T) == 8 && p.wts && p.wts_dd) ? 1 : 0);
    };
    if constexpr (sizeof(T) == 4)
        if (p.cl_phi == 1 && sm <= kTwoCtaSmem) return args(k_phi_fwd<T, SPIN, 1, 2>);
    return p.cl_phi == 4   ? args(k_phi_fwd<T, SPIN, 4>)
           : p.cl_phi == 2 ? args(k_phi_fwd<T, SPIN, 2>)
                           : args(k_phi_fwd<T, SPIN, 1>);
}

template <typename T, bool SPIN>
cudaError_t phi_adj_t(const Plan &p, const void *grid, void *X, cudaStream_t st)
{
    using C = cplx<T>;
    const size_t sm = phi_smem_bytes(p);
    const int chunk = (int)(sm / sizeof(C));
    const int nvec = SPIN ? p.R : (p.R + 1) / 2;
    auto args = [&](auto kern) {
        return launch_team(kern, p.cl_phi, nvec, phi_threads(p), sm, st, (const void *)grid, (C *)X, p.fN2, p.mmax,
                           p.ncol, p.R, p.pitch, p.W, chunk);
    };
    if constexpr (sizeof(T) == 4)
        if (p.cl_phi == 1 && sm <= kTwoCtaSmem) return args(k_phi_adj<T, SPIN, 1, 2>);
    return p.cl_phi == 4   ? args(k_phi_adj<T, SPIN, 4>)
           : p.cl_phi == 2 ? args(k_phi_adj<T, SPIN, 2>)
                           : args(k_phi_adj<T, SPIN, 1>);
}

}  // namespace

cudaError_t launch_theta_fwd(const Plan &p, const void *ring, void *X, cudaStream_t st)
{
    return p.prec == LENS_FP32 ? theta_fwd_t<float>(p, ring, X, st) : theta_fwd_t<double>(p, ring, X, st);
}

cudaError_t launch_theta_coeffs(const Plan &p, const void *ring, void *out, cudaStream_t st)
{
    if (p.cl_theta != 1) return cudaErrorNotSupported;
    const size_t sm = theta_smem_bytes(p);
    if (p.prec == LENS_FP32) {
        cudaError_t e = cudaFuncSetAttribute(k_theta_coeffs<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        k_theta_coeffs<float><<<p.ncol, kThetaThreads, sm, st>>>((const float2 *)ring, (float2 *)out, p.fM, p.ntheta,
                                                                p.lmax, p.mmax, p.spin);
    } else {
        cudaError_t e = cudaFuncSetAttribute(k_theta_coeffs<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        k_theta_coeffs<double><<<p.ncol, kThetaThreads, sm, st>>>((const double2 *)ring, (double2 *)out, p.fM,
                                                                 p.ntheta, p.lmax, p.mmax, p.spin);
    }
    return cudaGetLastError();
}

cudaError_t launch_theta_adj(const Plan &p, const void *X, void *ring, cudaStream_t st)
{
    return p.prec == LENS_FP32 ? theta_adj_t<float>(p, X, ring, st) : theta_adj_t<double>(p, X, ring, st);
}

cudaError_t launch_phi_fwd(const Plan &p, const void *X, void *grid, cudaStream_t st)
{
    if (p.prec == LENS_FP32) return p.spin ? phi_fwd_t<float, true>(p, X, grid, st) : phi_fwd_t<float, false>(p, X, grid, st);
    return p.spin ? phi_fwd_t<double, true>(p, X, grid, st) : phi_fwd_t<double, false>(p, X, grid, st);
}

cudaError_t launch_phi_adj(const Plan &p, const void *grid, void *X, cudaStream_t st)
{
    if (p.prec == LENS_FP32) return p.spin ? phi_adj_t<float, true>(p, grid, X, st) : phi_adj_t<float, false>(p, grid, X, st);
    return p.spin ? phi_adj_t<double, true>(p, grid, X, st) : phi_adj_t<double, false>(p, grid, X, st);
}

}  // namespace gsl
