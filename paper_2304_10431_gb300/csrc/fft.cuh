// Shared-memory mixed-radix FFT used by the torus transforms (Sect. 3 "FFT").
//
// One CTA transforms one vector held in shared memory.  The algorithm is the
// iterative decimation-in-time Cooley-Tukey scheme: the input is stored in
// digit-reversed order (element i at position perm[i]); stage k combines
// r_k sub-transforms of length L_{k-1} into length L_k = L_{k-1} r_k with
// twiddles W_{L_k}^{j q}; the output comes out in natural order.  Within a
// stage the butterflies touch disjoint positions, so one barrier per stage
// suffices.  Radices 2, 3, 4, 5, 7, 8; odd radices use the symmetric-pair
// form y_k = x_0 + sum_q (x_q + x_{p-q}) cos(2 pi qk/p) -+ i (x_q - x_{p-q}) sin(2 pi qk/p);
// FP32 transforms also use the composite radices 6, 9, 14 and 21 (two small
// DFTs in registers per stage, fewer shared-memory passes).
//
// DIR = -1: forward, sum x_n e^{-2 pi i nk/N};  DIR = +1: inverse (unnormalised).
//
// Vectors longer than one CTA's shared memory are split over a cluster of
// two or four CTAs (Blackwell distributed shared memory): elements
// [r chunk, (r+1) chunk) live in rank r's shared memory, the butterflies of
// all CTAs address any part through the cluster's shared window, and the
// stage barrier is a cluster barrier.  Team<CL> and Buf<C, CL> hide the
// difference; CL = 1 is the plain single-CTA path.
#pragma once

#include <cooperative_groups.h>
#include <type_traits>

#include "common.cuh"
#include "internal.h"

namespace gsl {

// The threads that share one vector: one CTA (CL = 1) or a cluster of two.
template <int CL> struct Team;
template <> struct Team<1> {
    int tid, nthr;
    __device__ Team() : tid(threadIdx.x), nthr(blockDim.x) {}
    __device__ __forceinline__ void sync() const { __syncthreads(); }
    __device__ __forceinline__ int vec() const { return blockIdx.x; }
};
template <int CL> struct Team {  // CL = 2 or 4: a cluster of CL CTAs
    static_assert(CL == 2 || CL == 4, "teams of 1, 2 or 4 CTAs");
    int tid, nthr;
    __device__ Team()
    {
        const int rank = (int)cooperative_groups::this_cluster().block_rank();
        tid = rank * blockDim.x + threadIdx.x;
        nthr = CL * blockDim.x;
    }
    __device__ __forceinline__ void sync() const { cooperative_groups::this_cluster().sync(); }
    __device__ __forceinline__ int vec() const { return blockIdx.x / CL; }
};

// Element access of the vector: a shared-memory array, or two halves.
template <typename C, int CL> struct Buf;
template <typename C> struct Buf<C, 1> {
    C *p;
    __device__ explicit Buf(C *local) : p(local) {}
    __device__ __forceinline__ C &operator[](int i) const { return p[i]; }
};
// One CTA, padded (theta transforms, FP32): one element skipped after every
// 16 (index i + i/16), so that the stride-2 butterfly accesses of the first
// stages do not put two lanes of a half-warp on the same banks (measured:
// theta transforms 5-7% faster; the phi transforms, whose rows are read and
// written in natural order, gain nothing and keep the plain buffer).  Size:
// fft_smem_elems(n, 8).
template <typename C> struct PadBuf {
    C *p;
    __device__ explicit PadBuf(C *local) : p(local) {}
    __device__ __forceinline__ C &operator[](int i) const { return p[i + (i >> 4)]; }
};

template <typename C> struct Buf<C, 2> {
    C *p0, *p1;
    int chunk;
    __device__ Buf(C *local, int chunk_) : chunk(chunk_)
    {
        auto cl = cooperative_groups::this_cluster();
        p0 = cl.map_shared_rank(local, 0);
        p1 = cl.map_shared_rank(local, 1);
    }
    __device__ __forceinline__ C &operator[](int i) const { return i < chunk ? p0[i] : p1[i - chunk]; }
};
template <typename C> struct Buf<C, 4> {
    C *p0, *p1, *p2, *p3;
    int chunk;
    __device__ Buf(C *local, int chunk_) : chunk(chunk_)
    {
        auto cl = cooperative_groups::this_cluster();
        p0 = cl.map_shared_rank(local, 0);
        p1 = cl.map_shared_rank(local, 1);
        p2 = cl.map_shared_rank(local, 2);
        p3 = cl.map_shared_rank(local, 3);
    }
    __device__ __forceinline__ C &operator[](int i) const
    {
        if (i < 2 * chunk) return i < chunk ? p0[i] : p1[i - chunk];
        return i < 3 * chunk ? p2[i - 2 * chunk] : p3[i - 3 * chunk];
    }
};

template <typename T> struct FftConst;
#define GSL_FFT_CONSTS(T)                                                                                  \
    template <> struct FftConst<T> {                                                                       \
        static __device__ __forceinline__ T c3() { return T(-0.5); }                                       \
        static __device__ __forceinline__ T s3() { return T(0.866025403784438646764); }                     \
        static __device__ __forceinline__ T c5(int t)                                                      \
        {                                                                                                  \
            return (t == 1 || t == 4) ? T(0.309016994374947424102) : T(-0.809016994374947424102);         \
        }                                                                                                  \
        static __device__ __forceinline__ T s5(int t)                                                      \
        {                                                                                                  \
            return t == 1 ? T(0.951056516295153572116)                                                     \
                          : t == 2 ? T(0.587785252292473129169)                                            \
                                   : t == 3 ? T(-0.587785252292473129169) : T(-0.951056516295153572116);   \
        }                                                                                                  \
        static __device__ __forceinline__ T c7(int t)                                                      \
        {                                                                                                  \
            return (t == 1 || t == 6) ? T(0.623489801858733530525)                                         \
                                      : (t == 2 || t == 5) ? T(-0.222520933956314404289)                   \
                                                           : T(-0.900968867902419126236);                  \
        }                                                                                                  \
        static __device__ __forceinline__ T s7(int t)                                                      \
        {                                                                                                  \
            return t == 1 ? T(0.781831482468029808708)                                                     \
                          : t == 2 ? T(0.974927912181823607018)                                            \
                                   : t == 3 ? T(0.433883739117558120476)                                   \
                                            : t == 4 ? T(-0.433883739117558120476)                         \
                                                     : t == 5 ? T(-0.974927912181823607018)                \
                                                              : T(-0.781831482468029808708);               \
        }                                                                                                  \
        static __device__ __forceinline__ T r2() { return T(0.707106781186547524401); }                    \
    };
GSL_FFT_CONSTS(float)
GSL_FFT_CONSTS(double)
#undef GSL_FFT_CONSTS

// multiply by -i (DIR=-1) or +i (DIR=+1)
template <int DIR, typename C> __device__ __forceinline__ C mul_dir_i(C a)
{
    return DIR < 0 ? cmul_mi(a) : cmul_i(a);
}

template <int R, int DIR, typename T> struct SmallDft;

template <int DIR, typename T> struct SmallDft<2, DIR, T> {
    static __device__ __forceinline__ void run(cplx<T> *x)
    {
        cplx<T> a = x[0], b = x[1];
        x[0] = cadd(a, b);
        x[1] = csub(a, b);
    }
};

template <int DIR, typename T> struct SmallDft<4, DIR, T> {
    static __device__ __forceinline__ void run(cplx<T> *x)
    {
        cplx<T> s02 = cadd(x[0], x[2]), d02 = csub(x[0], x[2]);
        cplx<T> s13 = cadd(x[1], x[3]), d13 = mul_dir_i<DIR>(csub(x[1], x[3]));
        x[0] = cadd(s02, s13);
        x[2] = csub(s02, s13);
        x[1] = cadd(d02, d13);
        x[3] = csub(d02, d13);
    }
};

template <int DIR, typename T> struct SmallDft<8, DIR, T> {
    static __device__ __forceinline__ void run(cplx<T> *x)
    {
        cplx<T> e[4] = {x[0], x[2], x[4], x[6]};
        cplx<T> o[4] = {x[1], x[3], x[5], x[7]};
        SmallDft<4, DIR, T>::run(e);
        SmallDft<4, DIR, T>::run(o);
        const T r = FftConst<T>::r2();
        // W8^1 = (1 + DIR i) r,  W8^2 = DIR i,  W8^3 = (-1 + DIR i) r
        cplx<T> t1 = mkc(r * (o[1].x - DIR * o[1].y), r * (o[1].y + DIR * o[1].x));
        cplx<T> t2 = mul_dir_i<DIR>(o[2]);
        cplx<T> t3 = mkc(r * (-o[3].x - DIR * o[3].y), r * (-o[3].y + DIR * o[3].x));
        x[0] = cadd(e[0], o[0]);
        x[4] = csub(e[0], o[0]);
        x[1] = cadd(e[1], t1);
        x[5] = csub(e[1], t1);
        x[2] = cadd(e[2], t2);
        x[6] = csub(e[2], t2);
        x[3] = cadd(e[3], t3);
        x[7] = csub(e[3], t3);
    }
};

template <int DIR, typename T> struct SmallDft<3, DIR, T> {
    static __device__ __forceinline__ void run(cplx<T> *x)
    {
        cplx<T> s = cadd(x[1], x[2]), d = csub(x[1], x[2]);
        cplx<T> a = mkc(x[0].x + FftConst<T>::c3() * s.x, x[0].y + FftConst<T>::c3() * s.y);
        cplx<T> b = cscale(d, FftConst<T>::s3());
        // forward: y1 = a - i b, y2 = a + i b
        cplx<T> ib = mul_dir_i<DIR>(b);  // DIR=-1: -i b
        x[0] = cadd(x[0], s);
        x[1] = cadd(a, ib);
        x[2] = csub(a, ib);
    }
};

template <int P, int DIR, typename T> struct OddDft {
    static __device__ __forceinline__ T cs(int t) { return P == 5 ? FftConst<T>::c5(t) : FftConst<T>::c7(t); }
    static __device__ __forceinline__ T sn(int t) { return P == 5 ? FftConst<T>::s5(t) : FftConst<T>::s7(t); }
    static __device__ __forceinline__ void run(cplx<T> *x)
    {
        constexpr int H = (P - 1) / 2;
        cplx<T> s[H], d[H];
        cplx<T> y0 = x[0];
#pragma unroll
        for (int q = 1; q <= H; ++q) {
            s[q - 1] = cadd(x[q], x[P - q]);
            d[q - 1] = csub(x[q], x[P - q]);
            y0 = cadd(y0, s[q - 1]);
        }
        cplx<T> out[P];
        out[0] = y0;
#pragma unroll
        for (int k = 1; k <= H; ++k) {
            cplx<T> a = x[0], b = mkc(T(0), T(0));
#pragma unroll
            for (int q = 1; q <= H; ++q) {
                const int t = (q * k) % P;
                const T c = cs(t), sv = sn(t);
                a.x += c * s[q - 1].x; a.y += c * s[q - 1].y;
                b.x += sv * d[q - 1].x; b.y += sv * d[q - 1].y;
            }
            cplx<T> ib = mul_dir_i<DIR>(b);
            out[k] = cadd(a, ib);
            out[P - k] = csub(a, ib);
        }
#pragma unroll
        for (int k = 0; k < P; ++k) x[k] = out[k];
    }
};
template <int DIR, typename T> struct SmallDft<5, DIR, T> {
    static __device__ __forceinline__ void run(cplx<T> *x) { OddDft<5, DIR, T>::run(x); }
};
template <int DIR, typename T> struct SmallDft<7, DIR, T> {
    static __device__ __forceinline__ void run(cplx<T> *x) { OddDft<7, DIR, T>::run(x); }
};

// cos (sine = false) or sin of 2 pi t / R, t < R, for the composite radices
template <int R> __host__ __device__ constexpr double root_cs(int t, bool sine)
{
    if (R == 6) {
        constexpr double c[6] = {1.00000000000000000000, 0.50000000000000011102, -0.49999999999999977796, -1.00000000000000000000, -0.50000000000000044409, 0.50000000000000011102};
        constexpr double s[6] = {0.00000000000000000000, 0.86602540378443859659, 0.86602540378443870761, 0.00000000000000012246, -0.86602540378443837454, -0.86602540378443859659};
        return sine ? s[t] : c[t];
    }
    if (R == 9) {
        constexpr double c[9] = {1.00000000000000000000, 0.76604444311897801345, 0.17364817766693041445, -0.49999999999999977796, -0.93969262078590831688, -0.93969262078590842791, -0.50000000000000044409, 0.17364817766692997036, 0.76604444311897779141};
        constexpr double s[9] = {0.00000000000000000000, 0.64278760968653925190, 0.98480775301220802032, 0.86602540378443870761, 0.34202014332566887944, -0.34202014332566865740, -0.86602540378443837454, -0.98480775301220813134, -0.64278760968653958496};
        return sine ? s[t] : c[t];
    }
    if (R == 14) {
        constexpr double c[14] = {1.00000000000000000000, 0.90096886790241914600, 0.62348980185873359439, 0.22252093395631444839, -0.22252093395631433737, -0.62348980185873348336, -0.90096886790241903498, -1.00000000000000000000, -0.90096886790241914600, -0.62348980185873370541, -0.22252093395631458717, 0.22252093395631333816, 0.62348980185873337234, 0.90096886790241936804};
        constexpr double s[14] = {0.00000000000000000000, 0.43388373911755812040, 0.78183148246802980363, 0.97492791218182361934, 0.97492791218182361934, 0.78183148246802991466, 0.43388373911755823142, 0.00000000000000012246, -0.43388373911755800938, -0.78183148246802969261, -0.97492791218182361934, -0.97492791218182384139, -0.78183148246802991466, -0.43388373911755750978};
        return sine ? s[t] : c[t];
    }
    if (R == 21) {
        constexpr double c[21] = {1.00000000000000000000, 0.95557280578614067768, 0.82623877431599490606, 0.62348980185873359439, 0.36534102436639498412, 0.07473009358642439259, -0.22252093395631433737, -0.49999999999999977796, -0.73305187182982634031, -0.90096886790241903498, -0.98883082622512852300, -0.98883082622512863402, -0.90096886790241914600, -0.73305187182982622929, -0.50000000000000044409, -0.22252093395631458717, 0.07473009358642436484, 0.36534102436639537270, 0.62348980185873337234, 0.82623877431599446197, 0.95557280578614056665};
        constexpr double s[21] = {0.00000000000000000000, 0.29475517441090420823, 0.56332005806362206446, 0.78183148246802980363, 0.93087374864420424636, 0.99720379718118012935, 0.97492791218182361934, 0.86602540378443870761, 0.68017273777091935560, 0.43388373911755823142, 0.14904226617617472028, -0.14904226617617402639, -0.43388373911755800938, -0.68017273777091946663, -0.86602540378443837454, -0.97492791218182361934, -0.99720379718118012935, -0.93087374864420413534, -0.78183148246802991466, -0.56332005806362273059, -0.29475517441090470783};
        return sine ? s[t] : c[t];
    }
    return 0.0;
}

// Composite radix R = P Q in registers (Cooley-Tukey with n = Q n1 + n2,
// k = k1 + P k2): Q DFTs of length P, twiddles W_R^(n2 k1), P DFTs of length
// Q.  One shared-memory pass instead of two.
template <int P, int Q, int DIR, typename T> struct CompositeDft {
    static __device__ __forceinline__ void run(cplx<T> *x)
    {
        constexpr int R = P * Q;
        cplx<T> y[Q][P];
#pragma unroll
        for (int n2 = 0; n2 < Q; ++n2) {
            cplx<T> t[P];
#pragma unroll
            for (int n1 = 0; n1 < P; ++n1) t[n1] = x[Q * n1 + n2];
            SmallDft<P, DIR, T>::run(t);
#pragma unroll
            for (int k1 = 0; k1 < P; ++k1) {
                if (n2 > 0 && k1 > 0) {
                    const int e = (n2 * k1) % R;
                    const T c = (T)root_cs<R>(e, false), s = (T)(DIR * root_cs<R>(e, true));
                    t[k1] = mkc(t[k1].x * c - t[k1].y * s, t[k1].x * s + t[k1].y * c);
                }
                y[n2][k1] = t[k1];
            }
        }
#pragma unroll
        for (int k1 = 0; k1 < P; ++k1) {
            cplx<T> u[Q];
#pragma unroll
            for (int n2 = 0; n2 < Q; ++n2) u[n2] = y[n2][k1];
            SmallDft<Q, DIR, T>::run(u);
#pragma unroll
            for (int k2 = 0; k2 < Q; ++k2) x[k1 + P * k2] = u[k2];
        }
    }
};
template <int DIR, typename T> struct SmallDft<6, DIR, T> {
    static __device__ __forceinline__ void run(cplx<T> *x) { CompositeDft<2, 3, DIR, T>::run(x); }
};
template <int DIR, typename T> struct SmallDft<9, DIR, T> {
    static __device__ __forceinline__ void run(cplx<T> *x) { CompositeDft<3, 3, DIR, T>::run(x); }
};
template <int DIR, typename T> struct SmallDft<14, DIR, T> {
    static __device__ __forceinline__ void run(cplx<T> *x) { CompositeDft<2, 7, DIR, T>::run(x); }
};
template <int DIR, typename T> struct SmallDft<21, DIR, T> {
    static __device__ __forceinline__ void run(cplx<T> *x) { CompositeDft<3, 7, DIR, T>::run(x); }
};

// x[q] *= w^q (DIR = -1) or conj(w)^q (DIR = +1) for q = 1 .. R-1, w = W_L^j
// = tw[e] with e = j N / L.  FP32: w read once and its powers formed by
// multiplication (q - 1 products, a few ulp; measured 5-8% faster torus
// transforms than one table read per power).  FP64: one table read per power
// (the products would run on the narrow FP64 pipe: measured 15% slower).
template <int R, int DIR, typename T>
__device__ __forceinline__ void twiddle(cplx<T> (&x)[R], const cplx<T> *__restrict__ tw, int64_t e)
{
    if constexpr (std::is_same<T, float>::value) {
        const cplx<T> w1 = __ldg(tw + e);
        cplx<T> w = w1;
#pragma unroll
        for (int q = 1; q < R; ++q) {
            x[q] = DIR < 0 ? cmul(x[q], w) : cmulc(x[q], w);
            if (q + 1 < R) w = cmul(w, w1);
        }
    } else {
#pragma unroll
        for (int q = 1; q < R; ++q) {
            const cplx<T> w = __ldg(tw + e * q);
            x[q] = DIR < 0 ? cmul(x[q], w) : cmulc(x[q], w);
        }
    }
}

// Butterfly b = g Lp + j of a stage, for b = tid, tid + nthr, ...: (g, j) are
// stepped by (nthr / Lp, nthr % Lp) with one carry instead of a division per
// butterfly.
struct BflyIndex {
    int g, j, dg, dj, Lp;
    __device__ __forceinline__ BflyIndex(int tid, int nthr, int Lp_) : Lp(Lp_)
    {
        g = tid / Lp;
        j = tid - g * Lp;
        dg = nthr / Lp;
        dj = nthr - dg * Lp;
    }
    __device__ __forceinline__ void next()
    {
        g += dg;
        j += dj;
        if (j >= Lp) {
            j -= Lp;
            ++g;
        }
    }
};

template <int R, int DIR, typename T, class B>
__device__ __forceinline__ void fft_stage(const B &buf, int N, int Lp, const cplx<T> *__restrict__ tw, int tid,
                                          int nthr)
{
    const int L = Lp * R;
    const int nb = N / R;
    const int tstep = N / L;
    BflyIndex ix(tid, nthr, Lp);
    for (int b = tid; b < nb; b += nthr, ix.next()) {
        const int g = ix.g;
        const int j = ix.j;
        const int base = g * L + j;
        cplx<T> x[R];
#pragma unroll
        for (int q = 0; q < R; ++q) x[q] = buf[base + q * Lp];
        if (j != 0) twiddle<R, DIR, T>(x, tw, (int64_t)j * tstep);
        SmallDft<R, DIR, T>::run(x);
#pragma unroll
        for (int q = 0; q < R; ++q) buf[base + q * Lp] = x[q];
    }
}

// Full transform of buf (digit-reversed input -> natural output).  Ends with
// a barrier of the team.
template <int DIR, typename T, int CL, class B>
__device__ void fft_smem(const B &buf, const FftDesc &d, const Team<CL> &tm)
{
    const cplx<T> *tw = (const cplx<T> *)d.tw;
    int Lp = 1;
    for (int st = 0; st < d.nst; ++st) {
        const int r = d.radix[st];
        switch (r) {
        case 2: fft_stage<2, DIR, T>(buf, d.n, Lp, tw, tm.tid, tm.nthr); break;
        case 3: fft_stage<3, DIR, T>(buf, d.n, Lp, tw, tm.tid, tm.nthr); break;
        case 4: fft_stage<4, DIR, T>(buf, d.n, Lp, tw, tm.tid, tm.nthr); break;
        case 5: fft_stage<5, DIR, T>(buf, d.n, Lp, tw, tm.tid, tm.nthr); break;
        case 7: fft_stage<7, DIR, T>(buf, d.n, Lp, tw, tm.tid, tm.nthr); break;
        case 6:
            if constexpr (std::is_same<T, float>::value) fft_stage<6, DIR, T>(buf, d.n, Lp, tw, tm.tid, tm.nthr);
            break;
        case 9:
            if constexpr (std::is_same<T, float>::value) fft_stage<9, DIR, T>(buf, d.n, Lp, tw, tm.tid, tm.nthr);
            break;
        case 14:
            if constexpr (std::is_same<T, float>::value) fft_stage<14, DIR, T>(buf, d.n, Lp, tw, tm.tid, tm.nthr);
            break;
        case 21:
            if constexpr (std::is_same<T, float>::value) fft_stage<21, DIR, T>(buf, d.n, Lp, tw, tm.tid, tm.nthr);
            break;
        default: fft_stage<8, DIR, T>(buf, d.n, Lp, tw, tm.tid, tm.nthr); break;
        }
        Lp *= r;
        tm.sync();
    }
}

template <int DIR, typename T> __device__ void fft_smem(cplx<T> *buf, const FftDesc &d)
{
    fft_smem<DIR, T, 1>(Buf<cplx<T>, 1>(buf), d, Team<1>());
}

// Decimation-in-frequency variant (the transpose of fft_smem): natural-order
// input, output element i at position perm[i].  Stages run in reverse order
// and the twiddles are applied after each small DFT.  Ends with a barrier.
template <int R, int DIR, typename T, class B>
__device__ __forceinline__ void fft_stage_dif(const B &buf, int N, int Lp, const cplx<T> *__restrict__ tw, int tid,
                                              int nthr)
{
    const int L = Lp * R;
    const int nb = N / R;
    const int tstep = N / L;
    BflyIndex ix(tid, nthr, Lp);
    for (int b = tid; b < nb; b += nthr, ix.next()) {
        const int g = ix.g;
        const int j = ix.j;
        const int base = g * L + j;
        cplx<T> x[R];
#pragma unroll
        for (int q = 0; q < R; ++q) x[q] = buf[base + q * Lp];
        SmallDft<R, DIR, T>::run(x);
        if (j != 0) twiddle<R, DIR, T>(x, tw, (int64_t)j * tstep);
#pragma unroll
        for (int q = 0; q < R; ++q) buf[base + q * Lp] = x[q];
    }
}

template <int DIR, typename T, int CL, class B>
__device__ void fft_smem_dif(const B &buf, const FftDesc &d, const Team<CL> &tm)
{
    const cplx<T> *tw = (const cplx<T> *)d.tw;
    int Lp = d.n;
    for (int st = d.nst - 1; st >= 0; --st) {
        const int r = d.radix[st];
        Lp /= r;
        switch (r) {
        case 2: fft_stage_dif<2, DIR, T>(buf, d.n, Lp, tw, tm.tid, tm.nthr); break;
        case 3: fft_stage_dif<3, DIR, T>(buf, d.n, Lp, tw, tm.tid, tm.nthr); break;
        case 4: fft_stage_dif<4, DIR, T>(buf, d.n, Lp, tw, tm.tid, tm.nthr); break;
        case 5: fft_stage_dif<5, DIR, T>(buf, d.n, Lp, tw, tm.tid, tm.nthr); break;
        case 7: fft_stage_dif<7, DIR, T>(buf, d.n, Lp, tw, tm.tid, tm.nthr); break;
        case 6:
            if constexpr (std::is_same<T, float>::value) fft_stage_dif<6, DIR, T>(buf, d.n, Lp, tw, tm.tid, tm.nthr);
            break;
        case 9:
            if constexpr (std::is_same<T, float>::value) fft_stage_dif<9, DIR, T>(buf, d.n, Lp, tw, tm.tid, tm.nthr);
            break;
        case 14:
            if constexpr (std::is_same<T, float>::value) fft_stage_dif<14, DIR, T>(buf, d.n, Lp, tw, tm.tid, tm.nthr);
            break;
        case 21:
            if constexpr (std::is_same<T, float>::value) fft_stage_dif<21, DIR, T>(buf, d.n, Lp, tw, tm.tid, tm.nthr);
            break;
        default: fft_stage_dif<8, DIR, T>(buf, d.n, Lp, tw, tm.tid, tm.nthr); break;
        }
        tm.sync();
    }
}

template <int DIR, typename T> __device__ void fft_smem_dif(cplx<T> *buf, const FftDesc &d)
{
    fft_smem_dif<DIR, T, 1>(Buf<cplx<T>, 1>(buf), d, Team<1>());
}

}  // namespace gsl
