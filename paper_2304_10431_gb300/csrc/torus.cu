// Torus steps of the general SHT (Sect. 3 "doubling" and "FFT", and their
// adjoints "FFT" and "undoubling").
//
// Forward, per m column (theta kernel):
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

__device__ __forceinline__ int pmod(int a, int n)
{
    int r = a % n;
    return r < 0 ? r + n : r;
}

// ----------------------------------------------------------------- theta fwd
template <typename T>
__global__ void __launch_bounds__(1024) k_theta_fwd(const cplx<T> *__restrict__ ring, cplx<T> *__restrict__ X,
                                                    FftDesc fM, FftDesc fN1, const T *__restrict__ w1,
                                                    const T *__restrict__ w2, int ntheta, int lmax, int mmax,
                                                    int spin, int ncol, int r_lo, int R)
{
    using C = cplx<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = reinterpret_cast<C *>(smem_raw);
    const int c = blockIdx.x;
    const int mc = spin == 0 ? c : c - mmax;
    const T par = ((mc + spin) & 1) ? T(-1) : T(1);
    const int M = fM.n, N1 = fN1.n;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const C *F = ring + (int64_t)c * ntheta;

    for (int i = tid; i < M; i += nthr) {
        C v = i < ntheta ? F[i] : cscale(F[M - i], par);
        buf[__ldg(fM.perm + i)] = v;
    }
    __syncthreads();
    fft_smem<-1, T>(buf, fM);  // natural order c_k * M

    // move k < 0 from M + k to N1 + k (top first: never overwrites an unread
    // source, since N1 >= M), scaling every kept k by w1(k) w2(m)
    const T wm = w2[c];
    for (int k0 = -1; k0 >= -lmax; k0 -= nthr) {
        const int k = k0 - tid;
        C v = mkc(T(0), T(0));
        if (k >= -lmax) v = cscale(buf[M + k], w1[k + lmax] * wm);
        __syncthreads();
        if (k >= -lmax) buf[N1 + k] = v;
        __syncthreads();
    }
    for (int k = tid; k <= lmax; k += nthr) buf[k] = cscale(buf[k], w1[k + lmax] * wm);
    for (int i = lmax + 1 + tid; i < N1 - lmax; i += nthr) buf[i] = mkc(T(0), T(0));
    __syncthreads();
    fft_smem_dif<+1, T>(buf, fN1);  // y_r at position perm_N1[r]

    for (int rr = tid; rr < R; rr += nthr) {
        const int r = pmod(r_lo + rr, N1);
        X[(int64_t)rr * ncol + c] = buf[__ldg(fN1.perm + r)];
    }
}

// ----------------------------------------------------------------- theta adj
template <typename T>
__global__ void __launch_bounds__(1024) k_theta_adj(const cplx<T> *__restrict__ X, cplx<T> *__restrict__ ring,
                                                    FftDesc fM, FftDesc fN1, const T *__restrict__ w1,
                                                    const T *__restrict__ w2, int ntheta, int lmax, int mmax,
                                                    int spin, int ncol, int r_lo, int R)
{
    using C = cplx<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = reinterpret_cast<C *>(smem_raw);
    const int c = blockIdx.x;
    const int mc = spin == 0 ? c : c - mmax;
    const T par = ((mc + spin) & 1) ? T(-1) : T(1);
    const int M = fM.n, N1 = fN1.n;
    const int tid = threadIdx.x, nthr = blockDim.x;

    for (int i = tid; i < N1; i += nthr) buf[i] = mkc(T(0), T(0));
    __syncthreads();
    for (int rr = tid; rr < R; rr += nthr) {
        const int r = pmod(r_lo + rr, N1);
        buf[__ldg(fN1.perm + r)] = X[(int64_t)rr * ncol + c];
    }
    __syncthreads();
    fft_smem<-1, T>(buf, fN1);  // natural order

    // move k < 0 from N1 + k down to M + k (lowest first), scale by w1 w2
    const T wm = w2[c];
    for (int k0 = -lmax; k0 <= -1; k0 += nthr) {
        const int k = k0 + tid;
        C v = mkc(T(0), T(0));
        if (k <= -1) v = cscale(buf[N1 + k], w1[k + lmax] * wm);
        __syncthreads();
        if (k <= -1) buf[M + k] = v;
        __syncthreads();
    }
    for (int k = tid; k <= lmax; k += nthr) buf[k] = cscale(buf[k], w1[k + lmax] * wm);
    for (int i = lmax + 1 + tid; i < M - lmax; i += nthr) buf[i] = mkc(T(0), T(0));
    __syncthreads();
    fft_smem_dif<+1, T>(buf, fM);  // H_j at position perm_M[j]

    C *F = ring + (int64_t)c * ntheta;
    for (int j = tid; j < ntheta; j += nthr) {
        C v = buf[__ldg(fM.perm + j)];
        if (j > 0 && j < ntheta - 1) v = cadd(v, cscale(buf[__ldg(fM.perm + (M - j))], par));
        F[j] = v;
    }
}

// ------------------------------------------------------------------- phi fwd
// spin 0: CTA = row pair (2b, 2b+1); spin s: CTA = one row.
template <typename T, bool SPIN>
__global__ void __launch_bounds__(512) k_phi_fwd(const cplx<T> *__restrict__ X, void *__restrict__ grid,
                                                 FftDesc fN2, int mmax, int ncol, int R, int pitch, int W)
{
    using C = cplx<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = reinterpret_cast<C *>(smem_raw);
    const int N2 = fN2.n;
    const int tid = threadIdx.x, nthr = blockDim.x;
    for (int i = tid; i < N2; i += nthr) buf[i] = mkc(T(0), T(0));
    __syncthreads();
    if (!SPIN) {
        const int ra = 2 * blockIdx.x, rb = ra + 1;
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
        __syncthreads();
        fft_smem<+1, T>(buf, fN2);
        T *ga = (T *)grid + (int64_t)ra * pitch;
        T *gb = (T *)grid + (int64_t)rb * pitch;
        for (int c = tid; c < N2 + W - 1; c += nthr) {
            C v = buf[c < N2 ? c : c - N2];
            ga[c] = v.x;
            if (hb) gb[c] = v.y;
        }
    } else {
        const int r = blockIdx.x;
        const C *xr = X + (int64_t)r * ncol;
        for (int i = tid; i < ncol; i += nthr) {
            const int m = i - mmax;
            buf[__ldg(fN2.perm + pmod(m, N2))] = xr[i];
        }
        __syncthreads();
        fft_smem<+1, T>(buf, fN2);
        C *gr = (C *)grid + (int64_t)r * pitch;
        for (int c = tid; c < N2 + W - 1; c += nthr) gr[c] = buf[c < N2 ? c : c - N2];
    }
}

// ------------------------------------------------------------------- phi adj
template <typename T, bool SPIN>
__global__ void __launch_bounds__(512) k_phi_adj(const void *__restrict__ grid, cplx<T> *__restrict__ X,
                                                 FftDesc fN2, int mmax, int ncol, int R, int pitch, int W)
{
    using C = cplx<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = reinterpret_cast<C *>(smem_raw);
    const int N2 = fN2.n;
    const int tid = threadIdx.x, nthr = blockDim.x;
    if (!SPIN) {
        const int ra = 2 * blockIdx.x, rb = ra + 1;
        const bool hb = rb < R;
        const T *ga = (const T *)grid + (int64_t)ra * pitch;
        const T *gb = (const T *)grid + (int64_t)rb * pitch;
        for (int c = tid; c < N2; c += nthr) {
            T a = ga[c], b = hb ? gb[c] : T(0);
            if (c < W - 1) { a += ga[N2 + c]; if (hb) b += gb[N2 + c]; }
            buf[__ldg(fN2.perm + c)] = mkc(a, b);
        }
        __syncthreads();
        fft_smem<-1, T>(buf, fN2);
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
        const int r = blockIdx.x;
        const C *gr = (const C *)grid + (int64_t)r * pitch;
        for (int c = tid; c < N2; c += nthr) {
            C v = gr[c];
            if (c < W - 1) v = cadd(v, gr[N2 + c]);
            buf[__ldg(fN2.perm + c)] = v;
        }
        __syncthreads();
        fft_smem<-1, T>(buf, fN2);
        C *xr = X + (int64_t)r * ncol;
        for (int i = tid; i < ncol; i += nthr) {
            const int m = i - mmax;
            xr[i] = buf[pmod(m, N2)];
        }
    }
}

template <typename T> size_t csz() { return sizeof(cplx<T>); }

}  // namespace

size_t theta_smem_bytes(const Plan &p) { return (size_t)(p.N1 > p.M ? p.N1 : p.M) * (p.prec == LENS_FP32 ? 8 : 16); }
size_t phi_smem_bytes(const Plan &p) { return (size_t)p.N2 * (p.prec == LENS_FP32 ? 8 : 16); }

static int theta_threads(const Plan &p) { return p.prec == LENS_FP32 ? 512 : 512; }
static int phi_threads(const Plan &p) { return p.prec == LENS_FP32 ? 512 : 256; }

template <typename T> static cudaError_t set_smem(const void *fn, size_t bytes)
{
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t launch_theta_fwd(const Plan &p, const void *ring, void *X, cudaStream_t st)
{
    const size_t sm = theta_smem_bytes(p);
    if (p.prec == LENS_FP32) {
        cudaError_t e = set_smem<float>((const void *)k_theta_fwd<float>, sm);
        if (e != cudaSuccess) return e;
        k_theta_fwd<float><<<p.ncol, theta_threads(p), sm, st>>>(
            (const float2 *)ring, (float2 *)X, p.fM, p.fN1, (const float *)p.w1, (const float *)p.w2, p.ntheta,
            p.lmax, p.mmax, p.spin, p.ncol, p.r_lo, p.R);
    } else {
        cudaError_t e = set_smem<double>((const void *)k_theta_fwd<double>, sm);
        if (e != cudaSuccess) return e;
        k_theta_fwd<double><<<p.ncol, theta_threads(p), sm, st>>>(
            (const double2 *)ring, (double2 *)X, p.fM, p.fN1, (const double *)p.w1, (const double *)p.w2, p.ntheta,
            p.lmax, p.mmax, p.spin, p.ncol, p.r_lo, p.R);
    }
    return cudaGetLastError();
}

cudaError_t launch_theta_adj(const Plan &p, const void *X, void *ring, cudaStream_t st)
{
    const size_t sm = theta_smem_bytes(p);
    if (p.prec == LENS_FP32) {
        cudaError_t e = set_smem<float>((const void *)k_theta_adj<float>, sm);
        if (e != cudaSuccess) return e;
        k_theta_adj<float><<<p.ncol, theta_threads(p), sm, st>>>(
            (const float2 *)X, (float2 *)ring, p.fM, p.fN1, (const float *)p.w1, (const float *)p.w2, p.ntheta,
            p.lmax, p.mmax, p.spin, p.ncol, p.r_lo, p.R);
    } else {
        cudaError_t e = set_smem<double>((const void *)k_theta_adj<double>, sm);
        if (e != cudaSuccess) return e;
        k_theta_adj<double><<<p.ncol, theta_threads(p), sm, st>>>(
            (const double2 *)X, (double2 *)ring, p.fM, p.fN1, (const double *)p.w1, (const double *)p.w2,
            p.ntheta, p.lmax, p.mmax, p.spin, p.ncol, p.r_lo, p.R);
    }
    return cudaGetLastError();
}

cudaError_t launch_phi_fwd(const Plan &p, const void *X, void *grid, cudaStream_t st)
{
    const size_t sm = phi_smem_bytes(p);
    const int nblk = p.spin ? p.R : (p.R + 1) / 2;
    cudaError_t e;
    if (p.prec == LENS_FP32) {
        if (p.spin) {
            if ((e = set_smem<float>((const void *)k_phi_fwd<float, true>, sm)) != cudaSuccess) return e;
            k_phi_fwd<float, true><<<nblk, phi_threads(p), sm, st>>>((const float2 *)X, grid, p.fN2, p.mmax, p.ncol,
                                                                     p.R, p.pitch, p.W);
        } else {
            if ((e = set_smem<float>((const void *)k_phi_fwd<float, false>, sm)) != cudaSuccess) return e;
            k_phi_fwd<float, false><<<nblk, phi_threads(p), sm, st>>>((const float2 *)X, grid, p.fN2, p.mmax,
                                                                      p.ncol, p.R, p.pitch, p.W);
        }
    } else {
        if (p.spin) {
            if ((e = set_smem<double>((const void *)k_phi_fwd<double, true>, sm)) != cudaSuccess) return e;
            k_phi_fwd<double, true><<<nblk, phi_threads(p), sm, st>>>((const double2 *)X, grid, p.fN2, p.mmax,
                                                                      p.ncol, p.R, p.pitch, p.W);
        } else {
            if ((e = set_smem<double>((const void *)k_phi_fwd<double, false>, sm)) != cudaSuccess) return e;
            k_phi_fwd<double, false><<<nblk, phi_threads(p), sm, st>>>((const double2 *)X, grid, p.fN2, p.mmax,
                                                                       p.ncol, p.R, p.pitch, p.W);
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_phi_adj(const Plan &p, const void *grid, void *X, cudaStream_t st)
{
    const size_t sm = phi_smem_bytes(p);
    const int nblk = p.spin ? p.R : (p.R + 1) / 2;
    cudaError_t e;
    if (p.prec == LENS_FP32) {
        if (p.spin) {
            if ((e = set_smem<float>((const void *)k_phi_adj<float, true>, sm)) != cudaSuccess) return e;
            k_phi_adj<float, true><<<nblk, phi_threads(p), sm, st>>>(grid, (float2 *)X, p.fN2,
                                                                     p.mmax, p.ncol, p.R, p.pitch, p.W);
        } else {
            if ((e = set_smem<float>((const void *)k_phi_adj<float, false>, sm)) != cudaSuccess) return e;
            k_phi_adj<float, false><<<nblk, phi_threads(p), sm, st>>>(grid, (float2 *)X, p.fN2, p.mmax, p.ncol, p.R, p.pitch, p.W);
        }
    } else {
        if (p.spin) {
            if ((e = set_smem<double>((const void *)k_phi_adj<double, true>, sm)) != cudaSuccess) return e;
            k_phi_adj<double, true><<<nblk, phi_threads(p), sm, st>>>(grid, (double2 *)X, p.fN2, p.mmax, p.ncol, p.R,
                                                                      p.pitch, p.W);
        } else {
            if ((e = set_smem<double>((const void *)k_phi_adj<double, false>, sm)) != cudaSuccess) return e;
            k_phi_adj<double, false><<<nblk, phi_threads(p), sm, st>>>(grid, (double2 *)X, p.fN2, p.mmax, p.ncol, p.R,
                                                                       p.pitch, p.W);
        }
    }
    return cudaGetLastError();
}

}  // namespace gsl
