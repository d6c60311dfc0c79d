// Quadrature grids, per-point weights and the magnification determinant.
//
// Lensed harmonic coefficients (Sect. 4): the lensed field is remapped onto
// an intermediate grid and sent back to harmonic space with a standard SHT.
// On a Gauss-Legendre grid (n rings at the roots of P_n, nphi equispaced
// longitudes) the backward SHT is the adjoint transform at the grid points
// applied to the map times the quadrature weights w_j 2 pi / nphi, exact for
// band limits below n.  lens_gl_grid builds the points and weights,
// lens_scale_points applies per-point weights.
//
// Inverse lensing (App. B): the adjoint applied to T |A|, with the
// magnification determinant
//   |A| = (sin a / a) ((1 - kappa)^2 + omega^2 - |gamma|^2)
//       + (cos a - sin a / a) (1 - kappa - cos(2 beta) gamma_1 - sin(2 beta) gamma_2),
// kappa + i omega = ethbar(1alpha) / 2 and gamma_1 + i gamma_2 = eth(1alpha) / 2,
// a = |alpha| and beta the angle of alpha from e_theta towards e_phi.  For a
// deflection that is the gradient of phi (1alpha = -eth phi) omega = 0,
//   kappa = spin-0 synthesis of l(l+1)/2 phi_lm,
//   gamma = spin-2 synthesis (P = -sum (G + iC) 2Y) of G = sqrt((l-1)l(l+1)(l+2))/2 phi_lm, C = 0.
#include <cuda_runtime.h>
#include <math.h>

#include <string>
#include <vector>
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace gsl {
namespace {

constexpr double kPiG = 3.141592653589793238462643383280;

__device__ __forceinline__ int64_t alm_base_g(int lmax, int m) { return (int64_t)m * (2 * lmax + 1 - m) / 2; }

// Gauss-Legendre nodes x_j (descending: theta ascending) and weights on the host
void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w)
{
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = cos(kPiG * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
        }
        x[i] = z;
        x[n - 1 - i] = -z;
        w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
    if (n & 1) x[n / 2] = 0.0;
}

__global__ void k_fill_grid(const double *__restrict__ th_r, const double *__restrict__ w_r, int nrings, int nphi,
                            double *__restrict__ th, double *__restrict__ ph, double *__restrict__ w)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)nrings * nphi) return;
    const int r = (int)(i / nphi), k = (int)(i - (int64_t)r * nphi);
    th[i] = th_r[r];
    ph[i] = 2.0 * kPiG * k / nphi;
    if (w) w[i] = w_r[r] * (2.0 * kPiG / nphi);
}

template <typename T>
__global__ void k_scale_points(int64_t n, int ncomp, const double *__restrict__ wt, const T *__restrict__ in,
                               T *__restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double f = wt[i];
    for (int c = 0; c < ncomp; ++c) out[c * n + i] = (T)(f * (double)in[c * n + i]);
}

// coefficient maps of the magnification: kappa (spin 0) and gamma (spin-2 G)
__global__ void k_lens_fields(const double2 *__restrict__ phi, double2 *__restrict__ kap, double2 *__restrict__ gam,
                              int lmax, int64_t nalm)
{
    const int m = blockIdx.y;
    const int64_t base = alm_base_g(lmax, m);
    for (int l = m + blockIdx.x * blockDim.x + threadIdx.x; l <= lmax; l += gridDim.x * blockDim.x) {
        const int64_t i = base + l;
        const double L = l;
        const double2 a = phi[i];
        const double fk = 0.5 * L * (L + 1.0);
        const double fg = 0.5 * sqrt(fmax((L - 1.0) * L * (L + 1.0) * (L + 2.0), 0.0));
        kap[i] = make_double2(fk * a.x, fk * a.y);
        gam[i] = make_double2(fg * a.x, fg * a.y);
        gam[nalm + i] = make_double2(0.0, 0.0);
    }
}

__global__ void k_det(int64_t n, const double *__restrict__ alpha, const double *__restrict__ kap,
                      const double *__restrict__ gam, double *__restrict__ det)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double at = alpha[i], ap = alpha[n + i];
    const double a = hypot(at, ap);
    const double k = kap[i], g1 = gam[i], g2 = gam[n + i];
    const double sa = a > 0.0 ? sin(a) / a : 1.0;
    double c2b = 1.0, s2b = 0.0;
    if (a > 0.0) {  // cos 2 beta, sin 2 beta from the direction of alpha
        const double ct = at / a, st = ap / a;
        c2b = ct * ct - st * st;
        s2b = 2.0 * ct * st;
    }
    const double cma = a > 0.0 ? cos(a) - sa : 0.0;
    det[i] = sa * ((1.0 - k) * (1.0 - k) - (g1 * g1 + g2 * g2)) + cma * (1.0 - k - c2b * g1 - s2b * g2);
}

int gerr(cudaError_t e, const char *where)
{
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return record_failure(e == cudaErrorMemoryAllocation ? LENS_ERR_NOMEM : LENS_ERR_CUDA, m.c_str());
}

}  // namespace
}  // namespace gsl

using namespace gsl;

extern "C" {

int lens_gl_grid(int nrings, int nphi, double *theta_d, double *phi_d, double *weight_d, void *stream)
{
    if (nrings < 1 || nphi < 1 || !theta_d || !phi_d)
        return record_failure(LENS_ERR_INVALID, "lens_gl_grid: bad sizes or NULL buffer");
    std::vector<double> x, w;
    gauss_legendre(nrings, x, w);
    std::vector<double> th(nrings);
    for (int j = 0; j < nrings; ++j) th[j] = acos(x[j]);
    cudaStream_t st = (cudaStream_t)stream;
    double *d_th = nullptr, *d_w = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&d_th, sizeof(double) * nrings, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&d_w, sizeof(double) * nrings, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_th, th.data(), sizeof(double) * nrings, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_w, w.data(), sizeof(double) * nrings, cudaMemcpyHostToDevice, st);
    const int64_t n = (int64_t)nrings * nphi;
    if (e == cudaSuccess) {
        k_fill_grid<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(d_th, d_w, nrings, nphi, theta_d, phi_d, weight_d);
        e = cudaGetLastError();
    }
    // the host vectors must outlive the copies
    const cudaError_t e2 = cudaStreamSynchronize(st);
    cudaFreeAsync(d_th, st);
    cudaFreeAsync(d_w, st);
    if (e == cudaSuccess) e = e2;
    return e == cudaSuccess ? LENS_OK : gerr(e, "lens_gl_grid");
}

int lens_scale_points(int64_t n, int ncomp, int prec, const double *weight_d, const void *in_d, void *out_d,
                      void *stream)
{
    if (n < 0 || ncomp < 1 || (prec != LENS_FP32 && prec != LENS_FP64))
        return record_failure(LENS_ERR_INVALID, "lens_scale_points: bad n, ncomp or precision");
    if (n == 0) return LENS_OK;
    if (!weight_d || !in_d || !out_d) return record_failure(LENS_ERR_INVALID, "lens_scale_points: NULL buffer");
    cudaStream_t st = (cudaStream_t)stream;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    if (prec == LENS_FP32)
        k_scale_points<float><<<blocks, 256, 0, st>>>(n, ncomp, weight_d, (const float *)in_d, (float *)out_d);
    else
        k_scale_points<double><<<blocks, 256, 0, st>>>(n, ncomp, weight_d, (const double *)in_d, (double *)out_d);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LENS_OK : gerr(e, "lens_scale_points");
}

int lens_magnification(lens_plan p0, lens_plan p2, const void *phi_lm_d, const double *alpha_d, double *det_d,
                       void *stream)
{
    if (!p0 || !p2 || !phi_lm_d || !alpha_d || !det_d)
        return record_failure(LENS_ERR_INVALID, "lens_magnification: NULL argument");
    const Plan &a = *reinterpret_cast<const Plan *>(p0), &b = *reinterpret_cast<const Plan *>(p2);
    if (a.spin != 0 || b.spin != 2 || a.prec != LENS_FP64 || b.prec != LENS_FP64 || a.lmax != b.lmax ||
        a.mmax != b.mmax || a.npts != b.npts || a.device != b.device)
        return record_failure(LENS_ERR_INVALID,
                              "lens_magnification: needs FP64 spin-0 and spin-2 plans on the same points and band limit");
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != a.device) cudaSetDevice(a.device);
    cudaStream_t st = stream ? (cudaStream_t)stream : a.stream;
    void *kc = nullptr, *gc = nullptr, *km = nullptr, *gm = nullptr;
    cudaError_t e = cudaMallocAsync(&kc, sizeof(double2) * (size_t)a.nalm, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&gc, 2 * sizeof(double2) * (size_t)a.nalm, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&km, sizeof(double) * (size_t)std::max<int64_t>(a.npts, 1), st);
    if (e == cudaSuccess) e = cudaMallocAsync(&gm, 2 * sizeof(double) * (size_t)std::max<int64_t>(a.npts, 1), st);
    int rc = LENS_OK;
    if (e == cudaSuccess) {
        k_lens_fields<<<dim3(4, a.mmax + 1), 256, 0, st>>>((const double2 *)phi_lm_d, (double2 *)kc, (double2 *)gc,
                                                           a.lmax, a.nalm);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) rc = run_forward(a, kc, km, st, 1.0);
    if (e == cudaSuccess && rc == LENS_OK) rc = run_forward(b, gc, gm, st, 1.0);
    if (e == cudaSuccess && rc == LENS_OK && a.npts > 0) {
        k_det<<<(unsigned)((a.npts + 255) / 256), 256, 0, st>>>(a.npts, alpha_d, (const double *)km,
                                                                (const double *)gm, det_d);
        e = cudaGetLastError();
    }
    cudaFreeAsync(kc, st);
    cudaFreeAsync(gc, st);
    cudaFreeAsync(km, st);
    cudaFreeAsync(gm, st);
    if (prev >= 0 && prev != a.device) cudaSetDevice(prev);
    if (rc != LENS_OK) return rc;
    return e == cudaSuccess ? LENS_OK : gerr(e, "lens_magnification");
}

}  // extern "C"
