// Differentiation with respect to the lensing potential.
//
// The forward model (Sect. 2 Eq. "deflect", the pointing formula of Sect. 3
// and the spin phase chi of Fig. 1, then Eq. "forward" / "forwardpol") is
//   alpha = spin-1 synthesis of G = sqrt(L(L+1)) phi_LM, C = 0 at the points n,
//   n' = exp_n(alpha),  P = Q + iU = e^{i s chi} sf(n').
// For a real loss with g = dL/dQ + i dL/dU (dL/dT for spin 0), the chain rule
// in the frame of n parallel-transported along the geodesic gives per point
//   dL/dalpha = J Y + K i ah,  Y = -1/2 [conj(g) A + g conj(B)],
//   K = -s c Im(conj(g) P),
// with a = |alpha|, ah = alpha / a, J = ah ah^T + (sin a / a)(1 - ah ah^T)
// the derivative of the exponential map, c = (1 - cos a) / a the holonomy of
// the transport, A = e^{i(s+1)chi} (eth sf)(n') and B = e^{i(s-1)chi}
// (ethbar sf)(n') the spin-raised and -lowered lensed syntheses (spin 0:
// B = conj A).  Then dL/dphi_LM = sqrt(L(L+1)) * (G part of the spin-1
// transform's gradient at n).  Every step below runs in the library's
// kernels; the lensed maps are recomputed rather than stored.
#include <cuda_runtime.h>
#include <math.h>

#include <string>
#include <type_traits>

#include "common.cuh"
#include "internal.h"

namespace gsl {
namespace {

__device__ __forceinline__ int64_t base_of(int lmax, int m) { return (int64_t)m * (2 * lmax + 1 - m) / 2; }

// eth (lower = 0) or ethbar (lower = 1) of a field of spin s as coefficients of
// a spin s +- 1 field in the convention sf = -sum (G + iC) sY:
//   s = 0 (f = sum a Y):  eth  -> G' = -sqrt(l(l+1)) a, C' = 0
//   s >= 1:               eth  -> (G', C') =  sqrt((l-s)(l+s+1)) (G, C)
//   s >= 2:               ethbar -> (G', C') = -sqrt((l+s)(l-s+1)) (G, C)
template <typename C>
__global__ void k_eth(const C *__restrict__ in, C *__restrict__ out, int lmax, int spin, int lower, int64_t nalm)
{
    const int m = blockIdx.y;
    const int64_t base = base_of(lmax, m);
    for (int l = m + blockIdx.x * blockDim.x + threadIdx.x; l <= lmax; l += gridDim.x * blockDim.x) {
        const int64_t i = base + l;
        const double L = l, s = spin;
        double f;
        if (spin == 0) f = -sqrt(L * (L + 1.0));
        else if (lower) f = -sqrt(fmax((L + s) * (L - s + 1.0), 0.0));
        else f = sqrt(fmax((L - s) * (L + s + 1.0), 0.0));
        using R = typename std::remove_const<typename std::remove_reference<decltype(in[0].x)>::type>::type;
        const C a = in[i];
        out[i] = mkc((R)(f * a.x), (R)(f * a.y));
        if (spin == 0) {
            out[nalm + i] = C{};
        } else {
            const C b = in[nalm + i];
            out[nalm + i] = mkc((R)(f * b.x), (R)(f * b.y));
        }
    }
}

// G = sqrt(L(L+1)) phi, C = 0 (Eq. "deflect" as a spin-1 forward operator)
__global__ void k_phi_to_g(const double2 *__restrict__ phi, double2 *__restrict__ out, int lmax, int64_t nalm)
{
    const int m = blockIdx.y;
    const int64_t base = base_of(lmax, m);
    for (int l = m + blockIdx.x * blockDim.x + threadIdx.x; l <= lmax; l += gridDim.x * blockDim.x) {
        const int64_t i = base + l;
        const double f = sqrt((double)l * (l + 1.0));
        const double2 a = phi[i];
        out[i] = make_double2(f * a.x, f * a.y);
        out[nalm + i] = make_double2(0.0, 0.0);
    }
}

// dL/dphi = sqrt(L(L+1)) dL/dG
__global__ void k_g_to_phi(const double2 *__restrict__ gg, double2 *__restrict__ out, int lmax)
{
    const int m = blockIdx.y;
    const int64_t base = base_of(lmax, m);
    for (int l = m + blockIdx.x * blockDim.x + threadIdx.x; l <= lmax; l += gridDim.x * blockDim.x) {
        const int64_t i = base + l;
        const double f = sqrt((double)l * (l + 1.0));
        const double2 a = gg[i];
        out[i] = make_double2(f * a.x, f * a.y);
    }
}

// dL/dalpha per point (FP64 arithmetic; inputs in the lensed plans' type T):
// alpha [2][n], g / p [ncomp][n], A / B [2][n]; out [2][n] (theta, phi parts).
template <typename T>
__global__ void k_deflection_vjp(int64_t n, int spin, const double *__restrict__ alpha, const T *__restrict__ g,
                                 const T *__restrict__ p, const T *__restrict__ A, const T *__restrict__ B,
                                 double *__restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double at = alpha[i], ap = alpha[n + i];
    const double a = hypot(at, ap);
    double hr = 1.0, hi = 0.0, k = 1.0, c = 0.0;
    if (a > 0.0) {
        hr = at / a;
        hi = ap / a;
        k = sin(a) / a;
        const double sh = sin(0.5 * a);
        c = 2.0 * sh * sh / a;
    }
    const double ar = A[i], ai = A[n + i];
    double yr, yi, K = 0.0;
    if (spin == 0) {
        const double gv = g[i];
        yr = -gv * ar;
        yi = -gv * ai;
    } else {
        const double gq = g[i], gu = g[n + i];
        const double br = B[i], bi = B[n + i];
        // conj(g) A + g conj(B)
        const double sr = (gq * ar + gu * ai) + (gq * br + gu * bi);
        const double si = (gq * ai - gu * ar) + (gu * br - gq * bi);
        yr = -0.5 * sr;
        yi = -0.5 * si;
        const double pr = p[i], pi = p[n + i];
        K = -spin * c * (gq * pi - gu * pr);
    }
    const double par = hr * yr + hi * yi;
    const double jr = par * hr + k * (yr - par * hr);
    const double ji = par * hi + k * (yi - par * hi);
    out[i] = jr - K * hi;
    out[n + i] = ji + K * hr;
}

const Plan *as_plan(lens_plan p) { return reinterpret_cast<const Plan *>(p); }

// stream-ordered scratch, released on destruction (on the same stream)
struct Scratch {
    cudaStream_t st;
    void *ptr[8] = {nullptr};
    int n = 0;
    explicit Scratch(cudaStream_t s) : st(s) {}
    cudaError_t get(void **out, size_t bytes)
    {
        cudaError_t e = cudaMallocAsync(out, bytes > 0 ? bytes : 16, st);
        if (e == cudaSuccess) ptr[n++] = *out;
        return e;
    }
    ~Scratch()
    {
        for (int i = 0; i < n; ++i) cudaFreeAsync(ptr[i], st);
    }
};

int cuda_err(cudaError_t e, const char *where)
{
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return record_failure(e == cudaErrorMemoryAllocation ? LENS_ERR_NOMEM : LENS_ERR_CUDA, m.c_str());
}

struct DevSwitch {
    int prev = -1;
    explicit DevSwitch(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DevSwitch()
    {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace
}  // namespace gsl

using namespace gsl;

extern "C" {

int lens_alm_eth(int lmax, int mmax, int spin, int lower, int prec, const void *alm_in_d, void *alm_out_d,
                 void *stream)
{
    if (lmax < 0 || mmax < 0 || mmax > lmax || spin < 0 || (prec != LENS_FP32 && prec != LENS_FP64))
        return record_failure(LENS_ERR_INVALID, "lens_alm_eth: bad lmax, mmax, spin or precision");
    if (lower && spin < 2)
        return record_failure(LENS_ERR_UNSUPPORTED, "lens_alm_eth: ethbar needs spin >= 2 (result spin >= 1)");
    if (!alm_in_d || !alm_out_d) return record_failure(LENS_ERR_INVALID, "lens_alm_eth: NULL buffer");
    const int64_t nalm = (int64_t)(mmax + 1) * (lmax + 1) - (int64_t)mmax * (mmax + 1) / 2;
    const dim3 grid(4, mmax + 1);
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == LENS_FP32)
        k_eth<float2><<<grid, 256, 0, st>>>((const float2 *)alm_in_d, (float2 *)alm_out_d, lmax, spin, lower, nalm);
    else
        k_eth<double2><<<grid, 256, 0, st>>>((const double2 *)alm_in_d, (double2 *)alm_out_d, lmax, spin, lower, nalm);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LENS_OK : cuda_err(e, "lens_alm_eth");
}

int lens_deflection(lens_plan defl, const void *phi_lm_d, double *alpha_d, void *stream)
{
    if (!defl || !phi_lm_d || (!alpha_d && as_plan(defl)->npts > 0))
        return record_failure(LENS_ERR_INVALID, "lens_deflection: NULL argument");
    const Plan &p = *as_plan(defl);
    if (p.spin != 1 || p.prec != LENS_FP64)
        return record_failure(LENS_ERR_INVALID, "lens_deflection: needs an FP64 spin-1 plan");
    DevSwitch g(p.device);
    cudaStream_t st = stream ? (cudaStream_t)stream : p.stream;
    Scratch sc(st);
    void *gc = nullptr;
    cudaError_t e = sc.get(&gc, 2 * (size_t)p.nalm * sizeof(double2));
    if (e != cudaSuccess) return cuda_err(e, "lens_deflection: scratch");
    k_phi_to_g<<<dim3(4, p.mmax + 1), 256, 0, st>>>((const double2 *)phi_lm_d, (double2 *)gc, p.lmax, p.nalm);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_err(e, "lens_deflection");
    return run_forward(p, gc, alpha_d, st, 1.0);
}

int lens_phi_gradient(lens_plan lensed, lens_plan lensed_up, lens_plan lensed_down, lens_plan defl,
                      const double *alpha_d, const void *x_alm_d, const void *map_d, const void *grad_map_d,
                      void *grad_phi_d, void *stream)
{
    if (!lensed || !lensed_up || !defl || !alpha_d || !x_alm_d || !grad_map_d || !grad_phi_d)
        return record_failure(LENS_ERR_INVALID, "lens_phi_gradient: NULL argument");
    const Plan &p = *as_plan(lensed), &pu = *as_plan(lensed_up), &pd = *as_plan(defl);
    const int s = p.spin;
    if (s == 1)
        return record_failure(LENS_ERR_UNSUPPORTED, "lens_phi_gradient: spin 1 fields are not supported");
    if (pu.spin != s + 1 || pd.spin != 1 || pd.prec != LENS_FP64 || pu.prec != p.prec || pu.lmax != p.lmax ||
        pu.mmax != p.mmax || pu.npts != p.npts || pd.npts != p.npts || pu.device != p.device || pd.device != p.device)
        return record_failure(LENS_ERR_INVALID,
                              "lens_phi_gradient: lensed_up must be spin s+1 with the lensed plan's points, band "
                              "limit and precision; defl an FP64 spin-1 plan on the same points");
    if (p.grad || pu.grad)
        return record_failure(LENS_ERR_INVALID, "lens_phi_gradient: lensed plans must not be LENS_GRAD_ONLY");
    const Plan *pdn = nullptr;
    if (s >= 2) {
        if (!lensed_down) return record_failure(LENS_ERR_INVALID, "lens_phi_gradient: spin s >= 2 needs lensed_down");
        pdn = as_plan(lensed_down);
        if (pdn->spin != s - 1 || pdn->grad || pdn->prec != p.prec || pdn->lmax != p.lmax || pdn->mmax != p.mmax ||
            pdn->npts != p.npts || pdn->device != p.device)
            return record_failure(LENS_ERR_INVALID, "lens_phi_gradient: lensed_down must be spin s-1 like lensed");
    }
    DevSwitch g(p.device);
    cudaStream_t st = stream ? (cudaStream_t)stream : p.stream;
    const size_t rsz = p.prec == LENS_FP32 ? 4 : 8, csz = 2 * rsz;
    const int64_t n = p.npts;
    Scratch sc(st);
    void *coef = nullptr, *A = nullptr, *B = nullptr, *map = nullptr, *ga = nullptr, *gg = nullptr;
    cudaError_t e;
    if ((e = sc.get(&coef, 2 * (size_t)p.nalm * csz)) != cudaSuccess ||
        (e = sc.get(&A, 2 * (size_t)n * rsz)) != cudaSuccess ||
        (s >= 2 && (e = sc.get(&B, 2 * (size_t)n * rsz)) != cudaSuccess) ||
        (!map_d && (e = sc.get(&map, (s ? 2 : 1) * (size_t)n * rsz)) != cudaSuccess) ||
        (e = sc.get(&ga, 2 * (size_t)n * sizeof(double))) != cudaSuccess ||
        (e = sc.get(&gg, 2 * (size_t)pd.nalm * sizeof(double2))) != cudaSuccess)
        return cuda_err(e, "lens_phi_gradient: scratch");
    int rc;
    if (!map_d) {
        if ((rc = run_forward(p, x_alm_d, map, st, 1.0)) != LENS_OK) return rc;
        map_d = map;
    }
    if ((rc = lens_alm_eth(p.lmax, p.mmax, s, 0, p.prec, x_alm_d, coef, st)) != LENS_OK) return rc;
    if ((rc = run_forward(pu, coef, A, st, 1.0)) != LENS_OK) return rc;
    if (s >= 2) {
        if ((rc = lens_alm_eth(p.lmax, p.mmax, s, 1, p.prec, x_alm_d, coef, st)) != LENS_OK) return rc;
        if ((rc = run_forward(*pdn, coef, B, st, 1.0)) != LENS_OK) return rc;
    }
    const unsigned blocks = (unsigned)((n + 255) / 256);
    if (n > 0) {
        if (p.prec == LENS_FP32)
            k_deflection_vjp<float><<<blocks, 256, 0, st>>>(n, s, alpha_d, (const float *)grad_map_d,
                                                             (const float *)map_d, (const float *)A,
                                                             (const float *)B, (double *)ga);
        else
            k_deflection_vjp<double><<<blocks, 256, 0, st>>>(n, s, alpha_d, (const double *)grad_map_d,
                                                              (const double *)map_d, (const double *)A,
                                                              (const double *)B, (double *)ga);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_err(e, "lens_phi_gradient: deflection vjp");
    }
    if ((rc = run_adjoint(pd, ga, gg, st, 2.0)) != LENS_OK) return rc;
    k_g_to_phi<<<dim3(4, pd.mmax + 1), 256, 0, st>>>((const double2 *)gg, (double2 *)grad_phi_d, pd.lmax);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_err(e, "lens_phi_gradient");
    return LENS_OK;
}

}  // extern "C"
