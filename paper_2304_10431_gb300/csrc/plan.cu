// Plan creation and the C ABI of libgslens (see include/gslens.h).
//
// Plan-time work (Sect. 4: excluded from the timed transform because the
// geometry is shared by many maps): grid sizes, the accuracy heuristic
// epsilon -> (sigma, W, beta), recursion-coefficient and ring tables, kernel
// deconvolution factors, FFT descriptors, and the sorted point tables.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace gsl {
int legendre_rpt(int prec, int spin, bool adjoint, bool rst);
int legendre_rpt_dd(int spin, bool adjoint);
bool legendre_rpt_supported(int prec, int spin, bool adjoint, int rpt, bool rst);
}

using namespace gsl;

namespace {

thread_local int g_last_status = LENS_OK;
thread_local char g_last_msg[512] = "";

int fail(int status, const std::string &msg)
{
    g_last_status = status;
    snprintf(g_last_msg, sizeof(g_last_msg), "%s", msg.c_str());
    return status;
}

int cuda_fail(cudaError_t e, const char *where)
{
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(e == cudaErrorMemoryAllocation ? LENS_ERR_NOMEM : LENS_ERR_CUDA, m);
}

constexpr double kPi = 3.141592653589793238462643383280;
constexpr size_t kSmemLimit = 227 * 1024;

bool smooth7(int n)
{
    if (n < 1) return false;
    for (int p : {2, 3, 5, 7})
        while (n % p == 0) n /= p;
    return n == 1;
}

int good_even(int n)
{
    if (n < 2) n = 2;
    if (n & 1) ++n;
    while (!smooth7(n)) n += 2;
    return n;
}

// ES kernel and its Fourier transform by Gauss-Legendre quadrature after
// z = (W/2) sin t, which removes the square-root endpoint behaviour:
//   psihat(xi) = W/2 int_{-pi/2}^{pi/2} exp(beta (cos t - 1)) cos(xi W/2 sin t) cos t dt
struct Quad {
    std::vector<double> x, w;
    explicit Quad(int n)
    {
        x.resize(n);
        w.resize(n);
        for (int i = 0; i < n; ++i) {  // Newton on P_n
            double z = cos(kPi * (i + 0.75) / (n + 0.5));
            for (int it = 0; it < 100; ++it) {
                double p0 = 1.0, p1 = z;
                for (int k = 2; k <= n; ++k) {
                    double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                    p0 = p1;
                    p1 = p2;
                }
                double dp = n * (z * p1 - p0) / (z * z - 1.0);
                double dz = p1 / dp;
                z -= dz;
                if (fabs(dz) < 1e-16) break;
            }
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            double dp = n * (z * p1 - p0) / (z * z - 1.0);
            x[i] = z;
            w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
        }
    }
};

double psihat(const Quad &q, double xi, int W, double beta)
{
    // integrate over t in [0, pi/2] (even integrand), nodes mapped from [-1, 1]
    double s = 0.0;
    const double h = 0.25 * kPi;
    for (size_t i = 0; i < q.x.size(); ++i) {
        const double t = h * (q.x[i] + 1.0);
        s += q.w[i] * exp(beta * (cos(t) - 1.0)) * cos(xi * 0.5 * W * sin(t)) * cos(t);
    }
    return 2.0 * 0.5 * W * h * s;
}

// FP32 plans: each tap's kernel weight phi(x) = exp(beta (sqrt(1 - x^2) - 1)), |x| < 1, with
// x = (t/2 + (W - 1)/2 - a) 2/W, as a polynomial in t in [-1, 1]: interpolated at the W + 2
// Chebyshev points of the first kind (coefficients c_k = (2 - [k = 0])/N sum_j y_j cos(pi k (j +
// 1/2)/N)) and rewritten in powers of t through T_{k+1} = 2 t T_k - T_{k-1}.  The device then
// evaluates W + 1 fused multiply-adds per weight instead of a square root and an exponential.
// Measured in double on a fine grid: the interpolant stays within e^-beta of phi (the kernel's
// own truncation step at |x| = 1) for sigma >= 1.25 and every W, and FP32 Horner evaluation
// adds ~6e-8; all monomial coefficients are below 1 in magnitude.
void ker_poly_fit(int W, double beta, KerPoly &kp)
{
    const int N = W + 2;
    double y[kMaxW + 2], c[kMaxW + 2], mono[kMaxW + 2], tk[kMaxW + 2], tk1[kMaxW + 2], tn[kMaxW + 2];
    for (int i = 0; i < kMaxW * (kMaxW + 2); ++i) kp.c[i] = 0.f;
    for (int a = 0; a < W; ++a) {
        for (int j = 0; j < N; ++j) {
            const double t = cos(kPi * (j + 0.5) / N);
            const double x = (0.5 * t + 0.5 * (W - 1) - a) * 2.0 / W;
            const double q = 1.0 - x * x;
            y[j] = q > 0 ? exp(beta * (sqrt(q) - 1.0)) : 0.0;
        }
        for (int k = 0; k < N; ++k) {
            double sum = 0;
            for (int j = 0; j < N; ++j) sum += y[j] * cos(kPi * k * (j + 0.5) / N);
            c[k] = (k ? 2.0 : 1.0) * sum / N;
        }
        for (int k = 0; k < N; ++k) mono[k] = tk[k] = tk1[k] = 0.0;
        tk[0] = 1.0;   // T_0
        tk1[1] = 1.0;  // T_1
        mono[0] = c[0];
        mono[1] = c[1];
        for (int k = 2; k < N; ++k) {  // T_k = 2 t T_{k-1} - T_{k-2}
            for (int i = 0; i < N; ++i) tn[i] = (i ? 2.0 * tk1[i - 1] : 0.0) - tk[i];
            for (int i = 0; i < N; ++i) {
                tk[i] = tk1[i];
                tk1[i] = tn[i];
                mono[i] += c[k] * tn[i];
            }
        }
        for (int k = 0; k < N; ++k) kp.c[a * (W + 2) + k] = (float)mono[k];
    }
}

// Largest |polynomial - phi| over the taps (polynomials evaluated in double at 256 points
// of t per tap).  With the default beta = pi W (1 - 1/(2 sigma)), sigma <= 2.5, it stays
// within e^-beta; a beta far from it at small W can leave the interpolant well above that.
double ker_poly_error(int W, double beta, const KerPoly &kp)
{
    double err = 0;
    for (int a = 0; a < W; ++a)
        for (int i = 0; i < 256; ++i) {
            const double t = -1.0 + (i + 0.5) / 128.0;
            double v = kp.c[a * (W + 2) + W + 1];
            for (int k = W; k >= 0; --k) v = v * t + kp.c[a * (W + 2) + k];
            const double x = (0.5 * t + 0.5 * (W - 1) - a) * 2.0 / W, q = 1.0 - x * x;
            err = std::max(err, std::fabs(v - (q > 0 ? exp(beta * (sqrt(q) - 1.0)) : 0.0)));
        }
    return err;
}

// Kernel support for a target accuracy at oversampling sigma:
// smallest W with 3 exp(-pi W sqrt(1 - 1/sigma)) <= eps (Barnett et al.'s
// estimate with a safety factor measured against direct summation).
int support_for(double eps, double sigma)
{
    const double r = kPi * sqrt(1.0 - 1.0 / sigma);
    int W = (int)ceil(log(3.0 / eps) / r);
    return std::max(W, 4);
}

// Radices of an FFT stage sequence.  composite (FP32): pairs of small primes
// are fused into radices 21, 14, 9 and 6 where possible (one shared-memory
// pass each; fft.cuh), measured on the 7-smooth lengths of lmax 4096.
std::vector<int> factorize(int n, bool composite)
{
    std::vector<int> f;
    while (n % 8 == 0) { f.push_back(8); n /= 8; }
    if (n % 4 == 0) { f.push_back(4); n /= 4; }
    int a2 = 0, a3 = 0, a5 = 0, a7 = 0;
    if (n % 2 == 0) { a2 = 1; n /= 2; }
    while (n % 3 == 0) { ++a3; n /= 3; }
    while (n % 5 == 0) { ++a5; n /= 5; }
    while (n % 7 == 0) { ++a7; n /= 7; }
    if (composite) {
        for (; a3 > 0 && a7 > 0; --a3, --a7) f.push_back(21);
        for (; a2 > 0 && a7 > 0; --a2, --a7) f.push_back(14);
        for (; a3 > 1; a3 -= 2) f.push_back(9);
        for (; a2 > 0 && a3 > 0; --a2, --a3) f.push_back(6);
    }
    for (; a2 > 0; --a2) f.push_back(2);
    for (; a3 > 0; --a3) f.push_back(3);
    for (; a5 > 0; --a5) f.push_back(5);
    for (; a7 > 0; --a7) f.push_back(7);
    return f;
}

struct Builder {
    Plan &p;
    explicit Builder(Plan &pl) : p(pl) {}
    cudaError_t alloc(void **ptr, size_t bytes, bool work)
    {
        *ptr = nullptr;
        if (bytes == 0) bytes = 16;
        if (p.nallocs >= (int)(sizeof(p.allocs) / sizeof(p.allocs[0]))) return cudaErrorMemoryAllocation;
        cudaError_t e = cudaMalloc(ptr, bytes);
        if (e != cudaSuccess) return e;
        p.allocs[p.nallocs++] = *ptr;
        (work ? p.work_bytes : p.plan_bytes) += bytes;
        return cudaSuccess;
    }
    template <typename V> cudaError_t upload(void **ptr, const std::vector<V> &v)
    {
        cudaError_t e = alloc(ptr, v.size() * sizeof(V), false);
        if (e != cudaSuccess) return e;
        return cudaMemcpy(*ptr, v.data(), v.size() * sizeof(V), cudaMemcpyHostToDevice);
    }
    cudaError_t fft(FftDesc &d, int n)
    {
        d.n = n;
        std::vector<int> f = factorize(n, p.prec == LENS_FP32);
        d.nst = (int)f.size();
        for (int i = 0; i < d.nst; ++i) d.radix[i] = f[i];
        std::vector<int> perm(n);
        for (int i = 0; i < n; ++i) {
            int v = i, scale = n, pos = 0;
            for (int st = d.nst - 1; st >= 0; --st) {
                const int r = f[st];
                scale /= r;
                pos += (v % r) * scale;
                v /= r;
            }
            perm[i] = pos;
        }
        void *dp = nullptr;
        cudaError_t e = upload(&dp, perm);
        if (e != cudaSuccess) return e;
        d.perm = (const int *)dp;
        void *tw = nullptr;
        if (p.prec == LENS_FP32) {
            std::vector<float2> t(n);
            for (int i = 0; i < n; ++i) t[i] = make_float2((float)cos(2 * kPi * i / n), (float)-sin(2 * kPi * i / n));
            e = upload(&tw, t);
        } else {
            std::vector<double2> t(n);
            for (int i = 0; i < n; ++i) t[i] = make_double2(cos(2 * kPi * i / n), -sin(2 * kPi * i / n));
            e = upload(&tw, t);
        }
        d.tw = tw;
        return e;
    }
};

struct Choice {
    double sigma = 0, beta = 0;
    int W = 0, N1 = 0, N2 = 0;
    double cost = 1e300;
};

// Grid sizes for a given sigma / W (N1 >= M so the theta kernels can move
// coefficients in place; N1 >= 4W + 4 so the kept rows never alias).
void sizes_for(int lmax, int mmax, int M, double sigma, int W, int &N1, int &N2)
{
    N1 = good_even(std::max({(int)ceil(sigma * (2 * lmax + 2)), M, 4 * W + 4}));
    N2 = good_even(std::max({(int)ceil(sigma * (2 * mmax + 2)), 4 * W + 4}));
}

}  // namespace

int gsl::record_failure(int status, const char *msg) { return fail(status, msg); }

extern "C" {

int64_t lens_nalm(int lmax, int mmax)
{
    if (lmax < 0 || mmax < 0 || mmax > lmax) return 0;
    return (int64_t)(mmax + 1) * (2 * lmax + 2 - mmax) / 2;
}

int lens_kernel_poly(int W, double beta, float *coef)
{
    if (W < 4 || W > kMaxW || !(beta > 0) || !coef) return fail(LENS_ERR_INVALID, "W in [4, 16], beta > 0, coef");
    KerPoly kp;
    ker_poly_fit(W, beta, kp);
    for (int i = 0; i < W * (W + 2); ++i) coef[i] = kp.c[i];
    return LENS_OK;
}

const char *lens_status_string(int s)
{
    switch (s) {
    case LENS_OK: return "ok";
    case LENS_ERR_INVALID: return "invalid argument";
    case LENS_ERR_DOMAIN: return "coordinate outside the domain";
    case LENS_ERR_PRECISION: return "accuracy not reachable at this precision";
    case LENS_ERR_NOMEM: return "out of memory";
    case LENS_ERR_CUDA: return "CUDA error";
    case LENS_ERR_TIMEOUT: return "device wait timed out";
    case LENS_ERR_UNSUPPORTED: return "size not supported by this build";
    default: return "unknown status";
    }
}

int lens_get_last_error(void) { return g_last_status; }
const char *lens_last_error_message(void) { return g_last_msg; }
int lens_version(void) { return 100; }

}  // extern "C"

// Legendre tables of an FP32 plan (lens_plan_params.legendre_tables): the
// degree at which each ring's monic values become non-negligible, the row
// layout (prefix sums on the host, once per plan), then the values.  Returns
// a lens_status (the caller destroys the plan on failure).
static int build_legendre_tables(Plan &p, Builder &B)
{
    cudaStream_t st = p.stream;
    if (cudaError_t e0 = tab_shape(p); e0 != cudaSuccess) return cuda_fail(e0, "table kernel attributes");
    int *first = nullptr;
    int64_t *rowlen = nullptr;
    cudaError_t e;
    auto done = [&](cudaError_t err, const char *what) {
        cudaFree(first);
        cudaFree(rowlen);
        return err == cudaSuccess ? LENS_OK : cuda_fail(err, what);
    };
    if ((e = cudaMalloc(&first, sizeof(int) * (size_t)(p.mmax + 1) * p.nnorth)) != cudaSuccess) return done(e, "table scratch");
    if ((e = cudaMalloc(&rowlen, sizeof(int64_t) * (size_t)p.nalm)) != cudaSuccess) return done(e, "table scratch");
    if ((e = B.alloc((void **)&p.tab_lstart, sizeof(int) * (size_t)(p.mmax + 1) * p.tab_ng, false)) != cudaSuccess ||
        (e = B.alloc((void **)&p.tab_jlo, sizeof(int) * (size_t)p.nalm, false)) != cudaSuccess)
        return done(e, "table index");
    if ((e = launch_tab_first(p, first)) != cudaSuccess) return done(e, "table degrees");
    if ((e = launch_tab_rows(p, first, p.tab_lstart, p.tab_jlo, rowlen)) != cudaSuccess) return done(e, "table rows");
    std::vector<int64_t> base(p.nalm);
    std::vector<int> jlo(p.nalm);
    if ((e = cudaMemcpyAsync(base.data(), rowlen, sizeof(int64_t) * p.nalm, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(jlo.data(), p.tab_jlo, sizeof(int) * p.nalm, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return done(e, "table rows");
    int64_t off = 0;
    for (int64_t i = 0; i < p.nalm; ++i) {
        const int64_t len = base[i];
        base[i] = off - jlo[i];
        off += len;
    }
    void *d = nullptr;
    if ((e = B.upload(&d, base)) != cudaSuccess) return done(e, "table rows");
    p.tab_rowbase = (int64_t *)d;
    const size_t esz = p.spin ? 8 : 4;
    p.tab_bytes = (size_t)off * esz;
    if ((e = B.alloc((void **)&p.tab_v, p.tab_bytes, false)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(first);
        cudaFree(rowlen);
        return fail(LENS_ERR_NOMEM, "Legendre tables: " + std::to_string(p.tab_bytes >> 20) + " MiB not available");
    }
    if ((e = launch_tab_fill(p)) != cudaSuccess) return done(e, "table values");
    return done(cudaStreamSynchronize(st), "table values");
}

extern "C" {

int lens_plan_destroy(lens_plan pl)
{
    if (!pl) return LENS_OK;
    Plan *p = reinterpret_cast<Plan *>(pl);
    int dev0 = 0;
    cudaGetDevice(&dev0);
    cudaSetDevice(p->device);
    cudaStreamSynchronize(p->stream);
    for (int i = 0; i < p->nallocs; ++i) cudaFree(p->allocs[i]);
    cudaSetDevice(dev0);
    delete p;
    return LENS_OK;
}

int lens_plan_create_ex(lens_plan *out, int lmax, int mmax, int spin, int64_t npoints, const double *theta_d,
                        const double *phi_d, const double *chi_d, double epsilon, int prec, unsigned flags,
                        void *stream, const lens_plan_params *prm)
{
    if (!out) return fail(LENS_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (lmax < 0 || mmax < 0 || mmax > lmax) return fail(LENS_ERR_INVALID, "need 0 <= mmax <= lmax");
    if (spin < 0 || spin > lmax) return fail(LENS_ERR_INVALID, "need 0 <= spin <= lmax");
    if (npoints < 0 || npoints > 0x7fffffffLL) return fail(LENS_ERR_INVALID, "npoints must be in [0, 2^31 - 1]");
    if (npoints > 0 && (!theta_d || !phi_d)) return fail(LENS_ERR_INVALID, "theta/phi pointers are NULL");
    if (prec != LENS_FP32 && prec != LENS_FP64) return fail(LENS_ERR_INVALID, "prec must be LENS_FP32 or LENS_FP64");
    if (flags & ~(unsigned)(LENS_GRAD_ONLY | LENS_DETERMINISTIC)) return fail(LENS_ERR_INVALID, "unknown flag");
    if ((flags & LENS_GRAD_ONLY) && spin == 0) return fail(LENS_ERR_INVALID, "LENS_GRAD_ONLY needs spin > 0");
    if (!(epsilon > 0) || !(epsilon < 1)) return fail(LENS_ERR_INVALID, "epsilon must be in (0, 1)");
    // FP32 floor: at lmax 4096 an FP32 plan with the narrowest kernel setting
    // measured eps_eff 1.2e-6 (forward), set by FP32 rounding of the sums
    if (prec == LENS_FP32 && epsilon < 2e-6)
        return fail(LENS_ERR_PRECISION, "FP32 plans reach epsilon >= 2e-6; use LENS_FP64");
    if (epsilon < 1e-13) return fail(LENS_ERR_PRECISION, "epsilon below 1e-13 is not supported");
    if (lmax > 16383) return fail(LENS_ERR_UNSUPPORTED, "lmax above 16383");

    Plan *p = new Plan();
    p->lmax = lmax; p->mmax = mmax; p->spin = spin; p->prec = prec;
    p->npts = npoints; p->eps = epsilon;
    p->grad = (flags & LENS_GRAD_ONLY) != 0;
    p->det = (flags & LENS_DETERMINISTIC) != 0;
    p->stream = (cudaStream_t)stream;
    cudaGetDevice(&p->device);
    p->nalm = lens_nalm(lmax, mmax);
    p->ncol = spin ? 2 * mmax + 1 : mmax + 1;
    Builder B(*p);
    auto bail = [&](int st, const std::string &m) { lens_plan_destroy(reinterpret_cast<lens_plan>(p)); return fail(st, m); };
    auto bailc = [&](cudaError_t e, const char *w) {
        lens_plan_destroy(reinterpret_cast<lens_plan>(p));
        return cuda_fail(e, w);
    };

    // ---- equiangular grid: ntheta >= lmax + 2, 2 ntheta - 2 7-smooth (Sect. 3, App. A)
    int nt = std::max(lmax + 2, 2);
    if (prm && prm->ntheta > 0) {
        if (prm->ntheta < lmax + 2 || !smooth7(2 * prm->ntheta - 2))
            return bail(LENS_ERR_INVALID, "ntheta must be >= lmax + 2 with 2 ntheta - 2 7-smooth");
        nt = prm->ntheta;
    } else {
        while (!smooth7(2 * nt - 2)) ++nt;
    }
    p->ntheta = nt;
    p->nnorth = (nt + 1) / 2;
    p->M = 2 * nt - 2;

    // ---- accuracy heuristic.  The NUFFT gets eps/2 of the error budget in FP64
    // plans and eps/4 in FP32 plans, where FP32 rounding in the Legendre sums and
    // the FFTs takes ~1e-6 at lmax ~ 4096.  sigma is then picked by a cost model.
    const size_t esz = prec == LENS_FP32 ? 8 : 16;
    // one CTA holds fft_one elements; a cluster of two or four CTAs 2x or 4x that
    // (FP32 single-CTA vectors carry one padding element per 16: fft_smem_elems)
    size_t fft_one = kSmemLimit / esz;
    while (fft_smem_elems(fft_one, esz) * esz > kSmemLimit) --fft_one;
    const size_t fft_max = 4 * fft_one;
    const int force_cl = prm ? prm->fft_cluster : 0;
    if (prm && prm->legendre_tables != 0) {
        if (prm->legendre_tables != 1) return bail(LENS_ERR_INVALID, "legendre_tables must be 0 or 1");
        if (prec != LENS_FP32) return bail(LENS_ERR_INVALID, "Legendre tables are built for FP32 plans only");
        p->tab = true;
    }
    if (force_cl != 0 && force_cl != 1 && force_cl != 2 && force_cl != 4)
        return bail(LENS_ERR_INVALID, "fft_cluster must be 0, 1, 2 or 4");
    const double eps_nufft = (prec == LENS_FP32 ? 0.25 : 0.5) * epsilon;
    const int ncomp = spin ? 2 : 1;
    Choice best;
    const double sig_cand[] = {1.2, 1.25, 1.3, 1.4, 1.5, 1.6, 1.75, 2.0, 2.25, 2.5};
    for (double sg : sig_cand) {
        if (prm && prm->sigma > 0 && fabs(prm->sigma - sg) > 1e-12) continue;
        int W = (prm && prm->W > 0) ? prm->W : support_for(eps_nufft, sg);
        if (W > 16) continue;
        int N1, N2;
        sizes_for(lmax, mmax, p->M, sg, W, N1, N2);
        const size_t lim = force_cl ? force_cl * fft_one : fft_max;
        if ((size_t)N1 > lim || (size_t)N2 > lim) continue;
        // per-point taps (+ kernel evaluations in FP32 plans; FP64 plans keep the
        // weights) against grid passes (FFTs).  Grid weight per cell, in taps, from
        // the stage times at lmax 4096: ~12 in FP32, ~60 in FP64 (FP64 butterflies
        // run on the narrow FP64 pipe).  FFTs split over a two-CTA cluster cost
        // more (remote shared-memory accesses).
        const bool f64 = prec == LENS_FP64;
        const double pts = (double)npoints * ncomp * ((double)W * W + (f64 ? 0.0 : 16.0 * W));
        const size_t nmax = std::max<size_t>(N1, N2);
        double clf = nmax > 2 * fft_one ? 2.0 : nmax > fft_one ? 1.5 : 1.0;
        // FP32 plans at epsilon >= 1e-5 spread through 32-bit fixed-point tiles (half the tap
        // cost of the float tiles): a grid cell then weighs ~32 taps (lmax 4096 stage times,
        // 50M points: sigma 1.5 / W 8 beats sigma 2.26 / W 6 by 3 ms per T + E/B pair); vectors
        // too long for two CTAs per SM (about 14k FP32 elements) run 1.3x slower per cell.
        // LENS_DETERMINISTIC plans take the same sigma, so that they match the atomic path
        // to rounding
        const bool fx32 = !f64 && epsilon >= 1e-5;
        if (fx32 && nmax * esz > 110000) clf *= 1.3;
        const double cell_w = f64 ? 60.0 : fx32 ? 32.0 : 12.0;
        const double grd = clf * (cell_w * ncomp * (double)N1 * 0.5 * N2 + 3.0 * (double)p->ncol * N1);
        const double cost = pts + grd;
        if (cost < best.cost) { best.cost = cost; best.sigma = sg; best.W = W; best.N1 = N1; best.N2 = N2; }
    }
    if (prm && prm->sigma > 0 && best.W == 0) {  // explicit sigma not in the candidate list
        int W = prm->W > 0 ? prm->W : support_for(eps_nufft, prm->sigma);
        sizes_for(lmax, mmax, p->M, prm->sigma, W, best.N1, best.N2);
        best.sigma = prm->sigma; best.W = W;
    }
    if (best.W == 0)
        return bail(LENS_ERR_UNSUPPORTED, "no oversampling factor fits the shared-memory FFT at this lmax/precision");
    if (best.W < 4 || best.W > 16) return bail(LENS_ERR_INVALID, "kernel support W must be in [4, 16]");
    if ((size_t)best.N1 > fft_max || (size_t)best.N2 > fft_max || (size_t)p->M > fft_max)
        return bail(LENS_ERR_UNSUPPORTED, "FFT length above the shared-memory limit of this build");
    p->W = best.W;
    p->N1 = best.N1;
    p->N2 = best.N2;
    {  // CTAs per FFT vector: the fewest of 1, 2, 4 that hold it (or the forced count)
        auto team = [&](size_t n) { return n <= fft_one ? 1 : n <= 2 * fft_one ? 2 : 4; };
        p->cl_theta = force_cl ? force_cl : team((size_t)std::max(p->N1, p->M));
        p->cl_phi = force_cl ? force_cl : team((size_t)p->N2);
        if ((size_t)std::max(p->N1, p->M) > (size_t)p->cl_theta * fft_one || (size_t)p->N2 > (size_t)p->cl_phi * fft_one)
            return bail(LENS_ERR_UNSUPPORTED, "FFT length above the forced fft_cluster's shared memory");
    }
    {
        const double s1 = (double)p->N1 / (2 * lmax + 2), s2 = (double)p->N2 / (2 * mmax + 2);
        p->sigma = std::min(s1, s2);
    }
    p->beta = (prm && prm->beta > 0) ? prm->beta : kPi * p->W * (1.0 - 0.5 / p->sigma);
    if (p->prec == LENS_FP32) {
        ker_poly_fit(p->W, p->beta, p->kpoly);
        // an explicit beta is checked; the default one stays within the kernel's own error
        // (at W <= 5 with the large sigma of tiny grids, ~1e-4 against the epsilon >= 7e-4
        // such plans serve)
        const double err = ker_poly_error(p->W, p->beta, p->kpoly), lim = 4.0 * std::max(exp(-p->beta), 1e-7);
        if (prm && prm->beta > 0 && err > lim) {
            char msg[200];
            snprintf(msg, sizeof msg,
                     "FP32 plans: beta %.3g at W %d is outside what the polynomial kernel weights reproduce "
                     "(error %.1e > %.1e); use the default beta or an FP64 plan", p->beta, p->W, err, lim);
            return bail(LENS_ERR_INVALID, msg);
        }
    }
    p->r_lo = -p->W;
    p->R = p->N1 / 2 + 2 * p->W + 1;
    p->pitch = ((p->N2 + p->W - 1) + 31) / 32 * 32;

    // ---- Legendre arithmetic: FP32 plans df32 for every m; FP64 plans native FP64
    // for m < m_df and df32 recursion + df32 accumulation for m >= m_df.  df32
    // loses ~2^-45 per operation and the recursion amplifies rounding most at
    // low m near the poles.  Measured eps_eff of the whole forward at lmax 4096,
    // HEALPix Nside 2048, eps 1e-10 (spin 0 / spin 2) against FP64 direct summation:
    //   df32 from m = 1: 2.3e-10 / 1.7e-10;  m = 64: 6.1e-11 / 5.1e-11;
    //   m = 128: 2.5e-11 / 2.3e-11;  m = 256: 8.3e-12 / 8.8e-12 (= all-FP64).
    // Hence m_df = 64 for epsilon >= 1e-9, 256 for epsilon >= 5e-11, none below,
    // times (lmax / 4096)^2 above lmax 4096 (lmax 8192, spin 0, eps 1e-10: adjoint
    // eps_eff 3.5e-10 with m_df = 256, 6.3e-11 with m_df = 1024 = all-FP64's).
    if (prec == LENS_FP32) {
        p->m_df = 0;
    } else {
        const int want = prm ? prm->legendre_df32_mmin : 0;
        if (want < 0) p->m_df = mmax + 1;
        else if (want > 0) p->m_df = std::min(want, mmax + 1);
        else {
            // the double-float recursion's error grows with lmax at a given m: at lmax 8192,
            // epsilon 1e-10, orders 256..1023 in df32 gave an adjoint eps_eff of 3.5e-10
            // against 6.3e-11 with FP64 up to m = 1024; so the FP64 orders scale as lmax^2
            const double g = std::max(1.0, ((double)lmax / 4096.0) * ((double)lmax / 4096.0));
            if (epsilon >= 1e-9) p->m_df = (int)std::min<double>(64.0 * g, mmax + 1);
            else if (epsilon >= 5e-11) p->m_df = (int)std::min<double>(256.0 * g, mmax + 1);
            else p->m_df = mmax + 1;
        }
    }
    // ---- FP32 plans: restarted FP32 recursion (legendre.cu, PolS / PolR) or df32
    {
        const int want = prm ? prm->legendre_restart : 0;
        if (want < -1 || (want > 0 && (want < 8 || want > 4096 || (want & (want - 1)) != 0)))
            return bail(LENS_ERR_INVALID, "legendre_restart must be -1, 0 or a power of two in [8, 4096]");
        if (prec == LENS_FP32 && !p->tab && want != -1 && (want > 0 || epsilon >= 1e-5)) {
            int K = want > 0 ? want : 64;
            const size_t esz_ck = spin ? 16 : 8;
            auto bytes_for = [&](int k) {
                size_t n = 0;
                for (int m = 0; m <= mmax; ++m) n += (size_t)ck_count(lmax, std::max(m, spin) + 1, k);
                return n * p->nnorth * esz_ck;
            };
            size_t b = bytes_for(K);
            while (want == 0 && b > ((size_t)20 << 30) && K < 4096) b = bytes_for(K *= 2);
            p->rst = true;
            p->ck.K = K;
            p->ck_bytes = b;
            // Reinsch's form on the rings with cos theta >= 0.7, rounded up to a multiple of 128 rings
            // (beyond 0.7 down to cos theta = 0.5 it is still the more accurate form).  The kernels
            // choose the form per warp (32 x 1, 2 or 4 rings) and the restart values were written for
            // the form of each ring, so no warp of any rings-per-thread setting may straddle jb.
            const double jr = acos(0.7) / kPi * (nt - 1);
            p->ck.jb = (int)std::ceil(jr / 128.0) * 128;
        }
        // FP64 plans whose epsilon admits df32 orders: every order in df32 (PolDDR), restarted
        // every K = 128 degrees from the FP64 recursion, so that no order runs on the FP64 pipe
        // (1/60 of the FP32 rate on GB300); the FP64 orders of m_df are not needed then
        const bool mdf_set = prm && prm->legendre_df32_mmin != 0;  // explicit FP64 orders: no restarts
        // (FP32 plans: the step table's FP32 rounding needs Reinsch's form near the poles; the df32
        // recursion runs the monic form everywhere, whose rounding grows quadratically with the
        // degrees since the last restart on rings near the poles, most at low orders: measured
        // ring-synthesis errors at lmax 2000 with K = 128 for every order: 6e-11 (m < 16),
        // 8e-12 (16 <= m < 128), 3e-12 (m >= 128); K = 16 / 64 / 128 by those bands: 1.2e-12,
        // 3.2e-12, 2.7e-12.  So orders below 16 g restart every 16 degrees, below 128 g every 64
        // and the others every 128, g = lmax / 4096 above lmax 4096 (lmax 8192, epsilon 1e-10:
        // adjoint eps_eff 1.1e-10 / 1.9e-10 with g = 1 and K = 256 / 512 above m = 128); an
        // explicit K applies to every order
        if (prec == LENS_FP64 && want != -1 && !mdf_set && p->m_df <= mmax && epsilon >= 5e-11) {
            int K = want > 0 ? want : 128;
            const size_t esz_ck = spin ? 32 : 16;
            const int g = std::max(1, lmax / 4096);
            auto k_of = [&](int m, int k) {
                return want > 0 ? k : std::min(k, m < 16 * g ? 16 : m < 128 * g ? 64 : k);
            };
            auto bytes_for = [&](int k) {
                size_t n = 0;
                for (int m = 0; m <= mmax; ++m) n += (size_t)ck_count(lmax, std::max(m, spin) + 1, k_of(m, k));
                return n * p->nnorth * esz_ck;
            };
            size_t b = bytes_for(K);
            while (want == 0 && b > ((size_t)40 << 30) && K < 4096) b = bytes_for(K *= 2);
            p->rst = true;
            p->ck.K = K;
            p->ck_bytes = b;
            p->ck.jb = 0;
            p->m_df = 0;
            p->ck_klog.resize(mmax + 1);
            for (int m = 0; m <= mmax; ++m) p->ck_klog[m] = (unsigned char)std::log2(k_of(m, K));
        }
    }
    // ---- Legendre launch shapes: RPT rings per thread; warps per CTA chosen
    // for occupancy of the kernel variant (legendre_shape)
    for (int adj = 0; adj < 2; ++adj) {
        const int want = prm ? (adj ? prm->legendre_rpt_adj : prm->legendre_rpt_fwd) : 0;
        if (want && !legendre_rpt_supported(prec, spin, adj != 0, want, p->rst))
            return bail(LENS_ERR_INVALID, "unsupported Legendre rings-per-thread setting");
        (adj ? p->leg_a : p->leg_f) =
            legendre_shape(*p, adj != 0, false, want ? want : legendre_rpt(prec, spin, adj != 0, p->rst));
        if (prec == LENS_FP64)
            (adj ? p->leg_ad : p->leg_fd) =
                legendre_shape(*p, adj != 0, true, (want && want <= 2) ? want : legendre_rpt_dd(spin, adj != 0));
    }
    if (prec == LENS_FP32) {  // synthesis of 2 / 4 maps sharing one recursion
        p->leg_fb[0] = legendre_shape(*p, false, false, p->leg_f.rpt, 2);
        p->leg_fb[1] = legendre_shape(*p, false, false, 1, 4);
    }

    cudaError_t e;
    // ---- device buffers
    if ((e = B.alloc((void **)&p->flags, sizeof(unsigned) * 4, false)) != cudaSuccess) return bailc(e, "alloc flags");
    if ((e = cudaMemset(p->flags, 0, sizeof(unsigned) * 4)) != cudaSuccess) return bailc(e, "clear flags");
    // FP32 spin plans interleave alpha and tau in rec_a (16 bytes per entry)
    const size_t ra_b = (prec == LENS_FP32 && spin) ? 16 : 8;
    if ((e = B.alloc(&p->rec_a, (size_t)p->nalm * ra_b, false)) != cudaSuccess) return bailc(e, "alloc rec_a");
    if (spin && prec == LENS_FP64 && (e = B.alloc(&p->rec_t, (size_t)p->nalm * 8, false)) != cudaSuccess)
        return bailc(e, "alloc rec_t");
    if ((e = B.alloc((void **)&p->scale, (size_t)p->nalm * 8, false)) != cudaSuccess) return bailc(e, "alloc scale");
    if (p->rst) {
        if (prec == LENS_FP32 && (e = B.alloc(&p->rec_s, (size_t)p->nalm * 16, false)) != cudaSuccess)
            return bailc(e, "alloc rec_s");
        std::vector<int64_t> cb(mmax + 1);
        int64_t off = 0;
        for (int m = 0; m <= mmax; ++m) {
            cb[m] = off;
            const int Km = p->ck_klog.empty() ? p->ck.K : 1 << p->ck_klog[m];
            off += (int64_t)ck_count(lmax, std::max(m, spin) + 1, Km) * p->nnorth;
        }
        void *d = nullptr;
        if ((e = B.upload(&d, cb)) != cudaSuccess) return bailc(e, "upload restart offsets");
        p->ck.base = (const int64_t *)d;
        if (!p->ck_klog.empty()) {
            if ((e = B.upload(&d, p->ck_klog)) != cudaSuccess) return bailc(e, "upload restart intervals");
            p->ck.klog = (const unsigned char *)d;
        }
        p->ck.ngrp = (p->nnorth + 31) / 32;
        if ((e = B.alloc(&d, sizeof(short) * (size_t)(mmax + 1) * p->ck.ngrp, false)) != cudaSuccess)
            return bailc(e, "alloc restart starts");
        p->ck.kstart = (const short *)d;
        if (p->ck_bytes > 0) {
            // values (FP32 plans 8 / 16 bytes, FP64 plans 16 / 32) and exponents (2 / 4 bytes) per entry
            const size_t ebytes = p->ck_bytes / (prec == LENS_FP32 ? 4 : 8);
            void *dv = nullptr, *de = nullptr;
            if ((e = B.alloc(&dv, p->ck_bytes, false)) != cudaSuccess || (e = B.alloc(&de, ebytes, false)) != cudaSuccess) {
                if (e == cudaErrorMemoryAllocation) {
                    cudaGetLastError();
                    return bail(LENS_ERR_NOMEM, "Legendre restart values: " + std::to_string((p->ck_bytes + ebytes) >> 20) +
                                                    " MiB not available (legendre_restart = -1 runs without them)");
                }
                return bailc(e, "alloc restart values");
            }
            p->ck.v = dv;
            p->ck.e = de;
            p->ck_bytes += ebytes;
        }
    }
    if (prec == LENS_FP64 && p->m_df <= mmax) {
        if ((e = B.alloc(&p->rec_a_df, (size_t)p->nalm * (spin ? 16 : 8), false)) != cudaSuccess)
            return bailc(e, "alloc rec_a_df");
    }
    if ((e = B.alloc(&p->coef, (size_t)p->nalm * esz * ncomp, true)) != cudaSuccess) return bailc(e, "alloc coef");
    if (p->rst && prec == LENS_FP32) {  // monic plain-form rings: c_l a_lm and the (c_l, 1/c_l) table
        void *d = nullptr;
        if ((e = B.alloc(&p->coef_m, (size_t)p->nalm * esz * ncomp, true)) != cudaSuccess ||
            (e = B.alloc(&d, (size_t)p->nalm * sizeof(float2), false)) != cudaSuccess)
            return bailc(e, "alloc monic coefficients");
        p->ck.cs = (const float2 *)d;
    }
    const ScratchSizes scr = plan_scratch_sizes(*p);
    if ((e = B.alloc(&p->ring, scr.ring, true)) != cudaSuccess) return bailc(e, "alloc ring");
    if ((e = B.alloc(&p->X, scr.X, true)) != cudaSuccess) return bailc(e, "alloc X");
    if ((e = B.alloc(&p->grid, scr.grid, true)) != cudaSuccess) return bailc(e, "alloc grid");
    if (p->det) {  // fixed-point sums; the small scalars share one allocation
        if ((e = B.alloc((void **)&p->fx_scale, sizeof(double) * ((size_t)mmax + 2), false)) != cudaSuccess ||
            (e = B.alloc((void **)&p->fx_maxbits, 64, false)) != cudaSuccess)
            return bailc(e, "alloc fixed-point units");
        p->fx_kmax = reinterpret_cast<uint32_t *>(p->fx_maxbits + 1);
        if ((e = cudaMemset(p->fx_maxbits, 0, 64)) != cudaSuccess) return bailc(e, "clear fixed-point units");
        if (prec == LENS_FP32) {
            if ((e = B.alloc(&p->fx_grid, 8 * (size_t)ncomp * p->R * p->pitch, true)) != cudaSuccess ||
                (e = B.alloc(&p->fx_alm, 16 * (size_t)p->nalm * p->alm_ncomp(), true)) != cudaSuccess)
                return bailc(e, "alloc fixed-point sums");
        }
    }
    if (npoints > 0) {
        if ((e = B.alloc((void **)&p->cell, sizeof(uint32_t) * npoints, false)) != cudaSuccess) return bailc(e, "alloc cell");
        if ((e = B.alloc(&p->frac, esz * npoints, false)) != cudaSuccess) return bailc(e, "alloc frac");
        if ((e = B.alloc((void **)&p->perm, sizeof(int32_t) * npoints, false)) != cudaSuccess) return bailc(e, "alloc perm");
        const int tr = prm ? prm->spread_tile_rows : 0;
        if (tr != 0 && tr != 16 && tr != 32 && tr != 64)
            return bail(LENS_ERR_INVALID, "spread_tile_rows must be 0, 16, 32 or 64");
        p->tile_r = tr ? tr : kTileR;
        p->ntile_c = (p->N2 + kTileC - 1) / kTileC;
        p->ntiles = (p->R + p->tile_r - 1) / p->tile_r * p->ntile_c;
        if ((e = B.alloc((void **)&p->tile_start, sizeof(uint32_t) * ((size_t)p->ntiles + 1), false)) != cudaSuccess)
            return bailc(e, "alloc tile table");
        if (spin && (e = B.alloc(&p->phase, esz * npoints, false)) != cudaSuccess) return bailc(e, "alloc phase");
        // FP32 plans at epsilon >= 1e-5 accumulate the spreading tiles in 32-bit fixed point,
        // FP64 plans in 64-bit fixed point (nufft.cu, k_spread); FP32 plans at smaller epsilon
        // and deterministic plans keep their own paths
        if (!p->det && (prec == LENS_FP64 || epsilon >= 1e-5)) {
            if ((e = B.alloc((void **)&p->tile_kmax, sizeof(unsigned short) * (size_t)p->ntiles, false)) != cudaSuccess ||
                (e = B.alloc((void **)&p->maxbits, sizeof(unsigned long long), true)) != cudaSuccess)
                return bailc(e, "alloc spreading bounds");
        }
        // FP64 plans keep the 2W kernel weights of every point (GB300's FP64 pipe makes
        // evaluating exp/sqrt per tap far dearer than reading 16 W bytes per point),
        // unless the table would exceed 48 GB (e.g. 805M points at W = 16: 206 GB);
        // then the taps are evaluated per call
        const size_t wbytes = sizeof(double) * 2 * (size_t)p->W * npoints;
        const int pw = prm ? prm->point_weights : 0;
        if (pw < -1 || pw > 1) return bail(LENS_ERR_INVALID, "point_weights must be -1, 0 or 1");
        if (prec == LENS_FP64 && (pw == 1 || (pw == 0 && wbytes <= (size_t)48 << 30)) &&
            (e = B.alloc((void **)&p->wts, wbytes, false)) != cudaSuccess) {
            if (e == cudaErrorMemoryAllocation) {
                cudaGetLastError();
                return bail(LENS_ERR_NOMEM, "point kernel weights: " + std::to_string(wbytes >> 20) + " MiB not available");
            }
            return bailc(e, "alloc weights");
        }
        // with the weights kept, FP64 plans at epsilon >= 5e-11 compute the interpolation and
        // spreading taps in double-float on the FP32 pipe (~2^-46 relative per term; lmax 4096,
        // 50M points, W = 13: interpolation 30.1 -> 13.4 ms for spin 2); smaller epsilon keeps FP64
        p->wts_dd = p->wts && epsilon >= 5e-11;
    }

    // ---- host tables: start-value norms, rings, deconvolution factors
    {
        // lognorm[m] = log2 sqrt((2 l0 + 1)/(4 pi) C(2 l0, k)),
        //   m >= s: l0 = m, C(2m, m + s) via the running ratio (2m)(2m-1)/((m+s)(m-s))
        //   m <  s: l0 = s, C(2s, s + m)
        std::vector<double> ln(mmax + 1);
        double lb = 0.0, cmp = 0.0;  // log2 C(2m, m+s), Neumaier-compensated running sum
        for (int m = 0; m <= mmax; ++m) {
            int l0;
            double logbin;
            if (m < spin) {
                l0 = spin;
                logbin = 0.0;
                for (int i = 1; i <= spin + m; ++i) logbin += log2((double)(2 * spin - (spin + m) + i) / i);
            } else {
                l0 = m;
                if (m == spin) {
                    lb = 0.0; cmp = 0.0;  // C(2s, 2s) = 1
                } else {
                    const double term = log2((2.0 * m) * (2.0 * m - 1.0) / ((double)(m + spin) * (m - spin)));
                    const double t = lb + term;
                    if (fabs(lb) >= fabs(term)) cmp += (lb - t) + term; else cmp += (term - t) + lb;
                    lb = t;
                }
                logbin = lb + cmp;
            }
            ln[m] = 0.5 * (log2((2.0 * l0 + 1.0) / (4.0 * kPi)) + logbin);
        }
        void *d = nullptr;
        if ((e = B.upload(&d, ln)) != cudaSuccess) return bailc(e, "upload lognorm");
        p->lognorm = (double *)d;

        std::vector<double> x(p->nnorth), ls(p->nnorth), lc(p->nnorth);
        std::vector<float2> xdf(p->nnorth);
        std::vector<float> y1(p->nnorth);
        for (int j = 0; j < p->nnorth; ++j) {
            const double th = kPi * j / (nt - 1);
            x[j] = cos(th);
            if (2 * j == nt - 1) x[j] = 0.0;
            const float h = (float)x[j];
            xdf[j] = make_float2(h, (float)(x[j] - (double)h));
            const double sh = sin(0.5 * th);
            y1[j] = (float)(2.0 * sh * sh);
            ls[j] = j == 0 ? -INFINITY : log2(sin(0.5 * th));
            lc[j] = log2(cos(0.5 * th));
        }
        if ((e = B.upload(&d, x)) != cudaSuccess) return bailc(e, "upload rings");
        p->rings.x = (const double *)d;
        if ((e = B.upload(&d, xdf)) != cudaSuccess) return bailc(e, "upload rings");
        p->rings.xdf = (const float2 *)d;
        if ((e = B.upload(&d, ls)) != cudaSuccess) return bailc(e, "upload rings");
        p->rings.lsin2 = (const double *)d;
        if ((e = B.upload(&d, lc)) != cudaSuccess) return bailc(e, "upload rings");
        p->rings.lcos2 = (const double *)d;
        if ((e = B.upload(&d, y1)) != cudaSuccess) return bailc(e, "upload rings");
        p->rings.y1 = (const float *)d;

        Quad q(std::max(64, 4 * p->W + 40));
        std::vector<double> w1(2 * lmax + 1), w2(p->ncol);
        for (int k = 0; k <= lmax; ++k) {
            const double v = 1.0 / psihat(q, 2 * kPi * k / p->N1, p->W, p->beta);
            w1[lmax + k] = v;
            w1[lmax - k] = v;
        }
        for (int c = 0; c < p->ncol; ++c) {
            const int m = spin ? c - mmax : c;
            w2[c] = 1.0 / (p->M * psihat(q, 2 * kPi * m / p->N2, p->W, p->beta));
        }
        if (prec == LENS_FP32) {
            std::vector<float> f1(w1.begin(), w1.end()), f2(w2.begin(), w2.end());
            if ((e = B.upload(&p->w1, f1)) != cudaSuccess) return bailc(e, "upload w1");
            if ((e = B.upload(&p->w2, f2)) != cudaSuccess) return bailc(e, "upload w2");
        } else {
            if ((e = B.upload(&p->w1, w1)) != cudaSuccess) return bailc(e, "upload w1");
            if ((e = B.upload(&p->w2, w2)) != cudaSuccess) return bailc(e, "upload w2");
        }
    }
    if ((e = B.fft(p->fM, p->M)) != cudaSuccess) return bailc(e, "fft tables");
    if ((e = B.fft(p->fN1, p->N1)) != cudaSuccess) return bailc(e, "fft tables");
    if ((e = B.fft(p->fN2, p->N2)) != cudaSuccess) return bailc(e, "fft tables");

    if ((e = launch_rec_tables(*p)) != cudaSuccess) return bailc(e, "recursion tables");
    if (p->rst) {  // (FP32: step table, then) restart values from the FP64 recursion
        if (prec == LENS_FP32 && (e = launch_rec_tables_s(*p)) != cudaSuccess) return bailc(e, "restart step table");
        if (p->ck_bytes > 0) {
            // temporaries: FP64 alpha and tau [nalm] each (FP32 plans; FP64 plans have their own),
            // first significant degree [mmax + 1][nnorth]
            const size_t tb = (size_t)p->nalm * 16 + sizeof(int) * (size_t)(mmax + 1) * p->nnorth;
            double *tmp = nullptr;
            if ((e = cudaMalloc((void **)&tmp, tb)) != cudaSuccess) {
                cudaGetLastError();
                return bail(LENS_ERR_NOMEM, "Legendre restart values: temporary tables not available");
            }
            if (prec == LENS_FP32)
                e = launch_ck_build(*p, tmp, tmp + p->nalm, const_cast<void *>(p->ck.v), const_cast<void *>(p->ck.e),
                                    reinterpret_cast<int *>(tmp + 2 * p->nalm), const_cast<short *>(p->ck.kstart));
            else
                e = launch_ck_build64(*p, const_cast<void *>(p->ck.v), const_cast<void *>(p->ck.e),
                                      reinterpret_cast<int *>(tmp + 2 * p->nalm), const_cast<short *>(p->ck.kstart));
            if (e == cudaSuccess) {  // non-negligible triples (the Legendre steps' algorithmic work)
                std::vector<int> lt((size_t)(mmax + 1) * p->nnorth);
                e = cudaMemcpyAsync(lt.data(), tmp + 2 * p->nalm, sizeof(int) * lt.size(), cudaMemcpyDeviceToHost,
                                    p->stream);
                if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
                if (e == cudaSuccess) {
                    int64_t n = 0;
                    for (int m = 0; m <= mmax; ++m) {
                        const int l0 = std::max(m, spin);
                        for (int j = 0; j < p->nnorth; ++j)
                            n += std::max(0, lmax + 1 - std::max(lt[(size_t)m * p->nnorth + j], l0));
                    }
                    p->leg_triples = n;
                }
            }
            cudaFree(tmp);
            if (e != cudaSuccess) return bailc(e, "restart values");
        } else if ((e = cudaMemsetAsync(const_cast<short *>(p->ck.kstart), 0,
                                        sizeof(short) * (size_t)(mmax + 1) * p->ck.ngrp, p->stream)) != cudaSuccess) {
            return bailc(e, "restart starts");
        }
    }
    if (p->tab) {
        const int rc = build_legendre_tables(*p, B);
        if (rc != LENS_OK) {
            lens_plan_destroy(reinterpret_cast<lens_plan>(p));
            return rc;
        }
    }
    {
        std::string err;
        e = launch_prep_points(*p, theta_d, phi_d, spin ? chi_d : nullptr, p->stream, err);
        if (e != cudaSuccess) {
            if (!err.empty()) return bail(err.find("internal") == 0 ? LENS_ERR_CUDA : LENS_ERR_DOMAIN, err);
            return bailc(e, "point preparation");
        }
    }
    if ((e = cudaStreamSynchronize(p->stream)) != cudaSuccess) return bailc(e, "plan sync");
    *out = reinterpret_cast<lens_plan>(p);
    return LENS_OK;
}

int lens_plan_create(lens_plan *out, int lmax, int mmax, int spin, int64_t npoints, const double *theta_d,
                     const double *phi_d, const double *chi_d, double epsilon, int prec, unsigned flags, void *stream)
{
    return lens_plan_create_ex(out, lmax, mmax, spin, npoints, theta_d, phi_d, chi_d, epsilon, prec, flags, stream,
                               nullptr);
}

int lens_plan_info(lens_plan pl, lens_plan_info_t *info)
{
    if (!pl || !info) return fail(LENS_ERR_INVALID, "NULL argument");
    const Plan *p = reinterpret_cast<const Plan *>(pl);
    info->lmax = p->lmax; info->mmax = p->mmax; info->spin = p->spin; info->prec = p->prec;
    info->npoints = p->npts; info->epsilon = p->eps;
    info->ntheta = p->ntheta; info->ntheta_fft = p->M; info->n1 = p->N1; info->n2 = p->N2;
    info->W = p->W; info->beta = p->beta; info->sigma = p->sigma;
    info->rows_kept = p->R; info->row_pitch = p->pitch;
    info->workspace_bytes = p->work_bytes; info->plan_bytes = p->plan_bytes;
    info->flags = (p->grad ? (unsigned)LENS_GRAD_ONLY : 0u) | (p->det ? (unsigned)LENS_DETERMINISTIC : 0u);
    info->alm_ncomp = p->alm_ncomp();
    info->legendre_table_bytes = p->tab_bytes;
    info->legendre_restart = p->rst ? p->ck.K : 0;
    info->restart_bytes = p->ck_bytes;
    info->legendre_df32_mmin = p->prec == LENS_FP64 ? p->m_df : 0;
    info->legendre_triples = p->leg_triples;
    info->point_weight_bytes = p->wts ? sizeof(double) * 2 * (size_t)p->W * p->npts : 0;
    return LENS_OK;
}

}  // extern "C"

namespace {

// ------------------------------------------------------------ stage timers
struct Profiler {
    bool on = false;
    double ms[32] = {0};
    int64_t cnt[32] = {0};
    struct Rec { int slot; cudaEvent_t a, b; };
    std::vector<Rec> pending;
    std::vector<cudaEvent_t> pool;
    cudaEvent_t get()
    {
        if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    void drain()
    {
        for (auto &r : pending) {
            float t = 0.f;
            if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
                ms[r.slot] += t;
                cnt[r.slot] += 1;
            }
            pool.push_back(r.a);
            pool.push_back(r.b);
        }
        pending.clear();
    }
};
Profiler g_prof;

// Runs one stage launch, bracketed by events when the profiler is on.
template <class F> cudaError_t staged(const Plan &p, int stage, cudaStream_t st, F &&launch)
{
    if (!g_prof.on) return launch();
    const int slot = stage + 8 * (p.spin > 0) + 16 * (p.prec == LENS_FP64);
    cudaEvent_t a = g_prof.get(), b = g_prof.get();
    cudaEventRecord(a, st);
    cudaError_t e = launch();
    cudaEventRecord(b, st);
    g_prof.pending.push_back({slot, a, b});
    if (g_prof.pending.size() > 4096) g_prof.drain();
    return e;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

int forward_one(const Plan &p, const void *alm, void *map, cudaStream_t st, double wpos = 1.0)
{
    cudaError_t e;
    if ((e = staged(p, 0, st, [&] { return launch_legendre_fwd(p, alm, p.ring, st, wpos); })) != cudaSuccess)
        return cuda_fail(e, "legendre synthesis");
    if ((e = staged(p, 1, st, [&] { return launch_theta_fwd(p, p.ring, p.X, st); })) != cudaSuccess)
        return cuda_fail(e, "theta transform");
    if ((e = staged(p, 2, st, [&] { return launch_phi_fwd(p, p.X, p.grid, st); })) != cudaSuccess)
        return cuda_fail(e, "phi transform");
    if ((e = staged(p, 3, st, [&] { return launch_interp(p, p.grid, map, st); })) != cudaSuccess)
        return cuda_fail(e, "interpolation");
    return LENS_OK;
}

int adjoint_one(const Plan &p, const void *map, void *alm, cudaStream_t st, double wpos = 1.0)
{
    cudaError_t e;
    if ((e = staged(p, 4, st, [&] { return launch_spread(p, map, p.grid, st); })) != cudaSuccess)
        return cuda_fail(e, "spreading");
    if ((e = staged(p, 5, st, [&] { return launch_phi_adj(p, p.grid, p.X, st); })) != cudaSuccess)
        return cuda_fail(e, "phi transform");
    if ((e = staged(p, 6, st, [&] { return launch_theta_adj(p, p.X, p.ring, st); })) != cudaSuccess)
        return cuda_fail(e, "theta transform");
    if ((e = staged(p, 7, st, [&] { return launch_legendre_adj(p, p.ring, alm, st, wpos); })) != cudaSuccess)
        return cuda_fail(e, "adjoint legendre");
    return LENS_OK;
}

size_t alm_bytes(const Plan &p) { return plan_alm_bytes(p); }
size_t map_bytes(const Plan &p) { return (size_t)p.npts * (p.spin ? 2 : 1) * (p.prec == LENS_FP32 ? 4 : 8); }
size_t ring_bytes(const Plan &p) { return (size_t)p.ncol * p.ntheta * 8; }

// Workspace of the grouped synthesis (FP32 plans): ring and prepared
// coefficients of four maps, allocated on the first call with two or more
// maps.  Not inside a stream capture (an allocation there would not be
// replayed): such calls then run map by map.
bool group_workspace(Plan &p, cudaStream_t st)
{
    if (p.ring_batch) return true;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return false;
    if (p.nallocs + 2 > (int)(sizeof(p.allocs) / sizeof(p.allocs[0]))) return false;
    void *r = nullptr, *c = nullptr;
    if (cudaMalloc(&r, 4 * ring_bytes(p)) != cudaSuccess) { cudaGetLastError(); return false; }
    if (cudaMalloc(&c, 4 * alm_bytes(p)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(r);
        return false;
    }
    p.ring_batch = r;
    p.coef_batch = c;
    p.allocs[p.nallocs++] = r;
    p.allocs[p.nallocs++] = c;
    p.work_bytes += 4 * (ring_bytes(p) + alm_bytes(p));
    return true;
}

// Workspace of the tensor-core synthesis: ring coefficients of 64 maps (32 per launch), their
// prepared coefficient tiles and the chunk offsets; allocated on the first call
// that uses it, not inside a stream capture (false: run the other paths).
bool tc_workspace(Plan &p, cudaStream_t st)
{
    if (p.tc_ring) return true;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return false;
    if (p.nallocs + 3 > (int)(sizeof(p.allocs) / sizeof(p.allocs[0]))) return false;
    std::vector<int64_t> cb(p.mmax + 1);
    int64_t tot = 0;
    for (int m = 0; m <= p.mmax; ++m) {
        cb[m] = tot;
        tot += tc_chunks(p.lmax, m);
    }
    const size_t rb = 64 * ring_bytes(p), cbytes = sizeof(float) * tc_coef_floats(64, tot > 0 ? tot : 1);
    void *r = nullptr, *c = nullptr, *o = nullptr;
    if (cudaMalloc(&r, rb) != cudaSuccess || cudaMalloc(&c, cbytes) != cudaSuccess ||
        cudaMalloc(&o, sizeof(int64_t) * cb.size()) != cudaSuccess ||
        cudaMemcpy(o, cb.data(), sizeof(int64_t) * cb.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(r);
        cudaFree(c);
        cudaFree(o);
        return false;
    }
    p.tc_ring = r;
    p.tc_coef = c;
    p.tc_cbase = (int64_t *)o;
    p.allocs[p.nallocs++] = r;
    p.allocs[p.nallocs++] = c;
    p.allocs[p.nallocs++] = o;
    p.work_bytes += rb + cbytes + sizeof(int64_t) * cb.size();
    return true;
}

// Synthesis of nm (<= 64) consecutive maps with the tensor-core Legendre step,
// then the Fourier stages and the interpolation per map.
int forward_tc(const Plan &p, const char *alm, char *map, int nm, cudaStream_t st)
{
    const int nb = nm <= 16 ? 16 : nm <= 32 ? 32 : 64;
    cudaError_t e;
    if ((e = staged(p, 0, st, [&] {
             cudaError_t e2 = cudaMemsetAsync(p.tc_ring, 0, nm * ring_bytes(p), st);
             if (e2 != cudaSuccess) return e2;
             return launch_legendre_fwd_tc(p, alm, nm, p.tc_ring, p.tc_coef, p.tc_cbase, nb, st);
         })) != cudaSuccess)
        return cuda_fail(e, "tensor-core legendre synthesis");
    for (int b = 0; b < nm; ++b) {
        const void *ring = (const char *)p.tc_ring + b * ring_bytes(p);
        if ((e = staged(p, 1, st, [&] { return launch_theta_fwd(p, ring, p.X, st); })) != cudaSuccess)
            return cuda_fail(e, "theta transform");
        if ((e = staged(p, 2, st, [&] { return launch_phi_fwd(p, p.X, p.grid, st); })) != cudaSuccess)
            return cuda_fail(e, "phi transform");
        if ((e = staged(p, 3, st, [&] { return launch_interp(p, p.grid, map + b * map_bytes(p), st); })) !=
            cudaSuccess)
            return cuda_fail(e, "interpolation");
    }
    return LENS_OK;
}

// Synthesis of nm = 2 or 4 consecutive maps: one Legendre launch shares the
// recursion among them, then the Fourier stages and the interpolation per map.
int forward_group(const Plan &p, const char *alm, char *map, int nm, cudaStream_t st, double wpos)
{
    cudaError_t e;
    if ((e = staged(p, 0, st, [&] {
             return launch_legendre_fwd_batch(p, alm, p.ring_batch, p.coef_batch, nm, st, wpos);
         })) != cudaSuccess)
        return cuda_fail(e, "legendre synthesis");
    for (int b = 0; b < nm; ++b) {
        const void *ring = (const char *)p.ring_batch + b * ring_bytes(p);
        if ((e = staged(p, 1, st, [&] { return launch_theta_fwd(p, ring, p.X, st); })) != cudaSuccess)
            return cuda_fail(e, "theta transform");
        if ((e = staged(p, 2, st, [&] { return launch_phi_fwd(p, p.X, p.grid, st); })) != cudaSuccess)
            return cuda_fail(e, "phi transform");
        if ((e = staged(p, 3, st, [&] { return launch_interp(p, p.grid, map + b * map_bytes(p), st); })) !=
            cudaSuccess)
            return cuda_fail(e, "interpolation");
    }
    return LENS_OK;
}

}  // namespace

bool gsl::profile_swap(bool on)
{
    const bool was = g_prof.on;
    g_prof.on = on;
    return was;
}

int gsl::run_forward(const Plan &p, const void *alm, void *map, cudaStream_t st, double wpos)
{
    return forward_one(p, alm, map, st, wpos);
}

int gsl::run_adjoint(const Plan &p, const void *map, void *alm, cudaStream_t st, double wpos)
{
    return adjoint_one(p, map, alm, st, wpos);
}

extern "C" {

static int device_call(lens_plan pl, const void *in_d, void *out_d, int nmaps, void *stream, bool fwd, double wpos)
{
    if (!pl || nmaps < 0) return fail(LENS_ERR_INVALID, "bad plan or nmaps");
    Plan &p = *reinterpret_cast<Plan *>(pl);
    const void *alm_d = fwd ? in_d : out_d, *map_d = fwd ? out_d : in_d;
    if (nmaps > 0 && (!alm_d || (!map_d && p.npts > 0))) return fail(LENS_ERR_INVALID, "NULL buffer");
    DeviceGuard g(p.device);
    cudaStream_t st = stream ? (cudaStream_t)stream : p.stream;
    const size_t ib = fwd ? alm_bytes(p) : map_bytes(p), ob = fwd ? map_bytes(p) : alm_bytes(p);
    int i = 0;
    // spin-0 FP32 synthesis of 16 or more maps (restarted recursion): the Legendre step on the
    // tensor cores, 32 maps at a time (at lmax 4096: 16 maps 32.4 ms, 32 maps 34.1 ms, 64 maps
    // 70.2 ms per launch; the 64-map tiles need 128 KB of shared memory, one CTA per SM)
    if (fwd && wpos == 1.0 && p.prec == LENS_FP32 && p.rst && p.spin == 0 && !p.grad && p.tc_on && nmaps >= 16 &&
        tc_workspace(p, st)) {
        for (; nmaps - i >= 16; ) {
            const int nm = std::min(32, nmaps - i);
            const int r = forward_tc(p, (const char *)in_d + i * ib, (char *)out_d + i * ob, nm, st);
            if (r != LENS_OK) return r;
            i += nm;
        }
    }
    // FP32 synthesis of several maps: groups of 4, then 2, share the recursion
    // (plans with Legendre tables: one table read serves the group; spin s groups of 2)
    if (fwd && p.prec == LENS_FP32 && !p.grad && nmaps >= 2 && p.group_maps && group_workspace(p, st)) {
        for (int nm = (p.tab && p.spin) ? 2 : 4; nm >= 2; nm /= 2)
            for (; nmaps - i >= nm; i += nm) {
                const int r = forward_group(p, (const char *)in_d + i * ib, (char *)out_d + i * ob, nm, st, wpos);
                if (r != LENS_OK) return r;
            }
    }
    for (; i < nmaps; ++i) {
        const void *in = (const char *)in_d + i * ib;
        void *out = (char *)out_d + i * ob;
        int r = fwd ? forward_one(p, in, out, st, wpos) : adjoint_one(p, in, out, st, wpos);
        if (r != LENS_OK) return r;
    }
    return LENS_OK;
}

int lens_plan_status(lens_plan pl, void *stream)
{
    if (!pl) return fail(LENS_ERR_INVALID, "bad plan");
    Plan &p = *reinterpret_cast<Plan *>(pl);
    DeviceGuard g(p.device);
    cudaStream_t st = stream ? (cudaStream_t)stream : p.stream;
    unsigned f = 0;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(&f, p.flags + 1, sizeof(unsigned), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_fail(e, "status read");
    if (f == 0) return LENS_OK;
    if ((e = cudaMemsetAsync(p.flags + 1, 0, sizeof(unsigned), st)) != cudaSuccess) return cuda_fail(e, "status reset");
    return fail(LENS_ERR_TIMEOUT, "a device-side wait gave up: the results of earlier calls are incomplete");
}

int lens_selftest_bounded_wait(void *stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    unsigned *d = nullptr, h = 0;
    cudaError_t e = cudaMalloc(&d, sizeof(unsigned));
    if (e != cudaSuccess) return cuda_fail(e, "selftest alloc");
    if ((e = cudaMemsetAsync(d, 0, sizeof(unsigned), st)) == cudaSuccess &&
        (e = launch_wait_selftest(d, 20000000LL, st)) == cudaSuccess &&  // ~10 ms
        (e = cudaMemcpyAsync(&h, d, sizeof(unsigned), cudaMemcpyDeviceToHost, st)) == cudaSuccess)
        e = cudaStreamSynchronize(st);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(e, "selftest");
    if (!(h & FLAG_TIMEOUT)) return fail(LENS_ERR_CUDA, "bounded wait did not report its timeout");
    return LENS_OK;
}

int lens_plan_set_grouping(lens_plan pl, int on)
{
    if (!pl) return fail(LENS_ERR_INVALID, "bad plan");
    reinterpret_cast<Plan *>(pl)->group_maps = on != 0;
    return LENS_OK;
}

int lens_plan_set_tensor_cores(lens_plan pl, int on)
{
    if (!pl) return fail(LENS_ERR_INVALID, "bad plan");
    reinterpret_cast<Plan *>(pl)->tc_on = on != 0;
    return LENS_OK;
}

int lens_synthesis(lens_plan pl, const void *alm_d, void *map_d, int nmaps, void *stream)
{
    return device_call(pl, alm_d, map_d, nmaps, stream, true, 1.0);
}

int lens_adjoint(lens_plan pl, const void *map_d, void *alm_d, int nmaps, void *stream)
{
    return device_call(pl, map_d, alm_d, nmaps, stream, false, 1.0);
}

// Gradients: lens_synthesis counts every m > 0 coefficient for +m and -m, so
// with respect to the weighted a_lm product the adjoint is exact and the
// gradients carry the weight 2 (or 1/2) on m > 0.
int lens_synthesis_vjp(lens_plan pl, const void *grad_map_d, void *grad_alm_d, int nmaps, void *stream)
{
    return device_call(pl, grad_map_d, grad_alm_d, nmaps, stream, false, 2.0);
}

int lens_adjoint_vjp(lens_plan pl, const void *grad_alm_d, void *grad_map_d, int nmaps, void *stream)
{
    return device_call(pl, grad_alm_d, grad_map_d, nmaps, stream, true, 0.5);
}

static int host_call(lens_plan pl, const void *in_h, void *out_h, int nmaps, void *stream, bool fwd,
                     bool sync = true)
{
    if (!pl || nmaps < 0) return fail(LENS_ERR_INVALID, "bad plan or nmaps");
    Plan &p = *reinterpret_cast<Plan *>(pl);
    if (nmaps > 0 && (!in_h || !out_h)) return fail(LENS_ERR_INVALID, "NULL buffer");
    DeviceGuard g(p.device);
    cudaStream_t st = stream ? (cudaStream_t)stream : p.stream;
    const size_t ab = alm_bytes(p), mb = map_bytes(p);
    cudaError_t e;
    if (!p.stage_in) {  // one alm-sized and one map-sized buffer, kept by the plan
        if (p.nallocs + 2 > (int)(sizeof(p.allocs) / sizeof(p.allocs[0])))
            return fail(LENS_ERR_NOMEM, "plan allocation table full");
        const size_t big = std::max(ab, mb) > 0 ? std::max(ab, mb) : 16;
        if ((e = cudaMalloc(&p.stage_in, big)) != cudaSuccess) { p.stage_in = nullptr; return cuda_fail(e, "staging alloc"); }
        if ((e = cudaMalloc(&p.stage_out, big)) != cudaSuccess) {
            cudaFree(p.stage_in);
            p.stage_in = nullptr;
            return cuda_fail(e, "staging alloc");
        }
        p.allocs[p.nallocs++] = p.stage_in;
        p.allocs[p.nallocs++] = p.stage_out;
        p.work_bytes += 2 * big;
    }
    void *d_in = p.stage_in, *d_out = p.stage_out;
    int rc = LENS_OK;
    for (int i = 0; i < nmaps && rc == LENS_OK; ++i) {
        const size_t ib = fwd ? ab : mb, ob = fwd ? mb : ab;
        if ((e = cudaMemcpyAsync(d_in, (const char *)in_h + i * ib, ib, cudaMemcpyHostToDevice, st)) != cudaSuccess) {
            rc = cuda_fail(e, "host to device copy");
            break;
        }
        rc = fwd ? forward_one(p, d_in, d_out, st) : adjoint_one(p, d_in, d_out, st);
        if (rc != LENS_OK) break;
        if ((e = cudaMemcpyAsync((char *)out_h + i * ob, d_out, ob, cudaMemcpyDeviceToHost, st)) != cudaSuccess) {
            rc = cuda_fail(e, "device to host copy");
            break;
        }
    }
    if (!sync) return rc;
    e = cudaStreamSynchronize(st);
    if (rc == LENS_OK && e != cudaSuccess) rc = cuda_fail(e, "stream sync");
    return rc;
}

int lens_synthesis_host(lens_plan p, const void *alm_h, void *map_h, int nmaps, void *stream)
{
    return host_call(p, alm_h, map_h, nmaps, stream, true);
}

int lens_adjoint_host(lens_plan p, const void *map_h, void *alm_h, int nmaps, void *stream)
{
    return host_call(p, map_h, alm_h, nmaps, stream, false);
}

int lens_synthesis_host_async(lens_plan p, const void *alm_h, void *map_h, int nmaps, void *stream)
{
    return host_call(p, alm_h, map_h, nmaps, stream, true, false);
}

int lens_adjoint_host_async(lens_plan p, const void *map_h, void *alm_h, int nmaps, void *stream)
{
    return host_call(p, map_h, alm_h, nmaps, stream, false, false);
}

int lens_ring_synthesis(lens_plan pl, const void *alm_d, void *ring_d, void *stream)
{
    if (!pl || !alm_d || !ring_d) return fail(LENS_ERR_INVALID, "NULL argument");
    const Plan &p = *reinterpret_cast<const Plan *>(pl);
    DeviceGuard g(p.device);
    cudaStream_t st = stream ? (cudaStream_t)stream : p.stream;
    cudaError_t e = launch_legendre_fwd(p, alm_d, ring_d, st);
    return e == cudaSuccess ? LENS_OK : cuda_fail(e, "legendre synthesis");
}

int lens_torus_coefficients(lens_plan pl, const void *alm_d, void *coef_d, void *stream)
{
    if (!pl || !alm_d || !coef_d) return fail(LENS_ERR_INVALID, "NULL argument");
    const Plan &p = *reinterpret_cast<const Plan *>(pl);
    if (p.cl_theta != 1) return fail(LENS_ERR_UNSUPPORTED, "torus coefficients of cluster-sized theta vectors");
    DeviceGuard g(p.device);
    cudaStream_t st = stream ? (cudaStream_t)stream : p.stream;
    cudaError_t e = launch_legendre_fwd(p, alm_d, p.ring, st);
    if (e == cudaSuccess) e = launch_theta_coeffs(p, p.ring, coef_d, st);
    return e == cudaSuccess ? LENS_OK : cuda_fail(e, "torus coefficients");
}

int lens_ring_adjoint(lens_plan pl, const void *ring_d, void *alm_d, void *stream)
{
    if (!pl || !alm_d || !ring_d) return fail(LENS_ERR_INVALID, "NULL argument");
    const Plan &p = *reinterpret_cast<const Plan *>(pl);
    DeviceGuard g(p.device);
    cudaStream_t st = stream ? (cudaStream_t)stream : p.stream;
    cudaError_t e = launch_legendre_adj(p, ring_d, alm_d, st);
    return e == cudaSuccess ? LENS_OK : cuda_fail(e, "adjoint legendre");
}

int lens_profile_enable(int on)
{
    g_prof.on = on != 0;
    return LENS_OK;
}

int lens_profile_read(double *ms, int64_t *counts, int n)
{
    if (n < 0 || n > 32) return fail(LENS_ERR_INVALID, "n must be in [0, 32]");
    g_prof.drain();
    for (int i = 0; i < n; ++i) {
        if (ms) ms[i] = g_prof.ms[i];
        if (counts) counts[i] = g_prof.cnt[i];
    }
    return LENS_OK;
}

int lens_profile_reset(void)
{
    g_prof.drain();
    for (int i = 0; i < 32; ++i) { g_prof.ms[i] = 0; g_prof.cnt[i] = 0; }
    return LENS_OK;
}

int lens_pointing(int64_t n, const double *theta_d, const double *phi_d, const double *ath_d, const double *aph_d,
                  double *theta_out_d, double *phi_out_d, double *chi_out_d, void *stream)
{
    if (n < 0) return fail(LENS_ERR_INVALID, "n < 0");
    if (n > 0 && (!theta_d || !phi_d || !ath_d || !aph_d || !theta_out_d || !phi_out_d))
        return fail(LENS_ERR_INVALID, "NULL argument");
    cudaError_t e = launch_pointing(n, theta_d, phi_d, ath_d, aph_d, theta_out_d, phi_out_d, chi_out_d,
                                    (cudaStream_t)stream);
    return e == cudaSuccess ? LENS_OK : cuda_fail(e, "pointing");
}

}  // extern "C"
