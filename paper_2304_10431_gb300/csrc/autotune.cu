// Autotuner: measured choice of the plan parameters for one geometry.
//
// The paper picks its kernel parameters with a "simple heuristic"; a plan here
// uses a cost model (plan.cu).  lens_autotune instead builds candidate plans
// for the caller's points and times them on the GPU, one parameter group at a
// time, each at the best values found so far:
//   1. the oversampling factor sigma with the smallest kernel support W that
//      meets epsilon (the accuracy frontier of (sigma, W));
//   2. W + 1 at that sigma (a wider kernel: more taps per point, a better
//      conditioned deconvolution);
//   3. the rows of the grid tiles that sort the points and hold the spreading
//      accumulators (16, 32, 64; 32 columns);
//   4. the Legendre rings per thread of the forward and adjoint kernels (1, 2,
//      and 4 for FP32 plans with the restarted recursion).
// Each candidate is timed over `reps` forward + adjoint pairs after one warm-up
// pair, with CUDA events on the caller's stream.  No counterpart in the paper.
#include <cuda_runtime.h>

#include <string>

#include "internal.h"

using namespace gsl;

namespace {

__global__ void k_fill(float *p, int64_t n, uint32_t seed)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t h = (uint32_t)i * 2654435761u ^ seed;
    h ^= h >> 15;
    h *= 2246822519u;
    h ^= h >> 13;
    p[i] = ((float)(h & 0xffff) - 32768.0f) * (1.0f / 32768.0f);
}

// fills n floats, or n / 2 doubles, with values in [-1, 1)
cudaError_t fill(void *p, size_t bytes, bool f64, cudaStream_t st)
{
    if (!f64) {
        const int64_t n = (int64_t)(bytes / 4);
        if (n > 0) k_fill<<<(unsigned)((n + 255) / 256), 256, 0, st>>>((float *)p, n, 12345u);
        return cudaGetLastError();
    }
    // doubles: every value 2^-15 (top byte 0x3f, the rest zero) is enough for timing
    const int64_t n = (int64_t)(bytes / 8);
    cudaError_t e = cudaMemsetAsync(p, 0, bytes, st);
    if (e != cudaSuccess || n == 0) return e;
    return cudaMemset2DAsync((char *)p + 7, 8, 0x3f, 1, (size_t)n, st);
}

struct Timer {
    cudaEvent_t a = nullptr, b = nullptr;
    Timer() { cudaEventCreate(&a); cudaEventCreate(&b); }
    ~Timer() { cudaEventDestroy(a); cudaEventDestroy(b); }
};

// milliseconds of one forward + adjoint pair, or a negative value on failure
double time_plan(lens_plan pl, void *alm, void *map, int reps, cudaStream_t st)
{
    if (lens_synthesis(pl, alm, map, 1, st) != LENS_OK || lens_adjoint(pl, map, alm, 1, st) != LENS_OK) return -1.0;
    Timer t;
    cudaEventRecord(t.a, st);
    for (int r = 0; r < reps; ++r) {
        if (lens_synthesis(pl, alm, map, 1, st) != LENS_OK || lens_adjoint(pl, map, alm, 1, st) != LENS_OK)
            return -1.0;
    }
    cudaEventRecord(t.b, st);
    if (cudaEventSynchronize(t.b) != cudaSuccess) return -1.0;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, t.a, t.b);
    return (double)ms / reps;
}

}  // namespace

extern "C" int lens_autotune(int lmax, int mmax, int spin, int64_t npoints, const double *theta_d,
                             const double *phi_d, const double *chi_d, double epsilon, int prec, void *stream,
                             int reps, lens_plan_params *best, double *best_ms)
{
    if (!best || reps < 1) return record_failure(LENS_ERR_INVALID, "lens_autotune: NULL best or reps < 1");
    cudaStream_t st = (cudaStream_t)stream;
    const bool f64 = prec == LENS_FP64;
    const int ncomp = spin ? 2 : 1;
    const int64_t nalm = lens_nalm(lmax, mmax);
    if (nalm <= 0) return record_failure(LENS_ERR_INVALID, "lens_autotune: bad lmax / mmax");
    const size_t alm_b = (size_t)nalm * ncomp * (f64 ? 16 : 8), map_b = (size_t)npoints * ncomp * (f64 ? 8 : 4);
    void *alm = nullptr, *map = nullptr;
    cudaError_t e = cudaMalloc(&alm, alm_b);
    if (e == cudaSuccess) e = cudaMalloc(&map, map_b > 0 ? map_b : 16);
    if (e == cudaSuccess) e = fill(alm, alm_b, f64, st);
    if (e != cudaSuccess) {
        cudaFree(alm);
        cudaFree(map);
        return record_failure(e == cudaErrorMemoryAllocation ? LENS_ERR_NOMEM : LENS_ERR_CUDA,
                              "lens_autotune: buffers");
    }
    lens_plan_params cur = {};
    lens_plan_params win = {};
    double win_ms = -1.0;
    int win_W = 0;  // kernel support of the winning plan
    auto trial = [&](const lens_plan_params &prm) {
        lens_plan pl = nullptr;
        if (lens_plan_create_ex(&pl, lmax, mmax, spin, npoints, theta_d, phi_d, chi_d, epsilon, prec, 0, stream,
                                &prm) != LENS_OK)
            return;  // candidate outside this build's limits
        const double ms = time_plan(pl, alm, map, reps, st);
        lens_plan_info_t inf;
        const int w = lens_plan_info(pl, &inf) == LENS_OK ? inf.W : 0;
        lens_plan_destroy(pl);
        if (ms > 0 && (win_ms < 0 || ms < win_ms)) { win_ms = ms; win = prm; win_W = w; }
    };
    const double sig_cand[] = {1.25, 1.5, 1.75, 2.0, 2.25, 2.5};
    for (double sg : sig_cand) {
        cur = {};
        cur.sigma = sg;
        trial(cur);
    }
    if (win_ms > 0 && win_W > 0 && win_W < 16) {  // 2. one tap wider at the best sigma
        cur = win;
        cur.W = win_W + 1;
        trial(cur);
    }
    if (win_ms > 0) {  // 3. tile rows of the point sort / spreading accumulators
        const lens_plan_params base = win;
        for (int tr : {16, 64}) {
            cur = base;
            cur.spread_tile_rows = tr;
            trial(cur);
        }
    }
    if (win_ms > 0) {  // 4. Legendre rings per thread (4: restarted FP32 recursion only)
        const lens_plan_params base = win;
        const int rmax = prec == LENS_FP32 ? 4 : 2;
        for (int rf = 1; rf <= rmax; rf *= 2)
            for (int ra = 1; ra <= rmax; ra *= 2) {
                cur = base;
                cur.legendre_rpt_fwd = rf;
                cur.legendre_rpt_adj = ra;
                trial(cur);
            }
    }
    cudaFree(alm);
    cudaFree(map);
    if (win_ms < 0) return record_failure(LENS_ERR_UNSUPPORTED, "lens_autotune: no candidate plan could be built");
    *best = win;
    if (best->W == 0) best->W = win_W;  // report the support the winning plan used
    if (best_ms) *best_ms = win_ms;
    return LENS_OK;
}
