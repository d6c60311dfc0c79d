// FMA throughput of the CUDA-core pipes, measured: the denominator of the
// ALU rooflines (the Legendre recursion is ALU work, not a contraction).
//
// Every thread runs NCH independent chains x <- fma(x, a, b) for `iters`
// steps, so the measured rate is the issue rate of FMA instructions (2 flops
// per lane each) with the latency hidden by NCH-way independence and several
// warps per scheduler.  The grid is a whole number of waves over the SMs.
#include <cuda_runtime.h>

#include <string>

#include "internal.h"

namespace {

constexpr int kNch = 8;

template <typename T> __global__ void __launch_bounds__(256) k_fma_chain(T *out, int iters, T a, T b)
{
    T x[kNch];
#pragma unroll
    for (int i = 0; i < kNch; ++i) x[i] = (T)(threadIdx.x + 1) * (T)1e-3 + (T)i;
#pragma unroll 4
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kNch; ++i) x[i] = fma(x[i], a, b);
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < kNch; ++i) s += x[i];
    if (s == (T)-1) out[blockIdx.x] = s;  // never true (all chains stay positive): keeps the work live
}

template <typename T> cudaError_t time_chain(int sms, int iters, cudaStream_t st, double &flops_per_s)
{
    T *out = nullptr;  // written only if the impossible condition above holds: never dereferenced
    const int blocks = sms * 8, threads = 256;
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return e;
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) { cudaEventDestroy(e0); return e; }
    const T a = (T)0.999999, b = (T)1e-6;
    k_fma_chain<T><<<blocks, threads, 0, st>>>(out, iters / 4, a, b);  // warm-up (clocks ramp up)
    cudaEventRecord(e0, st);
    k_fma_chain<T><<<blocks, threads, 0, st>>>(out, iters, a, b);
    cudaEventRecord(e1, st);
    if ((e = cudaGetLastError()) == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return e;
    flops_per_s = 2.0 * kNch * (double)iters * blocks * threads / (ms * 1e-3);
    return cudaSuccess;
}

}  // namespace

extern "C" int lens_measure_fma_peak(int prec, double *flops_per_s, void *stream)
{
    using namespace gsl;
    if (!flops_per_s || (prec != LENS_FP32 && prec != LENS_FP64))
        return record_failure(LENS_ERR_INVALID, "lens_measure_fma_peak: prec must be LENS_FP32 or LENS_FP64");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) {
        cudaStream_t st = (cudaStream_t)stream;
        // about 0.25 s per timed launch on GB300 (FP32 ~80 TFLOP/s, FP64 ~1.3 TFLOP/s)
        e = prec == LENS_FP32 ? time_chain<float>(sms, 1 << 12, st, *flops_per_s)
                              : time_chain<double>(sms, 1 << 6, st, *flops_per_s);
    }
    if (e != cudaSuccess) {
        const std::string m = std::string("lens_measure_fma_peak: ") + cudaGetErrorString(e);
        return record_failure(LENS_ERR_CUDA, m.c_str());
    }
    return LENS_OK;
}
