// Shared device helpers: complex arithmetic on float2/double2 and
// double-float ("df32") arithmetic on pairs of FP32 numbers.
//
// df32 numbers represent x = h + l with |l| <= ulp(h)/2 after normalisation.
// Products use the FMA error-free transform (p = a*b, e = fma(a, b, -p)),
// sums use Knuth's two-sum; every rounding step is written with the
// __f*_rn intrinsics so the compiler cannot contract or reassociate it.
// The Legendre recursion of FP32 plans runs in df32 because a plain FP32
// three-term recursion loses 1e-5..1e-3 relative accuracy at lmax ~ 4096
// (rounding of the recursion state accumulates over thousands of steps),
// while GB300's FP64 pipe is a small fraction of its FP32 rate.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gsl {

template <typename T> struct cplx_of;
template <> struct cplx_of<float> { using type = float2; };
template <> struct cplx_of<double> { using type = double2; };
template <typename T> using cplx = typename cplx_of<T>::type;

__host__ __device__ __forceinline__ float2 mkc(float r, float i) { return make_float2(r, i); }
__host__ __device__ __forceinline__ double2 mkc(double r, double i) { return make_double2(r, i); }

template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) { return mkc(a.x + b.x, a.y + b.y); }
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) { return mkc(a.x - b.x, a.y - b.y); }
template <typename C> __host__ __device__ __forceinline__ C cconj(C a) { return mkc(a.x, -a.y); }
template <typename C, typename T> __host__ __device__ __forceinline__ C cscale(C a, T s) { return mkc(a.x * s, a.y * s); }
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b)
{
    return mkc(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename C> __host__ __device__ __forceinline__ C cmulc(C a, C b)
{
    return mkc(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
// multiply by +i or -i
template <typename C> __host__ __device__ __forceinline__ C cmul_i(C a) { return mkc(-a.y, a.x); }
template <typename C> __host__ __device__ __forceinline__ C cmul_mi(C a) { return mkc(a.y, -a.x); }

// ------------------------------------------------------------------ df32
struct df32 {
    float h, l;
};

// a * b for df32 a, b (result not renormalised: |l| is small but may exceed ulp(h)/2)
__device__ __forceinline__ df32 df_mul(df32 a, df32 b)
{
    float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    return {p, e};
}

// a - b, renormalised (two-sum on the high parts, low parts added to the error)
__device__ __forceinline__ df32 df_sub(df32 a, df32 b)
{
    float s = __fsub_rn(a.h, b.h);
    float bb = __fsub_rn(s, a.h);
    float err = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(-b.h, bb));
    err = __fadd_rn(err, __fsub_rn(a.l, b.l));
    float h = __fadd_rn(s, err);
    float l = __fsub_rn(err, __fsub_rn(h, s));
    return {h, l};
}

// a - b without the final renormalisation: (s, e) with s = fl(a.h - b.h) and
// e the exact two-sum error plus the low parts, so s + e carries the full
// df32 accuracy and |e| is at most a few ulp of max(|a|, |b|).  df_mul accepts
// such pairs; s alone is off from a - b by at most |e|.
__device__ __forceinline__ df32 df_sub_u(df32 a, df32 b)
{
    float s = __fsub_rn(a.h, b.h);
    float bb = __fsub_rn(s, a.h);
    float err = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(-b.h, bb));
    err = __fadd_rn(err, __fsub_rn(a.l, b.l));
    return {s, err};
}

__device__ __forceinline__ df32 df_scale_pow2(df32 a, float p2) { return {a.h * p2, a.l * p2}; }

// v as h + l (h = v rounded to FP32, l the rest rounded: relative error ~2^-48)
__device__ __forceinline__ df32 df_split(double v)
{
    const float h = (float)v;
    return {h, (float)(v - (double)h)};
}
__device__ __forceinline__ double df_value(df32 a) { return (double)a.h + (double)a.l; }

// s += (p, e) for a product (p, e) of df_mul: two-sum on the high words, the
// error and e into the low word (s not renormalised)
__device__ __forceinline__ void df_acc(df32 &s, df32 t)
{
    const float h = __fadd_rn(s.h, t.h);
    const float bb = __fsub_rn(h, s.h);
    const float err = __fadd_rn(__fsub_rn(s.h, __fsub_rn(h, bb)), __fsub_rn(t.h, bb));
    s.l = __fadd_rn(s.l, __fadd_rn(err, t.l));
    s.h = h;
}
// two-sum renormalisation (exact for any ordering of |h|, |l|)
__device__ __forceinline__ df32 df_renorm(df32 a)
{
    const float h = __fadd_rn(a.h, a.l);
    const float bb = __fsub_rn(h, a.h);
    return {h, __fadd_rn(__fsub_rn(a.h, __fsub_rn(h, bb)), __fsub_rn(a.l, bb))};
}

// Fixed-point accumulation (deterministic plans): a sum whose terms are
// bounded by `bound` in total is accumulated as integers in units of 2^-k,
// with k the largest integer up to 122 such that bound 2^k <= 2^62 (so the
// int64 sums cannot overflow); returns 2^k, 1 for a zero bound and NaN for a
// bound that is not finite.
__device__ __forceinline__ double fx_unit(double bound)
{
    if (!(bound <= 1.7976931348623157e308)) return __longlong_as_double(0x7ff8000000000000LL);
    if (bound <= 0.0) return 1.0;
    int e = ilogb(bound) + 1;  // bound < 2^e
    if (e < -60) e = -60;
    return ldexp(1.0, 62 - e);
}
// integer sum v in units of 1 / (inv) -> value, one rounding
template <typename T> __device__ __forceinline__ T fx_value(long long v, double inv);
template <> __device__ __forceinline__ float fx_value<float>(long long v, double inv) { return __ll2float_rn(v) * (float)inv; }
template <> __device__ __forceinline__ double fx_value<double>(long long v, double inv) { return __ll2double_rn(v) * inv; }

// ---- bulk copies (TMA, non-tensor form) into shared memory, completed on an mbarrier
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
// makes barrier initialisation and earlier generic-proxy accesses of shared
// memory visible to the async proxy (bulk copies)
__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
// bytes (a multiple of 16) from a 16-byte aligned global address to a 16-byte
// aligned shared address; completes `bytes` of the barrier's transaction count
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok)
                 : "r"(smem_addr(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}
// Whole-warp wait for phase `parity` of bar: every lane observes the
// completion itself; gives up (uniformly, returning false) after about
// kWaitCycles clock cycles.
constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz
__device__ __forceinline__ bool mbar_wait_warp(uint64_t *bar, uint32_t parity, long long limit = kWaitCycles)
{
    const long long t0 = clock64();
    for (;;) {
        const bool done = mbar_try_wait(bar, parity);
        if (__all_sync(0xffffffffu, done)) return true;
        const bool late = clock64() - t0 > limit;
        if (__shfl_sync(0xffffffffu, late, 0)) return false;
    }
}

// Status flags written by kernels (bitwise OR).  No kernel traps.
enum : unsigned {
    FLAG_DOMAIN = 1u,     // point coordinate not finite / theta outside [0, pi]
    FLAG_OOB = 2u,        // an index check failed; the access was skipped
    FLAG_TIMEOUT = 4u,    // a bounded wait on a bulk copy gave up; the result is incomplete
};

}  // namespace gsl
