// Batched Legendre synthesis on the tensor cores (tcgen05.mma, kind::tf32).
//
// Sect. 3's synthesis step for B maps of one geometry is, for every order m,
// the dense contraction
//     F_b(theta_j) = sum_l a_lm,b lambda_lm(theta_j)
// of a (rings x degrees) matrix of Legendre values with a (degrees x 2B)
// matrix of coefficients (real and imaginary parts of B maps).  Spin 0, FP32
// plans with the restarted FP32 recursion (legendre.cu): the Legendre values
// are generated on the fly, 128 rings per CTA (one ring per thread), in
// chunks of 32 degrees l = lf + 32 c .. lf + 32 c + 31 (lf = m + 1), written
// into shared memory in the tensor core's layout; the coefficients of a chunk
// arrive by one bulk copy from a buffer prepared per call (k_tc_prep).
//
// The degrees of a chunk are split by the parity of l - lf: north sums
// E + O and south sums s0 (E - O) (lambda(pi - theta) = (-1)^(l+m) lambda),
// so the two accumulators E and O (each 128 x 2B FP32 in tensor memory) give
// both hemispheres.  Degree l0 = m itself is added in the epilogue.
//
// Precision: TF32 keeps 11 significant bits, so every operand is split into
// hi = v rounded to TF32 and lo = v - hi (exact in FP32, |lo| <= 2^-12 |v|),
// and each product is hi*hi + hi*lo + lo*hi (three MMAs; the dropped lo*lo
// term and the TF32 truncation of lo are below 2^-23 relative): FP32-level
// products, accumulated in FP32 by the tensor core.
//
// Shared-memory operand layout (no swizzle, K-major): 8-row x 16-byte core
// matrices (8 rows x 4 TF32 values along K); core matrix (row group g,
// K group q) at byte (4 g + q) * 128 of a 16-column tile, so K neighbours are
// 128 bytes apart (leading byte offset) and row groups 512 bytes (stride byte
// offset).  One MMA (K = 8) covers two K groups; the second starts 256 bytes on.
//
// Pipeline: two stages.  While the tensor core multiplies chunk c (stage
// c & 1), the threads generate chunk c + 1 into the other stage; a stage is
// rewritten only after the MMAs that read it have completed (tcgen05.commit
// on an mbarrier).  Every wait is bounded (about 2 s); a wait that gives up
// sets FLAG_TIMEOUT in the plan's status word, the kernel stops issuing work,
// waits (bounded) for what it issued, frees its tensor memory and returns.
#include <cuda_runtime.h>
#include <math.h>

#include "common.cuh"
#include "internal.h"
#include "legendre_rec.cuh"

namespace gsl {
namespace {

constexpr int kTcRows = 128;     // rings per CTA (MMA M)
constexpr int kTcChunk = 32;     // degrees per chunk (16 per parity: the MMA K of a tile)
constexpr int kTcTileK = 16;     // K of one parity tile
constexpr int kTcABytes = kTcRows * kTcTileK * 4;  // one A tile (8 KB)

__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr)
{
    uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)(128 >> 4) << 16;  // leading byte offset: K neighbours
    d |= (uint64_t)(512 >> 4) << 32;  // stride byte offset: 8-row groups
    d |= (uint64_t)1 << 46;           // descriptor version of this architecture
    return d;                         // base offset 0, no swizzle
}

// kind::tf32 instruction descriptor: D F32, A and B TF32, both K-major, M x N
__host__ __device__ constexpr uint32_t tc_idesc(int m, int n)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
                 "l"(a), "l"(b), "r"(idesc), "r"(acc)
                 : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}

// 32 consecutive FP32 columns of this warp's 32 tensor-memory lanes
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                   "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                   "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                   "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// v rounded to TF32 (nearest, ties away from zero), as an FP32 value with the low 13 bits zero
__device__ __forceinline__ float tf32_hi(float v)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
    return __uint_as_float(r);
}

// Byte offset of (row r, K group q) in a 16-column tile (16-byte row of a core matrix).
__device__ __forceinline__ int tc_off(int r, int q) { return (((r >> 3) * 4 + q) << 7) + ((r & 7) << 4); }

// One block of 8 degrees from l (l - lf a multiple of 8): values of the even
// (rel +1) and odd (rel -1) degrees.  GUARD: degrees above lmax give 0 and do
// not advance the recursion.
template <class P, int REG, bool GUARD>
__device__ __forceinline__ void tc_block(Rings<P, 1, false> &st, const float4 *reca, int l, int lmax, float (&ev)[4],
                                         float (&od)[4])
{
#pragma unroll
    for (int j = 0; j < kBlk; ++j) {
        float v = 0.f;
        if (!GUARD || l + j <= lmax) {
            if (j & 1) {
                st.template advance<1, REG != 0>(reca, nullptr, l + j);
                if (REG != 1) v = st.template vplus<1, REG == 2>(0);
            } else {
                st.template advance<0, REG != 0>(reca, nullptr, l + j);
                if (REG != 1) v = st.template vplus<0, REG == 2>(0);
            }
        }
        if (j & 1) od[j >> 1] = v;
        else ev[j >> 1] = v;
    }
}

// Kernel body for one recursion form (P = PolS or PolR, uniform over the CTA:
// the Reinsch boundary is a multiple of 128 rings).  NB = maps (MMA N = 2 NB).
template <class P, int NB>
__device__ __forceinline__ void tc_body(const float *__restrict__ coefB, const int64_t *__restrict__ cbase,
                                        const float2 *__restrict__ alm, int64_t nalm, int nm, const void *rec_s,
                                        const double *__restrict__ lognorm, const RingTab &rt,
                                        float2 *__restrict__ ring, int64_t ring_stride, int lmax, int ntheta,
                                        int nnorth, const CkTab &ck, unsigned *status, unsigned char *smem)
{
    constexpr int N = 2 * NB;
    constexpr int BBYTES = N * kTcTileK * 4;          // one B tile
    constexpr int STAGE = 4 * kTcABytes + 4 * BBYTES;  // A: E hi, E lo, O hi, O lo; B likewise
    constexpr uint32_t COLS = 2 * N;                   // accumulators E | O
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m = blockIdx.y;
    const int l0 = m, lf = m + 1;
    const int jn = blockIdx.x * kTcRows + tid;  // north ring of this thread
    const int64_t base = alm_base(lmax, m);
    const float4 *reca = (const float4 *)rec_s + base;
    const int nch = lmax >= lf ? (lmax - lf + kTcChunk) / kTcChunk : 0;

    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + 2 * STAGE);  // b_full[2], mma_done[2]
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 4);
    __shared__ int c0_sh;

    // ---- recursion state: the warp's first restart, then the CTA's (the smallest)
    Rings<P, 1, false> st;
    int kj = first_restart<1>(ck, m);
    if (ck.K < kTcChunk) kj = 0;  // restarts finer than a chunk: start from the start value
    if (tid == 0) c0_sh = 0x7fffffff;
    __syncthreads();
    if (lane == 0) atomicMin(&c0_sh, kj);
    __syncthreads();
    const int kc = c0_sh;
    const int c0 = (int)min((int64_t)kc * ck.K / kTcChunk, (int64_t)nch);  // first chunk
    float lam0 = 0.f;
    if (kc == 0) {
        st.init(rt, jn, nnorth, m, 0, lognorm[m]);
        lam0 = st.template vplus<1, true>(0);
    } else {
        st.init_geom(rt, jn, nnorth);
    }

    if (tid == 0) {
        mbar_init(bars + 0, 1);
        mbar_init(bars + 1, 1);
        mbar_init(bars + 2, 1);
        mbar_init(bars + 3, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                     "r"(COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const uint32_t idesc = tc_idesc(kTcRows, N);
    const int64_t ckrow = __ldg(ck.base + m);
    bool ok = true;
    int issued = -1;  // last chunk whose MMAs were committed
    // Every decision to stop is taken by the whole CTA (__syncthreads_and), so no barrier is ever
    // reached by only some of its warps.
    for (int c = c0; c < nch; ++c) {
        const int t = c - c0, s = t & 1;
        unsigned char *stg = smem + s * STAGE;
        const bool free_ok = t < 2 || mbar_wait_warp(bars + 2 + s, ((t >> 1) - 1) & 1);  // MMAs of chunk c - 2
        if (!__syncthreads_and(free_ok ? 1 : 0)) {
            ok = false;
            break;
        }
        if (tid == 0) {
            mbar_expect_tx(bars + s, 4 * BBYTES);
            bulk_copy_g2s(stg + 4 * kTcABytes, coefB + (size_t)(cbase[m] + c) * (4 * BBYTES / 4), 4 * BBYTES,
                          bars + s);
        }
        // generate the chunk's Legendre values into the A tiles of stage s
#pragma unroll 1
        for (int q = 0; q < 4; ++q) {
            const int l = lf + c * kTcChunk + q * kBlk;
            const int dl = l - lf;
            if (dl != 0 && (dl & (ck.K - 1)) == 0 && l + kBlk <= lmax + 1)
                st.restart(ck, ckrow + (int64_t)(dl / ck.K - 1) * nnorth, jn, nnorth);
            float ev[4], od[4];
            const int reg = st.regime();
            if (l + kBlk <= lmax + 1) {
                if (reg == 0) tc_block<P, 0, false>(st, reca, l, lmax, ev, od);
                else if (reg == 1) tc_block<P, 1, false>(st, reca, l, lmax, ev, od);
                else tc_block<P, 2, false>(st, reca, l, lmax, ev, od);
            } else {
                tc_block<P, 2, true>(st, reca, l, lmax, ev, od);
            }
            float4 eh, el, oh, ol;
            eh.x = tf32_hi(ev[0]); eh.y = tf32_hi(ev[1]); eh.z = tf32_hi(ev[2]); eh.w = tf32_hi(ev[3]);
            el = make_float4(ev[0] - eh.x, ev[1] - eh.y, ev[2] - eh.z, ev[3] - eh.w);
            oh.x = tf32_hi(od[0]); oh.y = tf32_hi(od[1]); oh.z = tf32_hi(od[2]); oh.w = tf32_hi(od[3]);
            ol = make_float4(od[0] - oh.x, od[1] - oh.y, od[2] - oh.z, od[3] - oh.w);
            const int off = tc_off(tid, q);
            *reinterpret_cast<float4 *>(stg + 0 * kTcABytes + off) = eh;
            *reinterpret_cast<float4 *>(stg + 1 * kTcABytes + off) = el;
            *reinterpret_cast<float4 *>(stg + 2 * kTcABytes + off) = oh;
            *reinterpret_cast<float4 *>(stg + 3 * kTcABytes + off) = ol;
        }
        fence_async_shared();  // generic-proxy writes of the A tiles -> visible to the tensor core
        __syncthreads();
        bool got = true;
        if (warp == 0) {
            got = mbar_wait_warp(bars + s, (t >> 1) & 1);  // coefficients of chunk c arrived
            if (got) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                if (lane == 0) {
                    const uint32_t a0 = smem_addr(stg), b0 = smem_addr(stg + 4 * kTcABytes);
#pragma unroll
                    for (int par = 0; par < 2; ++par) {
                        const uint32_t d = tmem + par * N;
                        const uint32_t ah = a0 + (2 * par) * kTcABytes, al = ah + kTcABytes;
                        const uint32_t bh = b0 + (2 * par) * BBYTES, bl = bh + BBYTES;
#pragma unroll
                        for (int ks = 0; ks < kTcTileK / 8; ++ks) {
                            const uint32_t o = ks * 256;
                            tc_mma(d, tc_desc(ah + o), tc_desc(bh + o), idesc, (t > 0 || ks > 0) ? 1u : 0u);
                            tc_mma(d, tc_desc(ah + o), tc_desc(bl + o), idesc, 1u);
                            tc_mma(d, tc_desc(al + o), tc_desc(bh + o), idesc, 1u);
                        }
                    }
                    tc_commit(bars + 2 + s);
                }
                __syncwarp();
            }
        }
        if (!__syncthreads_and(got ? 1 : 0)) {  // warp 0 issued nothing for chunk c
            ok = false;
            break;
        }
        issued = c;
    }
    // wait for the last committed MMAs (bounded), then read the accumulators
    bool have = false;
    if (issued >= c0) {
        const int t = issued - c0;
        have = __syncthreads_and(mbar_wait_warp(bars + 2 + (t & 1), (t >> 1) & 1) ? 1 : 0) != 0;
        if (!have) ok = false;
    }
    if (!ok && tid == 0) atomicOr(status, FLAG_TIMEOUT);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    const bool real_m = m == 0;
    const bool write = jn < nnorth && ok;
    const int js = ntheta - 1 - jn;
#pragma unroll 1
    for (int g = 0; g < N / 32; ++g) {  // 16 maps per column group
        float ev[32], od[32];
        if (have) {
            tc_ld32(tmem + ((uint32_t)(warp * 32) << 16) + g * 32, ev);
            tc_ld32(tmem + ((uint32_t)(warp * 32) << 16) + N + g * 32, od);
        } else {
#pragma unroll
            for (int i = 0; i < 32; ++i) { ev[i] = 0.f; od[i] = 0.f; }
        }
        if (write) {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int b = g * 16 + i;
                if (b >= nm) break;
                float2 a0 = __ldg(alm + (int64_t)b * nalm + base + l0);
                if (real_m) a0.y = 0.f;
                float2 *col = ring + b * ring_stride + (int64_t)m * ntheta;
                // north E + O, south s0 (E - O) with s0 = (-1)^(lf - m) = -1; degree l0 = m adds a0 lambda_l0 to both
                col[jn] = make_float2(ev[2 * i] + od[2 * i] + a0.x * lam0, ev[2 * i + 1] + od[2 * i + 1] + a0.y * lam0);
                if (js != jn)
                    col[js] = make_float2(od[2 * i] - ev[2 * i] + a0.x * lam0, od[2 * i + 1] - ev[2 * i + 1] + a0.y * lam0);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(COLS) : "memory");
}

template <int NB>
__global__ void __launch_bounds__(kTcRows) k_leg_fwd_tc(const float *__restrict__ coefB, const int64_t *__restrict__ cbase,
                                                       const float2 *__restrict__ alm, int64_t nalm, int nm,
                                                       const void *rec_s, const double *__restrict__ lognorm, RingTab rt,
                                                       float2 *__restrict__ ring, int64_t ring_stride, int lmax,
                                                       int ntheta, int nnorth, CkTab ck, unsigned *status)
{
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    if (blockIdx.x * kTcRows < ck.jb)
        tc_body<PolR, NB>(coefB, cbase, alm, nalm, nm, rec_s, lognorm, rt, ring, ring_stride, lmax, ntheta, nnorth, ck,
                          status, tc_smem);
    else
        tc_body<PolS, NB>(coefB, cbase, alm, nalm, nm, rec_s, lognorm, rt, ring, ring_stride, lmax, ntheta, nnorth, ck,
                          status, tc_smem);
}

// Coefficient tiles of one call: for every order m and chunk c, four tiles
// (even hi, even lo, odd hi, odd lo) of 2 NB rows (map b: row 2b real part,
// 2b + 1 imaginary part; zero for b >= nm) x 16 degrees l = lf + 32 c + 2 k
// (+1 for odd), in the core-matrix layout above; zero beyond lmax; m = 0
// imaginary parts dropped (real fields).
template <int NB>
__global__ void k_tc_prep(const float2 *__restrict__ alm, int64_t nalm, int nm, int lmax,
                          const int64_t *__restrict__ cbase, float *__restrict__ out)
{
    constexpr int N = 2 * NB;
    const int m = blockIdx.y;
    const int lf = m + 1;
    const int nch = lmax >= lf ? (lmax - lf + kTcChunk) / kTcChunk : 0;
    const int64_t base = alm_base(lmax, m);
    const int per = N * kTcTileK;  // entries of one parity (rows x degrees)
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)nch * per; i += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(i / per), e = (int)(i % per);
        const int n = e / kTcTileK, k = e % kTcTileK;
        const int b = n >> 1;
        float v[2] = {0.f, 0.f};  // even, odd
#pragma unroll
        for (int par = 0; par < 2; ++par) {
            const int l = lf + c * kTcChunk + 2 * k + par;
            if (b < nm && l <= lmax) {
                const float2 a = __ldg(alm + (int64_t)b * nalm + base + l);
                v[par] = (n & 1) ? (m == 0 ? 0.f : a.y) : a.x;
            }
        }
        float *ch = out + (size_t)(cbase[m] + c) * (4 * N * kTcTileK);
        const int off = ((((n >> 3) * 4 + (k >> 2)) << 7) + ((n & 7) << 4) + ((k & 3) << 2)) >> 2;  // floats
#pragma unroll
        for (int par = 0; par < 2; ++par) {
            const float h = tf32_hi(v[par]);
            ch[(2 * par) * per + off] = h;
            ch[(2 * par + 1) * per + off] = v[par] - h;
        }
    }
}

template <int NB> size_t tc_smem()
{
    return 2 * (size_t)(4 * kTcABytes + 4 * 2 * NB * kTcTileK * 4) + 64;
}

}  // namespace

// Chunks of order m and the prepared-coefficient offsets (host)
int64_t tc_chunks(int lmax, int m) { return lmax >= m + 1 ? (lmax - m - 1 + kTcChunk) / kTcChunk : 0; }

size_t tc_coef_floats(int nb, int64_t chunks) { return (size_t)chunks * 4 * 2 * nb * kTcTileK; }

cudaError_t launch_legendre_fwd_tc(const Plan &p, const void *alm, int nm, void *ring, void *coefB,
                                   const int64_t *cbase, int nb, cudaStream_t st)
{
    const dim3 g((p.nnorth + kTcRows - 1) / kTcRows, p.mmax + 1);
    const dim3 gp(64, p.mmax + 1);
    const int64_t rs = (int64_t)p.ncol * p.ntheta;
    cudaError_t e = cudaSuccess;
    auto run = [&](auto prep, auto kern, size_t smem) {
        prep<<<gp, 256, 0, st>>>((const float2 *)alm, p.nalm, nm, p.lmax, cbase, (float *)coefB);
        if ((e = cudaGetLastError()) != cudaSuccess) return;
        if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
            return;
        kern<<<g, kTcRows, smem, st>>>((const float *)coefB, cbase, (const float2 *)alm, p.nalm, nm, p.rec_s,
                                       p.lognorm, p.rings, (float2 *)ring, rs, p.lmax, p.ntheta, p.nnorth, p.ck,
                                       p.flags + 1);
        e = cudaGetLastError();
    };
    if (nb == 16) run(k_tc_prep<16>, k_leg_fwd_tc<16>, tc_smem<16>());
    else if (nb == 32) run(k_tc_prep<32>, k_leg_fwd_tc<32>, tc_smem<32>());
    else if (nb == 64) run(k_tc_prep<64>, k_leg_fwd_tc<64>, tc_smem<64>());
    else return cudaErrorInvalidValue;
    return e;
}

}  // namespace gsl
