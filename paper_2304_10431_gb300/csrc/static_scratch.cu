// Forward lensing transform that allocates nothing.
//
// Some callers cannot call cudaMalloc once they are running: for example a
// host program whose device memory is owned by another framework's allocator,
// or a service that reserves a fixed device-memory budget at start-up and
// forbids allocation afterwards.  lens_synthesis_static serves them: it runs
// the same four stages as lens_synthesis (Legendre synthesis, theta and phi
// transforms, interpolation) but takes its scratch (ring coefficients, torus
// rows and the oversampled grid) from the fixed array below instead of the
// plan's workspace, and calls no allocating routine.
//
// The array lives in every GPU that loads the library, until the process
// exits.  Its device address is looked up once per device, on the first call
// made with that device current; that first call should come before any
// stream capture.  All calls share the array and it keeps the contents of the
// last call: calls that overlap on the GPU (different streams, or several
// host threads) race on it.  A call also writes the plan's own prepared
// coefficients and status flags (allocated with the plan), as every
// transform on that plan does, so it must not overlap another call on the
// same plan either.
#include <cuda_runtime.h>
#include <stdio.h>

#include <mutex>
#include <string>

#include "internal.h"

namespace {

constexpr size_t kStaticScratchBytes = 64ull << 20;  // 64 MiB
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
void *g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mutex;

size_t align256(size_t n) { return (n + 255) & ~size_t(255); }

}  // namespace

extern "C" int lens_synthesis_static(lens_plan pl, const void *alm_d, void *map_d, void *stream)
{
    using namespace gsl;
    if (!pl || !alm_d || (!map_d && reinterpret_cast<const Plan *>(pl)->npts > 0))
        return record_failure(LENS_ERR_INVALID, "lens_synthesis_static: NULL argument");
    const Plan &p = *reinterpret_cast<const Plan *>(pl);
    const ScratchSizes scr = plan_scratch_sizes(p);  // the plan builder's own workspace sizes
    const size_t ring_b = scr.ring, x_b = scr.X, grid_b = scr.grid;
    const size_t need = align256(ring_b) + align256(x_b) + align256(grid_b);
    if (need > kStaticScratchBytes) {
        char msg[256];
        snprintf(msg, sizeof msg,
                 "lens_synthesis_static: the plan needs %zu bytes of scratch, above the fixed %zu-byte array; "
                 "use lens_synthesis", need, kStaticScratchBytes);
        return record_failure(LENS_ERR_UNSUPPORTED, msg);
    }
    if (p.device < 0 || p.device >= kMaxDevices)
        return record_failure(LENS_ERR_UNSUPPORTED, "lens_synthesis_static: device index out of range");
    int dev0 = -1;
    cudaGetDevice(&dev0);
    if (dev0 != p.device) cudaSetDevice(p.device);
    void *base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_scratch_mutex);
        if (!g_scratch_addr[p.device]) {
            void *ptr = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
            if (e != cudaSuccess) {
                if (dev0 != p.device) cudaSetDevice(dev0);
                std::string m = std::string("lens_synthesis_static: cudaGetSymbolAddress: ") + cudaGetErrorString(e);
                return record_failure(LENS_ERR_CUDA, m.c_str());
            }
            g_scratch_addr[p.device] = ptr;
        }
        base = g_scratch_addr[p.device];
    }
    unsigned char *b = static_cast<unsigned char *>(base);
    void *ring = b;
    void *X = b + align256(ring_b);
    void *grid = b + align256(ring_b) + align256(x_b);
    cudaStream_t st = stream ? (cudaStream_t)stream : p.stream;
    cudaError_t e = launch_legendre_fwd(p, alm_d, ring, st);  // zeroes the ring coefficients first
    if (e == cudaSuccess) e = launch_theta_fwd(p, ring, X, st);
    if (e == cudaSuccess) e = launch_phi_fwd(p, X, grid, st);
    if (e == cudaSuccess) e = launch_interp(p, grid, map_d, st);
    if (dev0 != p.device) cudaSetDevice(dev0);
    if (e != cudaSuccess) {
        std::string m = std::string("lens_synthesis_static: ") + cudaGetErrorString(e);
        return record_failure(LENS_ERR_CUDA, m.c_str());
    }
    return LENS_OK;
}
