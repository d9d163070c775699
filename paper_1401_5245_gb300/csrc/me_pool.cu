// Scratch memory for the calls that need some (the staged form's mask, the
// in-place seams or image copy, the Otsu histogram): a stream-ordered memory
// pool the library owns per device.  CUDA's default pool gives its memory
// back to the system at every synchronisation, so a call made after one
// paid for mapping fresh memory (measured: 156 us for an in-place call on a
// 32768 x 32768 image that takes 50-59 us in a stream of calls).  This pool
// keeps up to kKeepBytes reserved between calls; me_shutdown() destroys it.
#include <mutex>

#include "me_internal.h"

namespace me {

namespace {

constexpr uint64_t kKeepBytes = 512ull << 20;

std::mutex g_pool_mu;
cudaMemPool_t g_pools[64] = {};

}  // namespace

cudaError_t scratch_alloc(void **p, size_t bytes, cudaStream_t s) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    cudaMemPool_t pool;
    {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        if (g_pools[dev] == nullptr) {
            cudaMemPoolProps props = {};
            props.allocType = cudaMemAllocationTypePinned;
            props.handleTypes = cudaMemHandleTypeNone;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            cudaMemPool_t np = nullptr;
            if ((e = cudaMemPoolCreate(&np, &props)) != cudaSuccess) return e;
            uint64_t keep = kKeepBytes;
            if ((e = cudaMemPoolSetAttribute(np, cudaMemPoolAttrReleaseThreshold, &keep)) !=
                cudaSuccess) {
                cudaMemPoolDestroy(np);
                return e;
            }
            g_pools[dev] = np;
        }
        pool = g_pools[dev];
    }
    return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

cudaError_t scratch_free(void *p, cudaStream_t s) { return cudaFreeAsync(p, s); }

int scratch_shutdown() {
    int cur = 0;
    cudaGetDevice(&cur);
    std::lock_guard<std::mutex> lk(g_pool_mu);
    for (int d = 0; d < 64; ++d) {
        if (g_pools[d] == nullptr) continue;
        cudaSetDevice(d);
        cudaDeviceSynchronize();
        cudaMemPoolDestroy(g_pools[d]);
        g_pools[d] = nullptr;
    }
    cudaGetLastError();
    cudaSetDevice(cur);
    return ME_OK;
}

}  // namespace me
