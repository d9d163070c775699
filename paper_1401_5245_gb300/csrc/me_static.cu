// me_edges_staged_static: the staged five-pass form with its mask image in
// a fixed, file-scope device array instead of memory taken from an
// allocator, for callers that must not allocate device memory once they
// are running.
//
// The array belongs to the library's CUDA module: every GPU that loads the
// library holds kStaticMaskWords * 4 bytes for it until the process exits.
// With CUDA's lazy module loading (the default) the driver places the module,
// and so the array, in device memory only when it is first used, which is
// the address lookup below: the first call on a device is therefore where
// the 4 MiB is taken, and a caller whose device memory is capped or handed
// to a caching allocator later must make that first call before then.
// In host code the name g_static_mask is only a host-side stand-in, never a
// device address, so its device address is looked up once per device with
// cudaGetSymbolAddress (on the first call with that device current) and
// cached.  A device reset (cudaDeviceReset) reloads the module, possibly
// elsewhere, so me_shutdown() forgets the cached addresses and the next call
// looks them up again.  Every call on a device shares the one array: it is
// fully rewritten by pass 1 before passes 2-5 read it, so nothing left by an
// earlier call is ever read, but two calls whose work overlaps on the GPU
// (different streams, no ordering between them) race on it.
#include <mutex>

#include "me_internal.h"

namespace me {

// Largest mask image the array holds: h * stride_words words (4 MiB).
constexpr size_t kStaticMaskWords = ME_STATIC_MASK_WORDS;

static __device__ __align__(256) uint32_t g_static_mask[kStaticMaskWords];

static std::mutex g_static_mu;
static uint32_t *g_static_ptr[64] = {};

// Device address of g_static_mask on the current device (set-up on first
// use per device).
static int static_mask_ptr(uint32_t **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return record_cuda(e);
    if (dev < 0 || dev >= 64) return ME_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (g_static_ptr[dev] == nullptr) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_mask);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return record_cuda(e != cudaSuccess ? e : cudaErrorInvalidSymbol);
        }
        g_static_ptr[dev] = static_cast<uint32_t *>(p);
    }
    *out = g_static_ptr[dev];
    return ME_OK;
}

// Forget every cached address (me_shutdown): after a device reset the next
// call looks the array up again in the reloaded module.
void static_forget_all() {
    std::lock_guard<std::mutex> lk(g_static_mu);
    for (auto &p : g_static_ptr) p = nullptr;
}

}  // namespace me

using namespace me;

extern "C" int me_edges_staged_static(const uint32_t *img, int32_t w, int32_t h,
                                      int32_t stride_words, uint32_t *edge,
                                      int32_t boundary, me_stream_t stream) {
    int rc = check_image_args(img, edge, w, h, stride_words, boundary);
    if (rc != ME_OK) return rc;
    if ((size_t)h * (size_t)stride_words > kStaticMaskWords) return ME_ERR_TOO_BIG;
    if ((rc = check_device_ptr(img)) != ME_OK) return rc;
    if ((rc = check_device_ptr(edge)) != ME_OK) return rc;
    uint32_t *mask = nullptr;
    if ((rc = static_mask_ptr(&mask)) != ME_OK) return rc;
    const Geo g = make_geo(img, w, h, stride_words, boundary, 1);
    cudaError_t e = launch_staged(g, mask, edge, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return record_cuda(e);
    }
    return ME_OK;
}
