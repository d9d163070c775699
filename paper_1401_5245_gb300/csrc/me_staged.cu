// The method of masks as five separate whole-image passes, the way Section 2
// runs it: one bit-block transfer with a raster operation per step, each
// reading its sources from and writing its destination to memory.
//   pass 1  M  = NOT I                 (Section 3, mask construction)
//   pass 2  E  = M AND I(x-1)          (Section 4, left edge)
//   pass 3  E |= M AND I(x+1)          (right edge, ORed in: Section 5)
//   pass 4  E |= M AND I(y-1)          (up edge)
//   pass 5  E |= M AND I(y+1)          (down edge)
// One thread per word, 32-bit accesses.  Kept as the baseline form.
#include <algorithm>

#include "me_internal.h"

namespace me {

struct StageGeo {
    int32_t h, stride, nw;
    uint32_t lastmask, fill;
    uint32_t words;          // h * stride (< 2^32, checked by the launcher)
};

// Word i of the image is word c of row y; every word of every row is
// visited, padding words included, so outputs are written whole (0 there).
__device__ __forceinline__ void stage_index(const StageGeo &g, uint32_t i, int &y, int &c) {
    y = (int)(i / (uint32_t)g.stride);
    c = (int)(i - (uint32_t)y * (uint32_t)g.stride);
}

// Image word with the outside colour in its padding bits.
__device__ __forceinline__ uint32_t stage_load(const StageGeo &g, const uint32_t *img,
                                               int y, int c) {
    if (y < 0 || y >= g.h || c < 0 || c >= g.nw) return g.fill;
    uint32_t x = img[(size_t)y * g.stride + c];
    if (c == g.nw - 1) x = (x & g.lastmask) | (g.fill & ~g.lastmask);
    return x;
}

__global__ void k_stage_not(const uint32_t *img, uint32_t *M, StageGeo g) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < g.words;
         i += gridDim.x * blockDim.x) {
        int y, c;
        stage_index(g, i, y, c);
        const size_t at = (size_t)y * g.stride + c;
        const uint32_t valid = c < g.nw - 1 ? kAllOnes : (c == g.nw - 1 ? g.lastmask : 0u);
        M[at] = ~img[at] & valid;
    }
}

__global__ void k_stage_left(const uint32_t *img, const uint32_t *M, uint32_t *E,
                             StageGeo g) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < g.words;
         i += gridDim.x * blockDim.x) {
        int y, c;
        stage_index(g, i, y, c);
        const size_t at = (size_t)y * g.stride + c;
        const uint32_t cur = stage_load(g, img, y, c);
        const uint32_t prev = stage_load(g, img, y, c - 1);
        E[at] = M[at] & ((cur << 1) | (prev >> 31));
    }
}

__global__ void k_stage_right(const uint32_t *img, const uint32_t *M, uint32_t *E,
                              StageGeo g) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < g.words;
         i += gridDim.x * blockDim.x) {
        int y, c;
        stage_index(g, i, y, c);
        const size_t at = (size_t)y * g.stride + c;
        const uint32_t cur = stage_load(g, img, y, c);
        const uint32_t next = stage_load(g, img, y, c + 1);
        E[at] |= M[at] & ((cur >> 1) | (next << 31));
    }
}

// dy = -1: the image moved down one row (up edge); dy = +1: moved up.
__global__ void k_stage_vertical(const uint32_t *img, const uint32_t *M, uint32_t *E,
                                 StageGeo g, int dy) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < g.words;
         i += gridDim.x * blockDim.x) {
        int y, c;
        stage_index(g, i, y, c);
        const size_t at = (size_t)y * g.stride + c;
        E[at] |= M[at] & stage_load(g, img, y + dy, c);
    }
}

cudaError_t launch_staged(const Geo &geo, uint32_t *mask, uint32_t *edge,
                          cudaStream_t s) {
    const uint64_t words = (uint64_t)geo.h * (uint64_t)geo.stride;
    if (words >= (1ull << 32)) return cudaErrorInvalidValue;
    StageGeo g{geo.h, geo.stride, geo.nw, geo.lastmask, geo.fill, (uint32_t)words};
    DevInfo di;
    if (device_info(&di) != ME_OK) return cudaErrorInvalidDevice;
    const int threads = 256;
    const uint64_t want = (words + threads - 1) / threads;
    const int grid = (int)std::max<uint64_t>(
        1, std::min<uint64_t>(want, (uint64_t)di.sm_count * 8));
    k_stage_not<<<grid, threads, 0, s>>>(geo.img, mask, g);
    k_stage_left<<<grid, threads, 0, s>>>(geo.img, mask, edge, g);
    k_stage_right<<<grid, threads, 0, s>>>(geo.img, mask, edge, g);
    k_stage_vertical<<<grid, threads, 0, s>>>(geo.img, mask, edge, g, -1);
    k_stage_vertical<<<grid, threads, 0, s>>>(geo.img, mask, edge, g, +1);
    return cudaGetLastError();
}

}  // namespace me
