// me_edges_inplace: the edge map written over the image it is computed from.
//
// Every output row needs the original rows above and below it, so a row may
// be overwritten only once nobody still has to read it.  The image is cut
// into bands of band_rows rows; one CTA owns a band across the whole row
// width and walks it top to bottom.  Each thread owns up to C vector
// columns of 4 words and reads and writes global memory only there: at row
// y it holds the original rows y-1 and y in registers and has already
// loaded the rows below up to y+PF+1, computes row y and overwrites it.
// The words just left and right of each thread's columns (the neighbouring
// columns' words of row y) are exchanged through shared memory, one
// barrier per row, double-buffered, so within a band no thread ever reads
// a row another thread has overwritten.
//
// Between CTAs the only shared rows are at the band seams: the last row of
// a band is the row above the next band, and the first row of a band is the
// row below the previous one.  A first kernel copies those two rows of
// every seam into scratch before any band starts, and bands read their
// outer halo rows from there.
#include <algorithm>

#include "me_internal.h"

namespace me {

namespace {

constexpr int kIpPF = 2;                // rows loaded ahead of the next row
constexpr int kIpMaxThreads = 1024;

struct IpGeo {
    uint32_t *img;
    const uint32_t *seam;               // rows 2k, 2k+1: seam k (bands k, k+1)
    int32_t h, stride, nw, nv;          // nv = vector columns of 4 words
    uint32_t lastmask, fill;
    int32_t band_rows, nbands;
};

__device__ __forceinline__ uint32_t ip_keep(const IpGeo &g, int c) {
    return (c >= 0 && c < g.nw - 1) ? kAllOnes : (c == g.nw - 1 ? g.lastmask : 0u);
}

// Where row y comes from for band b: the image inside the band, the seam
// copies for the rows just outside it, nothing (boundary colour) beyond.
__device__ __forceinline__ const uint32_t *ip_row(const IpGeo &g, int b, int y0, int y1, int y) {
    if (y >= y0 && y < y1) return g.img + (size_t)y * (size_t)g.stride;
    if (y == y0 - 1 && y >= 0) return g.seam + (size_t)(2 * (b - 1)) * (size_t)g.stride;
    if (y == y1 && y < g.h) return g.seam + (size_t)(2 * b + 1) * (size_t)g.stride;
    return nullptr;
}

// Row y's 4 words at column c0, outside words and padding replaced by the
// boundary colour.
template <bool V16>
__device__ __forceinline__ uint4 ip_load(const IpGeo &g, const uint32_t *row, int c0,
                                         bool active) {
    uint32_t raw[4] = {0u, 0u, 0u, 0u};
    if (row != nullptr && active) {
        if constexpr (V16) {
            if (c0 < g.nw) {
                const uint4 v = *reinterpret_cast<const uint4 *>(row + c0);
                raw[0] = v.x; raw[1] = v.y; raw[2] = v.z; raw[3] = v.w;
            }
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (c0 + k < g.nw) raw[k] = row[c0 + k];
        }
    }
    uint32_t o[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint32_t keep = row != nullptr ? ip_keep(g, c0 + k) : 0u;
        o[k] = (raw[k] & keep) | (g.fill & ~keep);
    }
    return make_uint4(o[0], o[1], o[2], o[3]);
}

__device__ __forceinline__ uint32_t q_at(const uint4 &q, int i) {
    return i == 0 ? q.x : i == 1 ? q.y : i == 2 ? q.z : q.w;
}

template <int C, bool V16>
__global__ void __launch_bounds__(kIpMaxThreads)
k_inplace(IpGeo g) {
    // first and last word of every vector column of the current row
    __shared__ uint32_t s_first[2][2 * kIpMaxThreads], s_last[2][2 * kIpMaxThreads];
    const int b = blockIdx.x;
    const int y0 = b * g.band_rows;
    const int y1 = min(y0 + g.band_rows, g.h);
    const int T = blockDim.x;

    int c0[C];
    bool active[C];
#pragma unroll
    for (int k = 0; k < C; ++k) {
        const int v = threadIdx.x + k * T;
        active[k] = v < g.nv;
        c0[k] = v * 4;
    }
    auto load = [&](int k, int y) {
        return ip_load<V16>(g, ip_row(g, b, y0, y1, y), c0[k], active[k]);
    };

    uint4 up[C], cur[C], q[C][kIpPF + 1];
#pragma unroll
    for (int k = 0; k < C; ++k) {
        up[k] = load(k, y0 - 1);
        cur[k] = load(k, y0);
#pragma unroll
        for (int i = 0; i <= kIpPF; ++i) q[k][i] = load(k, y0 + 1 + i);
    }

    int buf = 0;
#pragma unroll 1
    for (int y = y0; y < y1; y += kIpPF + 1) {
#pragma unroll
        for (int j = 0; j <= kIpPF; ++j) {
            const int yy = y + j;
            if (yy >= y1) break;
#pragma unroll
            for (int k = 0; k < C; ++k) {
                const int v = threadIdx.x + k * T;
                s_first[buf][v] = cur[k].x;
                s_last[buf][v] = cur[k].w;
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < C; ++k) {
                const uint4 dn = q[k][j];
                // rows up to y1 only: those further down belong to other bands
                q[k][j] = load(k, yy + kIpPF + 2 <= y1 ? yy + kIpPF + 2 : -2);
                const int v = threadIdx.x + k * T;
                const uint32_t prev = v > 0 ? s_last[buf][v - 1] : g.fill;
                const uint32_t next = v + 1 < C * T ? s_first[buf][v + 1] : g.fill;
                uint32_t e[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const uint32_t x = q_at(cur[k], i);
                    const uint32_t pv = i == 0 ? prev : q_at(cur[k], i - 1);
                    const uint32_t nx = i == 3 ? next : q_at(cur[k], i + 1);
                    const uint32_t L = __funnelshift_l(pv, x, 1);   // I(x-1, y)
                    const uint32_t R = __funnelshift_r(x, nx, 1);   // I(x+1, y)
                    e[i] = ~x & (L | R | q_at(up[k], i) | q_at(dn, i)) & ip_keep(g, c0[k] + i);
                }
                if (active[k]) {
                    uint32_t *out = g.img + (size_t)yy * (size_t)g.stride + c0[k];
                    if constexpr (V16) {
                        *reinterpret_cast<uint4 *>(out) = make_uint4(e[0], e[1], e[2], e[3]);
                    } else {
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            if (c0[k] + i < g.stride) out[i] = e[i];
                    }
                }
                up[k] = cur[k];
                cur[k] = dn;
            }
            buf ^= 1;
        }
    }
}

// Rows on both sides of every seam into scratch: seam k = rows
// (k+1) * band_rows - 1 and (k+1) * band_rows.
__global__ void k_inplace_seams(IpGeo g, uint32_t *seam) {
    const int rows = 2 * (g.nbands - 1);
    for (int r = blockIdx.x; r < rows; r += gridDim.x) {
        const int y = (r / 2 + 1) * g.band_rows - 1 + (r & 1);
        const uint32_t *src = g.img + (size_t)y * (size_t)g.stride;
        uint32_t *dst = seam + (size_t)r * (size_t)g.stride;
        for (int c = threadIdx.x; c < g.stride; c += blockDim.x) dst[c] = src[c];
    }
}

template <int C, bool V16>
cudaError_t launch_inplace(const IpGeo &g, int threads, cudaStream_t s) {
    k_inplace<C, V16><<<g.nbands, threads, 0, s>>>(g);
    return cudaGetLastError();
}

}  // namespace

}  // namespace me

using namespace me;

extern "C" int me_edges_inplace(uint32_t *img, int32_t w, int32_t h, int32_t stride_words,
                                int32_t boundary, me_stream_t stream) {
    if (img == nullptr || w <= 0 || h <= 0 || stride_words <= 0 ||
        stride_words < (int32_t)(((int64_t)w + 31) / 32) ||
        (boundary != ME_BOUNDARY_WHITE && boundary != ME_BOUNDARY_BLACK) ||
        ((uintptr_t)img & 3))
        return ME_ERR_ARG;
    int rc = check_device_ptr(img);
    if (rc != ME_OK) return rc;
    DevInfo di;
    if ((rc = device_info(&di)) != ME_OK) return rc;
    const Geo geo = make_geo(img, w, h, stride_words, boundary, 4,
                             vec16_ok(img, img, stride_words));
    const int nv = geo.nv;
    const int C = nv <= kIpMaxThreads ? 1 : 2;
    if (nv > 2 * kIpMaxThreads) return ME_ERR_TOO_BIG;
    const int threads = std::max(32, ((nv + C - 1) / C + 31) / 32 * 32);

    IpGeo g;
    g.img = img;
    g.seam = nullptr;
    g.h = h;
    g.stride = stride_words;
    g.nw = geo.nw;
    g.nv = nv;
    g.lastmask = geo.lastmask;
    g.fill = geo.fill;
    // bands: about four CTAs per SM, at least 32 rows (seam copies stay
    // below 2 rows in 32 of extra traffic)
    const int64_t want = (int64_t)di.sm_count * 4;
    g.band_rows = (int32_t)std::max<int64_t>(32, (h + want - 1) / want);
    g.nbands = (int32_t)(((int64_t)h + g.band_rows - 1) / g.band_rows);

    const cudaStream_t s = (cudaStream_t)stream;
    uint32_t *seam = nullptr;
    cudaError_t e = cudaSuccess;
    if (g.nbands > 1) {
        const size_t bytes = (size_t)2 * (g.nbands - 1) * (size_t)stride_words * 4;
        if ((e = cudaMallocAsync(reinterpret_cast<void **>(&seam), bytes, s)) != cudaSuccess) {
            cudaGetLastError();
            return record_cuda(e);
        }
        g.seam = seam;
        const int rows = 2 * (g.nbands - 1);
        k_inplace_seams<<<std::min(rows, di.sm_count * 8), 256, 0, s>>>(g, seam);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        if (geo.vec16)
            e = C == 1 ? launch_inplace<1, true>(g, threads, s) : launch_inplace<2, true>(g, threads, s);
        else
            e = C == 1 ? launch_inplace<1, false>(g, threads, s)
                       : launch_inplace<2, false>(g, threads, s);
    }
    if (seam != nullptr) {
        const cudaError_t f = cudaFreeAsync(seam, s);
        if (e == cudaSuccess) e = f;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return record_cuda(e);
    }
    return ME_OK;
}
