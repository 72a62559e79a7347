// Sort-free tile binning.
//
// 3DGS replicates each Gaussian into every tile its footprint touches and
// then sorts each tile's list by depth (Sec. 4.1, Fig. 2).  Eq. 7 is a sum,
// so the order inside a tile does not matter and the sort goes away; what is
// left is a counting pass, an exclusive scan over tiles and an unordered
// scatter (a counting sort by tile with arbitrary order inside each tile).
//
//   k_bin<false>   count: atomicAdd into every tile the footprint reaches
//   k_scan_*       exclusive scan of the per-tile counts (three phases)
//   k_bin<true>    scatter: claim a slot per (Gaussian, tile) and store
// A tile is listed when the footprint q <= 9 reaches one of its pixel
// centres (exact ellipse-rectangle test), not merely its bounding box.
#include "wsr_launch.h"

namespace wsr {
namespace {

// Pixel rectangle of a record: pixels whose centre lies within the 3-sigma
// extents, clipped to the image.  Returns false when it misses the image.
__device__ __forceinline__ bool pixel_rect(const float4 r0, const float4 r2, const View& V, int& jx0, int& jx1,
                                           int& jy0, int& jy1) {
    if (!(r2.y >= 0.0f)) return false;          // culled (or NaN)
    if (!(fabsf(r0.x) < 1e30f) || !(fabsf(r0.y) < 1e30f) || !(r2.y < 1e30f) || !(r2.z < 1e30f)) return false;
    // pixel j is inside when |j + 0.5 - mu| <= extent; bounds kept within [-1, W]
    const float fw = (float)V.W, fh = (float)V.H;
    const float xlo = fminf(fmaxf(r0.x - r2.y - 0.5f, -1.0f), fw), xhi = fmaxf(fminf(r0.x + r2.y - 0.5f, fw), -1.0f);
    const float ylo = fminf(fmaxf(r0.y - r2.z - 0.5f, -1.0f), fh), yhi = fmaxf(fminf(r0.y + r2.z - 0.5f, fh), -1.0f);
    jx0 = max((int)ceilf(xlo), 0);
    jx1 = min((int)floorf(xhi), V.W - 1);
    jy0 = max((int)ceilf(ylo), 0);
    jy1 = min((int)floorf(yhi), V.H - 1);
    return jx0 <= jx1 && jy0 <= jy1;
}

// Binning pass.  Each warp takes 32 consecutive Gaussians of one view; their
// tile rectangles are laid end to end (warp scan) and the lanes walk that
// list of candidate (Gaussian, tile) pairs together, 32 at a time, so a large
// footprint is spread over the warp.  A candidate counts when the footprint
// reaches a pixel centre of the tile.  COUNT: atomicAdd per tile.  SCATTER:
// claim a slot in the tile's segment and write the record index.
template <bool SCATTER>
__global__ void __launch_bounds__(256) k_bin(const float4* __restrict__ rec, long long n, const Views vs,
                                             unsigned* __restrict__ cursor, unsigned* __restrict__ list,
                                             unsigned long long capacity, WsHeader* hdr) {
    __shared__ int s_end[8][32];        // inclusive prefix of candidate counts
    __shared__ int s_rect[8][32][3];    // tx0, ty0, tiles across
    __shared__ float s_geo[8][32][5];   // mu_x, mu_y, qs, qw, qd
    const int v = blockIdx.y;
    const View& V = vs.v[v];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int tw = vs.tile_w, th = vs.tile_h;
    int cnt = 0, tx0 = 0, ty0 = 0, nx = 0;
    float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0;
    if (i < n) {
        const long long r = (long long)v * n + i;
        r0 = __ldg(rec + 3 * r);
        r1 = __ldg(rec + 3 * r + 1);
        const float4 r2 = __ldg(rec + 3 * r + 2);
        int jx0, jx1, jy0, jy1;
        if (pixel_rect(r0, r2, V, jx0, jx1, jy0, jy1)) {
            tx0 = jx0 / tw;
            ty0 = jy0 / th;
            nx = jx1 / tw - tx0 + 1;
            cnt = nx * (jy1 / th - ty0 + 1);
        }
    }
    int inc = cnt;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += y;
    }
    s_end[warp][lane] = inc;
    s_rect[warp][lane][0] = tx0;
    s_rect[warp][lane][1] = ty0;
    s_rect[warp][lane][2] = nx;
    s_geo[warp][lane][0] = r0.x;
    s_geo[warp][lane][1] = r0.y;
    s_geo[warp][lane][2] = r0.z;
    s_geo[warp][lane][3] = r0.w;
    s_geo[warp][lane][4] = r1.x;
    __syncwarp();
    const int total = __shfl_sync(0xffffffffu, inc, 31);
    for (int base = 0; base < total; base += 32) {
        const int c = base + lane;
        if (c < total) {
            // owner: first lane whose inclusive end exceeds c
            int lo = 0, hi = 31;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (s_end[warp][mid] > c) hi = mid;
                else lo = mid + 1;
            }
            const int k = c - (lo ? s_end[warp][lo - 1] : 0);   // candidate index within the owner's rectangle
            const int w = s_rect[warp][lo][2];
            const int tx = s_rect[warp][lo][0] + k % w;
            const int ty = s_rect[warp][lo][1] + k / w;
            const float x0 = (float)(tx * tw) + 0.5f, x1 = (float)min(tx * tw + tw, V.W) - 0.5f;
            const float y0 = (float)(ty * th) + 0.5f, y1 = (float)min(ty * th + th, V.H) - 0.5f;
            const float* geo = s_geo[warp][lo];
            if (footprint_hits(geo[0], geo[1], geo[2], geo[3], geo[4], x0, x1, y0, y1)) {
                unsigned* cur = cursor + V.tile_base + ty * V.tiles_x + tx;
                if constexpr (SCATTER) {
                    const unsigned slot = atomicAdd(cur, 1u);
                    const long long rid = (long long)v * n + (long long)blockIdx.x * blockDim.x + warp * 32 + lo;
                    if (slot < capacity) list[slot] = (unsigned)rid;
                    else set_error(hdr, WSR_ERR_CAPACITY);
                } else {
                    atomicAdd(cur, 1u);
                }
            }
        }
    }
}

// --------------------------------------------------------------------------
// Exclusive scan over tiles: (1) per-block totals, (2) one block scans the
// totals and writes the grand total, (3) per-block scan plus block offset.
// --------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long block_exclusive_scan(unsigned long long x, unsigned long long* s_warp,
                                                                   unsigned long long& total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long inc = x;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        unsigned long long t = lane < nw ? s_warp[lane] : 0ull;
        unsigned long long ti = t;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, ti, off);
            if (lane >= off) ti += y;
        }
        if (lane < nw) s_warp[lane] = ti - t;
        if (lane == 31) s_warp[32] = ti;
    }
    __syncthreads();
    total = s_warp[32];
    const unsigned long long r = s_warp[warp] + inc - x;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanBlock) k_scan_reduce(const unsigned* __restrict__ cnt, int n,
                                                            unsigned long long* __restrict__ bsum) {
    __shared__ unsigned long long s_warp[33];
    const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
    unsigned long long x = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < n) x += cnt[base + k];
    unsigned long long tot;
    block_exclusive_scan(x, s_warp, tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanBlock) k_scan_top(unsigned long long* __restrict__ bsum, int nb,
                                                         unsigned* __restrict__ offsets, int n_tiles,
                                                         unsigned long long capacity, WsHeader* hdr) {
    __shared__ unsigned long long s_warp[33];
    unsigned long long carry = 0;
    for (int base = 0; base < nb; base += kScanBlock) {
        const int j = base + threadIdx.x;
        const unsigned long long x = j < nb ? bsum[j] : 0ull;
        unsigned long long tot;
        const unsigned long long ex = block_exclusive_scan(x, s_warp, tot);
        if (j < nb) bsum[j] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) {
        // offsets never exceed the list capacity, so the renderers stay in
        // bounds even when the list overflowed; the true total goes to the
        // workspace header for the caller to size a larger list
        const unsigned long long lim = capacity < 0xffffffffull ? capacity : 0xffffffffull;
        offsets[n_tiles] = (unsigned)(carry < lim ? carry : lim);
        hdr->total = carry;
        if (carry > lim) set_error(hdr, WSR_ERR_CAPACITY);
    }
}

__global__ void __launch_bounds__(kScanBlock) k_scan_apply(unsigned* __restrict__ cursor, int n,
                                                           const unsigned long long* __restrict__ bsum,
                                                           unsigned* __restrict__ offsets,
                                                           unsigned long long capacity) {
    const unsigned long long lim = capacity < 0xffffffffull ? capacity : 0xffffffffull;
    __shared__ unsigned long long s_warp[33];
    const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
    unsigned c[kScanItems];
    unsigned long long x = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        c[k] = (base + k < n) ? cursor[base + k] : 0u;
        x += c[k];
    }
    unsigned long long tot;
    unsigned long long run = bsum[blockIdx.x] + block_exclusive_scan(x, s_warp, tot);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) {
            const unsigned o = (unsigned)(run < lim ? run : lim);
            offsets[base + k] = o;
            cursor[base + k] = o;   // scatter cursor starts at the tile's offset
        }
        run += c[k];
    }
}

// Longest-first tile order for the persistent schedule: tiles are bucketed by
// the magnitude of their instance count (floor(log2)), buckets taken from the
// largest down; the order inside a bucket is arbitrary.
__device__ __forceinline__ int cost_bucket(unsigned c) { return c ? 32 - __clz(c) : 0; }   // 0..32

__global__ void __launch_bounds__(256) k_order_hist(const unsigned* __restrict__ offsets, int n,
                                                    unsigned* __restrict__ hist) {
    __shared__ unsigned h[33];
    if (threadIdx.x < 33) h[threadIdx.x] = 0;
    __syncthreads();
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x)
        atomicAdd(&h[cost_bucket(offsets[t + 1] - offsets[t])], 1u);
    __syncthreads();
    if (threadIdx.x < 33 && h[threadIdx.x]) atomicAdd(hist + threadIdx.x, h[threadIdx.x]);
}

__global__ void k_order_scan(unsigned* __restrict__ hist) {
    // hist[0..32] -> cursors hist[33..65]: start of each bucket, largest bucket first
    if (threadIdx.x == 0) {
        unsigned run = 0;
        for (int b = 32; b >= 0; --b) {
            hist[33 + b] = run;
            run += hist[b];
        }
    }
}

__global__ void __launch_bounds__(256) k_order_scatter(const unsigned* __restrict__ offsets, int n,
                                                       unsigned* __restrict__ hist, unsigned* __restrict__ order) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const unsigned pos = atomicAdd(hist + 33 + cost_bucket(offsets[t + 1] - offsets[t]), 1u);
        order[pos] = (unsigned)t;
    }
}

}  // namespace

cudaError_t launch_tile_order(const Views& vs, const unsigned* offsets, unsigned* buckets, unsigned* order,
                              cudaStream_t s) {
    const int n = vs.total_tiles;
    cudaError_t e = cudaMemsetAsync(buckets, 0, sizeof(unsigned) * 33, s);
    if (e != cudaSuccess || n == 0) return e;
    const int nb = min((n + 255) / 256, 1024);
    k_order_hist<<<nb, 256, 0, s>>>(offsets, n, buckets);
    k_order_scan<<<1, 32, 0, s>>>(buckets);
    k_order_scatter<<<nb, 256, 0, s>>>(offsets, n, buckets, order);
    return cudaGetLastError();
}

cudaError_t launch_bin_count(const float* records, long long n, const Views& vs, unsigned* cursor,
                             cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(cursor, 0, sizeof(unsigned) * (size_t)vs.total_tiles, s);
    if (e != cudaSuccess || n == 0) return e;
    dim3 grid((unsigned)((n + 255) / 256), (unsigned)vs.n);
    k_bin<false><<<grid, 256, 0, s>>>(reinterpret_cast<const float4*>(records), n, vs, cursor, nullptr, 0ull,
                                      nullptr);
    return cudaGetLastError();
}

cudaError_t launch_scan(const Views& vs, unsigned* cursor, unsigned* block_sums, unsigned* offsets,
                        unsigned long long capacity, WsHeader* hdr, cudaStream_t s) {
    const int n = vs.total_tiles;
    const int nb = (n + kScanTile - 1) / kScanTile;
    unsigned long long* bsum = reinterpret_cast<unsigned long long*>(block_sums);
    k_scan_reduce<<<nb, kScanBlock, 0, s>>>(cursor, n, bsum);
    k_scan_top<<<1, kScanBlock, 0, s>>>(bsum, nb, offsets, n, capacity, hdr);
    k_scan_apply<<<nb, kScanBlock, 0, s>>>(cursor, n, bsum, offsets, capacity);
    return cudaGetLastError();
}

cudaError_t launch_bin_scatter(const float* records, long long n, const Views& vs, unsigned* cursor,
                               unsigned* list, unsigned long long capacity, WsHeader* hdr, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    dim3 grid((unsigned)((n + 255) / 256), (unsigned)vs.n);
    k_bin<true><<<grid, 256, 0, s>>>(reinterpret_cast<const float4*>(records), n, vs, cursor, list, capacity, hdr);
    return cudaGetLastError();
}

}  // namespace wsr
