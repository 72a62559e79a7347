// Sort-free tile binning.
//
// 3DGS replicates each Gaussian into every tile its footprint touches and
// then sorts each tile's list by depth (Sec. 4.1, Fig. 2).  Eq. 7 is a sum,
// so the order inside a tile does not matter and the sort goes away; what is
// left is a counting pass, an exclusive scan over tiles and an unordered
// scatter (a counting sort by tile with arbitrary order inside each tile).
//
//   k_bin_count    one thread per (view, Gaussian): atomicAdd into its tiles
//   k_scan_*       exclusive scan of the per-tile counts (three phases)
//   k_bin_scatter  one thread per (view, Gaussian): claim a slot per tile
#include "wsr_launch.h"

namespace wsr {
namespace {

// Tile rectangle of a record: tiles holding a pixel centre within the
// 3-sigma extents.  Returns false when the footprint misses the image.
__device__ __forceinline__ bool tile_rect(const float4 r0, const float4 r2, const View& V, int tw,
                                          int th, int& tx0, int& tx1, int& ty0, int& ty1) {
    if (!(r2.y >= 0.0f)) return false;          // culled (or NaN)
    if (!(fabsf(r0.x) < 1e30f) || !(fabsf(r0.y) < 1e30f) || !(r2.y < 1e30f) || !(r2.z < 1e30f)) return false;
    // pixel j is inside when |j + 0.5 - mu| <= extent; bounds kept within [-1, W]
    const float fw = (float)V.W, fh = (float)V.H;
    const float xlo = fminf(fmaxf(r0.x - r2.y - 0.5f, -1.0f), fw), xhi = fmaxf(fminf(r0.x + r2.y - 0.5f, fw), -1.0f);
    const float ylo = fminf(fmaxf(r0.y - r2.z - 0.5f, -1.0f), fh), yhi = fmaxf(fminf(r0.y + r2.z - 0.5f, fh), -1.0f);
    const int jx0 = max((int)ceilf(xlo), 0), jx1 = min((int)floorf(xhi), V.W - 1);
    const int jy0 = max((int)ceilf(ylo), 0), jy1 = min((int)floorf(yhi), V.H - 1);
    if (jx0 > jx1 || jy0 > jy1) return false;
    tx0 = jx0 / tw; tx1 = jx1 / tw;
    ty0 = jy0 / th; ty1 = jy1 / th;
    return true;
}

__global__ void __launch_bounds__(256) k_bin_count(const float4* __restrict__ rec, long long n, const Views vs,
                                                   unsigned* __restrict__ cursor) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int v = blockIdx.y;
    if (i >= n) return;
    const View& V = vs.v[v];
    const long long r = (long long)v * n + i;
    const float4 r0 = __ldg(rec + 3 * r), r2 = __ldg(rec + 3 * r + 2);
    int tx0, tx1, ty0, ty1;
    if (!tile_rect(r0, r2, V, vs.tile_w, vs.tile_h, tx0, tx1, ty0, ty1)) return;
    for (int ty = ty0; ty <= ty1; ++ty)
        for (int tx = tx0; tx <= tx1; ++tx) atomicAdd(cursor + V.tile_base + ty * V.tiles_x + tx, 1u);
}

__global__ void __launch_bounds__(256) k_bin_scatter(const float4* __restrict__ rec, long long n, const Views vs,
                                                     unsigned* __restrict__ cursor, unsigned* __restrict__ list,
                                                     unsigned long long capacity, WsHeader* hdr) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int v = blockIdx.y;
    if (i >= n) return;
    const View& V = vs.v[v];
    const long long r = (long long)v * n + i;
    const float4 r0 = __ldg(rec + 3 * r), r2 = __ldg(rec + 3 * r + 2);
    int tx0, tx1, ty0, ty1;
    if (!tile_rect(r0, r2, V, vs.tile_w, vs.tile_h, tx0, tx1, ty0, ty1)) return;
    for (int ty = ty0; ty <= ty1; ++ty)
        for (int tx = tx0; tx <= tx1; ++tx) {
            const unsigned slot = atomicAdd(cursor + V.tile_base + ty * V.tiles_x + tx, 1u);
            if (slot < capacity) list[slot] = (unsigned)r;
            else set_error(hdr, WSR_ERR_CAPACITY);
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

}  // namespace

cudaError_t launch_bin_count(const float* records, long long n, const Views& vs, unsigned* cursor,
                             cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(cursor, 0, sizeof(unsigned) * (size_t)vs.total_tiles, s);
    if (e != cudaSuccess || n == 0) return e;
    dim3 grid((unsigned)((n + 255) / 256), (unsigned)vs.n);
    k_bin_count<<<grid, 256, 0, s>>>(reinterpret_cast<const float4*>(records), n, vs, cursor);
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
    k_bin_scatter<<<grid, 256, 0, s>>>(reinterpret_cast<const float4*>(records), n, vs, cursor, list, capacity,
                                       hdr);
    return cudaGetLastError();
}

}  // namespace wsr
