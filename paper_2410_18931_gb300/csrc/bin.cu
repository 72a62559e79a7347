// Sort-free tile binning.
//
// 3DGS replicates each Gaussian into every tile its footprint touches and
// then sorts each tile's list by depth (Sec. 4.1, Fig. 2).  Eq. 7 is a sum,
// so the order inside a tile does not matter and the sort goes away; what is
// left is a counting pass, an exclusive scan over tiles and an unordered
// scatter (a counting sort by tile with arbitrary order inside each tile).
//
//   k_bin<false>   count: atomicAdd into every tile the footprint reaches
//   k_scan_*       exclusive scan of the per-tile counts (three phases; one
//                  block, with the persistent schedule's tile order, for up
//                  to kSmallScanTiles tiles)
//   k_bin<true>    scatter: claim a slot per (Gaussian, tile) and store
// A tile is listed when a pixel-centre column of it meets the footprint
// q <= 9 within the tile's band of pixel-centre rows (the ellipse's exact
// extent per tile row), not merely when it meets the bounding box.
#include <mutex>

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

// Binning pass.  Each warp takes 32 consecutive Gaussians of one view.  A
// Gaussian's work is cut into segments, one per tile row of its pixel
// rectangle (and, for footprints wider than kPiece tiles, one per kPiece
// tiles of that row); the warp lays its segments end to end and takes them
// 32 at a time, one per lane, so a large footprint is spread over the warp.
//
// A segment needs no per-tile test: the footprint q' <= QM is an ellipse, and
// its part inside the row's band of pixel-centre rows [y_a, y_b] is convex,
// so the tiles of the row it reaches are those whose pixel-centre columns
// meet that part's x-extent [x_l, x_r].  With A' = qw^2 + qd, B' = qs qw,
// C' = qs^2 the right edge of the ellipse at height dy is
//     x(dy) = (-B' dy + sqrt(A' QM - qd C' dy^2)) / A',
// a concave function whose maximum sqrt(QM / qd) lies at dy* = -(qw/qs)
// sqrt(QM / qd); x_r is x at the point of the band nearest dy*, and x_l
// follows by symmetry.  The extent is widened by a margin far above its FP32
// rounding error, so every pixel centre with q' <= QM is kept (a tile the
// ellipse only passes near is listed at worst).
//
// The 32 segments' tile ranges are then laid end to end again and the lanes
// take consecutive tiles, so the atomics of a warp fall on neighbouring
// counters of a few rows.  COUNT: atomicAdd per tile.  SCATTER: claim a slot
// in the tile's segment and write the record index.
constexpr int kPiece = 8;

template <bool SCATTER>
__global__ void __launch_bounds__(256) k_bin(const float4* __restrict__ rec, long long n, const Views vs,
                                             unsigned* __restrict__ cursor, unsigned* __restrict__ list,
                                             unsigned long long capacity, WsHeader* hdr) {
    __shared__ int s_start[8][32];      // each Gaussian's first segment (exclusive prefix of segment counts)
    __shared__ int s_gown[8][32];       // the lanes of the Gaussians with segments, in order
    __shared__ int4 s_rect[8][32];      // pixel rectangle: jx0, jx1, jy0, jy1
    __shared__ float4 s_geo[8][32][2];  // mu_x, mu_y, B'/A', A' QM | det', 1/A', dy*, margin
    __shared__ int2 s_run[8][32];       // per segment with tiles, in order: its first tile's counter, less
                                        // its first position in the batch, and the owning lane
    const int v = blockIdx.y;
    const View& V = vs.v[v];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int lw = __ffs(vs.tile_w) - 1, lh = __ffs(vs.tile_h) - 1;   // tile sides are powers of two
    const float QM = kQMax * 1.0001f + 1e-4f;
    int nseg = 0, jx0 = 0, jx1 = -1, jy0 = 0, jy1 = -1;
    float4 g0 = make_float4(0.f, 0.f, 0.f, 0.f), g1 = g0;
    if (i < n) {
        const long long r = (long long)v * n + i;
        const float4 r0 = __ldg(rec + 3 * r);
        const float qd = __ldg(reinterpret_cast<const float*>(rec + 3 * r + 1));
        const float4 r2 = __ldg(rec + 3 * r + 2);
        if (pixel_rect(r0, r2, V, jx0, jx1, jy0, jy1)) {
            const float qs = r0.z, qw = r0.w;
            // hardware reciprocal and square root (relative error ~2^-22, far below the margin below)
            const float A = fmaf(qw, qw, qd), ia = rcp_approx(A);
            const float dxm = sqrt_approx(QM * rcp_approx(qd));  // half-width of the ellipse
            g0 = make_float4(r0.x, r0.y, qs * qw * ia, A * QM);
            g1 = make_float4(qd * qs * qs, ia, -(qw * rcp_approx(qs)) * dxm, fminf(2e-3f * dxm, 1e6f) + 0.01f);
            const int pcs = ((jx1 >> lw) - (jx0 >> lw) + kPiece) / kPiece;
            nseg = ((jy1 >> lh) - (jy0 >> lh) + 1) * pcs;
        }
    }
    int inc = nseg;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += y;
    }
    const int gex = inc - nseg;                          // this Gaussian's first segment
    // the Gaussians with segments, in lane order: a segment's owner is found by counting starts (below)
    const unsigned gmask = __ballot_sync(0xffffffffu, nseg > 0);
    if (nseg > 0) s_gown[warp][__popc(gmask & ((1u << lane) - 1u))] = lane;
    s_start[warp][lane] = gex;
    s_rect[warp][lane] = make_int4(jx0, jx1, jy0, jy1);
    s_geo[warp][lane][0] = g0;
    s_geo[warp][lane][1] = g1;
    __syncwarp();
    const int total = __shfl_sync(0xffffffffu, inc, 31);
    for (int c0 = 0; c0 < total; c0 += 32) {
        // ---- this lane's segment c0 + lane: its owner is the last Gaussian with segments whose first
        // segment is at or before it (those starting before c0, plus the starts in the batch up to it) ----
        const unsigned gst = __reduce_or_sync(0xffffffffu, nseg > 0 && gex >= c0 && gex < c0 + 32 ? 1u << (gex - c0)
                                                                                               : 0u);
        const int gbefore = __popc(__ballot_sync(0xffffffffu, nseg > 0 && gex < c0));
        const int c = c0 + lane;
        int ta = 0, tb = -1, lo = 0, row = 0;
        if (c < total) {
            lo = s_gown[warp][gbefore + __popc(gst & ((2u << lane) - 1u)) - 1];
            const int k = c - s_start[warp][lo];                // segment index within the owner
            const int4 rc = s_rect[warp][lo];
            const float4 a = s_geo[warp][lo][0], b = s_geo[warp][lo][1];
            const int np = ((rc.y >> lw) - (rc.x >> lw) + kPiece) / kPiece;
            const int kr = np == 1 ? k : k / np, kp = k - kr * np;
            const int ty = (rc.z >> lh) + kr;
            // the row's band of pixel-centre rows, inside the footprint's rows
            const float dya = (float)max(ty << lh, rc.z) + 0.5f - a.y;
            const float dyb = (float)min(((ty + 1) << lh) - 1, rc.w) + 0.5f - a.y;
            auto edge = [&](float dy, float side) {
                return fmaf(-a.z, dy, side * sqrt_approx(fmaxf(fmaf(-b.x * dy, dy, a.w), 0.0f)) * b.y);
            };
            const float xr = edge(fminf(fmaxf(b.z, dya), dyb), 1.0f);
            const float xl = edge(fminf(fmaxf(-b.z, dya), dyb), -1.0f);
            // pixel columns whose centre lies in [mu_x + x_l, mu_x + x_r] (widened), clipped to the rectangle
            const float fa = fmaxf(ceilf(a.x + xl - b.w - 0.5f), (float)rc.x);
            const float fb = fminf(floorf(a.x + xr + b.w - 0.5f), (float)rc.y);
            if (fa <= fb) {
                const int p0 = (rc.x >> lw) + kp * kPiece;       // this segment's tiles of the row
                ta = max((int)fa >> lw, p0);
                tb = min((int)fb >> lw, p0 + kPiece - 1);
                row = V.tile_base + ty * V.tiles_x;
            }
        }
        // ---- the batch's tiles end to end, consecutive tiles to consecutive lanes; a tile's segment is
        // found the same way, by counting the segments that start at or before it ----
        const int wdt = max(tb - ta + 1, 0);   // a piece the band does not reach has none
        int winc = wdt;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, winc, off);
            if (lane >= off) winc += y;
        }
        const int nt = __shfl_sync(0xffffffffu, winc, 31);
        const int wex = winc - wdt;                      // this segment's first position in the batch
        const unsigned smask = __ballot_sync(0xffffffffu, wdt > 0);
        if (wdt > 0) s_run[warp][__popc(smask & ((1u << lane) - 1u))] = make_int2(row + ta - wex, lo);
        __syncwarp();
        for (int j0 = 0; j0 < nt; j0 += 32) {
            const unsigned sst = __reduce_or_sync(0xffffffffu, wdt > 0 && wex >= j0 && wex < j0 + 32 ? 1u << (wex - j0)
                                                                                                  : 0u);
            const int sbefore = __popc(__ballot_sync(0xffffffffu, wdt > 0 && wex < j0));
            const int j = j0 + lane;
            if (j < nt) {
                const int2 run = s_run[warp][sbefore + __popc(sst & ((2u << lane) - 1u)) - 1];
                unsigned* cur = cursor + run.x + j;
                if constexpr (SCATTER) {
                    const unsigned slot = atomicAdd(cur, 1u);
                    const long long rid = (long long)v * n + (long long)blockIdx.x * blockDim.x + warp * 32 + run.y;
                    if (slot < capacity) list[slot] = (unsigned)rid;
                    else set_error(hdr, WSR_ERR_CAPACITY);
                } else {
                    atomicAdd(cur, 1u);
                }
            }
        }
        __syncwarp();
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

// Exclusive scan over the tiles and, for the persistent schedule, the longest-first
// tile order (the buckets of k_order_*), in one block: for views of at most
// kSmallScanTiles tiles.  The counts pass through shared memory (dynamic, n + 1
// words) so that every global access is coalesced.  Warp w scans the
// consecutive tiles [w seg, (w + 1) seg), 32 at a time (lane l on tile 32 i + l
// of its range: no bank conflicts), after one block scan of the warps' totals.
constexpr int kSmallScanTiles = WSR_SCAN_ONE_BLOCK_TILES;
static_assert(kSmallScanTiles % kScanBlock == 0, "whole segments");

__global__ void __launch_bounds__(kScanBlock) k_scan_order_small(unsigned* __restrict__ cursor, int n,
                                                                 unsigned* __restrict__ offsets,
                                                                 unsigned long long capacity, WsHeader* hdr,
                                                                 unsigned* __restrict__ order) {
    extern __shared__ unsigned s_off[];         // [n + 1]: the counts, then the offsets
    __shared__ unsigned long long s_warp[33];
    __shared__ unsigned s_hist[33];
    const unsigned long long lim = capacity < 0xffffffffull ? capacity : 0xffffffffull;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int t = threadIdx.x; t < n; t += kScanBlock) s_off[t] = cursor[t];
    if (threadIdx.x < 33) s_hist[threadIdx.x] = 0u;
    __syncthreads();
    const int seg = (n + kScanBlock - 1) / kScanBlock * 32;             // tiles per warp, a multiple of 32
    const int w0 = min(warp * seg, n), w1 = min(w0 + seg, n);
    unsigned long long x = 0;
    for (int t = w0 + lane; t < w1; t += 32) x += s_off[t];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
    unsigned long long tot;
    unsigned long long carry = block_exclusive_scan(lane == 0 ? x : 0ull, s_warp, tot);   // ends with a barrier
    carry = __shfl_sync(0xffffffffu, carry, 0);
    for (int t0 = w0; t0 < w1; t0 += 32) {
        const int t = t0 + lane;
        const unsigned c = t < w1 ? s_off[t] : 0u;
        unsigned long long inc = c;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, off);
            if (lane >= off) inc += y;
        }
        const unsigned long long run = carry + inc - c;
        if (t < w1) s_off[t] = (unsigned)(run < lim ? run : lim);
        carry += __shfl_sync(0xffffffffu, inc, 31);
    }
    if (threadIdx.x == 0) {
        s_off[n] = (unsigned)(tot < lim ? tot : lim);
        hdr->total = tot;
        if (tot > lim) set_error(hdr, WSR_ERR_CAPACITY);
    }
    __syncthreads();
    for (int t = threadIdx.x; t <= n; t += kScanBlock) {
        const unsigned o = s_off[t];
        offsets[t] = o;
        if (t < n) cursor[t] = o;       // the scatter's cursor starts at the tile's offset
    }
    if (!order) return;
    for (int t = threadIdx.x; t < n; t += kScanBlock) atomicAdd(&s_hist[cost_bucket(s_off[t + 1] - s_off[t])], 1u);
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned r = 0;                 // bucket starts, largest bucket first
        for (int b = 32; b >= 0; --b) {
            const unsigned h = s_hist[b];
            s_hist[b] = r;
            r += h;
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < n; t += kScanBlock)
        order[atomicAdd(&s_hist[cost_bucket(s_off[t + 1] - s_off[t])], 1u)] = (unsigned)t;
}

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

// Deterministic mode: each tile's list sorted by record index, so that the
// per-pixel sums of the forward and the chunks of the backward do not depend
// on the order of the scatter's atomics.  A bitonic sort in shared memory over
// the segment padded to a power of two; a segment longer than kDetMaxSegment
// is left as it is and reported.
__global__ void __launch_bounds__(512) k_sort_segments(const unsigned* __restrict__ offsets,
                                                       unsigned* __restrict__ list, WsHeader* hdr) {
    __shared__ unsigned key[kDetMaxSegment];
    const unsigned a = offsets[blockIdx.x], len = offsets[blockIdx.x + 1] - a;
    if (len <= 1u) return;                                   // the whole block returns together
    if (len > (unsigned)kDetMaxSegment) {
        if (threadIdx.x == 0) set_error(hdr, WSR_ERR_UNSUPPORTED);
        return;
    }
    unsigned p = 2;
    while (p < len) p <<= 1;
    for (unsigned i = threadIdx.x; i < p; i += blockDim.x) key[i] = i < len ? list[a + i] : 0xffffffffu;
    __syncthreads();
    for (unsigned k = 2; k <= p; k <<= 1)
        for (unsigned j = k >> 1; j > 0; j >>= 1) {
            for (unsigned i = threadIdx.x; i < p; i += blockDim.x) {
                const unsigned l = i ^ j;                    // each element is in one pair of the stage
                if (l > i) {
                    const unsigned x = key[i], y = key[l];
                    if ((x > y) == ((i & k) == 0)) {
                        key[i] = y;
                        key[l] = x;
                    }
                }
            }
            __syncthreads();
        }
    for (unsigned i = threadIdx.x; i < len; i += blockDim.x) list[a + i] = key[i];
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
                        unsigned long long capacity, WsHeader* hdr, unsigned* buckets, unsigned* order,
                        cudaStream_t s) {
    const int n = vs.total_tiles;
    if (n <= kSmallScanTiles) {
        const size_t smem = sizeof(unsigned) * ((size_t)n + 1);
        if (smem > 48 * 1024) {
            // the dynamic shared-memory opt-in is a per-device attribute: set once per device (thread-safe)
            static std::once_flag once[64];
            static cudaError_t once_err[64];
            int dev = 0;
            cudaError_t e = cudaGetDevice(&dev);
            if (e != cudaSuccess) return e;
            if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
            std::call_once(once[dev], [&] {
                once_err[dev] = cudaFuncSetAttribute(k_scan_order_small, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     (int)(sizeof(unsigned) * (kSmallScanTiles + 1)));
            });
            if (once_err[dev] != cudaSuccess) return once_err[dev];
        }
        k_scan_order_small<<<1, kScanBlock, smem, s>>>(cursor, n, offsets, capacity, hdr, order);
        return cudaGetLastError();
    }
    const int nb = (n + kScanTile - 1) / kScanTile;
    unsigned long long* bsum = reinterpret_cast<unsigned long long*>(block_sums);
    k_scan_reduce<<<nb, kScanBlock, 0, s>>>(cursor, n, bsum);
    k_scan_top<<<1, kScanBlock, 0, s>>>(bsum, nb, offsets, n, capacity, hdr);
    k_scan_apply<<<nb, kScanBlock, 0, s>>>(cursor, n, bsum, offsets, capacity);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !order) return e;
    return launch_tile_order(vs, offsets, buckets, order, s);
}

cudaError_t launch_bin_scatter(const float* records, long long n, const Views& vs, unsigned* cursor,
                               unsigned* list, unsigned long long capacity, WsHeader* hdr, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    dim3 grid((unsigned)((n + 255) / 256), (unsigned)vs.n);
    k_bin<true><<<grid, 256, 0, s>>>(reinterpret_cast<const float4*>(records), n, vs, cursor, list, capacity, hdr);
    return cudaGetLastError();
}

cudaError_t launch_sort_segments(const Views& vs, const unsigned* offsets, unsigned* list, WsHeader* hdr,
                                 cudaStream_t s) {
    if (vs.total_tiles == 0) return cudaSuccess;
    k_sort_segments<<<(unsigned)vs.total_tiles, 512, 0, s>>>(offsets, list, hdr);
    return cudaGetLastError();
}

}  // namespace wsr
