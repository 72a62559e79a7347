// Per-pixel Weighted Sum Rendering, forward and backward (Eq. 7).
//
// One thread block per tile.  The tile's Gaussian list (unordered: Eq. 7 is
// a sum) is streamed through shared memory in chunks of one record per
// thread; every thread owns PPT vertically adjacent pixels of the tile and
// accumulates, in FP32 registers,
//     N += (c u w) e,   D += (u w) e,   e = exp(-q/2) = 2^(-q'),   q <= 9
// with q' = q log2(e)/2 evaluated from the prescaled conic of the record.
// There is no early termination (App. D: every covering Gaussian counts).
// The epilogue writes C = (c_B w_B + N) / (w_B + D) and the denominator.
//
// The backward recomputes every (pixel, Gaussian) term from the records and
// the stored C and denominator (no per-pixel lists are kept).  It walks the
// pixels inside each Gaussian's footprint (per-row spans) with the work split
// evenly over the threads, so no lane idles on pixels outside a footprint and
// no per-pair reduction across lanes is needed.
#include "wsr_launch.h"

namespace wsr {
namespace {

template <int TW, int TH, int PPT>
struct TileShape {
    static constexpr int NT = TW * TH / PPT;    // threads per block
    static constexpr int ROWS = TH / PPT;       // thread rows
    static_assert(TH % PPT == 0, "PPT must divide the tile height");
    static_assert(NT % 32 == 0, "whole warps");
};

struct TileCoord {
    int v, tx, ty;
};

__device__ __forceinline__ TileCoord tile_coord(const Views& vs, int tile) {
    TileCoord t;
    t.v = view_of_tile(vs, tile);
    const View& V = vs.v[t.v];
    const int lt = tile - V.tile_base;
    t.ty = lt / V.tiles_x;
    t.tx = lt - t.ty * V.tiles_x;
    return t;
}

template <int TW, int TH, int PPT>
__global__ void __launch_bounds__(TileShape<TW, TH, PPT>::NT)
    k_render_fwd(const float4* __restrict__ rec, const unsigned* __restrict__ offsets,
                 const unsigned* __restrict__ list, const Views vs, const float* __restrict__ wparams,
                 float* __restrict__ out_rgb, float* __restrict__ out_den) {
    using S = TileShape<TW, TH, PPT>;
    constexpr int NT = S::NT;
    __shared__ float4 s0[NT];
    __shared__ float4 s1[NT];
    __shared__ float s2[NT];

    const int tile = blockIdx.x;
    const TileCoord tc = tile_coord(vs, tile);
    const View& V = vs.v[tc.v];
    const int tid = threadIdx.x;
    const int lx = tid % TW, ly = tid / TW;
    const int x = tc.tx * TW + lx;
    const int y0 = tc.ty * TH + ly * PPT;
    const float px = (float)x + 0.5f;
    float py[PPT];
#pragma unroll
    for (int k = 0; k < PPT; ++k) py[k] = (float)(y0 + k) + 0.5f;

    float nr[PPT], ng[PPT], nb[PPT], dd[PPT];
#pragma unroll
    for (int k = 0; k < PPT; ++k) nr[k] = ng[k] = nb[k] = dd[k] = 0.0f;

    const unsigned start = offsets[tile], end = offsets[tile + 1];
    for (unsigned base = start; base < end; base += NT) {
        const int cnt = (int)min((unsigned)NT, end - base);
        __syncthreads();
        if (tid < cnt) {
            const unsigned r = list[base + tid];
            const float4* p = rec + 3ull * r;
            s0[tid] = __ldg(p);
            s1[tid] = __ldg(p + 1);
            s2[tid] = __ldg(reinterpret_cast<const float*>(p + 2));
        }
        __syncthreads();
        for (int j = 0; j < cnt; ++j) {
            const float4 a = s0[j];   // mu_x, mu_y, A', 2B'
            const float4 b = s1[j];   // C', uw, cuw_r, cuw_g
            const float cb = s2[j];   // cuw_b
            const float dx = px - a.x;
            const float P = a.z * dx * dx;
            const float Q = a.w * dx;
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                const float dy = py[k] - a.y;
                const float q = fmaf(dy, fmaf(b.x, dy, Q), P);
                if (q <= kQMax) {
                    const float e = ex2_approx(-q);
                    nr[k] = fmaf(b.z, e, nr[k]);
                    ng[k] = fmaf(b.w, e, ng[k]);
                    nb[k] = fmaf(cb, e, nb[k]);
                    dd[k] = fmaf(b.y, e, dd[k]);
                }
            }
        }
    }

    const float wB = __ldg(wparams + 2);
    const float cB0 = __ldg(wparams + 3) * wB, cB1 = __ldg(wparams + 4) * wB, cB2 = __ldg(wparams + 5) * wB;
    if (x < V.W) {
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            const int y = y0 + k;
            if (y < V.H) {
                const long long pix = V.pix_base + (long long)y * V.W + x;
                const float D = wB + dd[k];
                const float inv = 1.0f / D;
                out_rgb[3 * pix + 0] = (cB0 + nr[k]) * inv;
                out_rgb[3 * pix + 1] = (cB1 + ng[k]) * inv;
                out_rgb[3 * pix + 2] = (cB2 + nb[k]) * inv;
                out_den[pix] = D;
            }
        }
    }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// a*b - c*d with one rounding error (Kahan's fma form)
__device__ __forceinline__ float diff_of_products(float a, float b, float c, float d) {
    const float w = c * d;
    const float e = fmaf(-c, d, w);
    const float f = fmaf(a, b, -w);
    return f + e;
}

// Backward, one block per tile, balanced over (pixel, Gaussian) pairs.
//
// For each chunk of up to kBwdThreads Gaussians of the tile:
//   A. thread j computes, for every row of the tile, the span of pixels whose
//      centre can lie inside Gaussian j's footprint (the roots of the
//      quadratic q(dx) = 9 on that row, widened slightly);
//   B. a block scan lays the spans of all Gaussians end to end;
//   C. every thread takes an equal slice of that pair list and walks it,
//      accumulating the nine partial derivatives of the current Gaussian in
//      registers and adding them to shared memory when the Gaussian changes;
//   D. thread j adds Gaussian j's totals to its global 2D gradient record.
// Every pair is still tested with the forward's exact arithmetic (q <= 9), so
// forward and backward agree on which pairs exist.
constexpr int kBwdThreads = 256;

template <int TW, int TH>
__global__ void __launch_bounds__(kBwdThreads)
    k_render_bwd(const float4* __restrict__ rec, const unsigned* __restrict__ offsets,
                 const unsigned* __restrict__ list, const Views vs, const float* __restrict__ wparams,
                 const float* __restrict__ out_rgb, const float* __restrict__ out_den,
                 const float* __restrict__ grad_rgb, float* __restrict__ grec, float* __restrict__ gw) {
    constexpr int NT = kBwdThreads;
    constexpr int NW = NT / 32;
    constexpr int NPIX = TW * TH;
    static_assert(TW <= 32 && TH <= 32, "span encoding");
    __shared__ float4 spix[NPIX];               // per pixel: G/D (3), (G.C)/D
    __shared__ float4 s0[NT];
    __shared__ float4 s1[NT];
    __shared__ float s2[NT];
    __shared__ unsigned sidx[NT];
    __shared__ unsigned short sspan[NT][TH];    // first pixel | count << 8, per row
    __shared__ unsigned char sly0[NT];          // first non-empty row (rows are contiguous)
    __shared__ unsigned soff[NT + 1];
    // partial sums per (thread, Gaussian) segment of the pair list: a thread's
    // slice covers Gaussians jfirst[t] .. jfirst[t] + nseg - 1, stored from
    // segment sbase[t] on; at most NT + NT segments per chunk
    __shared__ float sseg[2 * NT][9];
    __shared__ unsigned short sjfirst[NT];
    __shared__ unsigned short ssbase[NT];
    __shared__ unsigned swarp[NW];
    __shared__ float sbg[4][NW];

    const int tile = blockIdx.x;
    const TileCoord tc = tile_coord(vs, tile);
    const View& V = vs.v[tc.v];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int x_org = tc.tx * TW, y_org = tc.ty * TH;
    const int x_lim = min(TW, V.W - x_org);    // pixels of the tile inside the image
    const int y_lim = min(TH, V.H - y_org);
    const float wB = __ldg(wparams + 2);
    const float cB0 = __ldg(wparams + 3), cB1 = __ldg(wparams + 4), cB2 = __ldg(wparams + 5);

    float bg[4] = {0.f, 0.f, 0.f, 0.f};
    for (int p = tid; p < NPIX; p += NT) {
        const int lx = p % TW, ly = p / TW;
        float4 f = make_float4(0.f, 0.f, 0.f, 0.f);
        if (lx < x_lim && ly < y_lim) {
            const long long pix = V.pix_base + (long long)(y_org + ly) * V.W + x_org + lx;
            const float inv = 1.0f / out_den[pix];
            const float G0 = grad_rgb[3 * pix], G1 = grad_rgb[3 * pix + 1], G2 = grad_rgb[3 * pix + 2];
            const float C0 = out_rgb[3 * pix], C1 = out_rgb[3 * pix + 1], C2 = out_rgb[3 * pix + 2];
            f = make_float4(G0 * inv, G1 * inv, G2 * inv, (G0 * C0 + G1 * C1 + G2 * C2) * inv);
            // dL/dw_B = G.(c_B - C)/D,  dL/dc_B = G w_B / D
            bg[0] += f.x * cB0 + f.y * cB1 + f.z * cB2 - f.w;
            bg[1] += f.x * wB;
            bg[2] += f.y * wB;
            bg[3] += f.z * wB;
        }
        spix[p] = f;
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const float t = warp_sum(bg[c]);
        if (lane == 0) sbg[c][warp] = t;
    }
    const float QM = kQMax * 1.0001f + 1e-4f;
    const unsigned start = offsets[tile], end = offsets[tile + 1];
    for (unsigned base = start; base < end; base += NT) {
        const int cnt = (int)min((unsigned)NT, end - base);
        __syncthreads();
        // ---- A: record and per-row spans of Gaussian tid ----
        unsigned npairs = 0;
        if (tid < cnt) {
            const unsigned r = list[base + tid];
            const float4* pr = rec + 3ull * r;
            const float4 a = __ldg(pr);
            const float4 b = __ldg(pr + 1);
            const float cb = __ldg(reinterpret_cast<const float*>(pr + 2));
            s0[tid] = a;
            s1[tid] = b;
            s2[tid] = cb;
            sidx[tid] = r;
            // row y: the footprint is mu_x + c(dy) +- h(dy) with
            // c = -(B''/2) dy / A', h = sqrt(A' QM - det' dy^2) / A',
            // det' = A' C' - (B''/2)^2 (both terms of the root are positive)
            const float hb = 0.5f * a.w;
            const float det = diff_of_products(a.z, b.x, hb, hb);
            const float ia = 1.0f / a.z;
            int first = TH;
#pragma unroll 4
            for (int ly = 0; ly < TH; ++ly) {
                unsigned short sp = 0;
                if (ly < y_lim) {
                    const float dy = (float)(y_org + ly) + 0.5f - a.y;
                    const float d4 = fmaf(-det * dy, dy, a.z * QM);
                    if (d4 >= 0.0f) {
                        const float h = sqrtf(d4) * ia;
                        const float cx = a.x - hb * dy * ia;
                        const float fx0 = fmaxf(ceilf(cx - h - 0.52f), (float)x_org);
                        const float fx1 = fminf(floorf(cx + h - 0.48f), (float)(x_org + x_lim - 1));
                        if (fx0 <= fx1) {
                            const int xs = (int)fx0 - x_org, len = (int)fx1 - (int)fx0 + 1;
                            sp = (unsigned short)(xs | (len << 8));
                            npairs += (unsigned)len;
                            first = min(first, ly);
                        }
                    }
                }
                sspan[tid][ly] = sp;
            }
            // the footprint within the tile is convex, so its rows are contiguous
            sly0[tid] = (unsigned char)(first < TH ? first : 0);
        }
        // ---- B: exclusive scan of the pair counts ----
        unsigned inc = npairs;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, inc, off);
            if (lane >= off) inc += y;
        }
        if (lane == 31) swarp[warp] = inc;
        __syncthreads();
        unsigned wbase = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) wbase += (w < warp) ? swarp[w] : 0u;
        soff[tid] = wbase + inc - npairs;
        if (tid == NT - 1) soff[NT] = wbase + inc;
        __syncthreads();
        // ---- C: an equal slice of the pairs per thread ----
        const unsigned total = soff[NT];
        const unsigned p0 = (unsigned)(((unsigned long long)tid * total) / NT);
        const unsigned p1 = (unsigned)(((unsigned long long)(tid + 1) * total) / NT);
        // owner(p): the last Gaussian whose first pair is <= p
        auto owner = [&](unsigned p) {
            int lo = 0, hi = cnt - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (soff[mid] <= p) lo = mid;
                else hi = mid - 1;
            }
            return lo;
        };
        int j = 0, jlast = -1;
        if (p0 < p1) {
            j = owner(p0);
            jlast = owner(p1 - 1);
        }
        {
            // segment slots: a block scan of the per-thread Gaussian counts
            const unsigned nseg = (unsigned)(jlast - j + 1);
            unsigned sinc = nseg;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, sinc, off);
                if (lane >= off) sinc += y;
            }
            __syncthreads();                       // swarp reuse
            if (lane == 31) swarp[warp] = sinc;
            __syncthreads();
            unsigned sb = 0;
#pragma unroll
            for (int w = 0; w < NW; ++w) sb += (w < warp) ? swarp[w] : 0u;
            sjfirst[tid] = (unsigned short)j;
            ssbase[tid] = (unsigned short)(sb + sinc - nseg);
        }
        if (p0 < p1) {
            float* seg = sseg[ssbase[tid]];
            float4 a = s0[j], b = s1[j];
            float cb = s2[j];
            // -ln2 (c u w, u w): dL/dq' = e * -ln2 (G/D . c u w - s u w)
            float cwr = -kLn2 * b.z, cwg = -kLn2 * b.w, cwb = -kLn2 * cb, cwu = -kLn2 * b.y;
            unsigned k = p0 - soff[j];
            int ly = sly0[j];
            unsigned sp = sspan[j][ly];
            while (k >= (sp >> 8)) {
                k -= sp >> 8;
                sp = sspan[j][++ly];
            }
            int lx = (int)(sp & 0xffu) + (int)k;
            int lx_end = (int)(sp & 0xffu) + (int)(sp >> 8);
            float xf = (float)(x_org + lx) + 0.5f;
            float dy = (float)(y_org + ly) + 0.5f - a.y;
            float g[9];
#pragma unroll
            for (int c = 0; c < 9; ++c) g[c] = 0.0f;
            for (unsigned left = p1 - p0; left > 0; --left) {
                const float4 P = spix[ly * TW + lx];
                const float dx = xf - a.x;
                const float Pq = a.z * dx * dx;
                const float Q = a.w * dx;
                const float q = fmaf(dy, fmaf(b.x, dy, Q), Pq);   // the forward's arithmetic
                // outside the cutoff the pair contributes nothing (a select, not a branch)
                const float e = (q <= kQMax) ? ex2_approx(-q) : 0.0f;
                g[0] = fmaf(P.x, e, g[0]);                          // d/d(c u w)
                g[1] = fmaf(P.y, e, g[1]);
                g[2] = fmaf(P.z, e, g[2]);
                g[3] = fmaf(-P.w, e, g[3]);                         // d/d(u w) at fixed c u w
                const float gq = e * fmaf(P.x, cwr, fmaf(P.y, cwg, fmaf(P.z, cwb, -P.w * cwu)));  // dL/dq'
                const float t = gq * dx, u = gq * dy;
                g[4] = fmaf(t, dx, g[4]);                           // dL/dA'
                g[5] = fmaf(t, dy, g[5]);                           // dL/d(2B')
                g[6] = fmaf(u, dy, g[6]);                           // dL/dC'
                g[7] += t;                                          // sum dL/dq' dx
                g[8] += u;                                          // sum dL/dq' dy
                // advance: next pixel of the row, else the next row (selects)
                ++lx;
                xf += 1.0f;
                const bool row_end = lx >= lx_end;
                ly += row_end ? 1 : 0;
                if (row_end) sp = (ly < TH) ? (unsigned)sspan[j][ly] : 0u;   // 0: past the last row
                if (row_end && (sp >> 8) == 0) {
                    // end of Gaussian j: store its partial sums in its segment
#pragma unroll
                    for (int c = 0; c < 9; ++c) {
                        seg[c] = g[c];
                        g[c] = 0.0f;
                    }
                    seg += 9;
                    if (left > 1) {
                        ++j;
                        while (soff[j + 1] == soff[j]) {     // Gaussians without pairs here
#pragma unroll
                            for (int c = 0; c < 9; ++c) seg[c] = 0.0f;
                            seg += 9;
                            ++j;
                        }
                        a = s0[j];
                        b = s1[j];
                        cb = s2[j];
                        cwr = -kLn2 * b.z;
                        cwg = -kLn2 * b.w;
                        cwb = -kLn2 * cb;
                        cwu = -kLn2 * b.y;
                        ly = sly0[j];
                        sp = sspan[j][ly];
                    }
                }
                const int xs = (int)(sp & 0xffu);
                lx = row_end ? xs : lx;
                lx_end = row_end ? xs + (int)(sp >> 8) : lx_end;
                xf = row_end ? (float)(x_org + xs) + 0.5f : xf;
                dy = row_end ? (float)(y_org + ly) + 0.5f - a.y : dy;
            }
            if (jlast >= 0 && seg < sseg[ssbase[tid]] + 9 * (jlast - sjfirst[tid] + 1)) {
#pragma unroll
                for (int c = 0; c < 9; ++c) seg[c] = g[c];
            }
        }
        __syncthreads();
        // ---- D: totals of Gaussian tid to its global record ----
        if (tid < cnt && soff[tid + 1] > soff[tid]) {
            // threads whose slices hold pairs of Gaussian tid: from the owner of
            // its first pair to the owner of its last pair
            auto slice_of = [&](unsigned p) {
                int t = (int)(((unsigned long long)p * NT) / total);
                while (t + 1 < NT && (unsigned)(((unsigned long long)(t + 1) * total) / NT) <= p) ++t;
                while (t > 0 && (unsigned)(((unsigned long long)t * total) / NT) > p) --t;
                return t;
            };
            const int t0 = slice_of(soff[tid]), t1 = slice_of(soff[tid + 1] - 1);
            float v[9];
#pragma unroll
            for (int c = 0; c < 9; ++c) v[c] = 0.0f;
            for (int t = t0; t <= t1; ++t) {
                // threads with an empty slice hold no segment
                const unsigned q0 = (unsigned)(((unsigned long long)t * total) / NT);
                const unsigned q1 = (unsigned)(((unsigned long long)(t + 1) * total) / NT);
                if (q0 == q1) continue;
                const float* sg = sseg[ssbase[t] + (tid - sjfirst[t])];
#pragma unroll
                for (int c = 0; c < 9; ++c) v[c] += sg[c];
            }
            const float4 a = s0[tid];
            const float Cp = s1[tid].x;
            // q' = A' dx^2 + B'' dx dy + C' dy^2, dx = px - mu_x, dy = py - mu_y
            const float gmx = -(2.0f * a.z * v[7] + a.w * v[8]);
            const float gmy = -(a.w * v[7] + 2.0f * Cp * v[8]);
            // prescaled -> unscaled conic: A' = k A, B'' = 2k B, C' = k C
            float4* o = reinterpret_cast<float4*>(grec + (size_t)WSR_GRAD_RECORD_FLOATS * sidx[tid]);
            atomicAdd(o, make_float4(gmx, gmy, kHalfLog2e * v[4], 2.0f * kHalfLog2e * v[5]));
            atomicAdd(o + 1, make_float4(kHalfLog2e * v[6], v[3], v[0], v[1]));
            atomicAdd(reinterpret_cast<float*>(o + 2), v[2]);
        }
    }
    __syncthreads();
    if (tid < 4) {
        float t = 0.0f;
        for (int w = 0; w < NW; ++w) t += sbg[tid][w];
        if (t != 0.0f) atomicAdd(gw + 2 + tid, t);
    }
}

template <int TW, int TH, int PPT>
cudaError_t fwd_t(const float* rec, const unsigned* off, const unsigned* list, const Views& vs, WeightDev w,
                  float* rgb, float* den, cudaStream_t s) {
    k_render_fwd<TW, TH, PPT><<<vs.total_tiles, TileShape<TW, TH, PPT>::NT, 0, s>>>(
        reinterpret_cast<const float4*>(rec), off, list, vs, w.params, rgb, den);
    return cudaGetLastError();
}

template <int TW, int TH>
cudaError_t bwd_t(const float* rec, const unsigned* off, const unsigned* list, const Views& vs, WeightDev w,
                  const float* rgb, const float* den, const float* grgb, float* grec, float* gw, cudaStream_t s) {
    k_render_bwd<TW, TH><<<vs.total_tiles, kBwdThreads, 0, s>>>(reinterpret_cast<const float4*>(rec), off, list, vs,
                                                                w.params, rgb, den, grgb, grec, gw);
    return cudaGetLastError();
}

// Diagnostic: (pixel, Gaussian) pairs inside the cutoff, i.e. the
// algorithmic work of the render kernels (same arithmetic as the forward).
template <int TW, int TH, int PPT>
__global__ void __launch_bounds__(TileShape<TW, TH, PPT>::NT)
    k_count_pairs(const float4* __restrict__ rec, const unsigned* __restrict__ offsets,
                  const unsigned* __restrict__ list, const Views vs, unsigned long long* __restrict__ count) {
    using S = TileShape<TW, TH, PPT>;
    constexpr int NT = S::NT;
    __shared__ float4 s0[NT];
    __shared__ float s1[NT];
    const int tile = blockIdx.x;
    const TileCoord tc = tile_coord(vs, tile);
    const View& V = vs.v[tc.v];
    const int tid = threadIdx.x;
    const int lx = tid % TW, ly = tid / TW;
    const int x = tc.tx * TW + lx;
    const int y0 = tc.ty * TH + ly * PPT;
    const float px = (float)x + 0.5f;
    unsigned long long cnt_pairs = 0;
    const unsigned start = offsets[tile], end = offsets[tile + 1];
    for (unsigned base = start; base < end; base += NT) {
        const int cnt = (int)min((unsigned)NT, end - base);
        __syncthreads();
        if (tid < cnt) {
            const float4* p = rec + 3ull * list[base + tid];
            s0[tid] = __ldg(p);
            s1[tid] = __ldg(reinterpret_cast<const float*>(p + 1));
        }
        __syncthreads();
        if (x >= V.W) continue;
        for (int j = 0; j < cnt; ++j) {
            const float4 a = s0[j];
            const float dx = px - a.x;
            const float P = a.z * dx * dx;
            const float Q = a.w * dx;
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                const float dy = (float)(y0 + k) + 0.5f - a.y;
                const float q = fmaf(dy, fmaf(s1[j], dy, Q), P);
                if (q <= kQMax && y0 + k < V.H) ++cnt_pairs;
            }
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) cnt_pairs += __shfl_xor_sync(0xffffffffu, cnt_pairs, off);
    if ((tid & 31) == 0 && cnt_pairs) atomicAdd(count, cnt_pairs);
}

__global__ void k_loss_l1(const float* __restrict__ rgb, const float* __restrict__ target, long long count,
                          float* __restrict__ loss, float* __restrict__ grad) {
    const float inv = 1.0f / (float)count;
    float acc = 0.0f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        const float d = rgb[i] - target[i];
        acc += fabsf(d);
        grad[i] = (d > 0.0f ? inv : (d < 0.0f ? -inv : 0.0f));
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, acc * inv);
}

}  // namespace

cudaError_t launch_render_fwd(const float* rec, const unsigned* off, const unsigned* list, const Views& vs,
                              WeightDev w, float* rgb, float* den, cudaStream_t s) {
    if (vs.total_tiles == 0) return cudaSuccess;
    if (vs.tile_w == 16 && vs.tile_h == 16) return fwd_t<16, 16, 2>(rec, off, list, vs, w, rgb, den, s);
    if (vs.tile_w == 8 && vs.tile_h == 8) return fwd_t<8, 8, 2>(rec, off, list, vs, w, rgb, den, s);
    if (vs.tile_w == 32 && vs.tile_h == 8) return fwd_t<32, 8, 2>(rec, off, list, vs, w, rgb, den, s);
    if (vs.tile_w == 16 && vs.tile_h == 8) return fwd_t<16, 8, 2>(rec, off, list, vs, w, rgb, den, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_render_bwd(const float* rec, const unsigned* off, const unsigned* list, const Views& vs,
                              WeightDev w, const float* rgb, const float* den, const float* grgb, float* grec,
                              float* gw, cudaStream_t s) {
    if (vs.total_tiles == 0) return cudaSuccess;
    if (vs.tile_w == 16 && vs.tile_h == 16) return bwd_t<16, 16>(rec, off, list, vs, w, rgb, den, grgb, grec, gw, s);
    if (vs.tile_w == 8 && vs.tile_h == 8) return bwd_t<8, 8>(rec, off, list, vs, w, rgb, den, grgb, grec, gw, s);
    if (vs.tile_w == 32 && vs.tile_h == 8) return bwd_t<32, 8>(rec, off, list, vs, w, rgb, den, grgb, grec, gw, s);
    if (vs.tile_w == 16 && vs.tile_h == 8) return bwd_t<16, 8>(rec, off, list, vs, w, rgb, den, grgb, grec, gw, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_count_pairs(const float* rec, const unsigned* off, const unsigned* list, const Views& vs,
                               unsigned long long* count, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess || vs.total_tiles == 0) return e;
    const float4* r = reinterpret_cast<const float4*>(rec);
    if (vs.tile_w == 16 && vs.tile_h == 16) k_count_pairs<16, 16, 2><<<vs.total_tiles, 128, 0, s>>>(r, off, list, vs, count);
    else if (vs.tile_w == 8 && vs.tile_h == 8) k_count_pairs<8, 8, 2><<<vs.total_tiles, 32, 0, s>>>(r, off, list, vs, count);
    else if (vs.tile_w == 32 && vs.tile_h == 8) k_count_pairs<32, 8, 2><<<vs.total_tiles, 128, 0, s>>>(r, off, list, vs, count);
    else if (vs.tile_w == 16 && vs.tile_h == 8) k_count_pairs<16, 8, 2><<<vs.total_tiles, 64, 0, s>>>(r, off, list, vs, count);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_loss_l1(const float* rgb, const float* target, long long count, float* loss, float* grad,
                           cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(float), s);
    if (e != cudaSuccess || count == 0) return e;
    long long nb = (count + 255) / 256;
    if (nb > 4096) nb = 4096;
    k_loss_l1<<<(unsigned)nb, 256, 0, s>>>(rgb, target, count, loss, grad);
    return cudaGetLastError();
}

}  // namespace wsr
