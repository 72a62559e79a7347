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
// the stored C and denominator (no per-pixel lists are kept), forms the nine
// per-Gaussian partial derivatives per pixel, reduces them across the warp
// with shuffles, across warps in shared memory, and adds one value per
// Gaussian, tile and component to the global 2D gradient records.
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

template <int TW, int TH, int PPT>
__global__ void __launch_bounds__(TileShape<TW, TH, PPT>::NT)
    k_render_bwd(const float4* __restrict__ rec, const unsigned* __restrict__ offsets,
                 const unsigned* __restrict__ list, const Views vs, const float* __restrict__ wparams,
                 const float* __restrict__ out_rgb, const float* __restrict__ out_den,
                 const float* __restrict__ grad_rgb, float* __restrict__ grec, float* __restrict__ gw) {
    using S = TileShape<TW, TH, PPT>;
    constexpr int NT = S::NT;
    constexpr int NW = NT / 32;
    __shared__ float4 s0[NT];
    __shared__ float4 s1[NT];
    __shared__ float s2[NT];
    __shared__ unsigned sidx[NT];
    __shared__ float sacc[9][NT];
    __shared__ float sbg[4][NW];

    const int tile = blockIdx.x;
    const TileCoord tc = tile_coord(vs, tile);
    const View& V = vs.v[tc.v];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int lx = tid % TW, ly = tid / TW;
    const int x = tc.tx * TW + lx;
    const int y0 = tc.ty * TH + ly * PPT;
    const float px = (float)x + 0.5f;
    const float wB = __ldg(wparams + 2);
    const float cB[3] = {__ldg(wparams + 3), __ldg(wparams + 4), __ldg(wparams + 5)};

    // per-pixel factors: Gd = G / D, s = (G . C) / D; background terms
    float py[PPT], gdr[PPT], gdg[PPT], gdb[PPT], sg[PPT];
    float bg[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int y = y0 + k;
        py[k] = (float)y + 0.5f;
        gdr[k] = gdg[k] = gdb[k] = sg[k] = 0.0f;
        if (x < V.W && y < V.H) {
            const long long pix = V.pix_base + (long long)y * V.W + x;
            const float inv = 1.0f / out_den[pix];
            const float G0 = grad_rgb[3 * pix], G1 = grad_rgb[3 * pix + 1], G2 = grad_rgb[3 * pix + 2];
            const float C0 = out_rgb[3 * pix], C1 = out_rgb[3 * pix + 1], C2 = out_rgb[3 * pix + 2];
            gdr[k] = G0 * inv;
            gdg[k] = G1 * inv;
            gdb[k] = G2 * inv;
            sg[k] = (G0 * C0 + G1 * C1 + G2 * C2) * inv;
            // dL/dw_B = G.(c_B - C)/D,  dL/dc_B = G w_B / D
            bg[0] += gdr[k] * cB[0] + gdg[k] * cB[1] + gdb[k] * cB[2] - sg[k];
            bg[1] += gdr[k] * wB;
            bg[2] += gdg[k] * wB;
            bg[3] += gdb[k] * wB;
        }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const float t = warp_sum(bg[c]);
        if (lane == 0) sbg[c][warp] = t;
    }
    for (int c = 0; c < 9; ++c) sacc[c][tid] = 0.0f;

    const unsigned start = offsets[tile], end = offsets[tile + 1];
    for (unsigned base = start; base < end; base += NT) {
        const int cnt = (int)min((unsigned)NT, end - base);
        __syncthreads();
        if (tid < cnt) {
            const unsigned r = list[base + tid];
            const float4* p = rec + 3ull * r;
            sidx[tid] = r;
            s0[tid] = __ldg(p);
            s1[tid] = __ldg(p + 1);
            s2[tid] = __ldg(reinterpret_cast<const float*>(p + 2));
        }
        __syncthreads();
        for (int j = 0; j < cnt; ++j) {
            const float4 a = s0[j];
            const float4 b = s1[j];
            const float cb = s2[j];
            const float dx = px - a.x;
            const float P = a.z * dx * dx;
            const float Q = a.w * dx;
            float g[9];
#pragma unroll
            for (int c = 0; c < 9; ++c) g[c] = 0.0f;
            bool act = false;
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                const float dy = py[k] - a.y;
                const float q = fmaf(dy, fmaf(b.x, dy, Q), P);   // same arithmetic as the forward
                if (q <= kQMax) {
                    act = true;
                    const float e = ex2_approx(-q);
                    g[6] = fmaf(gdr[k], e, g[6]);           // d/d(c u w)
                    g[7] = fmaf(gdg[k], e, g[7]);
                    g[8] = fmaf(gdb[k], e, g[8]);
                    g[5] = fmaf(-sg[k], e, g[5]);           // d/d(u w) at fixed c u w
                    const float ge = gdr[k] * b.z + gdg[k] * b.w + gdb[k] * cb - sg[k] * b.y;
                    const float gq = -kLn2 * e * ge;        // dL/dq'
                    g[2] = fmaf(gq, dx * dx, g[2]);         // dL/dA'
                    g[3] = fmaf(gq, dx * dy, g[3]);         // dL/d(2B')
                    g[4] = fmaf(gq, dy * dy, g[4]);         // dL/dC'
                    g[0] = fmaf(-gq, fmaf(2.0f * a.z, dx, a.w * dy), g[0]);   // dL/dmu_x
                    g[1] = fmaf(-gq, fmaf(2.0f * b.x, dy, a.w * dx), g[1]);   // dL/dmu_y
                }
            }
            if (__any_sync(0xffffffffu, act)) {
#pragma unroll
                for (int c = 0; c < 9; ++c) g[c] = warp_sum(g[c]);
                if (lane == 0) {
#pragma unroll
                    for (int c = 0; c < 9; ++c)
                        if (g[c] != 0.0f) atomicAdd(&sacc[c][j], g[c]);
                }
            }
        }
        __syncthreads();
        if (tid < cnt) {
            // prescaled -> unscaled conic: A' = k A, 2B' = 2k B, C' = k C
            float* o = grec + 9ull * sidx[tid];
            const float scale[9] = {1.f, 1.f, kHalfLog2e, 2.0f * kHalfLog2e, kHalfLog2e, 1.f, 1.f, 1.f, 1.f};
#pragma unroll
            for (int c = 0; c < 9; ++c) {
                const float v = sacc[c][tid];
                if (v != 0.0f) atomicAdd(o + c, v * scale[c]);
                sacc[c][tid] = 0.0f;
            }
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

template <int TW, int TH, int PPT>
cudaError_t bwd_t(const float* rec, const unsigned* off, const unsigned* list, const Views& vs, WeightDev w,
                  const float* rgb, const float* den, const float* grgb, float* grec, float* gw, cudaStream_t s) {
    k_render_bwd<TW, TH, PPT><<<vs.total_tiles, TileShape<TW, TH, PPT>::NT, 0, s>>>(
        reinterpret_cast<const float4*>(rec), off, list, vs, w.params, rgb, den, grgb, grec, gw);
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
    if (vs.tile_w == 16 && vs.tile_h == 16) return bwd_t<16, 16, 2>(rec, off, list, vs, w, rgb, den, grgb, grec, gw, s);
    if (vs.tile_w == 8 && vs.tile_h == 8) return bwd_t<8, 8, 2>(rec, off, list, vs, w, rgb, den, grgb, grec, gw, s);
    if (vs.tile_w == 32 && vs.tile_h == 8) return bwd_t<32, 8, 2>(rec, off, list, vs, w, rgb, den, grgb, grec, gw, s);
    if (vs.tile_w == 16 && vs.tile_h == 8) return bwd_t<16, 8, 2>(rec, off, list, vs, w, rgb, den, grgb, grec, gw, s);
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
