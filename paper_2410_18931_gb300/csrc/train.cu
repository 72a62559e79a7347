// Training step around the renderer: the 3DGS rendering loss the paper
// trains with (Sec. 4.4: L1 + 0.2 D-SSIM) with its gradient, and the Adam
// update of the parameters.
//
// Loss.  One block per 32 x 32 output tile of one view.  For each channel the
// block stages the rendered and target pixels of the tile plus a 10-pixel
// halo in shared memory (zero outside the image), filters the five local
// statistics (mu_x, mu_y, E[x^2], E[y^2], E[xy]) separably with the 11-tap
// Gaussian over the tile plus a 5-pixel halo, forms the SSIM map and the three
// partials of the loss with respect to (mu_x, E[x^2], E[xy]), and filters
// those back (the window is symmetric, so the filter is its own adjoint) to
// the gradient of the tile's pixels.  L1 and SSIM sums go to the loss with
// one atomic per block and quantity.
//
// Adam.  One pass over a flat parameter buffer in float4 units, groups of
// contiguous elements with their own learning rates.  The step count and the
// bias corrections live in device memory (a one-thread kernel advances them),
// so a captured CUDA graph replays correct steps; both kernels leave
// everything untouched when a guard workspace recorded an error (a tile list
// that overflowed in the same step).
#include <mutex>

#include "wsr_common.cuh"
#include "wsr_launch.h"

namespace wsr {
namespace {

constexpr int kR = 5;                       // window radius: 11 taps
constexpr int kLT = 32;                     // output tile side
constexpr int kIn = kLT + 4 * kR;           // staged input side (52)
constexpr int kSt = kLT + 2 * kR;           // statistics side (42)
constexpr int kLossThreads = 256;
constexpr int kStage = (kIn * kIn + kLossThreads - 1) / kLossThreads;   // staged pixels per thread
// Shared memory, in floats: the staged (rendered, target) pairs, then the horizontally filtered
// statistics as (mu_x, mu_y) and (E[x^2], E[y^2]) pairs and E[xy].  The loss partials with
// respect to (mu_x, E[x^2]) as pairs and E[xy] reuse the staged pixels (no longer needed after
// the statistics); the filtered partials reuse the statistics.  The partials' rows are kMP
// apart and the filtered partials' kFP apart (odd numbers of 8-byte words): the horizontal
// pass reads them a row per lane, and its lanes then fall on distinct banks.
constexpr int kMP = kSt + 1, kFP = kLT + 1;
constexpr int kStatOff = ((3 * kSt * kMP > 2 * kIn * kIn ? 3 * kSt * kMP : 2 * kIn * kIn) + 3) / 4 * 4;
constexpr int kLossSmemFloats = kStatOff + 5 * kIn * kSt;      // the statistics start at kStatOff
static_assert(3 * kSt * kFP <= 5 * kIn * kSt, "layout");
// register blocking of the four filter passes (outputs per item along the filtered axis)
constexpr int kH1 = kSt / 3;                // horizontal statistics: 3 columns
constexpr int kV2 = 7, kS2 = kSt / kV2;     // vertical statistics: 7 rows
constexpr int kH3 = 4, kB3 = kLT / kH3;     // horizontal partials: 4 columns
constexpr int kV4 = 4, kS4 = kLT / kV4;     // vertical partials: 4 rows
static_assert(kH1 * 3 == kSt && kS2 * kV2 == kSt && kB3 * kH3 == kLT && kS4 * kV4 == kLT, "exact blocking");

__device__ __forceinline__ float block_sum_to(float x, float* red) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) red[w] = x;
    __syncthreads();
    float t = 0.f;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
    return t;   // valid in thread 0
}

// Every filter step runs on two quantities at once where it can (paired FP32 ops on float2):
// the rendered and target values, their squares, and the first two loss partials; the cross
// terms E[xy] and its partial go alone.
__global__ void __launch_bounds__(kLossThreads, 3) k_loss_3dgs(const float* __restrict__ rgb,
                                                               const float* __restrict__ tgt, const LossViews L,
                                                               float* __restrict__ loss, float* __restrict__ grad) {
    extern __shared__ __align__(16) float sm[];
    float2* sxy = reinterpret_cast<float2*>(sm);                   // [kIn][kIn] (rendered, target)
    float2* h01 = reinterpret_cast<float2*>(sm + kStatOff);        // [kIn][kSt] filtered (x, y)
    float2* h23 = h01 + kIn * kSt;                                 // [kIn][kSt] filtered (x^2, y^2)
    float* h4 = reinterpret_cast<float*>(h23 + kIn * kSt);         // [kIn][kSt] filtered x y
    float2* m01 = reinterpret_cast<float2*>(sm);                   // [kSt][kMP] partials: mu_x, E[x^2]
    float* m2 = reinterpret_cast<float*>(m01 + kSt * kMP);         // [kSt][kMP] partial: E[xy]
    float2* f01 = h01;                                             // [kSt][kFP] horizontally filtered
    float* f2s = reinterpret_cast<float*>(f01 + kSt * kFP);        // [kSt][kFP]
    __shared__ float red[kLossThreads / 32];
    const int tid = threadIdx.x;

    int v = 0;
    while (v + 1 < L.n && (int)blockIdx.x >= L.tile_off[v + 1]) ++v;
    const int t = (int)blockIdx.x - L.tile_off[v];
    const int W = L.w[v], H = L.h[v];
    const int x0 = (t % L.tiles_x[v]) * kLT, y0 = (t / L.tiles_x[v]) * kLT;
    const long long base = L.pix_off[v];
    const float gs = -L.lam * L.inv_count;                 // dL / d(SSIM map value)
    const float gl1 = (1.0f - L.lam) * L.inv_count;        // dL / d|x - y|
    float l1 = 0.f, ss = 0.f;
    float2 g2[2 * kR + 1];                                 // the window's taps, paired
#pragma unroll
    for (int k = 0; k < 2 * kR + 1; ++k) g2[k] = f2(L.g[k], L.g[k]);

    for (int c = 0; c < 3; ++c) {
        {
            // all of a thread's loads first, then the stores: kStage independent loads in flight
            float2 ab[kStage];
#pragma unroll
            for (int k = 0; k < kStage; ++k) {
                const int i = tid + k * kLossThreads;
                const int iy = i / kIn, ix = i - iy * kIn;
                const int gx = x0 - 2 * kR + ix, gy = y0 - 2 * kR + iy;
                ab[k] = f2(0.f, 0.f);
                if (i < kIn * kIn && gx >= 0 && gx < W && gy >= 0 && gy < H) {
                    const long long p = (base + (long long)gy * W + gx) * 3 + c;
                    ab[k] = f2(__ldg(rgb + p), __ldg(tgt + p));
                }
            }
#pragma unroll
            for (int k = 0; k < kStage; ++k) {
                const int i = tid + k * kLossThreads;
                if (i < kIn * kIn) sxy[i] = ab[k];
            }
        }
        __syncthreads();
        // horizontal statistics: three neighbouring columns per item from one window of 13
        for (int it = tid; it < kIn * kH1; it += kLossThreads) {
            const int iy = it / kH1, jx0 = (it - iy * kH1) * 3;
            const float2* r = sxy + iy * kIn + jx0;
            float2 ab[2 * kR + 3], sq[2 * kR + 3];
            float xy[2 * kR + 3];
#pragma unroll
            for (int k = 0; k < 2 * kR + 3; ++k) {
                ab[k] = r[k];
                sq[k] = __fmul2_rn(ab[k], ab[k]);
                xy[k] = ab[k].x * ab[k].y;
            }
#pragma unroll
            for (int o = 0; o < 3; ++o) {
                float2 s01 = f2(0.f, 0.f), s23 = f2(0.f, 0.f);
                float s4 = 0.f;
#pragma unroll
                for (int k = 0; k < 2 * kR + 1; ++k) {
                    s01 = __ffma2_rn(g2[k], ab[o + k], s01);
                    s23 = __ffma2_rn(g2[k], sq[o + k], s23);
                    s4 = fmaf(g2[k].x, xy[o + k], s4);
                }
                const int i = iy * kSt + jx0 + o;
                h01[i] = s01;
                h23[i] = s23;
                h4[i] = s4;
            }
        }
        __syncthreads();
        // vertical statistics, SSIM map and the loss partials: seven rows per item
        for (int it = tid; it < kSt * kS2; it += kLossThreads) {
            const int strip = it / kSt, jx = it - strip * kSt, jy0 = strip * kV2;
            float2 st01[kV2], st23[kV2];
            float st4[kV2];
            {
                float2 h[kV2 + 2 * kR];
#pragma unroll
                for (int r = 0; r < kV2 + 2 * kR; ++r) h[r] = h01[(jy0 + r) * kSt + jx];
#pragma unroll
                for (int o = 0; o < kV2; ++o) {
                    float2 acc = f2(0.f, 0.f);
#pragma unroll
                    for (int k = 0; k < 2 * kR + 1; ++k) acc = __ffma2_rn(g2[k], h[o + k], acc);
                    st01[o] = acc;
                }
#pragma unroll
                for (int r = 0; r < kV2 + 2 * kR; ++r) h[r] = h23[(jy0 + r) * kSt + jx];
#pragma unroll
                for (int o = 0; o < kV2; ++o) {
                    float2 acc = f2(0.f, 0.f);
#pragma unroll
                    for (int k = 0; k < 2 * kR + 1; ++k) acc = __ffma2_rn(g2[k], h[o + k], acc);
                    st23[o] = acc;
                }
            }
            {
                float h[kV2 + 2 * kR];
#pragma unroll
                for (int r = 0; r < kV2 + 2 * kR; ++r) h[r] = h4[(jy0 + r) * kSt + jx];
#pragma unroll
                for (int o = 0; o < kV2; ++o) {
                    float acc = 0.f;
#pragma unroll
                    for (int k = 0; k < 2 * kR + 1; ++k) acc = fmaf(g2[k].x, h[o + k], acc);
                    st4[o] = acc;
                }
            }
            const int gx = x0 - kR + jx;
            const bool col_in = gx >= 0 && gx < W;
            const bool col_own = jx >= kR && jx < kR + kLT;
#pragma unroll
            for (int o = 0; o < kV2; ++o) {
                const int jy = jy0 + o, gy = y0 - kR + jy;
                float2 p01 = f2(0.f, 0.f);
                float p2 = 0.f;
                if (col_in && gy >= 0 && gy < H) {
                    const float mx = st01[o].x, my = st01[o].y;
                    const float sxx = st23[o].x - mx * mx, syy = st23[o].y - my * my, sxy_ = st4[o] - mx * my;
                    const float a1 = 2.f * mx * my + L.c1, a2 = 2.f * sxy_ + L.c2;
                    const float b1 = mx * mx + my * my + L.c1, b2 = sxx + syy + L.c2;
                    const float ib1 = rcp_approx(b1), ib2 = rcp_approx(b2);
                    const float sv = a1 * a2 * ib1 * ib2;
                    p01 = f2(gs * (2.f * my * (a2 - a1) * ib1 * ib2 + 2.f * mx * sv * (ib2 - ib1)), gs * (-sv * ib2));
                    p2 = gs * (2.f * a1 * ib1 * ib2);
                    if (col_own && jy >= kR && jy < kR + kLT) ss += sv;
                }
                const int i = jy * kMP + jx;
                m01[i] = p01;
                m2[i] = p2;
            }
        }
        __syncthreads();
        // horizontal pass of the partials: four columns per item, consecutive lanes on consecutive rows
        for (int it = tid; it < kSt * kB3; it += kLossThreads) {
            const int blk = it / kSt, jy = it - blk * kSt, ox0 = blk * kH3;
            float2 r[kH3 + 2 * kR];
            float r2[kH3 + 2 * kR];
#pragma unroll
            for (int k = 0; k < kH3 + 2 * kR; ++k) {
                r[k] = m01[jy * kMP + ox0 + k];
                r2[k] = m2[jy * kMP + ox0 + k];
            }
#pragma unroll
            for (int o = 0; o < kH3; ++o) {
                float2 acc = f2(0.f, 0.f);
                float acc2 = 0.f;
#pragma unroll
                for (int k = 0; k < 2 * kR + 1; ++k) {
                    acc = __ffma2_rn(g2[k], r[o + k], acc);
                    acc2 = fmaf(g2[k].x, r2[o + k], acc2);
                }
                f01[jy * kFP + ox0 + o] = acc;
                f2s[jy * kFP + ox0 + o] = acc2;
            }
        }
        __syncthreads();
        // vertical pass of the partials and the gradient: four rows per item
        for (int it = tid; it < kLT * kS4; it += kLossThreads) {
            const int strip = it / kLT, ox = it - strip * kLT, oy0 = strip * kV4;
            const int gx = x0 + ox;
            float2 cc[kV4 + 2 * kR];
            float c2[kV4 + 2 * kR];
#pragma unroll
            for (int r = 0; r < kV4 + 2 * kR; ++r) {
                cc[r] = f01[(oy0 + r) * kFP + ox];
                c2[r] = f2s[(oy0 + r) * kFP + ox];
            }
            float av[kV4], bv[kV4];            // the staged copies are overwritten by now: read them again
#pragma unroll
            for (int o = 0; o < kV4; ++o) {
                const int gy = y0 + oy0 + o;
                av[o] = bv[o] = 0.f;
                if (gx < W && gy < H) {
                    const long long pix = (base + (long long)gy * W + gx) * 3 + c;
                    av[o] = __ldg(rgb + pix);
                    bv[o] = __ldg(tgt + pix);
                }
            }
            float2 f[kV4];
            float fx[kV4];
#pragma unroll
            for (int o = 0; o < kV4; ++o) {
                float2 acc = f2(0.f, 0.f);
                float acc2 = 0.f;
#pragma unroll
                for (int k = 0; k < 2 * kR + 1; ++k) {
                    acc = __ffma2_rn(g2[k], cc[o + k], acc);
                    acc2 = fmaf(g2[k].x, c2[o + k], acc2);
                }
                f[o] = acc;
                fx[o] = acc2;
            }
            if (gx >= W) continue;
#pragma unroll
            for (int o = 0; o < kV4; ++o) {
                const int oy = oy0 + o, gy = y0 + oy;
                if (gy >= H) break;
                const long long pix = (base + (long long)gy * W + gx) * 3 + c;
                const float a = av[o], b = bv[o];
                const float d = a - b;
                l1 += fabsf(d);
                const float gd = d > 0.f ? gl1 : (d < 0.f ? -gl1 : 0.f);
                grad[pix] = f[o].x + 2.f * a * f[o].y + b * fx[o] + gd;
            }
        }
        __syncthreads();
    }
    const float tl1 = block_sum_to(l1, red);
    __syncthreads();
    const float tss = block_sum_to(ss, red);
    if (tid == 0) {
        atomicAdd(loss, gl1 * tl1 + gs * tss + (blockIdx.x == 0 ? L.lam : 0.f));
        atomicAdd(loss + 1, tl1 * L.inv_count);
        atomicAdd(loss + 2, tss * L.inv_count);
    }
}

__global__ void k_adam_tick(AdamState* st, const WsHeader* guard, double b1, double b2) {
    if (guard && guard->err != 0) {
        st->skipped += 1;
        return;
    }
    const int t = st->step + 1;
    st->step = t;
    st->c1 = (float)(1.0 / (1.0 - pow(b1, (double)t)));
    st->c2 = (float)(1.0 / sqrt(1.0 - pow(b2, (double)t)));
}

__global__ void __launch_bounds__(256) k_adam(float* __restrict__ p, const float* __restrict__ g,
                                              float* __restrict__ m, float* __restrict__ v, const AdamGroups G,
                                              const AdamState* __restrict__ st, const WsHeader* guard) {
    if (guard && guard->err != 0) return;
    const float c1 = st->c1, c2 = st->c2;
    const long long units = G.ubase[G.n];
    for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < units;
         u += (long long)gridDim.x * blockDim.x) {
        int gi = 0;
        while (u >= G.ubase[gi + 1]) ++gi;
        const unsigned e0 = (unsigned)(u - G.ubase[gi]) * 4u;
        const long long at = G.off[gi] + e0;
        const unsigned left = G.cnt[gi] - e0;
        const unsigned per = (unsigned)G.period[gi];
        const unsigned r0 = per ? e0 % per : 0u;
        float lr[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            unsigned r = r0 + (unsigned)k;
            if (per) r = (r >= per) ? r - per * (r / per) : r;
            lr[k] = (per && r >= (unsigned)G.head[gi]) ? G.lr_tail[gi] : G.lr[gi];
        }
        if (left >= 4) {
            float4 pp = *reinterpret_cast<const float4*>(p + at);
            const float4 gg = *reinterpret_cast<const float4*>(g + at);
            float4 mv = *reinterpret_cast<const float4*>(m + at);
            float4 vv = *reinterpret_cast<const float4*>(v + at);
            float* P = &pp.x;
            const float* Gr = &gg.x;
            float* M = &mv.x;
            float* V = &vv.x;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                M[k] = fmaf(G.b1, M[k], G.omb1 * Gr[k]);
                V[k] = fmaf(G.b2, V[k], G.omb2 * Gr[k] * Gr[k]);
                P[k] -= lr[k] * c1 * M[k] / (sqrtf(V[k]) * c2 + G.eps);
            }
            *reinterpret_cast<float4*>(p + at) = pp;
            *reinterpret_cast<float4*>(m + at) = mv;
            *reinterpret_cast<float4*>(v + at) = vv;
        } else {
            for (unsigned k = 0; k < left; ++k) {
                const float gk = g[at + k];
                const float mk = fmaf(G.b1, m[at + k], G.omb1 * gk);
                const float vk = fmaf(G.b2, v[at + k], G.omb2 * gk * gk);
                m[at + k] = mk;
                v[at + k] = vk;
                p[at + k] -= lr[k] * c1 * mk / (sqrtf(vk) * c2 + G.eps);
            }
        }
    }
}

}  // namespace

cudaError_t launch_loss_3dgs(const float* rgb, const float* target, const LossViews& L, float* loss, float* grad,
                             cudaStream_t s) {
    const size_t smem = (size_t)kLossSmemFloats * sizeof(float);
    // the shared-memory opt-in is a per-device function attribute: set it once per device (thread-safe)
    static std::once_flag once[64];
    static cudaError_t once_err[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::call_once(once[dev], [&] {
        once_err[dev] = cudaFuncSetAttribute(k_loss_3dgs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    });
    if (once_err[dev] != cudaSuccess) return once_err[dev];
    e = cudaMemsetAsync(loss, 0, 3 * sizeof(float), s);
    if (e != cudaSuccess) return e;
    const int tiles = L.tile_off[L.n];
    if (tiles == 0) return cudaSuccess;
    k_loss_3dgs<<<tiles, kLossThreads, smem, s>>>(rgb, target, L, loss, grad);
    return cudaGetLastError();
}

int loss_tile_side() { return kLT; }

cudaError_t launch_adam(float* p, const float* g, float* m, float* v, const AdamGroups& G, double beta1,
                        double beta2, AdamState* st, const WsHeader* guard, cudaStream_t s) {
    k_adam_tick<<<1, 1, 0, s>>>(st, guard, beta1, beta2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long units = G.ubase[G.n];
    if (units == 0) return cudaSuccess;
    int dev = 0, sms = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const long long want = (units + 255) / 256;
    const long long cap = (long long)sms * 8;
    k_adam<<<(unsigned)(want < cap ? want : cap), 256, 0, s>>>(p, g, m, v, G, st, guard);
    return cudaGetLastError();
}

}  // namespace wsr
