// Internal definitions shared by the WSR kernels (not part of the C ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "wsr.h"

namespace wsr {

// exp(-q/2) = 2^(-q log2(e)/2): the conic is stored pre-multiplied by
// log2(e)/2 so the hot loop needs one ex2 per (pixel, Gaussian) pair.
constexpr float kHalfLog2e = 0.72134752044448170f;
constexpr float kCutoff = 9.0f;                       // q <= 9: 3-sigma footprint
constexpr float kQMax = kCutoff * kHalfLog2e;         // the same cutoff, prescaled
constexpr float kLn2 = 0.69314718055994531f;
constexpr float kDilation = 0.3f;                     // low-pass term of 3DGS pre-processing
constexpr float kClamp = 1.3f;                        // Jacobian clamp: 1.3 tan(fov)
constexpr int kMaxK = 16;

// Per-view constants, passed by value in kernel parameters.
struct View {
    float R[9];
    float T[3];
    float fx, fy, cx, cy, znear;
    float campos[3];      // camera centre -R^t T
    float limx, limy;     // 1.3 tan(fov/2) per axis
    int W, H;
    int tiles_x, tiles_y;
    int tile_base;        // first global tile index of this view
    int pad;
    long long pix_base;   // first output pixel of this view
};

struct Views {
    int n;
    int tile_w, tile_h;
    int total_tiles;
    long long total_pix;
    int schedule;         // WSR_SCHEDULE_*
    int chunk;            // Gaussians per block of the backward (64 or 128)
    int det;              // deterministic mode (wsr_tiles.deterministic)
    View v[WSR_MAX_VIEWS];
};

// Workspace layout: [header 8 KB][cursor: total_tiles + 1 u32][block sums]
//                   [tile order: total_tiles u32][order buckets: 64 u32]
//                   [deterministic mode: background terms per tile, 4 floats]
// The header's first 256 bytes are the struct below; in deterministic mode the
// projection backward keeps its per-block sigma/beta sums after it.
struct WsHeader {
    int err;                   // first device-side error (wsr_status), 0 if none
    int pad0;
    float gw[8];               // gradient accumulators of sigma, beta, w_B, c_B (6 used)
    unsigned long long total;  // tile instances counted by the last binning
    unsigned int work[4];      // persistent-schedule counters: [0] forward, [1] backward
    unsigned int det_pmax;     // deterministic mode: the largest |pixel term| G/D, (G.C)/D (float bits)
};

constexpr size_t kWsHeader = 8192;
constexpr size_t kWsDetSB = 256;       // deterministic mode: sigma/beta per projection-backward block
constexpr int kDetSBBlocks = (int)((kWsHeader - kWsDetSB) / (2 * sizeof(float)));   // 992
// Deterministic mode: a record term is added as 64-bit fixed point in units of
// 2^(e - kDetBits), 2^e above an a-priori bound on the sum of the absolute
// values of all its partials (over every tile of the Gaussian), so the exact
// integer sum stays below 2^kDetBits < 2^63.
constexpr int kDetBits = 60;
constexpr int kDetRecordFloats = WSR_GRAD_RECORD_FLOATS_DET;
constexpr int kDetMaxSegment = WSR_DET_MAX_SEGMENT;
constexpr int kScanBlock = 1024;       // threads of a scan block
constexpr int kScanItems = 4;          // elements per scan thread
constexpr int kScanTile = kScanBlock * kScanItems;

__host__ __device__ inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

__device__ __forceinline__ void set_error(WsHeader* h, int code) { atomicCAS(&h->err, 0, code); }

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// Hardware square root and reciprocal (relative error ~2^-22): the backward's
// per-row spans (widened by 0.02 pixel, far above that), the footprint test's
// minimising points and the SSIM map's two quotients.
__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Does the footprint q' <= kQMax reach a pixel centre of the rectangle
// [x0, x1] x [y0, y1] (pixel-centre coordinates)?  The record holds the
// quadratic as a sum of squares, q' = (qs dy + qw dx)^2 + qd dx^2.  Its
// minimum over the rectangle is at the centre when the centre is inside,
// otherwise on an edge, where it is a one-dimensional quadratic.  The
// threshold is widened slightly so the test stays conservative with respect
// to the renderers' FP32 per-pixel test.
__device__ __forceinline__ bool footprint_hits(float mx, float my, float qs, float qw, float qd, float x0,
                                               float x1, float y0, float y1) {
    if (mx >= x0 && mx <= x1 && my >= y0 && my <= y1) return true;
    const float thr = kQMax * 1.0001f + 1e-4f;
    auto q = [&](float dx, float dy) {
        const float r = fmaf(qs, dy, qw * dx);
        return fmaf(r, r, qd * dx * dx);
    };
    float best = 3.4e38f;
    // The minimising points below come from hardware reciprocals (relative error ~2^-22): q is
    // evaluated exactly at a point of the edge either way, and a point that far from the minimiser
    // raises q by a relative ~1e-13 against the threshold's 1e-4 margin.
    // vertical edges x = x0, x1: the minimum over dy is at qs dy = -qw dx
    const float ex[2] = {x0 - mx, x1 - mx};
    const float kx = -qw * rcp_approx(qs);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float dx = ex[k];
        const float dy = fminf(fmaxf(kx * dx, y0 - my), y1 - my);
        best = fminf(best, q(dx, dy));
    }
    // horizontal edges y = y0, y1: the minimum over dx is at dx = -qw qs dy / (qw^2 + qd)
    const float ey[2] = {y0 - my, y1 - my};
    const float ky = -qw * qs * rcp_approx(fmaf(qw, qw, qd));
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float dy = ey[k];
        const float dx = fminf(fmaxf(ky * dy, x0 - mx), x1 - mx);
        best = fminf(best, q(dx, dy));
    }
    return best <= thr;
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ---------------------------------------------------------------------------
// Real spherical harmonics (Eqs. 4 and 11), degree <= 3, on a unit vector
// (x, y, z), with the Condon-Shortley phase; index l^2 + l + m.  Each
// constant is the closed form of the real SH normalisation given beside it.
// ---------------------------------------------------------------------------
constexpr float kSH0 = 0.28209479177387814f;    // sqrt(1 / (4 pi))
constexpr float kSH1 = 0.48860251190291992f;    // sqrt(3 / (4 pi))
constexpr float kSH2a = 1.0925484305920792f;    // sqrt(15 / pi) / 2
constexpr float kSH2b = 0.31539156525252005f;   // sqrt(5 / pi) / 4
constexpr float kSH2c = 0.54627421529603959f;   // sqrt(15 / pi) / 4
constexpr float kSH3a = 0.59004358992664352f;   // sqrt(35 / (2 pi)) / 4
constexpr float kSH3b = 2.8906114426405538f;    // sqrt(105 / pi) / 2
constexpr float kSH3c = 0.45704579946446572f;   // sqrt(21 / (2 pi)) / 4
constexpr float kSH3d = 0.37317633259011540f;   // sqrt(7 / pi) / 4
constexpr float kSH3e = 1.4453057213202769f;    // sqrt(105 / pi) / 4

template <int DEG>
__device__ __forceinline__ void sh_basis(float x, float y, float z, float* Y) {
    Y[0] = kSH0;
    if (DEG >= 1) {
        Y[1] = -kSH1 * y;
        Y[2] = kSH1 * z;
        Y[3] = -kSH1 * x;
    }
    if (DEG >= 2) {
        const float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = kSH2a * x * y;
        Y[5] = -kSH2a * y * z;
        Y[6] = kSH2b * (3.0f * zz - 1.0f);
        Y[7] = -kSH2a * x * z;
        Y[8] = kSH2c * (xx - yy);
        if (DEG >= 3) {
            Y[9] = -kSH3a * y * (3.0f * xx - yy);
            Y[10] = kSH3b * x * y * z;
            Y[11] = -kSH3c * y * (5.0f * zz - 1.0f);
            Y[12] = kSH3d * z * (5.0f * zz - 3.0f);
            Y[13] = -kSH3c * x * (5.0f * zz - 1.0f);
            Y[14] = kSH3e * z * (xx - yy);
            Y[15] = -kSH3a * x * (xx - 3.0f * yy);
        }
    }
}

// Polynomial gradient of every basis function, contracted with per-basis
// weights: g += sum_k wk[k] * dY_k/d(x, y, z).  Only the tangential part is
// meaningful on the sphere; callers project it.
template <int DEG>
__device__ __forceinline__ void sh_grad_dot(float x, float y, float z, const float* wk, float& gx,
                                            float& gy, float& gz) {
    if (DEG >= 1) {
        gy += -kSH1 * wk[1];
        gz += kSH1 * wk[2];
        gx += -kSH1 * wk[3];
    }
    if (DEG >= 2) {
        gx += kSH2a * y * wk[4];
        gy += kSH2a * x * wk[4];
        gy += -kSH2a * z * wk[5];
        gz += -kSH2a * y * wk[5];
        gz += 6.0f * kSH2b * z * wk[6];
        gx += -kSH2a * z * wk[7];
        gz += -kSH2a * x * wk[7];
        gx += 2.0f * kSH2c * x * wk[8];
        gy += -2.0f * kSH2c * y * wk[8];
        if (DEG >= 3) {
            const float xx = x * x, yy = y * y, zz = z * z;
            gx += -6.0f * kSH3a * x * y * wk[9];
            gy += -3.0f * kSH3a * (xx - yy) * wk[9];
            gx += kSH3b * y * z * wk[10];
            gy += kSH3b * x * z * wk[10];
            gz += kSH3b * x * y * wk[10];
            gy += -kSH3c * (5.0f * zz - 1.0f) * wk[11];
            gz += -10.0f * kSH3c * y * z * wk[11];
            gz += kSH3d * (15.0f * zz - 3.0f) * wk[12];
            gx += -kSH3c * (5.0f * zz - 1.0f) * wk[13];
            gz += -10.0f * kSH3c * x * z * wk[13];
            gx += 2.0f * kSH3e * x * z * wk[14];
            gy += -2.0f * kSH3e * y * z * wk[14];
            gz += kSH3e * (xx - yy) * wk[14];
            gx += -3.0f * kSH3a * (xx - yy) * wk[15];
            gy += 6.0f * kSH3a * x * y * wk[15];
        }
    }
}

// ---------------------------------------------------------------------------
// Parameter loads: float32, or the reduced-precision storage (bf16 scales and
// quaternions, f16 SH and opacity).
// ---------------------------------------------------------------------------
template <bool RED>
struct Store;
template <>
struct Store<false> {
    using sq_t = float;
    using sh_t = float;
};
template <>
struct Store<true> {
    using sq_t = __nv_bfloat16;
    using sh_t = __half;
};

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__half v) { return __half2float(v); }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }

// Load N consecutive elements of type T starting at p into floats, using
// 16-byte loads when the span is a whole number of 16-byte units (the caller
// guarantees 16-byte alignment of p in that case).
template <typename T, int N>
__device__ __forceinline__ void load_n(const T* __restrict__ p, float* out) {
    constexpr int bytes = N * (int)sizeof(T);
    if constexpr (bytes % 16 == 0) {
        constexpr int vec = bytes / 16;
        constexpr int per = 16 / (int)sizeof(T);
        const uint4* q = reinterpret_cast<const uint4*>(p);
#pragma unroll
        for (int k = 0; k < vec; ++k) {
            uint4 u = __ldg(q + k);
            const T* e = reinterpret_cast<const T*>(&u);
#pragma unroll
            for (int j = 0; j < per; ++j) out[k * per + j] = to_f(e[j]);
        }
    } else {
#pragma unroll
        for (int k = 0; k < N; ++k) out[k] = to_f(p[k]);
    }
}

// Rotation matrix of a unit quaternion (w, x, y, z).
__device__ __forceinline__ void quat_rot(float w, float x, float y, float z, float* R) {
    R[0] = 1.f - 2.f * (y * y + z * z);
    R[1] = 2.f * (x * y - w * z);
    R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z);
    R[4] = 1.f - 2.f * (x * x + z * z);
    R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y);
    R[7] = 2.f * (y * z + w * x);
    R[8] = 1.f - 2.f * (x * x + y * y);
}

// Global tile -> view (views are few; a linear scan is enough).
__device__ __forceinline__ int view_of_tile(const Views& vs, int tile) {
    int v = vs.n - 1;
    while (v > 0 && tile < vs.v[v].tile_base) --v;
    return v;
}

}  // namespace wsr
