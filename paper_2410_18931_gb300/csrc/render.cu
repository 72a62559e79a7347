// Per-pixel Weighted Sum Rendering, forward and backward (Eq. 7).
//
// One thread block per tile (or, with the persistent schedule, one per
// resident slot taking tiles longest first).  Each warp of the block streams
// the tile's Gaussian list (unordered: Eq. 7 is a sum) through shared memory
// on its own, 32 records at a time, keeping those whose footprint reaches its
// rows; every thread owns a 2x2 block of pixels (two columns share each
// paired float2 FP32 instruction) and accumulates, in FP32 registers,
//     N += (c u w) e,   D += (u w) e,   e = exp(-q/2) = 2^(-q'),   q <= 9
// with q' = q log2(e)/2 evaluated from the record's sum of squares
// q' = (qs dy + qw dx)^2 + qd dx^2, which has no cancellation even for
// needle-like footprints.
// There is no early termination (App. D: every covering Gaussian counts).
// The epilogue writes C = (c_B w_B + N) / (w_B + D) and the denominator.
//
// The backward recomputes every (pixel, Gaussian) term from the records and
// the stored C and denominator (no per-pixel lists are kept).  It walks the
// pixels of each Gaussian's footprint row by row (per-row spans), a group of
// lanes per Gaussian, and per Gaussian adds d/d(u w), d/d(c u w) and moments
// of dL/dq' to a gradient record.
#include "wsr_launch.h"

namespace wsr {
namespace {

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

// Threads per block of the backward for chunks of CH Gaussians: 2 CH, at most 256.
template <int CH>
struct BwdThreads {
    static constexpr int value = CH < 128 ? 2 * CH : 256;
};

// Asynchronous 16-byte global-to-shared copies (both addresses 16-byte aligned).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// A lane count as a type, to instantiate one walk of the backward per group size.
template <int N>
struct Lanes {
    static constexpr int value = N;
};

// The backward's pixel spans of one record on the rows of a tile: on row y the
// footprint q' <= QM is mu_x + c(dy) +- h(dy) with the conic entries
// A' = qw^2 + qd, B' = qs qw, C' = qs^2, det' = A' C' - B'^2 = qd qs^2:
// c = -B' dy / A', h = sqrt(A' QM - det' dy^2) / A' (no cancellation anywhere),
// widened by 0.02 pixel.  `row` gives the span of a local row as
// (first column, rounded down to even) | (column pairs << 8): the pairs from
// that even column that hold the span (a padding pixel at either end lies
// outside the footprint or in the tile's zero column).
struct RowSpans {
    float Ap, hb, det, ia, ext, apqm, hbia;
    __device__ __forceinline__ RowSpans(const float4 a, const float qd, const float QM) {
        Ap = fmaf(a.w, a.w, qd);
        hb = a.z * a.w;
        det = qd * a.z * a.z;
        ia = rcp_approx(Ap);
        apqm = Ap * QM;
        hbia = hb * ia;
        // rows the footprint can reach: |dy| <= sqrt(A' QM / det'), with a pixel of slack
        ext = fminf(sqrt_approx(fmaxf(Ap * QM * rcp_approx(det), 0.0f)), 1e6f) + 1.0f;
    }
    // local rows [lo, hi] of the block [first, first + count) that the footprint can reach
    __device__ __forceinline__ void rows(const float4 a, int y_org, int first, int count, int& lo, int& hi) const {
        lo = max(first, (int)floorf(a.y - ext - 0.5f) - y_org);
        hi = min(first + count - 1, (int)ceilf(a.y + ext - 0.5f) - y_org);
    }
    __device__ __forceinline__ unsigned short row(const float4 a, const float QM, int x_org, int y_org, int x_lim,
                                                  int ly) const {
        const float dy = (float)(y_org + ly) + 0.5f - a.y;
        const float d4 = fmaf(-det * dy, dy, Ap * QM);
        if (d4 < 0.0f) return 0;
        const float h = sqrt_approx(d4) * ia;
        const float cx = a.x - hb * dy * ia;
        const float fx0 = fmaxf(ceilf(cx - h - 0.52f), (float)x_org);
        const float fx1 = fminf(floorf(cx + h - 0.48f), (float)(x_org + x_lim - 1));
        if (!(fx0 <= fx1)) return 0;
        const int xs = (int)fx0 - x_org, len = (int)fx1 - (int)fx0 + 1, xe = xs & ~1;
        return (unsigned short)(xe | (((xs - xe + len + 1) >> 1) << 8));    // even start, column pairs
    }
    // the spans of local rows ly and ly + 1 (low and high half), two rows per paired FP32 op
    __device__ __forceinline__ unsigned row2(const float4 a, int x_org, int y_org, int x_lim, int ly) const {
        const float dy0 = (float)(y_org + ly) + 0.5f - a.y;
        const float2 dy = f2(dy0, dy0 + 1.0f);
        const float2 d4 = __ffma2_rn(__fmul2_rn(f2(-det, -det), dy), dy, f2(apqm, apqm));
        const float2 h = __fmul2_rn(f2(sqrt_approx(fmaxf(d4.x, 0.0f)), sqrt_approx(fmaxf(d4.y, 0.0f))), f2(ia, ia));
        const float2 cx = __ffma2_rn(f2(-hbia, -hbia), dy, f2(a.x, a.x));
        const float2 l = __fadd2_rn(__ffma2_rn(h, f2(-1.0f, -1.0f), cx), f2(-0.52f, -0.52f));
        const float2 r = __fadd2_rn(__fadd2_rn(cx, h), f2(-0.48f, -0.48f));
        const float xlo = (float)x_org, xhi = (float)(x_org + x_lim - 1);
        unsigned out = 0;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const float fx0 = fmaxf(ceilf(k ? l.y : l.x), xlo), fx1 = fminf(floorf(k ? r.y : r.x), xhi);
            if ((k ? d4.y : d4.x) >= 0.0f && fx0 <= fx1) {
                const int xs = (int)fx0 - x_org, len = (int)fx1 - (int)fx0 + 1, xe = xs & ~1;
                out |= (unsigned)(xe | (((xs - xe + len + 1) >> 1) << 8)) << (16 * k);
            }
        }
        return out;
    }
};

// Pixel-per-thread layout of the pair-count diagnostic.
template <int TW, int TH, int PPT>
struct TileShape {
    static constexpr int NT = TW * TH / PPT;
    static_assert(TH % PPT == 0 && NT % 32 == 0, "whole warps");
};

// Forward tile shape: each thread owns a PX x 2 block of pixels (PX = 2 or 1),
// so two horizontally adjacent pixels share one paired (float2) FP32 op.
template <int TW, int TH, int PX>
struct FwdShape {
    static constexpr int PY = 2;
    static constexpr int BX = TW / PX;                  // thread columns
    static constexpr int NT = (TW / PX) * (TH / PY);    // threads per block
    static constexpr int NW = NT / 32;
    static_assert(NT % 32 == 0 && 32 % BX == 0, "whole warps of whole thread rows");
    // first and last pixel row (within the tile) of warp w
    __host__ __device__ static constexpr int row_lo(int w) { return (32 * w / BX) * PY; }
    __host__ __device__ static constexpr int row_hi(int w) { return ((32 * w + 31) / BX) * PY + PY - 1; }
};

template <int TW, int TH, int PX>
__device__ __forceinline__ void fwd_tile(const int tile, const float4* __restrict__ rec,
                                         const unsigned* __restrict__ offsets, const unsigned* __restrict__ list,
                                         const Views& vs, const float* __restrict__ wparams,
                                         float* __restrict__ out_rgb, float* __restrict__ out_den) {
    using S = FwdShape<TW, TH, PX>;
    constexpr int NW = S::NW;
    // per warp, the Gaussians of its current batch that reach its rows
    __shared__ float4 s0[NW][32];   // qs, qw, c_r u w, c_g u w
    __shared__ float2 s2[NW][32];   // c_b u w, u w
    __shared__ float4 s3[NW][32];   // at the tile's first pixel centre: r, qd dx^2, 2 qd dx; and qd
    __shared__ float4 sraw[NW][2][32][3];   // per warp, two batches of records in flight (cp.async)

    const TileCoord tc = tile_coord(vs, tile);
    const View& V = vs.v[tc.v];
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const int x0 = tc.tx * TW + (tid % S::BX) * PX;
    const int y0 = tc.ty * TH + (tid / S::BX) * S::PY;
    // offsets of the block's pixels from the tile's first pixel (PX == 1: the first column only, its two
    // rows paired instead)
    const float2 ox = f2((float)(x0 - tc.tx * TW), (float)(x0 - tc.tx * TW + 1));
    const float oy0 = (float)(y0 - tc.ty * TH), oy1 = oy0 + 1.0f;
    // the warp's pixel-centre rectangle
    const float xl = (float)(tc.tx * TW) + 0.5f, xh = xl + (float)(TW - 1);
    const float yl = (float)(tc.ty * TH + S::row_lo(w)) + 0.5f, yh = (float)(tc.ty * TH + S::row_hi(w)) + 0.5f;

    // accumulators per pixel (column c, row r): (N_r, N_g) and (N_b, D)
    float2 rg[2][2], bd[2][2];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 2; ++c) rg[r][c] = bd[r][c] = f2(0.f, 0.f);

    // Each warp takes the tile's list 32 Gaussians at a time on its own (no block barrier): a lane
    // takes one record and, with several warps per tile, tests whether the footprint reaches a pixel
    // centre of the warp's rows (exact ellipse-rectangle test); the hits are compacted and walked.
    // The next batch's records are copied into shared memory (cp.async) while the warp walks this one.
    const unsigned start = offsets[tile], end = offsets[tile + 1];
    unsigned nidx = start + lane < end ? list[start + lane] : 0u;       // the next batch's record index
    auto fetch = [&](unsigned b, int buf) {
        if (b + lane < end) {
            const float4* p = rec + 3ull * nidx;
#pragma unroll
            for (int q = 0; q < 3; ++q) cp_async16(&sraw[w][buf][lane][q], p + q);
        }
        cp_async_commit();
        nidx = b + 32 + lane < end ? list[b + 32 + lane] : 0u;
    };
    fetch(start, 0);
    int buf = 0;
    for (unsigned base = start; base < end; base += 32, buf ^= 1) {
        const int cnt = (int)min(32u, end - base);
        fetch(base + 32, buf ^ 1);                      // an empty group past the end
        cp_async_wait<1>();                             // this batch's copies have landed
        __syncwarp();
        bool hit = false;
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
        float cb = 0.f;
        if (lane < cnt) {
            a = sraw[w][buf][lane][0];
            b = sraw[w][buf][lane][1];
            cb = sraw[w][buf][lane][2].x;
            hit = NW == 1 || footprint_hits(a.x, a.y, a.z, a.w, b.x, xl, xh, yl, yh);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, hit);
        const int nj = __popc(bal);
        __syncwarp();                                   // the previous batch's walk is done with the arrays
        if (hit) {
            const int k = __popc(bal & ((1u << lane) - 1u));
            s0[w][k] = make_float4(a.z, a.w, b.z, b.w);
            s2[w][k] = f2(cb, b.y);
            const float gx = (float)(tc.tx * TW) + 0.5f - a.x, gy = (float)(tc.ty * TH) + 0.5f - a.y;
            s3[w][k] = make_float4(fmaf(a.z, gy, a.w * gx), b.x * gx * gx, 2.0f * b.x * gx, b.x);
        }
        __syncwarp();
#pragma unroll 8
        for (int k = 0; k < nj; ++k) {
            const float4 g = s0[w][k];
            const float2 cbuw = s2[w][k];
            const float4 t = s3[w][k];
            const float qs = g.x, qw = g.y;
            const float2 crg = f2(g.z, g.w);
            // q' = r^2 + qd dx^2 with dx = g_x + o_x: qd dx^2 = qd g_x^2 + o_x (2 qd g_x + o_x qd) and
            // r = r_0 + qs o_y + qw o_x from the values at the tile's first pixel centre
            if constexpr (PX == 1) {
                // one column, its two rows paired: the same dx, so the same qd dx^2
                const float P1 = fmaf(ox.x, fmaf(ox.x, t.w, t.z), t.y);
                const float base = fmaf(qw, ox.x, t.x);
                const float2 rr = __ffma2_rn(f2(qs, qs), f2(oy0, oy1), f2(base, base));
                const float2 q = __ffma2_rn(rr, rr, f2(P1, P1));
                if (q.x <= kQMax) {
                    const float e = ex2_approx(-q.x);
                    rg[0][0] = __ffma2_rn(crg, f2(e, e), rg[0][0]);
                    bd[0][0] = __ffma2_rn(cbuw, f2(e, e), bd[0][0]);
                }
                if (q.y <= kQMax) {
                    const float e = ex2_approx(-q.y);
                    rg[1][0] = __ffma2_rn(crg, f2(e, e), rg[1][0]);
                    bd[1][0] = __ffma2_rn(cbuw, f2(e, e), bd[1][0]);
                }
                continue;
            }
            const float2 P = __ffma2_rn(ox, __ffma2_rn(ox, f2(t.w, t.w), f2(t.z, t.z)), f2(t.y, t.y));
            const float rys[2] = {fmaf(qs, oy0, t.x), fmaf(qs, oy1, t.x)};
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const float2 rr = __ffma2_rn(f2(qw, qw), ox, f2(rys[r], rys[r]));
                const float2 q = __ffma2_rn(rr, rr, P);
                if (q.x <= kQMax) {
                    const float e = ex2_approx(-q.x);
                    rg[r][0] = __ffma2_rn(crg, f2(e, e), rg[r][0]);
                    bd[r][0] = __ffma2_rn(cbuw, f2(e, e), bd[r][0]);
                }
                if (q.y <= kQMax) {
                    const float e = ex2_approx(-q.y);
                    rg[r][1] = __ffma2_rn(crg, f2(e, e), rg[r][1]);
                    bd[r][1] = __ffma2_rn(cbuw, f2(e, e), bd[r][1]);
                }
            }
        }
    }

    const float wB = __ldg(wparams + 2);
    const float cB0 = __ldg(wparams + 3) * wB, cB1 = __ldg(wparams + 4) * wB, cB2 = __ldg(wparams + 5) * wB;
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < PX; ++c) {
            const int x = x0 + c, y = y0 + r;
            if (x < V.W && y < V.H) {
                const long long pix = V.pix_base + (long long)y * V.W + x;
                const float D = wB + bd[r][c].y;
                const float inv = 1.0f / D;
                out_rgb[3 * pix + 0] = (cB0 + rg[r][c].x) * inv;
                out_rgb[3 * pix + 1] = (cB1 + rg[r][c].y) * inv;
                out_rgb[3 * pix + 2] = (cB2 + bd[r][c].x) * inv;
                out_den[pix] = D;
            }
        }
}

// Persistent schedule: blocks take tiles order[0..n) through *counter.
template <typename F>
__device__ __forceinline__ void for_each_tile(const unsigned* __restrict__ order, unsigned* __restrict__ counter,
                                              int n_tiles, F&& body) {
    if (order == nullptr) {
        body((int)blockIdx.x);
        return;
    }
    __shared__ int s_item;
    for (;;) {
        __syncthreads();                      // the previous tile is done with shared memory
        if (threadIdx.x == 0) s_item = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int item = s_item;
        if (item >= n_tiles) break;
        body((int)order[item]);
    }
}

template <int TW, int TH, int PX>
__global__ void __launch_bounds__(FwdShape<TW, TH, PX>::NT)
    k_render_fwd(const float4* __restrict__ rec, const unsigned* __restrict__ offsets,
                 const unsigned* __restrict__ list, const Views vs, const float* __restrict__ wparams,
                 float* __restrict__ out_rgb, float* __restrict__ out_den, const unsigned* __restrict__ order,
                 unsigned* __restrict__ counter) {
    for_each_tile(order, counter, vs.total_tiles, [&](int tile) {
        fwd_tile<TW, TH, PX>(tile, rec, offsets, list, vs, wparams, out_rgb, out_den);
    });
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// Backward, one block per tile, a group of lanes per Gaussian.
//
// The tile's pixel terms P = (G/D, -(G.C)/D) sit in shared memory by column
// pairs, two float4 planes (x0, x1, y0, y1) and (z0, z1, w0, w1), with zero
// pairs past the tile's right edge as far as a lane reads.  For each chunk of
// CH Gaussians of the tile:
//   A. two threads per Gaussian compute, for their half of the tile's rows
//      (two rows per paired op), the span of pixels whose centre can lie
//      inside the footprint (the roots of q(dx) = 9 on each row, widened
//      slightly), kept as its first column rounded down to even and a number
//      of column pairs, and the first and last rows with a span, and take
//      the Gaussian's rank in its bucket of the sort below;
//   B. the chunk's Gaussians are ordered wide ones first (a row span longer
//      than TW / 2 pixels), each class by its number of rows, longest first
//      (a counting sort: the buckets' starts from one warp suffix scan); each
//      warp takes the next Gaussians of a class whenever it is free (a shared
//      counter per class), so that the groups of a warp walk for the same
//      number of steps and the warps stay busy;
//   C. a group of L consecutive lanes takes one Gaussian at a time and walks
//      its rows one per step, L = TW / (2 M) for the wide class and TW / (4 M)
//      for the narrow one (whose spans all fit in 2 M L columns), M = 4 column
//      pairs per lane and row (2 for 8-pixel-wide tiles); lane k takes column
//      pairs start / 2 + k + m L (m < M) of the row, so the lanes of a group
//      read consecutive entries of each plane, 2 M pixels per step from one
//      decode of the row's span, every quantity of a column pair in one
//      paired FP32 op.  The nine record terms stay in registers until
//      the Gaussian's last row; then log2(L) shuffle steps sum them over the
//      group and its first lane adds them to the Gaussian's global record (in
//      the deterministic mode: as fixed point, in units that a per-Gaussian
//      bound fixes).  A Gaussian's sums over a tile are thus formed in one
//      fixed order, whichever group takes it.
// Every pair is tested against the forward's cutoff (q' <= kQMax, FP32, from
// the same record values).  The forward forms q' from values at the tile's
// first pixel centre, the walk from each pixel's own offsets, so a pair
// within rounding of the cutoff (a tie: its term is e^-4.5 of the
// Gaussian's peak there) may be counted by one and not the other.
// Gaussians per chunk: CH, a template parameter (64, 128, 256 or 512); threads
// per block: BwdThreads<CH> (2 CH up to 256).
template <int TW, int TH, int CH>
__device__ __forceinline__ void bwd_tile(const int tile, const float4* __restrict__ rec,
                                         const unsigned* __restrict__ offsets, const unsigned* __restrict__ list,
                                         const Views& vs, const float* __restrict__ wparams,
                                         const float* __restrict__ out_rgb, const float* __restrict__ out_den,
                                         const float* __restrict__ grad_rgb, float* __restrict__ grec,
                                         float* __restrict__ gw, const int pass, float* __restrict__ bg_tiles,
                                         const unsigned* __restrict__ det_pmax) {
    constexpr int NT = BwdThreads<CH>::value;
    constexpr int NW = NT / 32;
    constexpr int PASSES = 2 * CH / NT;                // step A: (Gaussian, half) items per thread
    // pixel-table row pitch in column pairs: the row's TW / 2 pairs, then zero pairs up to the farthest pair a
    // lane reads (start / 2 + k + m L <= (TW / 2 - 1) + (TW / 2 - 1)), so no index needs a clamp; odd, so that
    // the rows start in different banks
    constexpr int PP = TW - 1;
    constexpr int HR = TH / 2;                          // rows per thread in step A
    constexpr int NB = TH + 1;                          // row counts 0 .. TH
    constexpr int NK = 2 * NB;                          // sort keys: narrow 0 .. TH, wide NB .. NB + TH
    static_assert(PASSES * NT == 2 * CH && TH % 4 == 0 && TW % 8 == 0 && TW <= 64 && CH <= 512 && NK <= NT, "layout");
    constexpr int M = TW >= 16 ? 4 : 2;                 // column pairs per lane and row in step C
    // per pixel: G/D (3), -(G.C)/D, stored per column pair as (x0, x1, y0, y1) and (z0, z1, w0, w1)
    __shared__ float4 spA[PP * TH];
    __shared__ float4 spB[PP * TH];
    __shared__ float4 s0[CH];                   // mu_x, mu_y, qs, qw
    __shared__ float4 s1[CH];                   // qd, u w, c_r u w, c_g u w
    __shared__ float2 s2[CH];                   // c_b u w, u w
    __shared__ unsigned sidx[CH];
    __shared__ unsigned short sspan[CH][TH];    // per row: even first column | column pairs << 8
    __shared__ unsigned char sfirst[CH];        // first row with a span
    __shared__ unsigned char snst[CH];          // rows from there to the last row with a span
    __shared__ unsigned char skey[CH];          // sort key: rows, plus NB when wide
    __shared__ unsigned short srank[CH];        // rank among the chunk's Gaussians of the same key
    __shared__ unsigned short sord[CH];         // the chunk's Gaussians: wide ones first, most rows first
    __shared__ unsigned shist[NK];
    __shared__ unsigned snext[2];               // per class: the next position of the order a warp takes
    __shared__ float sbg[4][NW];

    const TileCoord tc = tile_coord(vs, tile);
    const View& V = vs.v[tc.v];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int x_org = tc.tx * TW, y_org = tc.ty * TH;
    const int x_lim = min(TW, V.W - x_org);    // pixels of the tile inside the image
    const int y_lim = min(TH, V.H - y_org);
    const float wB = __ldg(wparams + 2);
    const float cB0 = __ldg(wparams + 3), cB1 = __ldg(wparams + 4), cB2 = __ldg(wparams + 5);
    const float pmax = pass != 0 ? __int_as_float(*det_pmax) : 0.0f;    // deterministic mode

    float bg[4] = {0.f, 0.f, 0.f, 0.f};
    for (int p = tid; p < 2 * PP * TH; p += NT) {
        const int ly = p / (2 * PP), lx = p - ly * (2 * PP);
        float4 f = make_float4(0.f, 0.f, 0.f, 0.f);
        if (lx < x_lim && ly < y_lim) {
            const long long pix = V.pix_base + (long long)(y_org + ly) * V.W + x_org + lx;
            const float inv = 1.0f / out_den[pix];
            const float G0 = grad_rgb[3 * pix], G1 = grad_rgb[3 * pix + 1], G2 = grad_rgb[3 * pix + 2];
            const float C0 = out_rgb[3 * pix], C1 = out_rgb[3 * pix + 1], C2 = out_rgb[3 * pix + 2];
            f = make_float4(G0 * inv, G1 * inv, G2 * inv, -(G0 * C0 + G1 * C1 + G2 * C2) * inv);
            // dL/dw_B = G.(c_B - C)/D,  dL/dc_B = G w_B / D
            bg[0] += f.x * cB0 + f.y * cB1 + f.z * cB2 + f.w;
            bg[1] += f.x * wB;
            bg[2] += f.y * wB;
            bg[3] += f.z * wB;
        }
        const int pi = 4 * (ly * PP + (lx >> 1)) + (lx & 1);
        reinterpret_cast<float*>(spA)[pi] = f.x;
        reinterpret_cast<float*>(spA)[pi + 2] = f.y;
        reinterpret_cast<float*>(spB)[pi] = f.z;
        reinterpret_cast<float*>(spB)[pi + 2] = f.w;
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const float t = warp_sum(bg[c]);
        if (lane == 0) sbg[c][warp] = t;
    }

    const float QM = kQMax * 1.0001f + 1e-4f;
    const unsigned start = offsets[tile], end = offsets[tile + 1];
    if (tid < NK) shist[tid] = 0u;
    for (unsigned base = start; base < end; base += CH) {
        const int cnt = (int)min((unsigned)CH, end - base);
        __syncthreads();                                // the previous chunk is done with shared memory
        // ---- A: record, spans of half the rows of a Gaussian per item, first and last rows ----
#pragma unroll 1
        for (int ps = 0; ps < PASSES; ++ps) {
            const int u = tid + ps * NT;
            const int gj = u >> 1, half = u & 1;
            unsigned rows = 0u;                         // bit ly: row ly has a span
            unsigned umax = 0u;                         // the most column pairs of a row's span
            if (gj < cnt) {
                const unsigned r = list[base + gj];
                const float4* pr = rec + 3ull * r;
                const float4 a = __ldg(pr);
                const float4 b = __ldg(pr + 1);
                if (half == 0) {
                    const float cb = __ldg(reinterpret_cast<const float*>(pr + 2));
                    s0[gj] = a;
                    s1[gj] = b;
                    s2[gj] = f2(cb, b.y);
                    sidx[gj] = r;
                }
                const RowSpans rs(a, b.x, QM);
#pragma unroll
                for (int k = 0; k < HR; k += 2) {
                    const int ly = half * HR + k;
                    // rows the footprint does not reach have no span (no root: the square root's argument is
                    // negative); rows past the image's last have none either
                    unsigned sp2 = rs.row2(a, x_org, y_org, x_lim, ly);
                    if (ly + 1 >= y_lim) sp2 = ly < y_lim ? sp2 & 0x0000ffffu : 0u;
                    *reinterpret_cast<unsigned*>(&sspan[gj][ly]) = sp2;
                    rows |= ((sp2 & 0x0000ff00u) ? 1u : 0u) << ly;
                    rows |= ((sp2 & 0xff000000u) ? 2u : 0u) << ly;
                    umax = max(umax, max((sp2 >> 8) & 0xffu, sp2 >> 24));
                }
            }
            rows |= __shfl_xor_sync(0xffffffffu, rows, 1);           // the two halves of a Gaussian
            umax = max(umax, __shfl_xor_sync(0xffffffffu, umax, 1));
            const int row_lo = rows ? __ffs((int)rows) - 1 : TH, row_hi = rows ? 31 - __clz((int)rows) : -1;
            if (gj < cnt && half == 0) {
                const int nst = row_hi >= row_lo ? row_hi - row_lo + 1 : 0;
                const int key = nst + (2 * (int)umax > TW / 2 ? NB : 0);    // wide: a span longer than TW / 2 pixels
                sfirst[gj] = (unsigned char)max(row_lo, 0);
                snst[gj] = (unsigned char)nst;
                skey[gj] = (unsigned char)key;
                srank[gj] = (unsigned short)atomicAdd(&shist[key], 1u);
            }
        }
        if (tid < 2) snext[tid] = 0u;
        __syncthreads();
        // ---- B: the chunk's order, wide first, most rows first: each warp forms the buckets' starts (the
        // counts of all larger keys, a suffix scan over the NK <= 64 keys held two per lane), and a
        // Gaussian's position is its bucket's start plus its rank in the bucket ----
        const unsigned h0 = lane < NK ? shist[lane] : 0u, h1 = lane + 32 < NK ? shist[lane + 32] : 0u;
        unsigned s0i = h0, s1i = h1;                    // inclusive suffix sums of keys lane and lane + 32
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned y0 = __shfl_down_sync(0xffffffffu, s0i, off), y1 = __shfl_down_sync(0xffffffffu, s1i, off);
            if (lane + off < 32) {
                s0i += y0;
                s1i += y1;
            }
        }
        s0i += __shfl_sync(0xffffffffu, s1i, 0);        // keys 32.. lie above every key of the first half
        const unsigned start0 = s0i - h0, start1 = s1i - h1;
        const int nwide = (int)__shfl_sync(0xffffffffu, s0i, NB);   // Gaussians with keys NB and up: the wide
        static_assert(NB < 32, "the wide class starts in the first half of the keys");
        for (int g0 = warp * 32; g0 < cnt; g0 += NT) {
            const int gj = g0 + lane;
            const int key = gj < cnt ? (int)skey[gj] : 0;
            const unsigned a0 = __shfl_sync(0xffffffffu, start0, key & 31);
            const unsigned a1 = __shfl_sync(0xffffffffu, start1, key & 31);
            if (gj < cnt) sord[(key < 32 ? a0 : a1) + srank[gj]] = (unsigned short)gj;
        }
        __syncthreads();
        if (tid < NK) shist[tid] = 0u;                  // for the next chunk (step C does not read it)
        // ---- C: a group per Gaussian; each warp takes the next 32 / L Gaussians of a class ----
        auto walk = [&](auto lanes, const int lo, const int hi, unsigned* next) {
            constexpr int L = decltype(lanes)::value;
            constexpr int GW = 32 / L;                  // groups per warp
            const int grp = lane / L, gk = lane % L;    // group and lane within the group
            for (;;) {
                unsigned at0 = 0;
                if (lane == 0) at0 = atomicAdd(next, (unsigned)GW);
                at0 = __shfl_sync(0xffffffffu, at0, 0);
                if (lo + (int)at0 >= hi) break;
                const int so = lo + (int)at0 + grp;
                const bool act = so < hi;
                const int j = act ? (int)sord[so] : 0;
                const int steps = act ? (int)snst[j] : 0;
                const int r0 = act ? (int)sfirst[j] : 0;
                const float4 a = s0[j], b = s1[j];
                const float2 c2 = s2[j];
                const float gx0 = (float)x_org + 0.5f - a.x;                 // dx of column 0
                const float gy0 = (float)y_org + 0.5f - a.y;                 // dy of row 0
                const float qs = a.z;
                const float2 qw2 = f2(a.w, a.w), qd2 = f2(b.x, b.x), gx2 = f2(gx0, gx0);
                // dL/dq' = e (P . cw) with cw = -ln2 u w (c, 1): the walk uses the colour c = (c u w) / (u w)
                // (in both halves of a pair) and applies the factor -ln2 u w to the moments once, after it
                const float iuw = c2.y != 0.0f ? 1.0f / c2.y : 0.0f;
                const float2 ccr = f2(b.z * iuw, b.z * iuw), ccg = f2(b.w * iuw, b.w * iuw);
                const float2 ccb = f2(c2.x * iuw, c2.x * iuw);
                // accumulators, each over the two pixels of a column pair: d/d(c u w) per channel, d/d(u w);
                // and the moments of gq = dL/dq' in the record's own frame (r = qs dy + qw dx, dx):
                // sum gq r^2, sum gq r dx, sum gq dx^2, sum gq r, sum gq dx.  Kept apart, a thin
                // footprint's small along-axis terms (dx) are not rounded away under its large r terms.
                float2 gr = f2(0.f, 0.f), gg = gr, gb = gr, gu = gr;
                float2 srr = f2(0.f, 0.f), srx = srr, sxx = srr, sr = srr, sx = srr;
                // dx of this lane's two column pairs (2 (k + m L), +1) from the row's even first column, less
                // that column
                const float2 gxb = __fadd2_rn(f2((float)(2 * gk), (float)(2 * gk + 1)), gx2);
                for (int st = 0; st < steps; ++st) {
                    const int ly = r0 + st;
                    const unsigned sp = sspan[j][ly];
                    const int xe = (int)(sp & 0xffu);                           // even first column
                    const int pb = ly * PP + (xe >> 1) + gk;
                    const float xsf = (float)xe;
                    const float rb = qs * ((float)ly + gy0);                     // qs dy
                    const float2 xb = __fadd2_rn(f2(xsf, xsf), gxb);             // dx of the lane's first pair
                    const float2 rb2 = f2(rb, rb);
#pragma unroll
                    for (int m = 0; m < M; ++m) {
                        // Columns outside the span evaluate q > 9 (the span holds every pixel centre of the row
                        // with q' <= kQMax, with a margin), so the cutoff test zeroes them; pairs past the tile
                        // read zero pairs.  No per-pixel validity mask is needed.
                        const int pi = pb + m * L;
                        const float4 A = spA[pi], B = spB[pi];          // (x0, x1, y0, y1), (z0, z1, w0, w1)
                        const float2 dx = m == 0 ? xb : __fadd2_rn(xb, f2((float)(2 * m * L), (float)(2 * m * L)));
                        const float2 rr = __ffma2_rn(qw2, dx, rb2);
                        const float2 q = __ffma2_rn(rr, rr, __fmul2_rn(__fmul2_rn(qd2, dx), dx));
                        const float2 e = f2(ex2_approx(q.x <= kQMax ? -q.x : -256.0f),      // 2^-256 flushes to 0
                                            ex2_approx(q.y <= kQMax ? -q.y : -256.0f));
                        // d/d(c u w) and d/d(u w) at fixed c u w
                        gr = __ffma2_rn(f2(A.x, A.y), e, gr);
                        gg = __ffma2_rn(f2(A.z, A.w), e, gg);
                        gb = __ffma2_rn(f2(B.x, B.y), e, gb);
                        gu = __ffma2_rn(f2(B.z, B.w), e, gu);
                        // dL/dq' per pixel, less the factor -ln2 u w: e * (P_w + c . P_rgb)
                        const float2 pc = __ffma2_rn(f2(B.x, B.y), ccb, __ffma2_rn(f2(A.z, A.w), ccg,
                                                     __ffma2_rn(f2(A.x, A.y), ccr, f2(B.z, B.w))));
                        const float2 gq = __fmul2_rn(e, pc);
                        const float2 tr = __fmul2_rn(gq, rr), tx = __fmul2_rn(gq, dx);
                        srr = __ffma2_rn(tr, rr, srr);
                        srx = __ffma2_rn(tr, dx, srx);
                        sxx = __ffma2_rn(tx, dx, sxx);
                        sr = __fadd2_rn(sr, tr);
                        sx = __fadd2_rn(sx, tx);
                    }
                }
                // the group's sums: record order sum gq r, sum gq dx, sum gq r^2, sum gq r dx, sum gq dx^2,
                // d/d(u w), d/d(c u w)
                const float fq = -kLn2 * c2.y;
                float vals[9] = {fq * (sr.x + sr.y), fq * (sx.x + sx.y), fq * (srr.x + srr.y), fq * (srx.x + srx.y),
                                 fq * (sxx.x + sxx.y), gu.x + gu.y, gr.x + gr.y, gg.x + gg.y, gb.x + gb.y};
                __syncwarp();
#pragma unroll
                for (int off = L / 2; off > 0; off >>= 1)
#pragma unroll
                    for (int c = 0; c < 9; ++c) vals[c] += __shfl_xor_sync(0xffffffffu, vals[c], off);
                if (act && gk == 0 && steps > 0) {
                    if (pass == 0) {
                        float4* o = reinterpret_cast<float4*>(grec + (size_t)WSR_GRAD_RECORD_FLOATS * sidx[j]);
                        atomicAdd(o, make_float4(vals[0], vals[1], vals[2], vals[3]));
                        atomicAdd(o + 1, make_float4(vals[4], vals[5], vals[6], vals[7]));
                        atomicAdd(reinterpret_cast<float*>(o + 2), vals[8]);
                    } else {
                        // deterministic mode: a 128-byte record holds 9 int64 sums, then the 9 bounds (float
                        // bits) that fix their units.  A term's bound caps the sum of its absolute pixel
                        // terms over the whole footprint, the same in every tile of the Gaussian: at most
                        // (2 hx + 2)(2 hy + 2) pixels (hx, hy its half-extents), each with e <= 1, every
                        // pixel-table entry at most pmax, |r| <= sqrt(QM), |dx| <= hx inside the cutoff.
                        float* o = grec + (size_t)kDetRecordFloats * sidx[j];
                        int* mag = reinterpret_cast<int*>(o + 18);
                        const float qd = b.x, hx = sqrtf(QM / qd);
                        const float hy = sqrtf(QM * fmaf(a.w, a.w, qd) / (qd * a.z * a.z));
                        const float npx = fminf((2.0f * hx + 2.0f) * (2.0f * hy + 2.0f), 1e12f);
                        const float gqm = pmax * kLn2 * 1.0001f * (fabsf(b.z) + fabsf(b.w) + fabsf(c2.x) + fabsf(b.y));
                        const float sq = sqrtf(QM);
                        const float bound[9] = {npx * gqm * sq, npx * gqm * hx, npx * gqm * QM, npx * gqm * sq * hx,
                                                npx * gqm * hx * hx, npx * pmax, npx * pmax, npx * pmax, npx * pmax};
                        unsigned long long* sum = reinterpret_cast<unsigned long long*>(o);
#pragma unroll
                        for (int c = 0; c < 9; ++c) {
                            const float m = fminf(bound[c], 1e30f);
                            mag[c] = __float_as_int(m);     // every tile of the Gaussian writes the same value
                            if (m > 0.0f) {
                                int e;
                                frexpf(m, &e);              // m < 2^e
                                const long long q = __double2ll_rn(ldexp((double)vals[c], kDetBits - e));
                                atomicAdd(sum + c, (unsigned long long)q);
                            }
                        }
                    }
                }
            }
        };
        walk(Lanes<TW / (2 * M)>(), 0, nwide, &snext[0]);        // the wide class
        walk(Lanes<TW / (4 * M)>(), nwide, cnt, &snext[1]);      // the narrow class
    }
    __syncthreads();
    if (tid < 4) {
        float t = 0.0f;
        for (int w = 0; w < NW; ++w) t += sbg[tid][w];
        if (pass == 0) {
            if (t != 0.0f) atomicAdd(gw + 2 + tid, t);
        } else {
            bg_tiles[4 * (size_t)tile + tid] = t;      // summed in tile order afterwards
        }
    }
}

template <int TW, int TH, int CH>
__global__ void __launch_bounds__(BwdThreads<CH>::value, 1024 / BwdThreads<CH>::value)
    k_render_bwd(const float4* __restrict__ rec, const unsigned* __restrict__ offsets,
                 const unsigned* __restrict__ list, const Views vs, const float* __restrict__ wparams,
                 const float* __restrict__ out_rgb, const float* __restrict__ out_den,
                 const float* __restrict__ grad_rgb, float* __restrict__ grec, float* __restrict__ gw,
                 const int pass, float* __restrict__ bg_tiles, const unsigned* __restrict__ det_pmax,
                 const unsigned* __restrict__ order,
                 unsigned* __restrict__ counter) {
    for_each_tile(order, counter, vs.total_tiles, [&](int tile) {
        bwd_tile<TW, TH, CH>(tile, rec, offsets, list, vs, wparams, out_rgb, out_den, grad_rgb, grec, gw, pass,
                             bg_tiles, det_pmax);
    });
}

// Deterministic mode: the largest magnitude of the backward's pixel terms, G / D per channel and
// (G.C) / D, over all pixels (the same expressions as the backward's pixel table), as float bits
// with an order-independent integer atomicMax.
__global__ void __launch_bounds__(256) k_det_pmax(const float* __restrict__ out_rgb,
                                                  const float* __restrict__ out_den,
                                                  const float* __restrict__ grad_rgb, long long npix,
                                                  unsigned* __restrict__ pmax) {
    float m = 0.0f;
    for (long long pix = (long long)blockIdx.x * blockDim.x + threadIdx.x; pix < npix;
         pix += (long long)gridDim.x * blockDim.x) {
        const float inv = 1.0f / out_den[pix];
        const float G0 = grad_rgb[3 * pix], G1 = grad_rgb[3 * pix + 1], G2 = grad_rgb[3 * pix + 2];
        const float C0 = out_rgb[3 * pix], C1 = out_rgb[3 * pix + 1], C2 = out_rgb[3 * pix + 2];
        m = fmaxf(m, fmaxf(fmaxf(fabsf(G0 * inv), fabsf(G1 * inv)),
                           fmaxf(fabsf(G2 * inv), fabsf(-(G0 * C0 + G1 * C1 + G2 * C2) * inv))));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0 && m > 0.0f) atomicMax(pmax, __float_as_uint(m));
}

// Deterministic mode: the tiles' background terms summed in a fixed order.
__global__ void __launch_bounds__(256) k_det_bg_reduce(const float* __restrict__ bg, int n_tiles,
                                                       float* __restrict__ gw) {
    __shared__ float part[4][256];
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int t = threadIdx.x; t < n_tiles; t += 256)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[c] += bg[4 * (size_t)t + c];
#pragma unroll
    for (int c = 0; c < 4; ++c) part[c][threadIdx.x] = acc[c];
    __syncthreads();
    if (threadIdx.x < 4) {
        float sum = 0.0f;
        for (int k = 0; k < 256; ++k) sum += part[threadIdx.x][k];
        gw[2 + threadIdx.x] = sum;
    }
}

// Grid of a launch: one block per tile, or, persistent, as many blocks as
// fit on the device at once, up to max_warps_per_sm warps per SM.
template <typename K>
unsigned grid_for(K kernel, int threads, const Views& vs, const Sched& sched, int max_warps_per_sm = 64) {
    if (!sched.order) return (unsigned)vs.total_tiles;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0);
    per_sm = min(per_sm, max(1, max_warps_per_sm * 32 / threads));
    return (unsigned)min(max(1, sms * max(per_sm, 1)), vs.total_tiles);
}

// The forward's persistent grid holds 16 warps per SM (8 blocks of 16x16 tiles), not the 28 that its
// registers allow: at 1M Gaussians and 1920x1080 it ran in 0.49 ms at 16 warps against 0.51 at 12,
// 0.55 at 20 and 0.58 at 28.
constexpr int kFwdWarpsPerSM = 16;

template <int TW, int TH, int PX>
cudaError_t fwd_t(const float* rec, const unsigned* off, const unsigned* list, const Views& vs, WeightDev w,
                  float* rgb, float* den, Sched sched, cudaStream_t s) {
    constexpr int NT = FwdShape<TW, TH, PX>::NT;
    const unsigned grid = grid_for(k_render_fwd<TW, TH, PX>, NT, vs, sched, kFwdWarpsPerSM);
    if (sched.order) {
        cudaError_t e = cudaMemsetAsync(sched.counter, 0, sizeof(unsigned), s);
        if (e != cudaSuccess) return e;
    }
    k_render_fwd<TW, TH, PX><<<grid, NT, 0, s>>>(reinterpret_cast<const float4*>(rec), off, list, vs, w.params, rgb,
                                                 den, sched.order, sched.counter);
    return cudaGetLastError();
}

template <int TW, int TH, int CH>
cudaError_t bwd_chunk(const float* rec, const unsigned* off, const unsigned* list, const Views& vs, WeightDev w,
                      const float* rgb, const float* den, const float* grgb, float* grec, float* gw, int pass,
                      float* bg_tiles, const unsigned* det_pmax, Sched sched, cudaStream_t s) {
    constexpr int NT = BwdThreads<CH>::value;
    const unsigned grid = grid_for(k_render_bwd<TW, TH, CH>, NT, vs, sched);
    if (sched.order) {
        cudaError_t e = cudaMemsetAsync(sched.counter, 0, sizeof(unsigned), s);
        if (e != cudaSuccess) return e;
    }
    k_render_bwd<TW, TH, CH><<<grid, NT, 0, s>>>(reinterpret_cast<const float4*>(rec), off, list, vs, w.params,
                                                     rgb, den, grgb, grec, gw, pass, bg_tiles, det_pmax,
                                                     sched.order, sched.counter);
    return cudaGetLastError();
}

template <int TW, int TH>
cudaError_t bwd_t(const float* rec, const unsigned* off, const unsigned* list, const Views& vs, WeightDev w,
                  const float* rgb, const float* den, const float* grgb, float* grec, float* gw, int pass,
                  float* bg_tiles, const unsigned* det_pmax, Sched sched, cudaStream_t s) {
    const int ch = vs.chunk;
    auto k = ch == 64 ? bwd_chunk<TW, TH, 64> : ch == 256 ? bwd_chunk<TW, TH, 256>
                                              : ch == 512 ? bwd_chunk<TW, TH, 512> : bwd_chunk<TW, TH, 128>;
    return k(rec, off, list, vs, w, rgb, den, grgb, grec, gw, pass, bg_tiles, det_pmax, sched, s);
}

// Diagnostic: the work of the render kernels, three counts added to count[0..2]:
//   [0] (pixel, Gaussian) pairs inside the cutoff, i.e. the algorithmic work
//       (q' from each pixel's own dx, dy; the renderers may decide pairs
//       within rounding of the cutoff differently);
//   [1] the (pixel, Gaussian) slots the forward evaluates: for every Gaussian
//       of a tile, the pixels of each warp whose region its footprint reaches
//       (the forward's per-warp test; all the tile's pixel slots with one warp);
//   [2] the backward's pixel slots (per tile instance, the rows from the first
//       to the last with a span, TW columns each, or TW / 2 when no span is
//       longer than TW / 2 pixels), from the backward's own span arithmetic.
template <int TW, int TH, int PPT, int PX>
__global__ void __launch_bounds__(TileShape<TW, TH, PPT>::NT)
    k_count_pairs(const float4* __restrict__ rec, const unsigned* __restrict__ offsets,
                  const unsigned* __restrict__ list, const Views vs, unsigned long long* __restrict__ count) {
    using S = TileShape<TW, TH, PPT>;
    using F = FwdShape<TW, TH, PX>;
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
    const int x_org = tc.tx * TW, y_org = tc.ty * TH;
    const int x_lim = min(TW, V.W - x_org), y_lim = min(TH, V.H - y_org);
    const float QM = kQMax * 1.0001f + 1e-4f;
    unsigned long long cnt_pairs = 0, cnt_fwd = 0, cnt_bwd = 0;
    const unsigned start = offsets[tile], end = offsets[tile + 1];
    for (unsigned base = start; base < end; base += NT) {
        const int cnt = (int)min((unsigned)NT, end - base);
        __syncthreads();
        if (tid < cnt) {
            const float4* p = rec + 3ull * list[base + tid];
            const float4 a = __ldg(p);
            const float qd = __ldg(reinterpret_cast<const float*>(p + 1));
            s0[tid] = a;
            s1[tid] = qd;
            // the forward's slots: 32 threads x PX x 2 pixels per warp whose rows the footprint reaches
            if constexpr (F::NW > 1) {
                const float xl = (float)x_org + 0.5f, xh = xl + (float)(TW - 1);
#pragma unroll
                for (int w = 0; w < F::NW; ++w) {
                    const float yl = (float)(y_org + F::row_lo(w)) + 0.5f;
                    const float yh = (float)(y_org + F::row_hi(w)) + 0.5f;
                    if (footprint_hits(a.x, a.y, a.z, a.w, qd, xl, xh, yl, yh)) cnt_fwd += 32ull * PX * 2;
                }
            } else {
                cnt_fwd += (unsigned long long)F::NT * PX * 2;
            }
            // the backward's pixel slots: the rows from its first span to its last, TW columns each, or
            // TW / 2 when no span is longer than TW / 2 pixels
            const RowSpans rs(a, qd, QM);
            int lo, hi, r_lo = TH, r_hi = -1, umax = 0;
            rs.rows(a, y_org, 0, y_lim, lo, hi);
            for (int r = lo; r <= hi; ++r) {
                const int u = rs.row(a, QM, x_org, y_org, x_lim, r) >> 8;
                if (u) {
                    r_lo = min(r_lo, r);
                    r_hi = max(r_hi, r);
                    umax = max(umax, u);
                }
            }
            if (r_hi >= r_lo) cnt_bwd += (unsigned long long)(r_hi - r_lo + 1) * (2 * umax > TW / 2 ? TW : TW / 2);
        }
        __syncthreads();
        if (x >= V.W) continue;
        for (int j = 0; j < cnt; ++j) {
            const float4 a = s0[j];
            const float dx = px - a.x;
            const float P = s1[j] * dx * dx;
            const float Q = a.w * dx;
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                const float dy = (float)(y0 + k) + 0.5f - a.y;
                const float rr = fmaf(a.z, dy, Q);
                const float q = fmaf(rr, rr, P);
                if (q <= kQMax && y0 + k < V.H) ++cnt_pairs;
            }
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        cnt_pairs += __shfl_xor_sync(0xffffffffu, cnt_pairs, off);
        cnt_fwd += __shfl_xor_sync(0xffffffffu, cnt_fwd, off);
        cnt_bwd += __shfl_xor_sync(0xffffffffu, cnt_bwd, off);
    }
    if ((tid & 31) == 0) {
        if (cnt_pairs) atomicAdd(count, cnt_pairs);
        if (cnt_fwd) atomicAdd(count + 1, cnt_fwd);
        if (cnt_bwd) atomicAdd(count + 2, cnt_bwd);
    }
}

// Mean absolute error and its gradient: float4 loads and stores (the arrays are 16-byte aligned;
// a scalar tail covers count % 4), then a block reduction and one atomic per block.
__global__ void __launch_bounds__(256) k_loss_l1(const float* __restrict__ rgb, const float* __restrict__ target,
                                                 long long count, float* __restrict__ loss,
                                                 float* __restrict__ grad) {
    __shared__ float red[8];
    const float inv = 1.0f / (float)count;
    auto sgn = [&](float d) { return d > 0.0f ? inv : (d < 0.0f ? -inv : 0.0f); };
    float acc = 0.0f;
    const long long n4 = count >> 2;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
        const float4 a = reinterpret_cast<const float4*>(rgb)[i];
        const float4 b = reinterpret_cast<const float4*>(target)[i];
        const float4 d = make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
        acc += (fabsf(d.x) + fabsf(d.y)) + (fabsf(d.z) + fabsf(d.w));
        reinterpret_cast<float4*>(grad)[i] = make_float4(sgn(d.x), sgn(d.y), sgn(d.z), sgn(d.w));
    }
    for (long long i = 4 * n4 + (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
        const float d = rgb[i] - target[i];
        acc += fabsf(d);
        grad[i] = sgn(d);
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        atomicAdd(loss, t * inv);
    }
}

}  // namespace

cudaError_t launch_render_fwd(const float* rec, const unsigned* off, const unsigned* list, const Views& vs,
                              WeightDev w, float* rgb, float* den, Sched sc, cudaStream_t s) {
    if (vs.total_tiles == 0) return cudaSuccess;
    if (vs.tile_w == 16 && vs.tile_h == 16) return fwd_t<16, 16, 2>(rec, off, list, vs, w, rgb, den, sc, s);
    if (vs.tile_w == 8 && vs.tile_h == 8) return fwd_t<8, 8, 1>(rec, off, list, vs, w, rgb, den, sc, s);
    if (vs.tile_w == 32 && vs.tile_h == 8) return fwd_t<32, 8, 2>(rec, off, list, vs, w, rgb, den, sc, s);
    if (vs.tile_w == 16 && vs.tile_h == 8) return fwd_t<16, 8, 2>(rec, off, list, vs, w, rgb, den, sc, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_render_bwd(const float* rec, const unsigned* off, const unsigned* list, const Views& vs,
                              WeightDev w, const float* rgb, const float* den, const float* grgb, float* grec,
                              float* gw, int pass, float* bg_tiles, const unsigned* det_pmax, Sched sc,
                              cudaStream_t s) {
    if (vs.total_tiles == 0) return cudaSuccess;
    if (vs.tile_w == 16 && vs.tile_h == 16)
        return bwd_t<16, 16>(rec, off, list, vs, w, rgb, den, grgb, grec, gw, pass, bg_tiles, det_pmax, sc, s);
    if (vs.tile_w == 8 && vs.tile_h == 8)
        return bwd_t<8, 8>(rec, off, list, vs, w, rgb, den, grgb, grec, gw, pass, bg_tiles, det_pmax, sc, s);
    if (vs.tile_w == 32 && vs.tile_h == 8)
        return bwd_t<32, 8>(rec, off, list, vs, w, rgb, den, grgb, grec, gw, pass, bg_tiles, det_pmax, sc, s);
    if (vs.tile_w == 16 && vs.tile_h == 8)
        return bwd_t<16, 8>(rec, off, list, vs, w, rgb, den, grgb, grec, gw, pass, bg_tiles, det_pmax, sc, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_det_pmax(const float* out_rgb, const float* out_den, const float* grad_rgb, long long npix,
                            unsigned* pmax, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(pmax, 0, sizeof(unsigned), s);
    if (e != cudaSuccess || npix == 0) return e;
    int dev = 0, sms = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const long long blocks = min((npix + 255) / 256, (long long)sms * 8);
    k_det_pmax<<<(unsigned)blocks, 256, 0, s>>>(out_rgb, out_den, grad_rgb, npix, pmax);
    return cudaGetLastError();
}

cudaError_t launch_det_bg_reduce(const float* bg_tiles, int n_tiles, float* gw, cudaStream_t s) {
    k_det_bg_reduce<<<1, 256, 0, s>>>(bg_tiles, n_tiles, gw);
    return cudaGetLastError();
}

cudaError_t launch_count_pairs(const float* rec, const unsigned* off, const unsigned* list, const Views& vs,
                               unsigned long long* count, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(count, 0, 3 * sizeof(unsigned long long), s);
    if (e != cudaSuccess || vs.total_tiles == 0) return e;
    const float4* r = reinterpret_cast<const float4*>(rec);
    // the forward's pixels per thread (PX) as launch_render_fwd picks them
    if (vs.tile_w == 16 && vs.tile_h == 16) k_count_pairs<16, 16, 2, 2><<<vs.total_tiles, 128, 0, s>>>(r, off, list, vs, count);
    else if (vs.tile_w == 8 && vs.tile_h == 8) k_count_pairs<8, 8, 2, 1><<<vs.total_tiles, 32, 0, s>>>(r, off, list, vs, count);
    else if (vs.tile_w == 32 && vs.tile_h == 8) k_count_pairs<32, 8, 2, 2><<<vs.total_tiles, 128, 0, s>>>(r, off, list, vs, count);
    else if (vs.tile_w == 16 && vs.tile_h == 8) k_count_pairs<16, 8, 2, 2><<<vs.total_tiles, 64, 0, s>>>(r, off, list, vs, count);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_loss_l1(const float* rgb, const float* target, long long count, float* loss, float* grad,
                           cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(float), s);
    if (e != cudaSuccess || count == 0) return e;
    int dev = 0, sms = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    long long nb = (count / 4 + 255) / 256;
    const long long cap = 4ll * sms;
    if (nb > cap) nb = cap;
    if (nb < 1) nb = 1;
    k_loss_l1<<<(unsigned)nb, 256, 0, s>>>(rgb, target, count, loss, grad);
    return cudaGetLastError();
}

}  // namespace wsr
