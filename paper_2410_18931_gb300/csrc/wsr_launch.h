// Host-side launch interface between the C ABI (api.cu) and the kernels.
#pragma once

#include <cuda_runtime.h>

#include "wsr_common.cuh"

namespace wsr {

struct GaussPtrs {
    long long n;
    int deg;       // 0..3
    int vd;        // opacity from SH (Eq. 11) instead of a logit
    int red;       // reduced-precision storage (bf16 scales/quats, f16 SH/opacity)
    const float* means;
    const void* log_scales;
    const void* quats;
    const void* sh;
    const void* opacity;
    const float* lc_v;
};

struct WeightDev {
    int kind;
    const float* params;   // device [6]: sigma, beta, w_B, c_B
};

cudaError_t launch_project(const GaussPtrs& g, const Views& vs, WeightDev w, float* records,
                           cudaStream_t s);
// det_sb: nullptr, or (deterministic mode) room for kDetSBBlocks pairs of sigma/beta block sums; the
// records are then WSR_GRAD_RECORD_FLOATS_DET floats of fixed-point sums and their scales
cudaError_t launch_project_bwd(const GaussPtrs& g, const Views& vs, WeightDev w,
                               const float* grad_records, const wsr_grads& out, float* det_sb, cudaStream_t s);

cudaError_t launch_bin_count(const float* records, long long n, const Views& vs,
                             unsigned* cursor, cudaStream_t s);
// the scan of the per-tile counts into offsets (and the scatter's cursors); with `order`, also
// the persistent schedule's longest-first tile order (`buckets`: 66 words of scratch)
cudaError_t launch_scan(const Views& vs, unsigned* cursor, unsigned* block_sums,
                        unsigned* tile_offsets, unsigned long long capacity, WsHeader* hdr,
                        unsigned* buckets, unsigned* order, cudaStream_t s);
cudaError_t launch_bin_scatter(const float* records, long long n, const Views& vs,
                               unsigned* cursor, unsigned* tile_list,
                               unsigned long long capacity, WsHeader* hdr, cudaStream_t s);

// deterministic mode: each tile's list sorted by record index
cudaError_t launch_sort_segments(const Views& vs, const unsigned* tile_offsets, unsigned* tile_list,
                                 WsHeader* hdr, cudaStream_t s);

// Work distribution of a render launch: order == nullptr means one block per
// tile; otherwise a persistent grid takes tiles order[0..total) via *counter
// (reset by the launcher).
struct Sched {
    const unsigned* order;
    unsigned* counter;
};

cudaError_t launch_render_fwd(const float* records, const unsigned* tile_offsets,
                              const unsigned* tile_list, const Views& vs, WeightDev w,
                              float* out_rgb, float* out_den, Sched sched, cudaStream_t s);
// pass 0: float atomics into WSR_GRAD_RECORD_FLOATS records and grad_wparams.  Deterministic mode
// (pass 1, WSR_GRAD_RECORD_FLOATS_DET records): the record terms added as fixed point in units set by
// a per-Gaussian bound from *det_pmax (launch_det_pmax first), each tile's background terms stored in
// bg_tiles[4 tile + c].
cudaError_t launch_render_bwd(const float* records, const unsigned* tile_offsets,
                              const unsigned* tile_list, const Views& vs, WeightDev w,
                              const float* out_rgb, const float* out_den, const float* grad_rgb,
                              float* grad_records, float* grad_wparams, int pass, float* bg_tiles,
                              const unsigned* det_pmax, Sched sched, cudaStream_t s);
// deterministic mode: grad_wparams[2..5] = the tiles' background terms summed in tile order
cudaError_t launch_det_pmax(const float* out_rgb, const float* out_den, const float* grad_rgb, long long npix,
                            unsigned* pmax, cudaStream_t s);
cudaError_t launch_det_bg_reduce(const float* bg_tiles, int n_tiles, float* grad_wparams, cudaStream_t s);

cudaError_t launch_count_pairs(const float* records, const unsigned* tile_offsets, const unsigned* tile_list,
                               const Views& vs, unsigned long long* count, cudaStream_t s);

cudaError_t launch_loss_l1(const float* rgb, const float* target, long long count,
                           float* loss, float* grad, cudaStream_t s);

// Views of the 3DGS loss: tiles of loss_tile_side() square per view, in view
// order; the Gaussian window taps g[] are normalised to sum 1.
struct LossViews {
    int n;
    int tile_off[WSR_MAX_VIEWS + 1];
    int tiles_x[WSR_MAX_VIEWS];
    int w[WSR_MAX_VIEWS];
    int h[WSR_MAX_VIEWS];
    long long pix_off[WSR_MAX_VIEWS];
    float g[11];
    float lam, inv_count, c1, c2;
};

int loss_tile_side();
cudaError_t launch_loss_3dgs(const float* rgb, const float* target, const LossViews& L, float* loss,
                             float* grad, cudaStream_t s);

// Adam groups in float4 units: group k covers units [ubase[k], ubase[k+1])
// and elements [off[k], off[k] + cnt[k]) of the flat buffers.
struct AdamGroups {
    int n;
    long long ubase[WSR_ADAM_MAX_GROUPS + 1];
    long long off[WSR_ADAM_MAX_GROUPS];
    unsigned cnt[WSR_ADAM_MAX_GROUPS];
    float lr[WSR_ADAM_MAX_GROUPS];
    float lr_tail[WSR_ADAM_MAX_GROUPS];
    int period[WSR_ADAM_MAX_GROUPS];
    int head[WSR_ADAM_MAX_GROUPS];
    float b1, omb1, b2, omb2, eps;
};

// Device-resident Adam state (the wsr_adam_state of the C ABI).
struct AdamState {
    int step;
    float c1;      // 1 / (1 - beta1^step)
    float c2;      // 1 / sqrt(1 - beta2^step)
    int skipped;
};
static_assert(sizeof(AdamState) == sizeof(wsr_adam_state), "Adam state layout");

cudaError_t launch_adam(float* p, const float* g, float* m, float* v, const AdamGroups& G, double beta1,
                        double beta2, AdamState* st, const WsHeader* guard, cudaStream_t s);

}  // namespace wsr
