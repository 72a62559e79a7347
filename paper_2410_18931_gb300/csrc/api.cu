// C ABI of the WSR library: argument checks, view table, workspace layout and
// dispatch to the kernels.  Nothing here allocates device memory.
#include <math.h>
#include <string.h>

#include <mutex>

#include "wsr_launch.h"

using namespace wsr;

namespace {

constexpr int32_t kVersion = 1 * 10000 + 0 * 100 + 0;

bool tiles_ok(const wsr_tiles* t) {
    if (!t) return false;
    return (t->tile_w == 16 && t->tile_h == 16) || (t->tile_w == 8 && t->tile_h == 8) ||
           (t->tile_w == 32 && t->tile_h == 8) || (t->tile_w == 16 && t->tile_h == 8);
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }
bool aligned4(const void* p) { return ((uintptr_t)p & 3u) == 0; }
bool aligned8(const void* p) { return ((uintptr_t)p & 7u) == 0; }

// Builds the per-view constant table.  Returns WSR_OK or the argument error.
wsr_status make_views(const wsr_camera* cams, int32_t n_cams, const wsr_tiles* tiles, Views* vs) {
    if (!cams || n_cams < 1 || n_cams > WSR_MAX_VIEWS) return WSR_ERR_INVALID_ARG;
    int tw = 16, th = 16, sched = WSR_SCHEDULE_TILE_BLOCKS, chunk = 128, det = 0;
    if (tiles) {
        if (tiles->chunk < 0) return WSR_ERR_INVALID_ARG;
        if (tiles->deterministic != 0 && tiles->deterministic != 1) return WSR_ERR_INVALID_ARG;
        if (tiles->schedule != WSR_SCHEDULE_TILE_BLOCKS && tiles->schedule != WSR_SCHEDULE_PERSISTENT)
            return WSR_ERR_INVALID_ARG;
        if (!tiles_ok(tiles)) return WSR_ERR_UNSUPPORTED;
        if (tiles->chunk != 0 && tiles->chunk != 64 && tiles->chunk != 128 && tiles->chunk != 256 &&
            tiles->chunk != 512)
            return WSR_ERR_UNSUPPORTED;
        tw = tiles->tile_w;
        th = tiles->tile_h;
        sched = tiles->schedule;
        chunk = tiles->chunk ? tiles->chunk : 128;
        det = tiles->deterministic;
    }
    memset(vs, 0, sizeof(Views));
    vs->n = n_cams;
    vs->tile_w = tw;
    vs->tile_h = th;
    vs->schedule = sched;
    vs->chunk = chunk;
    vs->det = det;
    long long tile_base = 0, pix_base = 0;
    for (int v = 0; v < n_cams; ++v) {
        const wsr_camera& c = cams[v];
        if (c.width <= 0 || c.height <= 0 || c.width > 32768 || c.height > 32768) return WSR_ERR_INVALID_ARG;
        if (!(c.fx > 0.0f) || !(c.fy > 0.0f) || !(c.znear >= 0.0f) || !isfinite(c.cx) || !isfinite(c.cy))
            return WSR_ERR_INVALID_ARG;
        for (int k = 0; k < 9; ++k)
            if (!isfinite(c.R[k])) return WSR_ERR_INVALID_ARG;
        for (int k = 0; k < 3; ++k)
            if (!isfinite(c.T[k])) return WSR_ERR_INVALID_ARG;
        View& V = vs->v[v];
        memcpy(V.R, c.R, sizeof V.R);
        memcpy(V.T, c.T, sizeof V.T);
        V.fx = c.fx; V.fy = c.fy; V.cx = c.cx; V.cy = c.cy; V.znear = c.znear;
        for (int k = 0; k < 3; ++k)
            V.campos[k] = (float)(-((double)c.R[k] * c.T[0] + (double)c.R[3 + k] * c.T[1] +
                                    (double)c.R[6 + k] * c.T[2]));
        V.limx = (float)(1.3 * 0.5 * c.width / (double)c.fx);
        V.limy = (float)(1.3 * 0.5 * c.height / (double)c.fy);
        V.W = c.width;
        V.H = c.height;
        V.tiles_x = (c.width + tw - 1) / tw;
        V.tiles_y = (c.height + th - 1) / th;
        V.tile_base = (int)tile_base;
        V.pix_base = pix_base;
        tile_base += (long long)V.tiles_x * V.tiles_y;
        pix_base += (long long)c.width * c.height;
        if (tile_base > (1ll << 30)) return WSR_ERR_INVALID_ARG;
    }
    vs->total_tiles = (int)tile_base;
    vs->total_pix = pix_base;
    return WSR_OK;
}

struct WsLayout {
    size_t cursor, block_sums, order, buckets, bg_tiles, total;
};

// The tile order of the persistent schedule is only part of its layout.
WsLayout ws_layout(const Views& vs) {
    WsLayout L;
    const size_t nb = (size_t)(vs.total_tiles + kScanTile - 1) / kScanTile;
    L.cursor = kWsHeader;
    L.block_sums = L.cursor + align256(sizeof(unsigned) * ((size_t)vs.total_tiles + 1));
    L.total = L.block_sums + align256(sizeof(unsigned long long) * (nb + 1));
    L.order = L.buckets = L.bg_tiles = 0;
    if (vs.schedule == WSR_SCHEDULE_PERSISTENT) {
        L.order = L.total;
        L.buckets = L.order + align256(sizeof(unsigned) * (size_t)vs.total_tiles);
        L.total = L.buckets + align256(sizeof(unsigned) * 66);
    }
    if (vs.det) {
        L.bg_tiles = L.total;
        L.total = L.bg_tiles + align256(4 * sizeof(float) * (size_t)vs.total_tiles);
    }
    return L;
}

Sched sched_of(const Views& vs, void* workspace, int which) {
    Sched sc{nullptr, nullptr};
    if (vs.schedule == WSR_SCHEDULE_PERSISTENT) {
        const WsLayout L = ws_layout(vs);
        sc.order = (const unsigned*)((char*)workspace + L.order);
        sc.counter = &((WsHeader*)workspace)->work[which];
    }
    return sc;
}

wsr_status check_ws(const Views& vs, void* ws, size_t bytes) {
    if (!ws || !aligned16(ws)) return WSR_ERR_INVALID_ARG;
    if (bytes < ws_layout(vs).total) return WSR_ERR_INVALID_ARG;
    return WSR_OK;
}

wsr_status check_gauss(const wsr_gaussians* g, int32_t n_cams, int wkind, GaussPtrs* out) {
    if (!g || g->n < 0) return WSR_ERR_INVALID_ARG;
    if (g->sh_degree < 0 || g->sh_degree > 3) return WSR_ERR_INVALID_ARG;
    if (g->opacity_mode != WSR_OPACITY_LOGIT && g->opacity_mode != WSR_OPACITY_SH) return WSR_ERR_INVALID_ARG;
    const bool full = g->dtype_scales_quats == WSR_F32 && g->dtype_sh == WSR_F32;
    const bool red = g->dtype_scales_quats == WSR_BF16 && g->dtype_sh == WSR_F16;
    if (!full && !red) {
        const bool known = (g->dtype_scales_quats >= WSR_F32 && g->dtype_scales_quats <= WSR_BF16) &&
                           (g->dtype_sh >= WSR_F32 && g->dtype_sh <= WSR_BF16);
        return known ? WSR_ERR_UNSUPPORTED : WSR_ERR_INVALID_ARG;
    }
    if ((unsigned long long)g->n * (unsigned long long)n_cams > 0xffffffffull) return WSR_ERR_INVALID_ARG;
    if (g->n > 0) {
        if (!g->means || !g->log_scales || !g->quats || !g->sh || !g->opacity) return WSR_ERR_INVALID_ARG;
        if (wkind == WSR_WEIGHT_LC && !g->lc_v) return WSR_ERR_INVALID_ARG;
        if (!aligned16(g->means) || !aligned16(g->log_scales) || !aligned16(g->quats) || !aligned16(g->sh) ||
            !aligned16(g->opacity) || (g->lc_v && !aligned16(g->lc_v)))
            return WSR_ERR_INVALID_ARG;
    }
    out->n = g->n;
    out->deg = g->sh_degree;
    out->vd = g->opacity_mode == WSR_OPACITY_SH;
    out->red = red ? 1 : 0;
    out->means = g->means;
    out->log_scales = g->log_scales;
    out->quats = g->quats;
    out->sh = g->sh;
    out->opacity = g->opacity;
    out->lc_v = g->lc_v;
    return WSR_OK;
}

wsr_status check_weight(const wsr_weight* w, WeightDev* out) {
    if (!w || !w->params) return WSR_ERR_INVALID_ARG;
    if (w->kind < WSR_WEIGHT_DIR || w->kind > WSR_WEIGHT_LC) return WSR_ERR_INVALID_ARG;
    out->kind = w->kind;
    out->params = w->params;
    return WSR_OK;
}

wsr_status cuda_status(cudaError_t e) { return e == cudaSuccess ? WSR_OK : WSR_ERR_CUDA; }

#define WSR_TRY(expr)                         \
    do {                                      \
        const wsr_status st_ = (expr);        \
        if (st_ != WSR_OK) return st_;        \
    } while (0)
#define WSR_CUDA(expr)                                        \
    do {                                                      \
        const cudaError_t ce_ = (expr);                       \
        if (ce_ != cudaSuccess) return WSR_ERR_CUDA;          \
    } while (0)

// ---------------------------------------------------------------------------
// Fixed scratch for wsr_bin_static: the same layout as a workspace sized for
// WSR_BIN_STATIC_MAX_TILES tiles, in one device array of the library.
// ---------------------------------------------------------------------------
constexpr size_t align256c(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kStaticTiles = WSR_BIN_STATIC_MAX_TILES;
constexpr size_t kStaticBytes = kWsHeader + align256c(sizeof(unsigned) * (kStaticTiles + 1)) +
                                align256c(sizeof(unsigned long long) * ((kStaticTiles + kScanTile - 1) / kScanTile + 1));

static_assert(kStaticBytes == WSR_BIN_STATIC_BYTES, "the header states the scratch array's size");

static __device__ __align__(256) unsigned char g_bin_static_scratch[kStaticBytes];

constexpr int kMaxDevices = 128;
std::mutex g_static_mu;
void* g_static_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (host code cannot
// use the symbol itself as a device address).  Looked up afresh on every call
// outside stream capture, so that a device reset in between leaves no stale
// address behind; inside a capture the last address found on the device is
// reused (the lookup is not made while a stream captures).
wsr_status static_scratch(cudaStream_t s, void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return WSR_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return WSR_ERR_UNSUPPORTED;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return WSR_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (cs == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_bin_static_scratch) != cudaSuccess || !p) return WSR_ERR_CUDA;
        g_static_addr[dev] = p;
    } else if (!g_static_addr[dev]) {
        return WSR_ERR_UNSUPPORTED;
    }
    *out = g_static_addr[dev];
    return WSR_OK;
}

}  // namespace

extern "C" {

const char* wsr_status_string(wsr_status s) {
    switch (s) {
        case WSR_OK: return "ok";
        case WSR_ERR_INVALID_ARG: return "invalid argument";
        case WSR_ERR_CAPACITY: return "tile list capacity exceeded";
        case WSR_ERR_CUDA: return "CUDA error";
        case WSR_ERR_TIMEOUT: return "timeout";
        case WSR_ERR_UNSUPPORTED: return "unsupported configuration";
    }
    return "unknown status";
}

int32_t wsr_version(void) { return kVersion; }

int64_t wsr_num_tiles(const wsr_camera* cams, int32_t n_cams, const wsr_tiles* tiles) {
    static thread_local Views vs;
    if (!tiles || make_views(cams, n_cams, tiles, &vs) != WSR_OK) return 0;
    return vs.total_tiles;
}

int64_t wsr_num_pixels(const wsr_camera* cams, int32_t n_cams) {
    static thread_local Views vs;
    if (make_views(cams, n_cams, nullptr, &vs) != WSR_OK) return 0;
    return vs.total_pix;
}

size_t wsr_workspace_size(const wsr_camera* cams, int32_t n_cams, const wsr_tiles* tiles) {
    static thread_local Views vs;
    if (!tiles || make_views(cams, n_cams, tiles, &vs) != WSR_OK) return 0;
    return ws_layout(vs).total;
}

wsr_status wsr_project(const wsr_gaussians* g, const wsr_camera* cams, int32_t n_cams, const wsr_weight* w,
                       float* records, void* stream) {
    static thread_local Views vs;
    WeightDev wd;
    GaussPtrs gp;
    WSR_TRY(check_weight(w, &wd));
    WSR_TRY(make_views(cams, n_cams, nullptr, &vs));
    WSR_TRY(check_gauss(g, n_cams, wd.kind, &gp));
    if (gp.n > 0 && (!records || !aligned16(records))) return WSR_ERR_INVALID_ARG;
    return cuda_status(launch_project(gp, vs, wd, records, (cudaStream_t)stream));
}

static wsr_status bin_count_impl(const float* records, int64_t n, const Views& vs, uint32_t* tile_offsets,
                                 unsigned long long capacity, void* workspace, cudaStream_t s) {
    const WsLayout L = ws_layout(vs);
    char* ws = (char*)workspace;
    WsHeader* hdr = (WsHeader*)ws;
    unsigned* cursor = (unsigned*)(ws + L.cursor);
    unsigned* bsum = (unsigned*)(ws + L.block_sums);
    WSR_CUDA(cudaMemsetAsync(&hdr->err, 0, sizeof(int), s));
    WSR_CUDA(launch_bin_count(records, n, vs, cursor, s));
    const bool persistent = vs.schedule == WSR_SCHEDULE_PERSISTENT;
    WSR_CUDA(launch_scan(vs, cursor, bsum, tile_offsets, capacity, hdr, (unsigned*)(ws + L.buckets),
                         persistent ? (unsigned*)(ws + L.order) : nullptr, s));
    return WSR_OK;
}

wsr_status wsr_bin_count(const float* records, int64_t n, const wsr_camera* cams, int32_t n_cams,
                         const wsr_tiles* tiles, uint32_t* tile_offsets, void* workspace, size_t workspace_bytes,
                         void* stream) {
    static thread_local Views vs;
    if (!tiles) return WSR_ERR_INVALID_ARG;
    WSR_TRY(make_views(cams, n_cams, tiles, &vs));
    WSR_TRY(check_ws(vs, workspace, workspace_bytes));
    if (n < 0 || (n > 0 && (!records || !aligned16(records))) || !tile_offsets) return WSR_ERR_INVALID_ARG;
    if (!aligned4(tile_offsets)) return WSR_ERR_INVALID_ARG;
    if ((unsigned long long)n * (unsigned long long)n_cams > 0xffffffffull) return WSR_ERR_INVALID_ARG;
    return bin_count_impl(records, n, vs, tile_offsets, ~0ull, workspace, (cudaStream_t)stream);
}

wsr_status wsr_bin(const float* records, int64_t n, const wsr_camera* cams, int32_t n_cams, const wsr_tiles* tiles,
                   uint32_t* tile_offsets, uint32_t* tile_list, uint64_t list_capacity, uint64_t* total_dev,
                   void* workspace, size_t workspace_bytes, void* stream) {
    static thread_local Views vs;
    if (!tiles) return WSR_ERR_INVALID_ARG;
    WSR_TRY(make_views(cams, n_cams, tiles, &vs));
    WSR_TRY(check_ws(vs, workspace, workspace_bytes));
    if (n < 0 || (n > 0 && (!records || !aligned16(records))) || !tile_offsets) return WSR_ERR_INVALID_ARG;
    if (list_capacity > 0 && !tile_list) return WSR_ERR_INVALID_ARG;
    if (!aligned4(tile_offsets) || !aligned4(tile_list) || !aligned8(total_dev)) return WSR_ERR_INVALID_ARG;
    if ((unsigned long long)n * (unsigned long long)n_cams > 0xffffffffull) return WSR_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    WSR_TRY(bin_count_impl(records, n, vs, tile_offsets, list_capacity, workspace, s));
    const WsLayout L = ws_layout(vs);
    char* ws = (char*)workspace;
    WSR_CUDA(launch_bin_scatter(records, n, vs, (unsigned*)(ws + L.cursor), tile_list, list_capacity,
                                (WsHeader*)ws, s));
    if (vs.det) WSR_CUDA(launch_sort_segments(vs, tile_offsets, tile_list, (WsHeader*)ws, s));
    if (total_dev)
        WSR_CUDA(cudaMemcpyAsync(total_dev, &((WsHeader*)ws)->total, sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
    return WSR_OK;
}

wsr_status wsr_bin_static(const float* records, int64_t n, const wsr_camera* cams, int32_t n_cams,
                          const wsr_tiles* tiles, uint32_t* tile_offsets, uint32_t* tile_list, uint64_t list_capacity,
                          uint64_t* total_dev, int32_t* status_dev, void* stream) {
    static thread_local Views vs;
    if (!tiles) return WSR_ERR_INVALID_ARG;
    WSR_TRY(make_views(cams, n_cams, tiles, &vs));
    if ((size_t)vs.total_tiles > kStaticTiles) return WSR_ERR_UNSUPPORTED;
    if (vs.schedule != WSR_SCHEDULE_TILE_BLOCKS) return WSR_ERR_UNSUPPORTED;
    if (n < 0 || (n > 0 && (!records || !aligned16(records))) || !tile_offsets) return WSR_ERR_INVALID_ARG;
    if (list_capacity > 0 && !tile_list) return WSR_ERR_INVALID_ARG;
    if (!aligned4(tile_offsets) || !aligned4(tile_list) || !aligned8(total_dev) || !aligned4(status_dev))
        return WSR_ERR_INVALID_ARG;
    if ((unsigned long long)n * (unsigned long long)n_cams > 0xffffffffull) return WSR_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    void* scratch = nullptr;
    WSR_TRY(static_scratch(s, &scratch));
    Views vb = vs;                 // the binning's part of the layout (no backward regions)
    vb.det = 0;
    if (ws_layout(vb).total > kStaticBytes) return WSR_ERR_UNSUPPORTED;
    WSR_TRY(bin_count_impl(records, n, vs, tile_offsets, list_capacity, scratch, s));
    const WsLayout L = ws_layout(vs);
    char* ws = (char*)scratch;
    WSR_CUDA(launch_bin_scatter(records, n, vs, (unsigned*)(ws + L.cursor), tile_list, list_capacity,
                                (WsHeader*)ws, s));
    if (vs.det) WSR_CUDA(launch_sort_segments(vs, tile_offsets, tile_list, (WsHeader*)ws, s));
    if (total_dev)
        WSR_CUDA(cudaMemcpyAsync(total_dev, &((WsHeader*)ws)->total, sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
    if (status_dev)
        WSR_CUDA(cudaMemcpyAsync(status_dev, &((WsHeader*)ws)->err, sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    return WSR_OK;
}

wsr_status wsr_bin_total(const void* workspace, size_t workspace_bytes, uint64_t* total, void* stream) {
    if (!workspace || workspace_bytes < kWsHeader || !total) return WSR_ERR_INVALID_ARG;
    unsigned long long t = 0;
    cudaStream_t s = (cudaStream_t)stream;
    WSR_CUDA(cudaMemcpyAsync(&t, &((const WsHeader*)workspace)->total, sizeof t, cudaMemcpyDeviceToHost, s));
    WSR_CUDA(cudaStreamSynchronize(s));
    *total = t;
    return WSR_OK;
}

wsr_status wsr_render_fwd(const float* records, int64_t n, const uint32_t* tile_offsets, const uint32_t* tile_list,
                          const wsr_camera* cams, int32_t n_cams, const wsr_tiles* tiles, const wsr_weight* w,
                          float* out_rgb, float* out_den, void* workspace, size_t workspace_bytes, void* stream) {
    static thread_local Views vs;
    WeightDev wd;
    if (!tiles) return WSR_ERR_INVALID_ARG;
    WSR_TRY(check_weight(w, &wd));
    WSR_TRY(make_views(cams, n_cams, tiles, &vs));
    WSR_TRY(check_ws(vs, workspace, workspace_bytes));
    if (n < 0 || !tile_offsets || !out_rgb || !out_den) return WSR_ERR_INVALID_ARG;
    if (n > 0 && (!records || !tile_list)) return WSR_ERR_INVALID_ARG;
    // the records are read as float4; every other array as 32-bit words
    if (!aligned16(records) || !aligned4(tile_list) || !aligned4(tile_offsets) || !aligned4(out_rgb) ||
        !aligned4(out_den))
        return WSR_ERR_INVALID_ARG;
    return cuda_status(launch_render_fwd(records, tile_offsets, tile_list, vs, wd, out_rgb, out_den,
                                         sched_of(vs, workspace, 0), (cudaStream_t)stream));
}

wsr_status wsr_render_bwd_tiles(const float* records, int64_t n, const uint32_t* tile_offsets,
                                const uint32_t* tile_list, const wsr_camera* cams, int32_t n_cams,
                                const wsr_tiles* tiles, const wsr_weight* w, const float* out_rgb,
                                const float* out_den, const float* grad_rgb, float* grad_records, void* workspace,
                                size_t workspace_bytes, void* stream) {
    static thread_local Views vs;
    WeightDev wd;
    if (!tiles) return WSR_ERR_INVALID_ARG;
    WSR_TRY(check_weight(w, &wd));
    WSR_TRY(make_views(cams, n_cams, tiles, &vs));
    WSR_TRY(check_ws(vs, workspace, workspace_bytes));
    if (n < 0 || !tile_offsets || !out_rgb || !out_den || !grad_rgb) return WSR_ERR_INVALID_ARG;
    if (n > 0 && (!records || !tile_list || !grad_records)) return WSR_ERR_INVALID_ARG;
    // records are read and gradient records added to as float4 (as 64-bit integers in the deterministic mode)
    if (!aligned16(records) || !aligned16(grad_records) || !aligned4(tile_list) || !aligned4(tile_offsets) ||
        !aligned4(out_rgb) || !aligned4(out_den) || !aligned4(grad_rgb))
        return WSR_ERR_INVALID_ARG;
    if ((unsigned long long)n * (unsigned long long)n_cams > 0xffffffffull) return WSR_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    WsHeader* hdr = (WsHeader*)workspace;
    WSR_CUDA(cudaMemsetAsync(hdr->gw, 0, sizeof hdr->gw, s));
    const size_t rec_floats = vs.det ? WSR_GRAD_RECORD_FLOATS_DET : WSR_GRAD_RECORD_FLOATS;
    if (n > 0) WSR_CUDA(cudaMemsetAsync(grad_records, 0, sizeof(float) * rec_floats * (size_t)n * n_cams, s));
    if (!vs.det) {
        WSR_CUDA(launch_render_bwd(records, tile_offsets, tile_list, vs, wd, out_rgb, out_den, grad_rgb, grad_records,
                                   hdr->gw, 0, nullptr, nullptr, sched_of(vs, workspace, 1), s));
        return WSR_OK;
    }
    // deterministic: the largest pixel term over the image, then the record terms as exact fixed-point sums
    // in units that a per-Gaussian bound fixes; the background terms per tile, then summed in tile order
    float* bg_tiles = (float*)((char*)workspace + ws_layout(vs).bg_tiles);
    WSR_CUDA(launch_det_pmax(out_rgb, out_den, grad_rgb, vs.total_pix, &hdr->det_pmax, s));
    WSR_CUDA(launch_render_bwd(records, tile_offsets, tile_list, vs, wd, out_rgb, out_den, grad_rgb, grad_records,
                               hdr->gw, 1, bg_tiles, &hdr->det_pmax, sched_of(vs, workspace, 1), s));
    WSR_CUDA(launch_det_bg_reduce(bg_tiles, vs.total_tiles, hdr->gw, s));
    return WSR_OK;
}

wsr_status wsr_project_bwd(const wsr_gaussians* g, const wsr_camera* cams, int32_t n_cams, const wsr_tiles* tiles,
                           const wsr_weight* w, const float* grad_records, const wsr_grads* grads, void* workspace,
                           size_t workspace_bytes, void* stream) {
    static thread_local Views vs;
    WeightDev wd;
    GaussPtrs gp;
    if (!grads || !workspace || workspace_bytes < kWsHeader || !aligned16(workspace)) return WSR_ERR_INVALID_ARG;
    if (tiles && tiles->deterministic != 0 && tiles->deterministic != 1) return WSR_ERR_INVALID_ARG;
    const bool det = tiles && tiles->deterministic == 1;
    WSR_TRY(check_weight(w, &wd));
    WSR_TRY(make_views(cams, n_cams, nullptr, &vs));
    WSR_TRY(check_gauss(g, n_cams, wd.kind, &gp));
    if (gp.n > 0 && (!grad_records || !aligned16(grad_records))) return WSR_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    WsHeader* hdr = (WsHeader*)workspace;
    wsr_grads inner = *grads;
    inner.weight_params = hdr->gw;
    float* sb = det ? (float*)((char*)workspace + kWsDetSB) : nullptr;   // sigma/beta per block
    WSR_CUDA(launch_project_bwd(gp, vs, wd, grad_records, inner, sb, s));
    if (grads->weight_params)
        WSR_CUDA(cudaMemcpyAsync(grads->weight_params, hdr->gw, 6 * sizeof(float), cudaMemcpyDeviceToDevice, s));
    return WSR_OK;
}

wsr_status wsr_render_bwd(const wsr_gaussians* g, const float* records, const uint32_t* tile_offsets,
                          const uint32_t* tile_list, const wsr_camera* cams, int32_t n_cams, const wsr_tiles* tiles,
                          const wsr_weight* w, const float* out_rgb, const float* out_den, const float* grad_rgb,
                          float* grad_records, const wsr_grads* grads, void* workspace, size_t workspace_bytes,
                          void* stream) {
    if (!g || !grads) return WSR_ERR_INVALID_ARG;
    {
        // validate the scene before enqueuing anything
        static thread_local Views vs;
        WeightDev wd;
        GaussPtrs gp;
        WSR_TRY(check_weight(w, &wd));
        WSR_TRY(make_views(cams, n_cams, tiles, &vs));
        WSR_TRY(check_gauss(g, n_cams, wd.kind, &gp));
    }
    WSR_TRY(wsr_render_bwd_tiles(records, g->n, tile_offsets, tile_list, cams, n_cams, tiles, w, out_rgb, out_den,
                                 grad_rgb, grad_records, workspace, workspace_bytes, stream));
    return wsr_project_bwd(g, cams, n_cams, tiles, w, grad_records, grads, workspace, workspace_bytes, stream);
}

wsr_status wsr_count_pairs(const float* records, int64_t n, const uint32_t* tile_offsets, const uint32_t* tile_list,
                           const wsr_camera* cams, int32_t n_cams, const wsr_tiles* tiles, uint64_t* count_dev,
                           void* stream) {
    static thread_local Views vs;
    if (!tiles || !count_dev || !tile_offsets || n < 0) return WSR_ERR_INVALID_ARG;
    if (n > 0 && (!records || !tile_list)) return WSR_ERR_INVALID_ARG;
    if (!aligned16(records) || !aligned4(tile_list) || !aligned4(tile_offsets) || ((uintptr_t)count_dev & 7u))
        return WSR_ERR_INVALID_ARG;
    WSR_TRY(make_views(cams, n_cams, tiles, &vs));
    return cuda_status(launch_count_pairs(records, tile_offsets, tile_list, vs, (unsigned long long*)count_dev,
                                          (cudaStream_t)stream));
}

wsr_status wsr_loss_l1(const float* rgb, const float* target, int64_t count, float* loss_out, float* grad_rgb,
                       void* stream) {
    if (count < 0 || !loss_out || (count > 0 && (!rgb || !target || !grad_rgb))) return WSR_ERR_INVALID_ARG;
    if (count > 0 && (!aligned16(rgb) || !aligned16(target) || !aligned16(grad_rgb))) return WSR_ERR_INVALID_ARG;
    return cuda_status(launch_loss_l1(rgb, target, count, loss_out, grad_rgb, (cudaStream_t)stream));
}

wsr_status wsr_loss_3dgs(const float* rgb, const float* target, const wsr_camera* cams, int32_t n_cams,
                         float lambda, float* loss_out, float* grad_rgb, void* stream) {
    if (!cams || n_cams < 1 || n_cams > WSR_MAX_VIEWS || !loss_out || !rgb || !target || !grad_rgb)
        return WSR_ERR_INVALID_ARG;
    if (!(lambda >= 0.0f && lambda <= 1.0f)) return WSR_ERR_INVALID_ARG;
    static thread_local LossViews L;
    memset(&L, 0, sizeof L);
    const int side = loss_tile_side();
    long long tiles = 0, pix = 0;
    L.n = n_cams;
    for (int v = 0; v < n_cams; ++v) {
        const int W = cams[v].width, H = cams[v].height;
        if (W <= 0 || H <= 0 || W > 32768 || H > 32768) return WSR_ERR_INVALID_ARG;
        L.w[v] = W;
        L.h[v] = H;
        L.tiles_x[v] = (W + side - 1) / side;
        L.tile_off[v] = (int)tiles;
        L.pix_off[v] = pix;
        tiles += (long long)L.tiles_x[v] * ((H + side - 1) / side);
        pix += (long long)W * H;
        if (tiles > (1ll << 30)) return WSR_ERR_INVALID_ARG;
    }
    L.tile_off[n_cams] = (int)tiles;
    // the normalised 11-tap Gaussian of standard deviation 1.5
    double g[11], sum = 0.0;
    for (int k = 0; k < 11; ++k) sum += (g[k] = exp(-(double)((k - 5) * (k - 5)) / (2.0 * 1.5 * 1.5)));
    for (int k = 0; k < 11; ++k) L.g[k] = (float)(g[k] / sum);
    L.lam = lambda;
    L.inv_count = (float)(1.0 / (3.0 * (double)pix));
    L.c1 = 0.01f * 0.01f;
    L.c2 = 0.03f * 0.03f;
    return cuda_status(launch_loss_3dgs(rgb, target, L, loss_out, grad_rgb, (cudaStream_t)stream));
}

wsr_status wsr_adam_step(float* params, const float* grads, float* exp_avg, float* exp_avg_sq,
                         const wsr_adam_group* groups, int32_t n_groups, const wsr_adam_hparams* hp,
                         wsr_adam_state* state, const void* guard_workspace, size_t guard_bytes, void* stream) {
    if (!params || !grads || !exp_avg || !exp_avg_sq || !hp || !state) return WSR_ERR_INVALID_ARG;
    if (!aligned16(params) || !aligned16(grads) || !aligned16(exp_avg) || !aligned16(exp_avg_sq) ||
        ((uintptr_t)state & 3u))
        return WSR_ERR_INVALID_ARG;
    if (n_groups < 0 || n_groups > WSR_ADAM_MAX_GROUPS || (n_groups > 0 && !groups)) return WSR_ERR_INVALID_ARG;
    if (!(hp->beta1 >= 0.0 && hp->beta1 < 1.0) || !(hp->beta2 >= 0.0 && hp->beta2 < 1.0) || !(hp->eps >= 0.0))
        return WSR_ERR_INVALID_ARG;
    if (guard_workspace && (guard_bytes < kWsHeader || !aligned16(guard_workspace))) return WSR_ERR_INVALID_ARG;
    static thread_local AdamGroups G;
    memset(&G, 0, sizeof G);
    G.n = n_groups;
    long long units = 0;
    for (int k = 0; k < n_groups; ++k) {
        const wsr_adam_group& q = groups[k];
        if (q.offset < 0 || (q.offset & 3) || q.count < 0 || q.count >= (1ll << 32)) return WSR_ERR_INVALID_ARG;
        if (q.period < 0 || (q.period > 0 && (q.head < 0 || q.head > q.period))) return WSR_ERR_INVALID_ARG;
        if (!isfinite(q.lr) || !isfinite(q.lr_tail)) return WSR_ERR_INVALID_ARG;
        for (int j = 0; j < k; ++j) {
            const wsr_adam_group& o = groups[j];
            if (q.offset < o.offset + o.count && o.offset < q.offset + q.count) return WSR_ERR_INVALID_ARG;
        }
        G.ubase[k] = units;
        G.off[k] = q.offset;
        G.cnt[k] = (unsigned)q.count;
        G.lr[k] = q.lr;
        G.lr_tail[k] = q.lr_tail;
        G.period[k] = q.period;
        G.head[k] = q.head;
        units += (q.count + 3) / 4;
    }
    G.ubase[n_groups] = units;
    G.b1 = (float)hp->beta1;
    G.omb1 = (float)(1.0 - hp->beta1);
    G.b2 = (float)hp->beta2;
    G.omb2 = (float)(1.0 - hp->beta2);
    G.eps = (float)hp->eps;
    return cuda_status(launch_adam(params, grads, exp_avg, exp_avg_sq, G, hp->beta1, hp->beta2,
                                   reinterpret_cast<AdamState*>(state),
                                   reinterpret_cast<const WsHeader*>(guard_workspace), (cudaStream_t)stream));
}

wsr_status wsr_check(void* workspace, size_t workspace_bytes, void* stream) {
    if (!workspace || workspace_bytes < kWsHeader) return WSR_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int err = 0;
    WSR_CUDA(cudaMemcpyAsync(&err, workspace, sizeof err, cudaMemcpyDeviceToHost, s));
    WSR_CUDA(cudaStreamSynchronize(s));
    if (err != 0) WSR_CUDA(cudaMemsetAsync(workspace, 0, sizeof(int), s));
    return (wsr_status)err;
}

}  // extern "C"
