// gs_api.cu -- host side of the C-ABI: plans, workspace layout, argument
// checks, counters.  The kernels live in the other translation units.
#include <string.h>

#include <atomic>

#include "gs_internal.cuh"

using namespace gs;

int gs::sm_count() {
    constexpr int kDevices = 64;
    static std::atomic<int> cache[kDevices];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 0;
    if (dev < kDevices) {
        const int c = cache[dev].load(std::memory_order_relaxed);
        if (c > 0) return c;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    if (dev < kDevices && sms > 0) cache[dev].store(sms, std::memory_order_relaxed);
    return sms > 0 ? sms : 0;
}

namespace {

int ilog2_exact(int x) {
    int l = 0;
    while ((1 << l) < x) ++l;
    return (1 << l) == x ? l : -1;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

bool plan_ok(const gs_plan* plan) { return plan && P(plan)->magic == kPlanMagic; }

}  // namespace

extern "C" gs_status gs_plan_init(gs_plan* plan, const gs_config* cfg, int32_t n_views,
                                  const gs_view* views_host, int32_t n_capacity,
                                  int64_t instance_capacity) {
    if (!plan || !cfg || !views_host) return GS_ERR_INVALID;
    if (n_views < 1 || n_views > GS_MAX_VIEWS || n_capacity < 1) return GS_ERR_INVALID;
    if (instance_capacity < 1 || instance_capacity > (int64_t(1) << 31)) return GS_ERR_INVALID;
    const int l2w = ilog2_exact(cfg->tile_w), l2h = ilog2_exact(cfg->tile_h);
    if (l2w < 0 || l2h < 0 || cfg->tile_w * cfg->tile_h < 64 || cfg->tile_w * cfg->tile_h > 256)
        return GS_ERR_UNSUPPORTED;
    auto batch_ok = [](int b) { return b >= 32 && b <= 256 && b % 32 == 0; };
    auto ppt_ok = [&](int q) {
        return (q == 1 || q == 2 || q == 4 || q == 8) && cfg->tile_w % q == 0 &&
               (cfg->tile_w * cfg->tile_h / q) % 32 == 0;
    };
    if (!batch_ok(cfg->smem_batch)) return GS_ERR_UNSUPPORTED;
    int ppt = cfg->pixels_per_thread;
    if (ppt == 0) ppt = 1;
    if (!ppt_ok(ppt)) return GS_ERR_UNSUPPORTED;
    const int batch_bwd = cfg->smem_batch_bwd ? cfg->smem_batch_bwd : cfg->smem_batch;
    const int ppt_bwd = cfg->pixels_per_thread_bwd ? cfg->pixels_per_thread_bwd : ppt;
    if (!batch_ok(batch_bwd) || !ppt_ok(ppt_bwd)) return GS_ERR_UNSUPPORTED;
    if (cfg->deterministic && cfg->tile_w * cfg->tile_h / ppt_bwd != 32) return GS_ERR_UNSUPPORTED;
    if (!(cfg->near_z > 0.0f)) return GS_ERR_INVALID;
    if ((int64_t)n_views * n_capacity > (int64_t(1) << 31)) return GS_ERR_INVALID;

    memset(plan, 0, sizeof(*plan));
    Plan* p = reinterpret_cast<Plan*>(plan);
    p->cfg = *cfg;
    p->cfg.pixels_per_thread = ppt;
    p->cfg.smem_batch_bwd = batch_bwd;
    p->cfg.pixels_per_thread_bwd = ppt_bwd;
    p->n_capacity = n_capacity;
    p->inst_capacity = instance_capacity;
    p->vt.n_views = n_views;
    p->vt.tile_w = cfg->tile_w;
    p->vt.tile_h = cfg->tile_h;
    p->vt.log2_tw = l2w;
    p->vt.log2_th = l2h;
    p->vt.tight_rect = cfg->tight_rect != 0;
    if (cfg->recompute < 0) return GS_ERR_INVALID;
    p->recompute = cfg->recompute;
    p->n_views_full = n_views;
    p->view_index = -1;
    // views per pass: all of them, or at most `recompute` in a recompute plan
    p->ws_views = (p->recompute && p->recompute < n_views) ? p->recompute : n_views;
    int64_t tiles = 0, pixels = 0, values = 0, max_pass_tiles = 0, pass_tiles = 0;
    for (int v = 0; v < n_views; ++v) {
        const gs_view& vw = views_host[v];
        if (vw.width < 1 || vw.height < 1 || vw.width > 16384 || vw.height > 16384)
            return GS_ERR_INVALID;
        if (vw.channels != 1 && vw.channels != 3) return GS_ERR_INVALID;
        ViewGeom& g = p->vt.v[v];
        g.width = vw.width;
        g.height = vw.height;
        g.channels = vw.channels;
        g.tiles_x = (vw.width + cfg->tile_w - 1) / cfg->tile_w;
        g.tiles_y = (vw.height + cfg->tile_h - 1) / cfg->tile_h;
        g.tile_offset = (int32_t)tiles;
        g.pixel_offset = pixels;
        g.value_offset = values;
        tiles += (int64_t)g.tiles_x * g.tiles_y;
        if (v % p->ws_views == 0) pass_tiles = 0;  // the first view of a pass
        pass_tiles += (int64_t)g.tiles_x * g.tiles_y;
        if (pass_tiles > max_pass_tiles) max_pass_tiles = pass_tiles;
        pixels += (int64_t)vw.width * vw.height;
        values += (int64_t)vw.width * vw.height * vw.channels;
    }
    if (tiles > (int64_t(1) << 24)) return GS_ERR_UNSUPPORTED;
    p->total_tiles = (int32_t)tiles;
    p->total_pixels = pixels;
    p->total_values = values;
    // tiles binned per call: all views', or one pass's in a recompute plan
    const int64_t bin_tiles = max_pass_tiles;
    int bits = 0;
    while ((int64_t(1) << bits) < bin_tiles) ++bits;
    p->tile_bits = bits < 1 ? 1 : bits;
    p->tile_passes = (p->tile_bits + kRadixBits - 1) / kRadixBits;

    // (view, Gaussian) pairs the workspace holds: all views', or one view's
    // in a recompute plan (views then go through it one pass at a time)
    const int64_t VN = (int64_t)p->ws_views * n_capacity;
    p->depth_sort_blocks = (int32_t)((VN + kSortTile - 1) / kSortTile);
    p->inst_sort_blocks = (int32_t)((instance_capacity + kSortTile - 1) / kSortTile);
    p->scan_blocks = (int32_t)((VN + kScanTile - 1) / kScanTile);
    // loss: 32x16 output tiles per channel plane
    int64_t lb = 0;
    for (int v = 0; v < n_views; ++v) {
        ViewGeom& g = p->vt.v[v];
        g.loss_block_offset = (int32_t)lb;
        lb += (int64_t)((g.width + kLossTileW - 1) / kLossTileW) *
              ((g.height + kLossTileH - 1) / kLossTileH) * g.channels;
    }
    p->loss_blocks = (int32_t)lb;

    size_t len[B_TOTAL] = {0};
    len[GS_BUF_COUNTERS] = 256;
    len[GS_BUF_PROJ] = (size_t)VN * kProjFloats * sizeof(float);
    len[GS_BUF_RECT] = (size_t)VN * 4 * sizeof(uint16_t);
    len[GS_BUF_TOUCHED] = (size_t)VN * sizeof(uint32_t);
    len[GS_BUF_RADIUS] = (size_t)VN * sizeof(int32_t);
    len[GS_BUF_DEPTH_ORDER] = (size_t)VN * sizeof(uint32_t);
    len[GS_BUF_TILE_KEYS] = (size_t)instance_capacity * sizeof(uint32_t);
    len[GS_BUF_TILE_VALUES] = (size_t)instance_capacity * sizeof(uint32_t);
    len[GS_BUF_RANGES] = (size_t)bin_tiles * 2 * sizeof(uint32_t);
    len[GS_BUF_GRAD2D] = (size_t)VN * kGrad2d * sizeof(float);
    len[GS_BUF_ABSGRAD] = cfg->density_stats ? (size_t)VN * 2 * sizeof(float) : 0;
    len[B_DKEY_A] = (size_t)VN * sizeof(uint32_t);
    len[B_DKEY_B] = (size_t)VN * sizeof(uint32_t);
    len[B_DVAL_B] = (size_t)VN * sizeof(uint32_t);
    len[B_DKEY_C] = (size_t)VN * sizeof(uint32_t);
    len[B_SCAN_BLOCKS] = (size_t)(p->scan_blocks + 1) * sizeof(uint32_t) * 2;
    {
        int mb = p->depth_sort_blocks > p->inst_sort_blocks ? p->depth_sort_blocks
                                                             : p->inst_sort_blocks;
        len[B_HIST] = ((size_t)kRadix * mb + kRadix) * sizeof(uint32_t);
    }
    len[B_IKEY_B] = (size_t)instance_capacity * sizeof(uint32_t);
    len[B_IVAL_B] = (size_t)instance_capacity * sizeof(uint32_t);
    len[B_LOSS_MAPS] = (size_t)values * 3 * sizeof(float);
    len[B_LOSS_BLOCKS] = (size_t)(p->loss_blocks + 1) * 2 * sizeof(float);
    len[B_GCOL] = (size_t)VN * 3 * sizeof(float);
    len[B_OFFSETS] = (size_t)(VN + 1) * sizeof(uint32_t);
    // the order, then the counts and cursors of its length buckets
    len[B_TILE_ORDER] = ((size_t)bin_tiles + 2 * kOrderBuckets) * sizeof(uint32_t);
    len[B_TILE_QUEUE] = 2 * sizeof(uint32_t);
    len[B_SPANS] = cfg->tight_rect ? (size_t)VN * kSpanRows * sizeof(uint32_t) : 0;
    // boxes of more than kSpanRows tile rows are rare (4 of 446k visible
    // Gaussians at 1M, 1200x680, 8x8 tiles): one row per 8 pairs, at least 64k
    {
        const int64_t rows = VN / 8 > 65536 ? VN / 8 : 65536;
        p->span_pool_rows = cfg->tight_rect ? (uint32_t)(rows < (int64_t(1) << 30) ? rows
                                                                                   : (int64_t(1) << 30))
                                            : 0u;
    }
    len[B_SPAN_POOL] = (size_t)p->span_pool_rows * sizeof(uint32_t);
    len[B_GID_OF] = cfg->deterministic ? (size_t)instance_capacity * sizeof(uint32_t) : 0;
    len[B_PARTIAL] = cfg->deterministic ? (size_t)instance_capacity * 11 * sizeof(float) : 0;
    // Layout.  A recompute plan keeps nothing of the projection and binning
    // from the forward to the backward (both are run again per view), so
    // the SSIM maps of the loss, which live only inside gs_loss_l1_ssim,
    // share their bytes with that region.
    auto persistent = [](int b) {
        return b == GS_BUF_COUNTERS || b == B_LOSS_BLOCKS || b == B_TILE_QUEUE ||
               b == B_LOSS_MAPS;
    };
    size_t off = 0;
    for (int b = 0; b < B_TOTAL; ++b) {
        if (!persistent(b)) continue;
        if (b == B_LOSS_MAPS && p->recompute) continue;
        p->off[b] = off;
        p->len[b] = len[b];
        off = align256(off + len[b]);
    }
    const size_t transient0 = off;
    for (int b = 0; b < B_TOTAL; ++b) {
        if (persistent(b)) continue;
        p->off[b] = off;
        p->len[b] = len[b];
        off = align256(off + len[b]);
    }
    if (p->recompute) {
        p->off[B_LOSS_MAPS] = transient0;
        p->len[B_LOSS_MAPS] = len[B_LOSS_MAPS];
        const size_t maps_end = align256(transient0 + len[B_LOSS_MAPS]);
        if (maps_end > off) off = maps_end;
    }
    p->ws_bytes = off;
    p->magic = kPlanMagic;
    return GS_OK;
}

extern "C" int32_t gs_plan_passes(const gs_plan* plan) {
    if (!plan_ok(plan)) return 0;
    const Plan* p = P(plan);
    if (p->view_index >= 0) return 1;
    return (p->n_views_full + p->ws_views - 1) / p->ws_views;
}

extern "C" gs_status gs_plan_view_pass(const gs_plan* plan, int32_t k, gs_plan* pass) {
    if (!plan_ok(plan) || !pass) return GS_ERR_INVALID;
    const Plan* p = P(plan);
    if (!p->recompute || p->view_index >= 0) return GS_ERR_INVALID;
    const int first = k * p->ws_views;
    if (k < 0 || first >= p->n_views_full) return GS_ERR_INVALID;
    const int count = p->n_views_full - first < p->ws_views ? p->n_views_full - first
                                                           : p->ws_views;
    ViewTable vt = p->vt;
    if (pass != plan) memcpy(pass, plan, sizeof(*plan));
    Plan* q = reinterpret_cast<Plan*>(pass);
    // views [first, first + count): their own tile ids and loss blocks from 0,
    // their offsets in the packed images kept
    int32_t tile = 0, blocks = 0;
    q->vt.n_views = count;
    for (int i = 0; i < count; ++i) {
        ViewGeom g = vt.v[first + i];
        g.tile_offset = tile;
        g.loss_block_offset = blocks;
        tile += g.tiles_x * g.tiles_y;
        blocks += ((g.width + kLossTileW - 1) / kLossTileW) *
                  ((g.height + kLossTileH - 1) / kLossTileH) * g.channels;
        q->vt.v[i] = g;
    }
    q->view_index = first;
    q->total_tiles = tile;
    int bits = 0;
    while ((int64_t(1) << bits) < q->total_tiles) ++bits;
    q->tile_bits = bits < 1 ? 1 : bits;
    q->tile_passes = (q->tile_bits + kRadixBits - 1) / kRadixBits;
    q->loss_blocks = blocks;
    return GS_OK;
}

extern "C" size_t gs_plan_workspace_bytes(const gs_plan* plan) {
    return plan_ok(plan) ? P(plan)->ws_bytes : 0;
}

extern "C" gs_status gs_plan_view(const gs_plan* plan, int32_t v, int64_t* value_offset,
                                  int64_t* pixel_offset, int32_t* tile_offset, int32_t* tiles_x,
                                  int32_t* tiles_y) {
    if (!plan_ok(plan) || v < 0 || v >= P(plan)->vt.n_views) return GS_ERR_INVALID;
    const ViewGeom& g = P(plan)->vt.v[v];
    if (value_offset) *value_offset = g.value_offset;
    if (pixel_offset) *pixel_offset = g.pixel_offset;
    if (tile_offset) *tile_offset = g.tile_offset;
    if (tiles_x) *tiles_x = g.tiles_x;
    if (tiles_y) *tiles_y = g.tiles_y;
    return GS_OK;
}

extern "C" gs_status gs_plan_totals(const gs_plan* plan, int64_t* total_values,
                                    int64_t* total_pixels, int32_t* total_tiles) {
    if (!plan_ok(plan)) return GS_ERR_INVALID;
    if (total_values) *total_values = P(plan)->total_values;
    if (total_pixels) *total_pixels = P(plan)->total_pixels;
    if (total_tiles) *total_tiles = P(plan)->total_tiles;
    return GS_OK;
}

extern "C" gs_status gs_plan_buffer(const gs_plan* plan, int32_t id, size_t* offset,
                                    size_t* bytes) {
    if (!plan_ok(plan) || id < 0 || id >= GS_BUF_COUNT) return GS_ERR_INVALID;
    const Plan* p = P(plan);
    if (id > GS_BUF_ABSGRAD) return GS_ERR_INVALID;
    size_t o = p->off[id], l = p->len[id];
    // The sorted instance arrays end in the A or B buffer depending on the
    // number of tile-id passes; report where the result is.
    if ((id == GS_BUF_TILE_KEYS || id == GS_BUF_TILE_VALUES) && (p->tile_passes & 1)) {
        o = p->off[id == GS_BUF_TILE_KEYS ? B_IKEY_B : B_IVAL_B];
    }
    if (offset) *offset = o;
    if (bytes) *bytes = l;
    return GS_OK;
}

// The workspace holds the projection of every view of the plan (not so for
// the whole of a multi-view recompute plan, whose views go through it one
// pass at a time).
static bool per_view_ok(const Plan* p) { return p->vt.n_views <= p->ws_views; }
// ... and the plan covers all views of the workspace's iteration at once.
static bool all_views_ok(const Plan* p) {
    return per_view_ok(p) && p->vt.n_views == p->n_views_full;
}
// The poses of a pass plan's view: views_dev[view_index] of the caller's array.
static const gs_view* pass_views(const Plan* p, const gs_view* views_dev) {
    return views_dev + (p->view_index > 0 ? p->view_index : 0);
}

static bool map_ok(const Plan* p, const gs_map* m) {
    return m && m->means && m->log_scales && m->quats && m->opacity_logits && m->sh &&
           m->n >= 1 && m->n <= p->n_capacity && m->sh_degree >= 0 && m->sh_degree <= 3;
}

extern "C" gs_status gs_project(const gs_plan* plan, const gs_map* map, const gs_view* views_dev,
                                void* ws, void* stream) {
    if (!plan_ok(plan) || !views_dev || !ws) return GS_ERR_INVALID;
    if (!map_ok(P(plan), map) || !per_view_ok(P(plan))) return GS_ERR_INVALID;
    return launch_project(P(plan), map, pass_views(P(plan), views_dev), ws, S(stream));
}

extern "C" gs_status gs_bin_sort(const gs_plan* plan, int32_t n, void* ws, void* stream) {
    if (!plan_ok(plan) || !ws || n < 1 || n > P(plan)->n_capacity) return GS_ERR_INVALID;
    if (!per_view_ok(P(plan))) return GS_ERR_INVALID;
    return launch_bin_sort(P(plan), n, ws, S(stream));
}

extern "C" gs_status gs_render_fwd(const gs_plan* plan, void* ws, float* images,
                                   float* final_T, int32_t* last_idx, void* stream) {
    if (!plan_ok(plan) || !ws || !images || !final_T || !last_idx) return GS_ERR_INVALID;
    if (!per_view_ok(P(plan))) return GS_ERR_INVALID;
    return launch_render_fwd(P(plan), ws, images, final_T, last_idx, S(stream));
}

extern "C" gs_status gs_loss_l1_ssim(const gs_plan* plan, const float* images,
                                     const float* targets, float lambda, float view_weight,
                                     float* loss_dev, float* dL_dimages, void* ws, void* stream) {
    if (!plan_ok(plan) || !images || !targets || !loss_dev || !dL_dimages || !ws)
        return GS_ERR_INVALID;
    if (!(lambda >= 0.0f && lambda <= 1.0f) || !(view_weight > 0.0f)) return GS_ERR_INVALID;
    return launch_loss(P(plan), images, targets, lambda, view_weight, loss_dev, dL_dimages, ws,
                       S(stream));
}

extern "C" gs_status gs_render_bwd(const gs_plan* plan, const gs_map* map,
                                   const gs_view* views_dev, void* ws, const float* final_T,
                                   const int32_t* last_idx, const float* dL_dimages,
                                   const gs_map_grad* grads, int32_t accumulate, void* stream) {
    if (!plan_ok(plan) || !views_dev || !ws || !final_T || !last_idx || !dL_dimages || !grads)
        return GS_ERR_INVALID;
    if (!map_ok(P(plan), map) || !per_view_ok(P(plan))) return GS_ERR_INVALID;
    if (!grads->means || !grads->log_scales || !grads->quats || !grads->opacity_logits ||
        !grads->sh)
        return GS_ERR_INVALID;
    return launch_render_bwd(P(plan), map, pass_views(P(plan), views_dev), ws, final_T, last_idx,
                             dL_dimages, grads, accumulate ? 1 : 0, S(stream));
}

extern "C" gs_status gs_render_bwd_pixels(const gs_plan* plan, void* ws, const float* final_T,
                                          const int32_t* last_idx, const float* dL_dimages,
                                          void* stream) {
    if (!plan_ok(plan) || !ws || !final_T || !last_idx || !dL_dimages) return GS_ERR_INVALID;
    if (!per_view_ok(P(plan))) return GS_ERR_INVALID;
    return launch_render_bwd_pixels(P(plan), ws, final_T, last_idx, dL_dimages, S(stream));
}

extern "C" gs_status gs_project_bwd(const gs_plan* plan, const gs_map* map,
                                    const gs_view* views_dev, const void* ws,
                                    const gs_map_grad* grads, int32_t accumulate, void* stream) {
    if (!plan_ok(plan) || !views_dev || !ws || !grads) return GS_ERR_INVALID;
    if (!map_ok(P(plan), map) || !per_view_ok(P(plan))) return GS_ERR_INVALID;
    if (!grads->means || !grads->log_scales || !grads->quats || !grads->opacity_logits ||
        !grads->sh)
        return GS_ERR_INVALID;
    return launch_project_bwd(P(plan), map, pass_views(P(plan), views_dev),
                              const_cast<void*>(ws), grads, accumulate ? 1 : 0, S(stream));
}

extern "C" gs_status gs_project_bwd_groups(const gs_plan* plan, const gs_map* map,
                                           const gs_view* views_dev, const void* ws,
                                           const gs_map_grad* grads, uint8_t* group_vis,
                                           void* stream) {
    if (!plan_ok(plan) || !views_dev || !ws || !grads || !group_vis) return GS_ERR_INVALID;
    if (!map_ok(P(plan), map) || !all_views_ok(P(plan))) return GS_ERR_INVALID;
    if (!grads->means || !grads->log_scales || !grads->quats || !grads->opacity_logits ||
        !grads->sh)
        return GS_ERR_INVALID;
    return launch_project_bwd(P(plan), map, views_dev, const_cast<void*>(ws), grads, 0,
                              S(stream), group_vis);
}

extern "C" gs_status gs_adam_step_groups(float* params, const float* grads, float* m, float* v,
                                         int64_t n_floats, int32_t n_groups,
                                         const int64_t* group_offsets_host,
                                         const float* group_lr_host,
                                         const int32_t* group_stride_host, int32_t n_gauss,
                                         const uint8_t* group_vis, float beta1, float beta2,
                                         float eps, int32_t* step_dev, void* stream) {
    if (!params || !grads || !m || !v || !step_dev || !group_offsets_host || !group_lr_host ||
        !group_stride_host || !group_vis || n_gauss < 1)
        return GS_ERR_INVALID;
    if (n_floats < 1 || n_groups < 1 || n_groups > GS_MAX_GROUPS) return GS_ERR_INVALID;
    if (group_offsets_host[0] != 0 || group_offsets_host[n_groups] != n_floats)
        return GS_ERR_INVALID;
    for (int g = 0; g < n_groups; ++g) {
        if (group_offsets_host[g + 1] < group_offsets_host[g]) return GS_ERR_INVALID;
        if (group_stride_host[g] < 1 ||
            (int64_t)group_stride_host[g] * n_gauss >= (int64_t(1) << 31))
            return GS_ERR_INVALID;
    }
    if (!(beta1 >= 0.0f && beta1 < 1.0f && beta2 >= 0.0f && beta2 < 1.0f && eps >= 0.0f))
        return GS_ERR_INVALID;
    return launch_adam_groups(params, grads, m, v, n_floats, n_groups, group_offsets_host,
                              group_lr_host, group_stride_host, n_gauss, group_vis, beta1, beta2,
                              eps, step_dev, S(stream));
}

static bool grad_ok(const gs_map_grad* g) {
    return g && g->means && g->log_scales && g->quats && g->opacity_logits && g->sh;
}

extern "C" gs_status gs_project_bwd_adam(const gs_plan* plan, const gs_map* map,
                                         const gs_view* views_dev, void* ws,
                                         const gs_map_grad* params, const gs_map_grad* m,
                                         const gs_map_grad* v, const gs_map_grad* grads_acc,
                                         const gs_map_grad* grads_out, const float* group_lr_host,
                                         float beta1, float beta2, float eps, int32_t* step_dev,
                                         void* stream) {
    if (!plan_ok(plan) || !views_dev || !ws || !group_lr_host || !step_dev) return GS_ERR_INVALID;
    if (!map_ok(P(plan), map) || !grad_ok(params) || !grad_ok(m) || !grad_ok(v))
        return GS_ERR_INVALID;
    if (!all_views_ok(P(plan))) return GS_ERR_INVALID;
    if ((grads_acc && !grad_ok(grads_acc)) || (grads_out && !grad_ok(grads_out)))
        return GS_ERR_INVALID;
    if (!(beta1 >= 0.0f && beta1 < 1.0f && beta2 >= 0.0f && beta2 < 1.0f && eps >= 0.0f))
        return GS_ERR_INVALID;
    return launch_project_bwd_adam(P(plan), map, views_dev, ws, params, m, v, grads_acc,
                                   grads_out, group_lr_host, beta1, beta2, eps, step_dev,
                                   S(stream));
}

extern "C" gs_status gs_adam_step(float* params, const float* grads, float* m, float* v,
                                  int64_t n_floats, int32_t n_groups,
                                  const int64_t* group_offsets_host, const float* group_lr_host,
                                  float beta1, float beta2, float eps, int32_t* step_dev,
                                  void* stream) {
    if (!params || !grads || !m || !v || !step_dev || !group_offsets_host || !group_lr_host)
        return GS_ERR_INVALID;
    if (n_floats < 1 || n_groups < 1 || n_groups > GS_MAX_GROUPS) return GS_ERR_INVALID;
    if (group_offsets_host[0] != 0 || group_offsets_host[n_groups] != n_floats)
        return GS_ERR_INVALID;
    for (int g = 0; g < n_groups; ++g)
        if (group_offsets_host[g + 1] < group_offsets_host[g]) return GS_ERR_INVALID;
    if (!(beta1 >= 0.0f && beta1 < 1.0f && beta2 >= 0.0f && beta2 < 1.0f && eps >= 0.0f))
        return GS_ERR_INVALID;
    return launch_adam(params, grads, m, v, n_floats, n_groups, group_offsets_host,
                       group_lr_host, beta1, beta2, eps, step_dev, S(stream));
}

extern "C" gs_status gs_visibility(const gs_plan* plan, int32_t n, const void* ws,
                                   uint8_t* vis, void* stream) {
    if (!plan_ok(plan) || !ws || !vis || n < 1 || n > P(plan)->n_capacity) return GS_ERR_INVALID;
    if (!all_views_ok(P(plan))) return GS_ERR_INVALID;
    return launch_visibility(n, P(plan)->vt.n_views, cbuf<uint32_t>(P(plan), ws, GS_BUF_TOUCHED),
                             vis, S(stream));
}

extern "C" gs_status gs_adam_step_sparse(float* params, const float* grads, float* m, float* v,
                                         int64_t n_floats, int32_t n_groups,
                                         const int64_t* group_offsets_host,
                                         const float* group_lr_host,
                                         const int32_t* group_stride_host, int32_t n_gauss,
                                         const uint8_t* vis, float beta1, float beta2, float eps,
                                         int32_t* step_dev, void* stream) {
    if (!params || !grads || !m || !v || !step_dev || !group_offsets_host || !group_lr_host ||
        !group_stride_host || !vis || n_gauss < 1)
        return GS_ERR_INVALID;
    if (n_floats < 1 || n_groups < 1 || n_groups > GS_MAX_GROUPS) return GS_ERR_INVALID;
    if (group_offsets_host[0] != 0 || group_offsets_host[n_groups] != n_floats)
        return GS_ERR_INVALID;
    for (int g = 0; g < n_groups; ++g) {
        if (group_offsets_host[g + 1] < group_offsets_host[g]) return GS_ERR_INVALID;
        if (group_stride_host[g] < 1 ||
            (int64_t)group_stride_host[g] * n_gauss >= (int64_t(1) << 31))
            return GS_ERR_INVALID;
    }
    if (!(beta1 >= 0.0f && beta1 < 1.0f && beta2 >= 0.0f && beta2 < 1.0f && eps >= 0.0f))
        return GS_ERR_INVALID;
    return launch_adam_sparse(params, grads, m, v, n_floats, n_groups, group_offsets_host,
                              group_lr_host, group_stride_host, n_gauss, vis, beta1, beta2, eps,
                              step_dev, S(stream));
}

extern "C" gs_status gs_read_counters(const gs_plan* plan, const void* ws, gs_counters* out,
                                      void* stream) {
    if (!plan_ok(plan) || !ws || !out) return GS_ERR_INVALID;
    DevCounters c;
    cudaStream_t st = S(stream);
    if (cudaMemcpyAsync(&c, cbuf<char>(P(plan), ws, GS_BUF_COUNTERS), sizeof(c),
                        cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return GS_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return GS_ERR_CUDA;
    memset(out, 0, sizeof(*out));
    out->status = c.status;
    out->n_instances = c.n_instances;
    out->n_instances_raw = c.n_raw;
    out->loss = c.loss;
    return GS_OK;
}

extern "C" const char* gs_status_string(gs_status s) {
    switch (s) {
        case GS_OK: return "GS_OK";
        case GS_ERR_INVALID: return "GS_ERR_INVALID: invalid argument";
        case GS_ERR_CUDA: return "GS_ERR_CUDA: CUDA launch or copy failed";
        case GS_ERR_CAPACITY: return "GS_ERR_CAPACITY: capacity exceeded";
        case GS_ERR_UNSUPPORTED: return "GS_ERR_UNSUPPORTED: unsupported configuration";
        case GS_ERR_TIMEOUT: return "GS_ERR_TIMEOUT: bounded device wait gave up";
    }
    return "unknown gs_status";
}
