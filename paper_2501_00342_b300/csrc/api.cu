// C ABI of the rasterizer (declared in include/sgs.h): argument checks, workspace layout
// and the order of the stage kernels.  Nothing here allocates; every launch goes to the
// caller's stream.
#include <cuda_runtime.h>

#include <cstring>

#include "common.cuh"
#include "kernels.h"
#include "sgs.h"

using namespace sgs;

namespace {

enum Region {
    O_STATUS, O_REC0, O_REC1, O_REC2, O_RECT, O_TILES, O_OFFS, O_K0, O_V0, O_K1, O_V1,
    O_RANGES, O_PIXT, O_PIXLAST, O_GRAD2D, O_PIXCOUNT, O_SPANS, O_SCANLB, O_HIST, O_GOFF, O_SORTLB,
    O_COUNTERS, O_RK0, O_RV0, O_RK1, O_RV1, O_RLB, O_TORDER, O_TTOP, O_BORDER, O_MASKS, O_FLAGS, O_END
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

int ceil_log2(int64_t x) {
    int b = 0;
    while (((int64_t)1 << b) < x) ++b;
    return b;
}

// Tile sides are powers of two of at least 8 (the blend's warps own 8-wide blocks of 4 or
// 8 rows), with 64-1024 pixels per tile; each blend pass runs one CTA of at most 512
// threads per tile, so a tile of more than 512 pixels needs 2 or more pixels per thread in
// both passes (fwd, bwd: the resolved pixels per thread).
bool valid_tile(int32_t w, int32_t h, int32_t fwd, int32_t bwd) {
    auto pow2 = [](int32_t x) { return x >= 8 && x <= 64 && (x & (x - 1)) == 0; };
    if (!pow2(w) || !pow2(h)) return false;
    const int32_t t = w * h;
    return t >= 64 && t <= 1024 && t / fwd <= 512 && t / bwd <= 512;
}

int32_t resolved_pixels(int32_t setting) { return setting ? setting : 2; }

sgs_status check_gaussians(const sgs_gaussians* g) {
    if (!g || g->n < 0 || g->stride < g->n || (g->stride & 3) != 0) return SGS_ERR_INVALID;
    if (g->sh_degree < 0 || g->sh_degree > SGS_MAX_SH_DEGREE) return SGS_ERR_INVALID;
    if (g->num_lobes < 0 || g->num_lobes > 4) return SGS_ERR_INVALID;
    if (g->axis_mode != SGS_AXIS_FREE && g->axis_mode != SGS_AXIS_ORTHO_FIXED &&
        g->axis_mode != SGS_AXIS_ORTHO_FRAME)
        return SGS_ERR_INVALID;
    if (g->axis_mode != SGS_AXIS_FREE && g->num_lobes > 3) return SGS_ERR_INVALID;
    if (g->sh_adaptive != 0 && g->sh_adaptive != 1) return SGS_ERR_INVALID;
    if (g->sh_adaptive && !(g->sh_radius[0] >= 0.0f && g->sh_radius[0] <= g->sh_radius[1]))
        return SGS_ERR_INVALID;  // also rejects NaN thresholds
    return SGS_OK;
}

sgs_status check_pointers(const sgs_gaussians* g) {
    if (g->n == 0) return SGS_OK;
    const float* need[] = {g->mean, g->scale, g->rot, g->opacity, g->sh};
    for (const float* p : need)
        if (!p || !aligned16(p)) return SGS_ERR_INVALID;
    if (g->num_lobes > 0) {
        if (!g->sg_amp || !g->sg_sharp || !aligned16(g->sg_amp) || !aligned16(g->sg_sharp))
            return SGS_ERR_INVALID;
        if (g->axis_mode != SGS_AXIS_ORTHO_FIXED && (!g->sg_axis || !aligned16(g->sg_axis))) return SGS_ERR_INVALID;
    }
    return SGS_OK;
}

bool same_layout(const sgs_plan* p, const sgs_gaussians* g) {
    return p->n == g->n && p->stride == g->stride && p->sh_degree == g->sh_degree &&
           p->num_lobes == g->num_lobes && p->axis_mode == g->axis_mode;
}

template <typename T>
T* region(const sgs_plan* p, int which) {
    return reinterpret_cast<T*>(static_cast<unsigned char*>(p->workspace) + p->offsets[which]);
}

ViewTable view_table(const sgs_plan* p) {
    ViewTable vt;
    std::memset(&vt, 0, sizeof(vt));
    vt.B = p->B;
    vt.tile_w = p->settings.tile_w;
    vt.tile_h = p->settings.tile_h;
    vt.inv_tile_w = 1.0f / (float)vt.tile_w;  // exact: powers of two
    vt.inv_tile_h = 1.0f / (float)vt.tile_h;
    vt.fwd_ppt = resolved_pixels(p->settings.fwd_pixels);
    vt.bwd_ppt = resolved_pixels(p->settings.bwd_pixels);
    vt.count_pairs = p->settings.count_pairs ? 1 : 0;
    vt.num_tiles = p->num_tiles;
    vt.order = p->workspace ? region<uint32_t>(p, O_TORDER) : nullptr;
    vt.tile_top = p->workspace ? region<uint32_t>(p, O_TTOP) : nullptr;
    vt.masks = p->workspace ? region<uint16_t>(p, O_MASKS) : nullptr;
    vt.persistent = p->settings.persistent ? 1 : 0;
    vt.work = p->workspace ? region<DeviceStatus>(p, O_STATUS)->work : nullptr;
    for (int v = 0; v < p->B; ++v) {
        const sgs_camera& c = p->cams[v];
        View& w = vt.v[v];
        std::memcpy(w.V, c.viewmat, sizeof(w.V));
        std::memcpy(w.campos, c.campos, sizeof(w.campos));
        w.fx = c.fx;
        w.fy = c.fy;
        w.cx = c.cx;
        w.cy = c.cy;
        w.W = c.width;
        w.H = c.height;
        w.near_plane = c.near_plane;
        // single-precision steps, each correctly rounded, as the FP32 projection orders them
        const float half_w = 0.5f * (float)c.width, half_h = 0.5f * (float)c.height;
        const float qx = half_w / c.fx, qy = half_h / c.fy;
        w.limx = 1.3f * qx;
        w.limy = 1.3f * qy;
        w.tiles_x = p->tiles_x[v];
        w.tiles_y = p->tiles_y[v];
        w.tile_base = (uint32_t)p->tile_base[v];
        w.pixel_base = p->pixel_base[v];
    }
    return vt;
}

RecordPtrs records(const sgs_plan* p) {
    RecordPtrs r;
    r.rec0 = region<float4>(p, O_REC0);
    r.rec1 = region<float4>(p, O_REC1);
    r.rec2 = region<float4>(p, O_REC2);
    r.rect = region<uint2>(p, O_RECT);
    r.tiles = region<uint32_t>(p, O_TILES);
    r.spans = region<uint4>(p, O_SPANS);
    r.flags = region<uint32_t>(p, O_FLAGS);
    r.sort_keys = region<uint32_t>(p, O_RK0);
    r.sort_vals = region<uint32_t>(p, O_RV0);
    r.rv = record_value(p->num_records);
    return r;
}

sgs_status cuda_status(cudaError_t e) { return e == cudaSuccess ? SGS_OK : SGS_ERR_CUDA; }

cudaError_t probe(const sgs_plan* p, int k, cudaStream_t s) {
    if (!p->events || !p->events[k]) return cudaSuccess;
    return record_probe(p->events[k], s);
}

#define SGS_TRY(expr)                                  \
    do {                                               \
        cudaError_t _e = (expr);                       \
        if (_e != cudaSuccess) return SGS_ERR_CUDA;    \
    } while (0)

}  // namespace

extern "C" {

const char* sgs_status_string(sgs_status s) {
    switch (s) {
        case SGS_OK: return "ok";
        case SGS_ERR_INVALID: return "invalid argument, size, alignment or layout";
        case SGS_ERR_CAPACITY: return "more (record, tile) instances than the workspace capacity";
        case SGS_ERR_TIMEOUT: return "a bounded device-side wait ran out";
        case SGS_ERR_CUDA: return "CUDA runtime error";
        default: return "unknown status";
    }
}

void sgs_abi_sizes(size_t* sizes) {
    sizes[0] = sizeof(sgs_plan);
    sizes[1] = sizeof(sgs_camera);
    sizes[2] = sizeof(sgs_gaussians);
    sizes[3] = sizeof(sgs_settings);
    sizes[4] = sizeof(sgs_adam_config);
    sizes[5] = sizeof(sgs_grads);
}

sgs_status sgs_workspace_size(const sgs_gaussians* g, const sgs_camera* cams, int32_t B,
                              const sgs_settings* settings, int64_t instance_capacity,
                              sgs_plan* plan, size_t* bytes) {
    if (!plan || !bytes || !cams || !settings) return SGS_ERR_INVALID;
    if (check_gaussians(g) != SGS_OK) return SGS_ERR_INVALID;
    if (B < 1 || B > SGS_MAX_VIEWS) return SGS_ERR_INVALID;
    if (settings->batch_depth < 32 || settings->batch_depth > 1024) return SGS_ERR_INVALID;
    if (settings->fwd_pixels < 0 || settings->fwd_pixels > 2) return SGS_ERR_INVALID;
    if (settings->bwd_pixels < 0 || settings->bwd_pixels == 3 || settings->bwd_pixels > 4) return SGS_ERR_INVALID;
    if (!valid_tile(settings->tile_w, settings->tile_h, resolved_pixels(settings->fwd_pixels),
                    resolved_pixels(settings->bwd_pixels)))
        return SGS_ERR_INVALID;
    if (settings->bwd_pixels == 4 && settings->tile_h % 16 != 0) return SGS_ERR_INVALID;
    if (settings->count_pairs != 0 && settings->count_pairs != 1) return SGS_ERR_INVALID;
    if (settings->digit_bits < kMinDigitBits || settings->digit_bits > kMaxDigitBits) return SGS_ERR_INVALID;
    if (settings->memory_mode != 0) return SGS_ERR_INVALID;
    if (settings->persistent != 0 && settings->persistent != 1) return SGS_ERR_INVALID;
    if (instance_capacity < 0 || instance_capacity > 0xffffffffll) return SGS_ERR_INVALID;
    std::memset(plan, 0, sizeof(*plan));
    plan->n = g->n;
    plan->stride = g->stride;
    plan->sh_degree = g->sh_degree;
    plan->num_lobes = g->num_lobes;
    plan->axis_mode = g->axis_mode;
    plan->B = B;
    plan->settings = *settings;
    int64_t tiles = 0, pixels = 0;
    for (int v = 0; v < B; ++v) {
        const sgs_camera& c = cams[v];
        if (c.width < 1 || c.height < 1 || !(c.fx > 0.0f) || !(c.fy > 0.0f) || !(c.near_plane > 0.0f))
            return SGS_ERR_INVALID;  // depth > near > 0 keeps the depth bits ordered as values
        const int32_t tx = (c.width + settings->tile_w - 1) / settings->tile_w;
        const int32_t ty = (c.height + settings->tile_h - 1) / settings->tile_h;
        if (tx > 65535 || ty > 65535) return SGS_ERR_INVALID;
        plan->cams[v] = c;
        plan->tiles_x[v] = tx;
        plan->tiles_y[v] = ty;
        plan->tile_base[v] = tiles;
        plan->pixel_base[v] = pixels;
        tiles += (int64_t)tx * ty;
        pixels += (int64_t)c.width * c.height;
    }
    plan->tile_base[B] = tiles;
    plan->pixel_base[B] = pixels;
    if (tiles >= 0xffffffffll) return SGS_ERR_INVALID;
    const int64_t R = (int64_t)B * g->n;
    if (R >= 0xffffffffll) return SGS_ERR_INVALID;
    plan->num_records = R;
    plan->num_tiles = tiles;
    plan->num_pixels = pixels;
    plan->instance_capacity = instance_capacity;
    plan->key_bits = 32 + ceil_log2(tiles < 1 ? 1 : tiles);
    // the depth half of the key is ordered by the record sort; the instance sort takes the
    // tile bits only
    plan->sort_passes = sort_passes(0, plan->key_bits - 32, settings->digit_bits);
    if (plan->sort_passes > kMaxSortPasses) return SGS_ERR_INVALID;

    size_t sz[O_END];
    const size_t cap = (size_t)instance_capacity;
    sz[O_STATUS] = 256;
    sz[O_REC0] = sz[O_REC1] = sz[O_REC2] = 16 * (size_t)R;
    sz[O_RECT] = 8 * (size_t)R;
    sz[O_TILES] = sz[O_OFFS] = 4 * (size_t)R;
    sz[O_K0] = sz[O_K1] = 4 * cap;  // tile ids
    sz[O_V0] = sz[O_V1] = 4 * cap;
    sz[O_RANGES] = 8 * (size_t)tiles;
    sz[O_PIXT] = sz[O_PIXLAST] = 4 * (size_t)pixels;
    sz[O_GRAD2D] = 36 * (size_t)R;  // float4[2][R], float[R]
    sz[O_PIXCOUNT] = 8 * (size_t)pixels;
    sz[O_SPANS] = 64 * (size_t)R;
    sz[O_SCANLB] = 8 * (size_t)((R + kScanTile - 1) / kScanTile + 1);
    sz[O_HIST] = sz[O_GOFF] = 4 * (size_t)kHistEntries;
    int ipasses, irb, rpasses, rrb;
    sort_digit_plan(0, plan->key_bits - 32, settings->digit_bits, &ipasses, &irb);
    sort_digit_plan(0, 32, settings->digit_bits, &rpasses, &rrb);
    sz[O_SORTLB] = 8 * sort_lookback_entries(instance_capacity, irb);
    sz[O_COUNTERS] = 4 * (size_t)kMaxSortPasses;
    sz[O_RK0] = sz[O_RK1] = 4 * (size_t)R;  // depth bits
    sz[O_RV0] = sz[O_RV1] = 4 * (size_t)R;
    sz[O_RLB] = 8 * sort_lookback_entries(R, rrb);
    // the blend's tile orders and the forward's per-tile last contributor
    sz[O_TORDER] = sz[O_TTOP] = sz[O_BORDER] = 4 * (size_t)tiles;
    sz[O_MASKS] = 2 * cap;  // per instance, the warp blocks its support reaches
    sz[O_FLAGS] = 4 * (size_t)R;  // per record, the decisions the backward reuses
    size_t off = 0;
    for (int k = 0; k < O_END; ++k) {
        plan->offsets[k] = off;
        off += align256(sz[k]);
    }
    plan->workspace_bytes = off;
    *bytes = off;
    return SGS_OK;
}

sgs_status sgs_preprocess(sgs_plan* plan, const sgs_gaussians* g, void* workspace,
                          size_t ws_bytes, cudaStream_t stream) {
    if (!plan || !workspace || check_gaussians(g) != SGS_OK || !same_layout(plan, g)) return SGS_ERR_INVALID;
    if (check_pointers(g) != SGS_OK) return SGS_ERR_INVALID;
    if (((uintptr_t)workspace & 255u) != 0 || ws_bytes < plan->workspace_bytes) return SGS_ERR_INVALID;
    const bool rebind = plan->workspace != workspace;
    plan->workspace = workspace;
    plan->stage = 0;
    DeviceStatus* st = region<DeviceStatus>(plan, O_STATUS);
    SGS_TRY(launch_sort_init(st, 0u, stream));
    // the forward's tile tops schedule the next forward of this plan (see sgs_bin_sort);
    // a newly bound workspace has none
    if (rebind && plan->num_tiles > 0)
        SGS_TRY(cudaMemsetAsync(region<uint32_t>(plan, O_TTOP), 0, 4 * (size_t)plan->num_tiles, stream));
    // the reverse blend adds into zeroed 2D gradients; after this clear every backward
    // leaves them zero again (the preprocess backward clears what it reads)
    if (rebind) SGS_TRY(launch_zero_grad2d(region<float4>(plan, O_GRAD2D), plan->num_records, stream));
    const ViewTable vt = view_table(plan);
    SGS_TRY(probe(plan, SGS_EV_PRE_BEGIN, stream));
    if (plan->n > 0) SGS_TRY(launch_preprocess(*g, vt, records(plan), stream));
    SGS_TRY(probe(plan, SGS_EV_PRE_END, stream));
    plan->stage = 1;
    return SGS_OK;
}

sgs_status sgs_bin_sort(sgs_plan* plan, int64_t* num_instances, cudaStream_t stream) {
    if (!plan || !plan->workspace || plan->stage < 1) return SGS_ERR_INVALID;
    DeviceStatus* st = region<DeviceStatus>(plan, O_STATUS);
    const ViewTable vt = view_table(plan);
    const RecordPtrs rp = records(plan);
    const int64_t R = plan->num_records;
    const int64_t cap = plan->instance_capacity;
    unsigned long long* scan_lb = region<unsigned long long>(plan, O_SCANLB);
    SGS_TRY(probe(plan, SGS_EV_BIN_BEGIN, stream));
    SGS_TRY(launch_fill_u32(st->tile_counter, 0u, 16, stream));
    SGS_TRY(launch_fill_u32(reinterpret_cast<uint32_t*>(scan_lb), 0u,
                            2 * (size_t)((R + kScanTile - 1) / kScanTile + 1), stream));
    // (c, depth half) stable sort of the records by view depth bits
    const int rpasses = sort_passes(0, 32, plan->settings.digit_bits);
    // the preprocess wrote the pairs (keys: depth bits; values: RecordValue)
    SGS_TRY(launch_record_hist(region<uint32_t>(plan, O_RK0), R, st, plan->settings.digit_bits,
                               region<uint32_t>(plan, O_HIST), stream));
    if (R > 0)
        SGS_TRY(launch_sort(region<uint32_t>(plan, O_RK0), region<uint32_t>(plan, O_RV0),
                            region<uint32_t>(plan, O_RK1), region<uint32_t>(plan, O_RV1),
                            &st->num_records, R, 0, 32, plan->settings.digit_bits, region<uint32_t>(plan, O_HIST),
                            region<uint32_t>(plan, O_GOFF), region<uint32_t>(plan, O_COUNTERS),
                            region<unsigned long long>(plan, O_RLB), st, stream, nullptr,
                            /*histogram_ready=*/true, &st->num_visible, /*drop_first=*/true));
    const uint32_t* perm = region<uint32_t>(plan, (rpasses & 1) ? O_RV1 : O_RV0);
    // (b) counts and instances in depth order
    SGS_TRY(launch_scan(rp.tiles, perm, region<uint32_t>(plan, O_OFFS), R, scan_lb, st, cap, stream));
    SGS_TRY(probe(plan, SGS_EV_SCAN_END, stream));
    int ipasses, irb;
    const int tile_bits = plan->key_bits - 32;
    sort_digit_plan(0, tile_bits, plan->settings.digit_bits, &ipasses, &irb);
    SGS_TRY(launch_duplicate(vt, rp, perm, region<uint32_t>(plan, O_OFFS), plan->n, R, st, cap,
                             region<uint32_t>(plan, O_K0), region<uint32_t>(plan, O_V0), irb,
                             ipasses, region<uint32_t>(plan, O_HIST), stream));
    SGS_TRY(probe(plan, SGS_EV_DUP_END, stream));
    // (c, tile half) stable sort of the instances by tile id
    cudaEvent_t hist_end = plan->events ? plan->events[SGS_EV_HIST_END] : nullptr;
    if (plan->sort_passes > 0) {
        SGS_TRY(launch_sort(region<uint32_t>(plan, O_K0), region<uint32_t>(plan, O_V0),
                            region<uint32_t>(plan, O_K1), region<uint32_t>(plan, O_V1),
                            &st->m_clamped, cap, 0, tile_bits, plan->settings.digit_bits,
                            region<uint32_t>(plan, O_HIST), region<uint32_t>(plan, O_GOFF),
                            region<uint32_t>(plan, O_COUNTERS), region<unsigned long long>(plan, O_SORTLB),
                            st, stream, hist_end, /*histogram_ready=*/true));
    } else if (hist_end) {
        SGS_TRY(record_probe(hist_end, stream));
    }
    SGS_TRY(probe(plan, SGS_EV_SORT_END, stream));
    const int kreg = (plan->sort_passes & 1) ? O_K1 : O_K0;
    SGS_TRY(launch_fill_u32(region<uint32_t>(plan, O_RANGES), 0u, 2 * (size_t)plan->num_tiles, stream));
    SGS_TRY(launch_ranges(region<uint32_t>(plan, kreg), st, cap, plan->num_tiles,
                          region<uint2>(plan, O_RANGES), stream));
    // most expensive tiles first: by the previous forward's last contributors where there
    // are some, else by list length
    SGS_TRY(launch_tile_order(region<uint2>(plan, O_RANGES), region<uint32_t>(plan, O_TTOP), plan->num_tiles,
                              region<uint32_t>(plan, O_TORDER), stream));
    SGS_TRY(probe(plan, SGS_EV_RANGES_END, stream));
    plan->stage = 2;
    if (num_instances) {
        unsigned long long m = 0;
        SGS_TRY(cudaMemcpyAsync(&m, &st->m, sizeof(m), cudaMemcpyDeviceToHost, stream));
        SGS_TRY(cudaStreamSynchronize(stream));
        *num_instances = (int64_t)m;
        if ((int64_t)m > cap) return SGS_ERR_CAPACITY;
    }
    return SGS_OK;
}

sgs_status sgs_render(sgs_plan* plan, float* out_rgb, float* out_T, cudaStream_t stream) {
    if (!plan || !plan->workspace || !out_rgb || plan->stage < 2) return SGS_ERR_INVALID;
    const ViewTable vt = view_table(plan);
    const int vreg = (plan->sort_passes & 1) ? O_V1 : O_V0;
    const sgs_settings& s = plan->settings;
    SGS_TRY(probe(plan, SGS_EV_BLEND_BEGIN, stream));
    SGS_TRY(launch_blend(vt, region<uint2>(plan, O_RANGES), region<uint32_t>(plan, vreg),
                         plan->num_records, records(plan),
                         s.batch_depth, s.bg[0], s.bg[1], s.bg[2], out_rgb, out_T,
                         region<float>(plan, O_PIXT), region<uint32_t>(plan, O_PIXLAST),
                         region<uint2>(plan, O_PIXCOUNT), region<DeviceStatus>(plan, O_STATUS), stream));
    SGS_TRY(probe(plan, SGS_EV_BLEND_END, stream));
    plan->stage = 3;
    return SGS_OK;
}

sgs_status sgs_render_backward(sgs_plan* plan, const sgs_gaussians* g, const float* dL_drgb,
                               sgs_grads* out, cudaStream_t stream) {
    if (!plan || !plan->workspace || !dL_drgb || !out || plan->stage < 3) return SGS_ERR_INVALID;
    if (check_gaussians(g) != SGS_OK || !same_layout(plan, g) || check_pointers(g) != SGS_OK)
        return SGS_ERR_INVALID;
    if (plan->n > 0) {
        if (!out->mean || !out->scale || !out->rot || !out->opacity || !out->sh) return SGS_ERR_INVALID;
        if (plan->num_lobes > 0 && (!out->sg_amp || !out->sg_sharp)) return SGS_ERR_INVALID;
        if (plan->num_lobes > 0 && plan->axis_mode != SGS_AXIS_ORTHO_FIXED && !out->sg_axis) return SGS_ERR_INVALID;
    }
    const ViewTable vt = view_table(plan);
    const RecordPtrs rp = records(plan);
    const int64_t R = plan->num_records;
    float4* grad2d = region<float4>(plan, O_GRAD2D);
    const int vreg = (plan->sort_passes & 1) ? O_V1 : O_V0;
    const sgs_settings& s = plan->settings;
    SGS_TRY(probe(plan, SGS_EV_BWD_BEGIN, stream));
    // the backward's tile order: tiles by decreasing position of their last contributor
    // (written by the forward), so the longest reverse walks start first
    SGS_TRY(launch_tile_order(nullptr, region<uint32_t>(plan, O_TTOP), plan->num_tiles,
                              region<uint32_t>(plan, O_BORDER), stream));
    SGS_TRY(probe(plan, SGS_EV_BWD_ZERO_END, stream));
    ViewTable vtb = vt;
    vtb.order = region<uint32_t>(plan, O_BORDER);
    vtb.work = region<DeviceStatus>(plan, O_STATUS)->work + 1;
    // the two-pixel kernels of both passes share warp blocks: the backward reads the masks
    // the forward stored
    if (!(vt.fwd_ppt == 2 && vt.bwd_ppt == 2)) vtb.masks = nullptr;
    SGS_TRY(launch_blend_backward(vtb, region<uint2>(plan, O_RANGES), region<uint32_t>(plan, vreg), rp,
                                  s.batch_depth, s.bg[0], s.bg[1], s.bg[2], region<float>(plan, O_PIXT),
                                  region<uint32_t>(plan, O_PIXLAST), dL_drgb, grad2d, R,
                                  region<DeviceStatus>(plan, O_STATUS), stream));
    SGS_TRY(probe(plan, SGS_EV_BWD_BLEND_END, stream));
    if (plan->n > 0) SGS_TRY(launch_preprocess_backward(*g, vt, rp, grad2d, R, *out, stream));
    SGS_TRY(probe(plan, SGS_EV_BWD_PRE_END, stream));
    return SGS_OK;
}

sgs_status sgs_set_events(sgs_plan* plan, cudaEvent_t* events) {
    if (!plan) return SGS_ERR_INVALID;
    plan->events = events;
    return SGS_OK;
}

sgs_status sgs_read_device_status(const sgs_plan* plan, int32_t* status, cudaStream_t stream) {
    if (!plan || !plan->workspace || !status) return SGS_ERR_INVALID;
    int32_t v = 0;
    SGS_TRY(cudaMemcpyAsync(&v, region<DeviceStatus>(plan, O_STATUS), sizeof(v), cudaMemcpyDeviceToHost, stream));
    SGS_TRY(cudaStreamSynchronize(stream));
    *status = v;
    return SGS_OK;
}

sgs_status sgs_region_info(const sgs_plan* plan, int32_t which, size_t* offset, size_t* bytes) {
    if (!plan || !offset || which < 0 || which >= SGS_REGION_COUNT) return SGS_ERR_INVALID;
    const bool odd = (plan->sort_passes & 1) != 0;
    int r;
    switch (which) {
        case SGS_REGION_STATUS: r = O_STATUS; break;
        case SGS_REGION_REC0: r = O_REC0; break;
        case SGS_REGION_REC1: r = O_REC1; break;
        case SGS_REGION_REC2: r = O_REC2; break;
        case SGS_REGION_RECT: r = O_RECT; break;
        case SGS_REGION_TILES: r = O_TILES; break;
        case SGS_REGION_OFFSETS: r = O_OFFS; break;
        case SGS_REGION_KEYS: r = odd ? O_K1 : O_K0; break;
        case SGS_REGION_VALS: r = odd ? O_V1 : O_V0; break;
        case SGS_REGION_KEYS_IN: r = O_K0; break;
        case SGS_REGION_VALS_IN: r = O_V0; break;
        case SGS_REGION_RANGES: r = O_RANGES; break;
        case SGS_REGION_PIX_T: r = O_PIXT; break;
        case SGS_REGION_PIX_LAST: r = O_PIXLAST; break;
        case SGS_REGION_GRAD2D: r = O_GRAD2D; break;
        case SGS_REGION_PIX_COUNT: r = O_PIXCOUNT; break;
        default: return SGS_ERR_INVALID;
    }
    *offset = plan->offsets[r];
    if (bytes) *bytes = plan->offsets[r + 1] - plan->offsets[r];
    return SGS_OK;
}

sgs_status sgs_sort_temp_bytes(int64_t m, int32_t key_bits, int32_t digit_bits, size_t* bytes) {
    if (!bytes || m < 0 || m > 0xffffffffll || key_bits < 1 || key_bits > 64 || digit_bits < kMinDigitBits ||
        digit_bits > kMaxDigitBits || sort_passes(key_bits, digit_bits) > kMaxSortPasses)
        return SGS_ERR_INVALID;
    int passes, rb;
    sort_digit_plan(0, key_bits, digit_bits, &passes, &rb);
    *bytes = 256 + align256(8 * (size_t)m) + align256(4 * (size_t)m) + 2 * align256(4 * (size_t)kHistEntries) +
             align256(4 * kMaxSortPasses) + align256(8 * sort_lookback_entries(m, rb));
    return SGS_OK;
}

sgs_status sgs_sort_pairs(uint64_t* keys, uint32_t* vals, int64_t m, int32_t key_bits,
                          int32_t digit_bits, void* temp, size_t temp_bytes, cudaStream_t stream) {
    size_t need = 0;
    if (sgs_sort_temp_bytes(m, key_bits, digit_bits, &need) != SGS_OK) return SGS_ERR_INVALID;
    if (m == 0) return SGS_OK;
    if (!keys || !vals || !temp || temp_bytes < need || ((uintptr_t)temp & 255u) != 0) return SGS_ERR_INVALID;
    unsigned char* t = static_cast<unsigned char*>(temp);
    DeviceStatus* st = reinterpret_cast<DeviceStatus*>(t);
    size_t off = 256;
    auto take = [&](size_t b) {
        unsigned char* p = t + off;
        off += align256(b);
        return p;
    };
    unsigned long long* k1 = reinterpret_cast<unsigned long long*>(take(8 * (size_t)m));
    uint32_t* v1 = reinterpret_cast<uint32_t*>(take(4 * (size_t)m));
    int passes, rb;
    sort_digit_plan(0, key_bits, digit_bits, &passes, &rb);
    uint32_t* hist = reinterpret_cast<uint32_t*>(take(4 * (size_t)kHistEntries));
    uint32_t* goff = reinterpret_cast<uint32_t*>(take(4 * (size_t)kHistEntries));
    uint32_t* counters = reinterpret_cast<uint32_t*>(take(4 * kMaxSortPasses));
    unsigned long long* lb = reinterpret_cast<unsigned long long*>(take(8 * sort_lookback_entries(m, rb)));
    unsigned long long* k0 = reinterpret_cast<unsigned long long*>(keys);
    SGS_TRY(launch_sort_init(st, (uint32_t)m, stream));
    SGS_TRY(launch_sort(k0, vals, k1, v1, &st->m_clamped, m, 0, key_bits, digit_bits, hist, goff, counters, lb,
                        st, stream, nullptr));
    if (sort_passes(key_bits, digit_bits) & 1) SGS_TRY(launch_copy_pairs(k1, v1, k0, vals, m, stream));
    return SGS_OK;
}

sgs_status sgs_sort_pairs32(uint32_t* keys, uint32_t* vals, int64_t m, int32_t key_bits,
                            int32_t digit_bits, void* temp, size_t temp_bytes, cudaStream_t stream) {
    size_t need = 0;
    if (key_bits > 32 || sgs_sort_temp_bytes(m, key_bits, digit_bits, &need) != SGS_OK) return SGS_ERR_INVALID;
    if (m == 0) return SGS_OK;
    if (!keys || !vals || !temp || temp_bytes < need || ((uintptr_t)temp & 255u) != 0) return SGS_ERR_INVALID;
    unsigned char* t = static_cast<unsigned char*>(temp);
    DeviceStatus* st = reinterpret_cast<DeviceStatus*>(t);
    size_t off = 256;
    auto take = [&](size_t b) {
        unsigned char* p = t + off;
        off += align256(b);
        return p;
    };
    // the same layout as sgs_sort_pairs (its 8-byte key slots hold 4-byte keys here)
    uint32_t* k1 = reinterpret_cast<uint32_t*>(take(8 * (size_t)m));
    uint32_t* v1 = reinterpret_cast<uint32_t*>(take(4 * (size_t)m));
    int passes, rb;
    sort_digit_plan(0, key_bits, digit_bits, &passes, &rb);
    uint32_t* hist = reinterpret_cast<uint32_t*>(take(4 * (size_t)kHistEntries));
    uint32_t* goff = reinterpret_cast<uint32_t*>(take(4 * (size_t)kHistEntries));
    uint32_t* counters = reinterpret_cast<uint32_t*>(take(4 * kMaxSortPasses));
    unsigned long long* lb = reinterpret_cast<unsigned long long*>(take(8 * sort_lookback_entries(m, rb)));
    SGS_TRY(launch_sort_init(st, (uint32_t)m, stream));
    SGS_TRY(launch_sort(keys, vals, k1, v1, &st->m_clamped, m, 0, key_bits, digit_bits, hist, goff, counters, lb,
                        st, stream, nullptr));
    if (passes & 1) SGS_TRY(launch_copy_pairs(k1, v1, keys, vals, m, stream));
    return SGS_OK;
}

sgs_status sgs_selftest_lookback(const uint64_t* slots, int64_t num_slots, uint64_t* sum,
                                 int32_t* status, cudaStream_t stream) {
    if (num_slots < 0 || !sum || !status || (num_slots > 0 && !slots)) return SGS_ERR_INVALID;
    SGS_TRY(launch_lookback_selftest(reinterpret_cast<const unsigned long long*>(slots), num_slots,
                                     reinterpret_cast<unsigned long long*>(sum), status, stream));
    return SGS_OK;
}

sgs_status sgs_adam_step(const sgs_gaussians* layout, const sgs_grads* raw, const sgs_grads* act,
                         const sgs_grads* grad, const sgs_grads* m, const sgs_grads* v,
                         const sgs_adam_config* cfg, cudaStream_t stream) {
    if (!layout || !raw || !act || !grad || !m || !v || !cfg || check_gaussians(layout) != SGS_OK)
        return SGS_ERR_INVALID;
    if (!(cfg->beta1 >= 0.0f && cfg->beta1 < 1.0f && cfg->beta2 >= 0.0f && cfg->beta2 < 1.0f && cfg->eps >= 0.0f))
        return SGS_ERR_INVALID;
    for (int gi = 0; gi < SGS_GROUP_COUNT; ++gi)
        if (!(cfg->lr[gi] >= 0.0f) || (cfg->lr[gi] > 0.0f && cfg->step[gi] < 1)) return SGS_ERR_INVALID;
    if (layout->n > 0) {
        const sgs_grads* sets[] = {raw, act, grad, m, v};
        for (const sgs_grads* q : sets) {
            const float* need[] = {q->mean, q->scale, q->rot, q->opacity, q->sh};
            for (const float* ptr : need)
                if (!ptr || !aligned16(ptr)) return SGS_ERR_INVALID;
            if (layout->num_lobes > 0 && (!q->sg_amp || !q->sg_sharp || !aligned16(q->sg_amp) || !aligned16(q->sg_sharp)))
                return SGS_ERR_INVALID;
            if (layout->num_lobes > 0 && layout->axis_mode != SGS_AXIS_ORTHO_FIXED &&
                (!q->sg_axis || !aligned16(q->sg_axis)))
                return SGS_ERR_INVALID;
        }
        if (act->scale == raw->scale || act->opacity == raw->opacity) return SGS_ERR_INVALID;
    }
    SGS_TRY(launch_adam(*layout, *raw, *act, *grad, *m, *v, *cfg, stream));
    return SGS_OK;
}

sgs_status sgs_l1_loss(const float* img, const float* target, int64_t count, float* loss,
                       float* dL_dimg, cudaStream_t stream) {
    if (count < 0 || !loss || (count > 0 && (!img || !target || !dL_dimg))) return SGS_ERR_INVALID;
    SGS_TRY(launch_l1_loss(img, target, count, count > 0 ? 1.0f / (float)count : 0.0f, loss, dL_dimg, stream));
    return SGS_OK;
}

sgs_status sgs_l1_loss_scaled(const float* img, const float* target, int64_t count, float scale, float* loss,
                              float* dL_dimg, cudaStream_t stream) {
    if (count < 0 || !loss || (count > 0 && (!img || !target || !dL_dimg)) || !(scale >= 0.0f)) return SGS_ERR_INVALID;
    SGS_TRY(launch_l1_loss(img, target, count, scale, loss, dL_dimg, stream));
    return SGS_OK;
}

}  // extern "C"
