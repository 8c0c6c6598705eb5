// C-ABI entry points of libsph: argument validation, the workspace plan, and
// dispatch to the kernels.  Every argument error is caught here, before any
// device work is issued.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include "sph_internal.cuh"

using namespace sph;

namespace {

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

bool layout_ok(const sph_aos_layout *L)
{
    if (!L || L->record_bytes <= 0 || L->record_bytes % 8 != 0 || L->record_bytes > 512) return false;
    if (L->offset[SPH_F_X] < 0 || L->type[SPH_F_X] != SPH_AOS_F64) return false;
    for (int f = 0; f < SPH_NFIELDS; ++f) {
        if (L->offset[f] < 0) continue;
        if (L->type[f] != SPH_AOS_F64 && L->type[f] != SPH_AOS_F32) return false;
        int es = L->type[f] == SPH_AOS_F64 ? 8 : 4;
        if (L->offset[f] % es != 0) return false;
        if (L->offset[f] + es * ncomp(f) > L->record_bytes) return false;
    }
    return true;
}

bool params_ok(const sph_params *p)
{
    if (!p) return false;
    for (int k = 0; k < 3; ++k)
        if (!(p->box[k] > 0.0) || !std::isfinite(p->box[k])) return false;
    if (!(p->gamma > 1.0) || !(p->eta > 0.0) || !(p->h_max > 0.0)) return false;
    if (!(p->alpha_av >= 0.0) || !(p->beta_av >= 0.0) || !(p->eps_av >= 0.0)) return false;
    return true;
}

// which storage formats each SoA field accepts
bool fmt_allowed(int f, int fmt)
{
    if ((fmt < SPH_P_FP32 || fmt > SPH_P_FP32_M10) && !fmt_trunc_any(fmt)) return false;
    switch (f) {
    case SPH_F_X: return fmt == SPH_P_FP32 || fmt == SPH_P_FP16;
    case SPH_F_V: case SPH_F_M: case SPH_F_H: case SPH_F_U: return true;
    case SPH_F_A: case SPH_F_DUDT: return fmt == SPH_P_FP32;    // the force writes, kick/drift reads, FP32
    default: return !fmt_packed(fmt);
    }
}

void default_tuning(sph_tuning *t)
{
    // the autotuner's choice on the 1M-particle Sod step (GB300): density
    // prefers a stage that holds a whole neighbourhood, force more resident
    // warps, and the costliest work items go first
    t->block_threads = 32;
    t->block_threads_force = 32;
    t->ctas_per_sm = 0;
    t->stage_density = 128;
    t->stage_force = 128;
    t->subcells = 2;
    t->item_order = 1;
    t->class_launches = 0;
    t->pair_kernel = 0;
}

}  // namespace

namespace sph {

bool make_plan(const sph_aos_layout &L, int64_t n, int64_t ncell_max, uint32_t ws_flags, Plan *p)
{
    if (n < 0 || n > (int64_t)INT32_MAX / 2 || ncell_max < 27 || ncell_max > (int64_t)INT32_MAX / 2)
        return false;
    std::memset(p, 0, sizeof(*p));
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    const size_t N = (size_t)n;
    for (int b = 0; b < 2; ++b) {
        p->keys[b] = take(4 * N);
        p->vals[b] = take(4 * N);
    }
    const int64_t nkeys = ncell_max * kMaxSub * kMaxSub * kMaxSub;   // sub-cells
    p->cell_count = take(4 * (size_t)nkeys);
    p->cell_start = take(4 * ((size_t)nkeys + 1));
    p->nblk_radix = (n + kRadixTile - 1) / kRadixTile;
    p->ghist = take(4 * (256 * (size_t)p->nblk_radix + 1));  // +1: the scan writes its total
    int64_t scan_len = 256 * p->nblk_radix;
    if (nkeys + 1 > scan_len) scan_len = nkeys + 1;
    if ((ws_flags & SPH_WS_LEVELS) && n + 1 > scan_len) scan_len = n + 1;   // per-slot scans of a level
    p->scan_part = take(4 * ((size_t)(scan_len + kScanTile - 1) / kScanTile + 2));
    // items of one binning: n/32 full tiles plus one partial tile per cell;
    // a level of the hierarchy may have a partial tile per particle
    const bool lv = (ws_flags & SPH_WS_LEVELS) != 0;
    p->item_max = n / 32 + (lv ? n : (n < ncell_max ? n : ncell_max)) + 1;
    p->item_cell = take(4 * (size_t)p->item_max);
    p->item_first = take(4 * (size_t)p->item_max);
    p->item_count = take(4 * (size_t)p->item_max);
    p->item_tmp = take(4 * ((size_t)ncell_max + 1));
    p->item_sorted = take(4 * 3 * (size_t)p->item_max);
    p->item_class = take(4 * (size_t)p->item_max);
    p->class_hist = take(4 * 3 * (kItemClasses + 1));
    p->nngb = take(4 * N);
    p->nngb_force = take(4 * N);
    p->dflags = take(N);
    p->stage = take(4 * N);
    p->key_hmax = take(4 * (size_t)nkeys);
    p->origin = take(sizeof(double) * 3 * kMaxCellsPerAxis);
    p->pack = take(3 * 16 * N);
    p->buf_origin = take(sizeof(double) * 3 * (N / 32 + 1));    // buffers of >= 32 records
    p->aos_tmp = (ws_flags & SPH_WS_REORDER) ? take((size_t)L.record_bytes * N) : 0;
    if (lv) {
        p->level = take(N);
        p->level_tmp = take(N);
        p->tlist = take(4 * N);
        p->tcode = take(4 * N);
        p->tscan = take(4 * (N + 1));
        p->iscan = take(4 * (N + 1));
        p->lstart = take(4 * (kLevelMax + 2));
        p->lpack = take(3 * 16 * N);
        // coarse indexes: at most 8^7 cells, and no more cells than particles
        p->cidx_lc = 1;
        while (p->cidx_lc < 7 && ((int64_t)1 << (3 * (p->cidx_lc + 1))) <= n) ++p->cidx_lc;
        p->cidx = take(4 * (size_t)(1 + SPH_LEVELS_MAX) * (((size_t)1 << (3 * p->cidx_lc)) + 1));
    }
    p->stats = take(sizeof(DevStats));
    for (int f = 0; f < SPH_NFIELDS; ++f)
        for (int c = 0; c < 3; ++c)
            p->soa[f][c] = c < ncomp(f) ? take(4 * N + 64) : 0;
    p->total = off;
    return true;
}

int max_dynamic_smem(const sph_ctx *c) { return (int)c->smem_optin; }

}  // namespace sph

extern "C" {

size_t sph_workspace_bytes(const sph_aos_layout *layout, int64_t n, int64_t ncell_max,
                           uint32_t ws_flags)
{
    if (!layout_ok(layout)) return 0;
    Plan p;
    if (!make_plan(*layout, n, ncell_max, ws_flags, &p)) return 0;
    return p.total;
}

sph_status sph_create(const sph_aos_layout *layout, const sph_params *params, int64_t n,
                      int64_t ncell_max, uint32_t ws_flags, void *d_aos, void *d_workspace,
                      size_t workspace_bytes, void *stream, sph_ctx **out)
{
    if (!out) return SPH_EINVAL;
    *out = nullptr;
    if (!layout_ok(layout) || !params_ok(params) || (!d_aos && n > 0) || !d_workspace) return SPH_EINVAL;
    if (((uintptr_t)d_aos & 15) != 0 || ((uintptr_t)d_workspace & 255) != 0) return SPH_EINVAL;
    Plan plan;
    if (!make_plan(*layout, n, ncell_max, ws_flags, &plan)) return SPH_EINVAL;
    if (workspace_bytes < plan.total) return SPH_ENOSPACE;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SPH_ECUDA;
    int sms = 0, optin = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return SPH_ECUDA;

    sph_ctx *c = new (std::nothrow) sph_ctx();
    if (!c) return SPH_ENOSPACE;
    c->layout = *layout;
    c->params = *params;
    c->n = n;
    c->ncell_max = ncell_max;
    c->ws_flags = ws_flags;
    c->aos = (uint8_t *)d_aos;
    if (d_aos) {
        cudaPointerAttributes pa;
        if (cudaPointerGetAttributes(&pa, d_aos) != cudaSuccess) {
            cudaGetLastError();
            delete c;
            return SPH_EINVAL;
        }
        c->aos_device = pa.type == cudaMemoryTypeDevice;
    }
    c->ws = (uint8_t *)d_workspace;
    c->ws_bytes = workspace_bytes;
    c->stream = (cudaStream_t)stream;
    c->device = dev;
    c->sm_count = sms;
    c->smem_optin = (size_t)optin;
    c->plan = plan;
    default_tuning(&c->tuning);
    uint8_t *w = c->ws;
    for (int b = 0; b < 2; ++b) {
        c->keys[b] = (int32_t *)(w + plan.keys[b]);
        c->vals[b] = (int32_t *)(w + plan.vals[b]);
    }
    c->cell_count = (int32_t *)(w + plan.cell_count);
    c->cell_start = (int32_t *)(w + plan.cell_start);
    c->scan_part = (int32_t *)(w + plan.scan_part);
    c->ghist = (uint32_t *)(w + plan.ghist);
    c->item_cell = (int32_t *)(w + plan.item_cell);
    c->item_first = (int32_t *)(w + plan.item_first);
    c->item_count = (int32_t *)(w + plan.item_count);
    c->item_tmp = (int32_t *)(w + plan.item_tmp);
    c->item_sorted = (int32_t *)(w + plan.item_sorted);
    c->item_class = (int32_t *)(w + plan.item_class);
    c->class_hist = (int32_t *)(w + plan.class_hist);
    c->nngb = (int32_t *)(w + plan.nngb);
    c->nngb_force = (int32_t *)(w + plan.nngb_force);
    c->dflags = (uint8_t *)(w + plan.dflags);
    c->stage = (float *)(w + plan.stage);
    c->key_hmax = (float *)(w + plan.key_hmax);
    c->origin = (double *)(w + plan.origin);
    c->pack = (float4 *)(w + plan.pack);
    c->buf_origin = (double *)(w + plan.buf_origin);
    c->aos_tmp = (ws_flags & SPH_WS_REORDER) ? w + plan.aos_tmp : nullptr;
    if (ws_flags & SPH_WS_LEVELS) {
        c->level = (int8_t *)(w + plan.level);
        c->level_tmp = (int8_t *)(w + plan.level_tmp);
        c->tlist = (int32_t *)(w + plan.tlist);
        c->tcode = (int32_t *)(w + plan.tcode);
        c->tscan = (int32_t *)(w + plan.tscan);
        c->iscan = (int32_t *)(w + plan.iscan);
        c->lpack = (float4 *)(w + plan.lpack);
        c->cidx = (int32_t *)(w + plan.cidx);
        c->cs_stride = ((int64_t)1 << (3 * plan.cidx_lc)) + 1;
        c->lstart = (int32_t *)(w + plan.lstart);
    }
    c->dstats = (DevStats *)(w + plan.stats);
    for (int f = 0; f < SPH_NFIELDS; ++f) {
        c->prec[f] = SPH_P_FP32;
        for (int k = 0; k < ncomp(f); ++k) c->soa[f][k] = w + plan.soa[f][k];
    }
    if (cudaMemsetAsync(c->dstats, 0, sizeof(DevStats), c->stream) != cudaSuccess) {
        delete c;
        return SPH_ECUDA;
    }
    *out = c;
    return SPH_OK;
}

sph_status sph_bin_cells(sph_ctx *c, double cell_edge, int32_t flags)
{
    if (!c || !(std::isfinite(cell_edge) || cell_edge <= 0.0)) return SPH_EINVAL;
    if (flags & ~(SPH_BIN_REORDER | SPH_BIN_DRIFT_KEYS)) return SPH_EINVAL;
    const bool reorder_aos = (flags & SPH_BIN_REORDER) != 0;
    if (reorder_aos && !c->aos_tmp) return SPH_ENOSPACE;
    double want = 2.0 * c->params.h_max;
    if (cell_edge > want) want = cell_edge;
    int32_t nc[3];
    int64_t ncell = 1;
    for (int k = 0; k < 3; ++k) {
        double f = std::floor(c->params.box[k] / want);
        if (f < 3.0) return SPH_ECAPACITY;
        if (f > (double)kMaxCellsPerAxis) f = kMaxCellsPerAxis;  // larger cells still cover 2 h_max
        nc[k] = (int32_t)f;
        ncell *= nc[k];
    }
    if (ncell > c->ncell_max) return SPH_ENOSPACE;
    for (int k = 0; k < 3; ++k) {
        c->nc[k] = nc[k];
        c->inv[k] = (double)nc[k] / c->params.box[k];
        c->edge[k] = c->params.box[k] / (double)nc[k];
    }
    c->ncell = ncell;
    c->sub = c->tuning.subcells;
    c->valid = 0;
    c->binned = false;
    c->buffer = 0;
    c->levels = false;
    // the drift's keys serve when the caller vouches for the records and the
    // grid is the one they were computed on
    const bool dk = (flags & SPH_BIN_DRIFT_KEYS) && c->drift_keys && c->dk_sub == c->sub && c->dk_nc[0] == nc[0] &&
                    c->dk_nc[1] == nc[1] && c->dk_nc[2] == nc[2];
    c->drift_keys = false;
    if (run_binning(c, reorder_aos ? 1 : 0, dk) != cudaSuccess) return SPH_ECUDA;
    if (run_items(c) != cudaSuccess) return SPH_ECUDA;
    c->binned = true;
    return SPH_OK;
}

sph_status sph_aos_to_soa(sph_ctx *c, uint32_t fields, const int32_t *prec)
{
    if (!c) return SPH_EINVAL;
    if (fields == 0 || (fields >> SPH_NFIELDS) != 0) return SPH_EINVAL;
    for (int f = 0; f < SPH_NFIELDS; ++f) {
        if (!(fields & SPH_BIT(f))) continue;
        if (c->layout.offset[f] < 0) return SPH_EINVAL;
        int fmt = prec ? prec[f] : SPH_P_FP32;
        if (!fmt_allowed(f, fmt)) return SPH_EINVAL;
    }
    if (!c->binned) return SPH_ESTATE;
    for (int f = 0; f < SPH_NFIELDS; ++f)
        if (fields & SPH_BIT(f)) c->prec[f] = prec ? prec[f] : SPH_P_FP32;
    if (run_aos_to_soa(c, fields) != cudaSuccess) return SPH_ECUDA;
    c->valid |= fields;
    if (fields & SPH_BIT(SPH_F_H)) c->levels_fixed = false;   // h no longer the density's
    return SPH_OK;
}

sph_status sph_set_field_scale(sph_ctx *c, const int32_t *exp2)
{
    if (!c || !exp2) return SPH_EINVAL;
    for (int f = 0; f < SPH_NFIELDS; ++f) {
        if (exp2[f] < -SPH_SCALE_MAX_EXP || exp2[f] > SPH_SCALE_MAX_EXP) return SPH_EINVAL;
        if ((f == SPH_F_A || f == SPH_F_DUDT) && exp2[f] != 0) return SPH_EINVAL;
    }
    for (int f = 0; f < SPH_NFIELDS; ++f) {
        if (c->scale_exp[f] != exp2[f]) c->valid &= ~SPH_BIT(f);   // stored under the old scale
        c->scale_exp[f] = exp2[f];
    }
    return SPH_OK;
}

size_t sph_host_stage_bytes(const sph_ctx *c) { return c ? host_stage_bytes(c) : 0; }

sph_status sph_aos_to_soa_host(sph_ctx *c, const void *host_aos, uint32_t fields, const int32_t *prec,
                               void *host_stage, size_t stage_bytes, int32_t nthreads)
{
    if (!c || (!host_aos && c->n > 0) || (!host_stage && c->n > 0)) return SPH_EINVAL;
    if (fields == 0 || (fields >> SPH_NFIELDS) != 0) return SPH_EINVAL;
    for (int f = 0; f < SPH_NFIELDS; ++f) {
        if (!(fields & SPH_BIT(f))) continue;
        if (c->layout.offset[f] < 0) return SPH_EINVAL;
        if (!fmt_allowed(f, prec ? prec[f] : SPH_P_FP32)) return SPH_EINVAL;
    }
    if (stage_bytes < host_stage_bytes(c)) return SPH_ENOSPACE;
    if (!c->binned) return SPH_ESTATE;
    for (int f = 0; f < SPH_NFIELDS; ++f)
        if (fields & SPH_BIT(f)) c->prec[f] = prec ? prec[f] : SPH_P_FP32;
    if (run_aos_to_soa_host(c, (const uint8_t *)host_aos, fields, (uint8_t *)host_stage, nthreads) != cudaSuccess)
        return SPH_ECUDA;
    c->valid |= fields;
    if (fields & SPH_BIT(SPH_F_H)) c->levels_fixed = false;
    return SPH_OK;
}

sph_status sph_soa_to_aos_host(sph_ctx *c, void *host_aos, uint32_t fields, void *host_stage, size_t stage_bytes,
                               int32_t nthreads)
{
    if (!c || (!host_aos && c->n > 0) || (!host_stage && c->n > 0)) return SPH_EINVAL;
    if (fields == 0 || (fields >> SPH_NFIELDS) != 0) return SPH_EINVAL;
    if ((fields & SPH_BIT(SPH_F_X)) && !c->buffer) return SPH_EINVAL;
    for (int f = 0; f < SPH_NFIELDS; ++f)
        if ((fields & SPH_BIT(f)) && c->layout.offset[f] < 0) return SPH_EINVAL;
    if (stage_bytes < host_stage_bytes(c)) return SPH_ENOSPACE;
    if (!c->binned) return SPH_ESTATE;
    if ((c->valid & fields) != fields) return SPH_ESTATE;
    if (fields & SPH_BIT(SPH_F_X)) c->drift_keys = false;
    if (run_soa_to_aos_host(c, (uint8_t *)host_aos, fields, (uint8_t *)host_stage, nthreads) != cudaSuccess)
        return SPH_ECUDA;
    return SPH_OK;
}

sph_status sph_get_field_scale(const sph_ctx *c, int32_t *exp2_out)
{
    if (!c || !exp2_out) return SPH_EINVAL;
    for (int f = 0; f < SPH_NFIELDS; ++f) exp2_out[f] = c->scale_exp[f];
    return SPH_OK;
}

sph_status sph_density(sph_ctx *c, int32_t newton_steps)
{
    if (!c || newton_steps < 0 || newton_steps > 32) return SPH_EINVAL;
    if (!c->binned || c->buffer || c->levels) return SPH_ESTATE;
    const uint32_t need = SPH_BIT(SPH_F_X) | SPH_BIT(SPH_F_M) | SPH_BIT(SPH_F_H);
    if ((c->valid & need) != need) return SPH_ESTATE;
    // outputs keep their current format; packed outputs are not supported for
    // rho / P / c (fmt_allowed), h may be packed (written through the stage)
    if (run_density(c, newton_steps) != cudaSuccess) return SPH_ECUDA;
    c->valid |= SPH_BIT(SPH_F_RHO) | SPH_BIT(SPH_F_H);
    if (c->valid & SPH_BIT(SPH_F_U)) c->valid |= SPH_BIT(SPH_F_P) | SPH_BIT(SPH_F_CS);
    return SPH_OK;
}

sph_status sph_force(sph_ctx *c)
{
    if (!c) return SPH_EINVAL;
    if (!c->binned || c->buffer || c->levels) return SPH_ESTATE;
    const uint32_t need = SPH_BIT(SPH_F_X) | SPH_BIT(SPH_F_V) | SPH_BIT(SPH_F_M) |
                          SPH_BIT(SPH_F_H) | SPH_BIT(SPH_F_RHO) | SPH_BIT(SPH_F_P) |
                          SPH_BIT(SPH_F_CS);
    if ((c->valid & need) != need) return SPH_ESTATE;
    c->prec[SPH_F_A] = SPH_P_FP32;
    c->prec[SPH_F_DUDT] = SPH_P_FP32;
    if (run_force(c) != cudaSuccess) return SPH_ECUDA;
    c->valid |= SPH_BIT(SPH_F_A) | SPH_BIT(SPH_F_DUDT);
    return SPH_OK;
}

namespace {

// after a kick/drift on the cell grid: keys[0] holds the keys of the new
// positions (run_kick_drift writes them there on that grid)
void note_drift_keys(sph_ctx *c)
{
    if (!c->binned || c->levels || c->buffer != 0) return;
    c->drift_keys = true;
    for (int k = 0; k < 3; ++k) c->dk_nc[k] = c->nc[k];
    c->dk_sub = c->sub;
}

}  // namespace

sph_status sph_kick_drift(sph_ctx *c, double dt_kick, double dt_drift)
{
    if (!c || !std::isfinite(dt_kick) || !std::isfinite(dt_drift)) return SPH_EINVAL;
    if (!c->binned) return SPH_ESTATE;
    const uint32_t need = SPH_BIT(SPH_F_V) | SPH_BIT(SPH_F_A) | SPH_BIT(SPH_F_U) |
                          SPH_BIT(SPH_F_DUDT);
    if ((c->valid & need) != need) return SPH_ESTATE;
    c->drift_keys = false;
    if (run_kick_drift(c, dt_kick, dt_drift, 0) != cudaSuccess) return SPH_ECUDA;
    note_drift_keys(c);
    c->valid &= ~SPH_BIT(SPH_F_X);   // SoA positions are stale after the drift
    return SPH_OK;
}

sph_status sph_kick_drift_writeback(sph_ctx *c, double dt_kick, double dt_drift, uint32_t fields)
{
    if (!c || !std::isfinite(dt_kick) || !std::isfinite(dt_drift)) return SPH_EINVAL;
    if (fields == 0 || (fields >> SPH_NFIELDS) != 0 || (fields & SPH_BIT(SPH_F_X))) return SPH_EINVAL;
    for (int f = 0; f < SPH_NFIELDS; ++f)
        if ((fields & SPH_BIT(f)) && c->layout.offset[f] < 0) return SPH_EINVAL;
    if (!c->binned) return SPH_ESTATE;
    const uint32_t need = SPH_BIT(SPH_F_V) | SPH_BIT(SPH_F_A) | SPH_BIT(SPH_F_U) | SPH_BIT(SPH_F_DUDT) | fields;
    if ((c->valid & need) != need) return SPH_ESTATE;
    c->drift_keys = false;
    if (run_kick_drift(c, dt_kick, dt_drift, fields) != cudaSuccess) return SPH_ECUDA;
    note_drift_keys(c);
    c->valid &= ~(SPH_BIT(SPH_F_X) | SPH_BIT(SPH_F_V) | SPH_BIT(SPH_F_U));   // kicked values went to the AoS only
    return SPH_OK;
}

sph_status sph_soa_to_aos(sph_ctx *c, uint32_t fields)
{
    if (!c) return SPH_EINVAL;
    if (fields == 0 || (fields >> SPH_NFIELDS) != 0) return SPH_EINVAL;
    if ((fields & SPH_BIT(SPH_F_X)) && !c->buffer) return SPH_EINVAL;   // positions: buffer mode only
    for (int f = 0; f < SPH_NFIELDS; ++f)
        if ((fields & SPH_BIT(f)) && c->layout.offset[f] < 0) return SPH_EINVAL;
    if (!c->binned) return SPH_ESTATE;
    if ((c->valid & fields) != fields) return SPH_ESTATE;
    if (fields & SPH_BIT(SPH_F_X)) c->drift_keys = false;
    if (run_soa_to_aos(c, fields) != cudaSuccess) return SPH_ECUDA;
    return SPH_OK;
}

sph_status sph_bin_buffers(sph_ctx *c, int32_t buffer_size)
{
    if (!c) return SPH_EINVAL;
    if (buffer_size < SPH_BUFFER_MIN || buffer_size > SPH_BUFFER_MAX || (buffer_size & (buffer_size - 1)))
        return SPH_EINVAL;
    c->valid = 0;
    c->binned = false;
    c->drift_keys = false;
    c->buffer = buffer_size;
    c->levels = false;
    if (run_bin_buffers(c) != cudaSuccess) return SPH_ECUDA;
    c->binned = true;
    return SPH_OK;
}

namespace {

// h_l = min_d (box_d / 2^l) / 2: the largest h whose support fits a level-l
// cell (exact in FP64: a power-of-two scaling)
double level_cap(const sph_ctx *c, int l)
{
    double e = std::ldexp(c->params.box[0], -l);
    for (int k = 1; k < 3; ++k) e = std::fmin(e, std::ldexp(c->params.box[k], -l));
    return 0.5 * e;
}

}  // namespace

sph_status sph_bin_levels(sph_ctx *c, int32_t level_min, int32_t level_max, double h_margin)
{
    if (!c) return SPH_EINVAL;
    if (level_min < SPH_LEVEL_MIN || level_max > SPH_LEVEL_MAX || level_min > level_max ||
        level_max - level_min >= SPH_LEVELS_MAX)
        return SPH_EINVAL;
    if (!std::isfinite(h_margin) || !(h_margin >= 0.0)) return SPH_EINVAL;
    if (c->layout.offset[SPH_F_H] < 0) return SPH_EINVAL;
    if (!(c->ws_flags & SPH_WS_LEVELS)) return SPH_ENOSPACE;
    if (c->params.h_max > level_cap(c, level_min)) return SPH_ECAPACITY;
    const int32_t F = 1 << level_max;
    for (int k = 0; k < 3; ++k) {
        c->nc[k] = F;
        c->inv[k] = (double)F / c->params.box[k];
        c->edge[k] = c->params.box[k] / (double)F;
    }
    c->ncell = (int64_t)F * F * F;
    c->sub = 1;
    c->valid = 0;
    c->drift_keys = false;
    c->binned = false;
    c->buffer = 0;
    c->levels = true;
    c->levels_fixed = false;
    c->lvl_min = level_min;
    c->lvl_max = level_max;
    c->items_by_class = false;
    if (run_bin_levels(c, 1.0 + h_margin) != cudaSuccess) return SPH_ECUDA;
    c->cs_lc = std::min((int32_t)c->plan.cidx_lc, level_max);
    c->cl_lc = std::min(c->cs_lc, (int32_t)6);
    if (run_coarse_index(c, c->slot_cell(), nullptr, 1, c->cs_lc, c->cidx) != cudaSuccess) return SPH_ECUDA;
    c->binned = true;
    return SPH_OK;
}

sph_status sph_density_levels(sph_ctx *c, int32_t newton_steps)
{
    if (!c || newton_steps < 0 || newton_steps > 32) return SPH_EINVAL;
    if (!c->binned || !c->levels) return SPH_ESTATE;
    const uint32_t need = SPH_BIT(SPH_F_X) | SPH_BIT(SPH_F_M) | SPH_BIT(SPH_F_H);
    if ((c->valid & need) != need) return SPH_ESTATE;
    if (run_density_levels(c, newton_steps) != cudaSuccess) return SPH_ECUDA;
    c->levels_fixed = true;
    c->valid |= SPH_BIT(SPH_F_RHO) | SPH_BIT(SPH_F_H);
    if (c->valid & SPH_BIT(SPH_F_U)) c->valid |= SPH_BIT(SPH_F_P) | SPH_BIT(SPH_F_CS);
    return SPH_OK;
}

sph_status sph_force_levels(sph_ctx *c)
{
    if (!c) return SPH_EINVAL;
    if (!c->binned || !c->levels || !c->levels_fixed) return SPH_ESTATE;
    const uint32_t need = SPH_BIT(SPH_F_X) | SPH_BIT(SPH_F_V) | SPH_BIT(SPH_F_M) | SPH_BIT(SPH_F_H) |
                          SPH_BIT(SPH_F_RHO) | SPH_BIT(SPH_F_P) | SPH_BIT(SPH_F_CS);
    if ((c->valid & need) != need) return SPH_ESTATE;
    c->prec[SPH_F_A] = SPH_P_FP32;
    c->prec[SPH_F_DUDT] = SPH_P_FP32;
    if (run_force_levels(c) != cudaSuccess) return SPH_ECUDA;
    c->valid |= SPH_BIT(SPH_F_A) | SPH_BIT(SPH_F_DUDT);
    return SPH_OK;
}

sph_status sph_level_counts(sph_ctx *c, int64_t *done, int64_t *promoted)
{
    if (!c || !done || !promoted) return SPH_EINVAL;
    DevStats d;
    if (cudaMemcpyAsync(&d, c->dstats, sizeof(d), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
        return SPH_ECUDA;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return SPH_ECUDA;
    for (int l = 0; l <= SPH_LEVEL_MAX; ++l) {
        done[l] = (int64_t)d.lvl_done[l];
        promoted[l] = (int64_t)d.lvl_promoted[l];
    }
    return SPH_OK;
}

namespace {

// a buffer call's checks: the source, the mode, and its inputs (in the
// layout for SPH_SRC_AOS, where its outputs must exist too; current in the
// SoA for SPH_SRC_SOA)
sph_status buffer_call_ok(const sph_ctx *c, int32_t source, uint32_t in, uint32_t out)
{
    if (source != SPH_SRC_AOS && source != SPH_SRC_SOA) return SPH_EINVAL;
    if (source == SPH_SRC_AOS) {
        for (int f = 0; f < SPH_NFIELDS; ++f)
            if (((in | out) & SPH_BIT(f)) && c->layout.offset[f] < 0) return SPH_EINVAL;
    }
    if (!c->binned || !c->buffer) return SPH_ESTATE;
    if (source == SPH_SRC_SOA && (c->valid & in) != in) return SPH_ESTATE;
    return SPH_OK;
}

// after a buffer call: SoA outputs are current; AoS outputs leave their SoA
// copies stale
void buffer_call_done(sph_ctx *c, int32_t source, uint32_t out)
{
    if (source == SPH_SRC_SOA) c->valid |= out;
    else c->valid &= ~out;
}

}  // namespace

sph_status sph_buffer_density(sph_ctx *c, int32_t source)
{
    if (!c) return SPH_EINVAL;
    const uint32_t in = SPH_BIT(SPH_F_X) | SPH_BIT(SPH_F_M) | SPH_BIT(SPH_F_H) | SPH_BIT(SPH_F_U);
    const uint32_t out = SPH_BIT(SPH_F_RHO) | SPH_BIT(SPH_F_P);
    const sph_status st = buffer_call_ok(c, source, in, out);
    if (st != SPH_OK) return st;
    if (run_buffer_density(c, source) != cudaSuccess) return SPH_ECUDA;
    buffer_call_done(c, source, out | SPH_BIT(SPH_F_CS));
    return SPH_OK;
}

sph_status sph_buffer_force(sph_ctx *c, int32_t source)
{
    if (!c) return SPH_EINVAL;
    const uint32_t in = SPH_BIT(SPH_F_X) | SPH_BIT(SPH_F_V) | SPH_BIT(SPH_F_M) | SPH_BIT(SPH_F_H) |
                        SPH_BIT(SPH_F_RHO) | SPH_BIT(SPH_F_P);
    const uint32_t out = SPH_BIT(SPH_F_A) | SPH_BIT(SPH_F_DUDT);
    const sph_status st = buffer_call_ok(c, source, in, out);
    if (st != SPH_OK) return st;
    if (source == SPH_SRC_SOA) {
        c->prec[SPH_F_A] = SPH_P_FP32;
        c->prec[SPH_F_DUDT] = SPH_P_FP32;
    }
    if (run_buffer_force(c, source) != cudaSuccess) return SPH_ECUDA;
    buffer_call_done(c, source, out);
    return SPH_OK;
}

sph_status sph_buffer_kick(sph_ctx *c, int32_t source, double dt)
{
    if (!c || !std::isfinite(dt)) return SPH_EINVAL;
    const uint32_t in = SPH_BIT(SPH_F_V) | SPH_BIT(SPH_F_A) | SPH_BIT(SPH_F_U) | SPH_BIT(SPH_F_DUDT);
    const uint32_t out = SPH_BIT(SPH_F_V) | SPH_BIT(SPH_F_U);
    const sph_status st = buffer_call_ok(c, source, in, out);
    if (st != SPH_OK) return st;
    if (run_buffer_kick(c, source, dt) != cudaSuccess) return SPH_ECUDA;
    buffer_call_done(c, source, out);
    return SPH_OK;
}

sph_status sph_buffer_drift(sph_ctx *c, int32_t source, double dt)
{
    if (!c || !std::isfinite(dt)) return SPH_EINVAL;
    const uint32_t in = SPH_BIT(SPH_F_X) | SPH_BIT(SPH_F_V);
    const uint32_t out = SPH_BIT(SPH_F_X);
    const sph_status st = buffer_call_ok(c, source, in, out);
    if (st != SPH_OK) return st;
    if (run_buffer_drift(c, source, dt) != cudaSuccess) return SPH_ECUDA;
    buffer_call_done(c, source, out);
    return SPH_OK;
}

sph_status sph_get_stats(sph_ctx *c, sph_stats *out)
{
    if (!c || !out) return SPH_EINVAL;
    DevStats d;
    if (cudaMemcpyAsync(&d, c->dstats, sizeof(d), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
        return SPH_ECUDA;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return SPH_ECUDA;
    std::memset(out, 0, sizeof(*out));
    out->pairs_density = d.pairs_density;
    out->pairs_force = d.pairs_force;
    out->tests_density = d.tests_density;
    out->tests_force = d.tests_force;
    out->hcap_clamps = d.hcap_clamps;
    out->error_bits = d.error_bits;
    for (int k = 0; k < 3; ++k) out->ncell[k] = c->nc[k];
    out->nitems = d.nitems;
    out->max_occupancy = d.max_occ;
    out->launches = c->launches;
    if (d.error_bits & (SPH_ERR_NONFINITE | SPH_ERR_OUTSIDE | SPH_ERR_TIMEOUT)) return SPH_ENUMERIC;
    return SPH_OK;
}

sph_status sph_set_kernel_events(sph_ctx *c, int32_t which, void *ev_begin, void *ev_end)
{
    if (!c || (which != SPH_KEV_DENSITY && which != SPH_KEV_FORCE)) return SPH_EINVAL;
    if ((ev_begin == nullptr) != (ev_end == nullptr)) return SPH_EINVAL;
    c->kev[which][0] = (cudaEvent_t)ev_begin;
    c->kev[which][1] = (cudaEvent_t)ev_end;
    return SPH_OK;
}

sph_status sph_reset_stats(sph_ctx *c)
{
    if (!c) return SPH_EINVAL;
    // keep nitems / max_occ (they describe the current binning)
    if (cudaMemsetAsync(c->dstats, 0, offsetof(DevStats, queue), c->stream) != cudaSuccess)
        return SPH_ECUDA;
    const size_t lv = offsetof(DevStats, lvl_done);
    if (cudaMemsetAsync(reinterpret_cast<uint8_t *>(c->dstats) + lv, 0, sizeof(DevStats) - lv, c->stream) !=
        cudaSuccess)
        return SPH_ECUDA;
    return SPH_OK;
}

sph_status sph_set_tuning(sph_ctx *c, const sph_tuning *t)
{
    if (!c || !t) return SPH_EINVAL;
    sph_tuning n = c->tuning;
    if (t->block_threads > 0) {
        if (t->block_threads % 32 != 0 || t->block_threads < 32 || t->block_threads > kMaxBlock)
            return SPH_EINVAL;
        n.block_threads = t->block_threads;
        n.block_threads_force = t->block_threads;
    }
    if (t->block_threads_force > 0) {
        if (t->block_threads_force % 32 != 0 || t->block_threads_force > kMaxBlock) return SPH_EINVAL;
        n.block_threads_force = t->block_threads_force;
    }
    if (t->ctas_per_sm > 0) n.ctas_per_sm = t->ctas_per_sm;
    if (t->stage_density > 0) n.stage_density = t->stage_density;
    if (t->stage_force > 0) n.stage_force = t->stage_force;
    if (t->subcells > 0) {
        if (t->subcells > kMaxSub) return SPH_EINVAL;
        n.subcells = t->subcells;
    }
    if (t->item_order >= 0) {
        if (t->item_order > 1) return SPH_EINVAL;
        n.item_order = t->item_order;
    }
    if (t->class_launches >= 0) {
        if (t->class_launches > 1) return SPH_EINVAL;
        n.class_launches = t->class_launches;
    }
    if (t->pair_kernel >= 0) {
        if (t->pair_kernel > 1) return SPH_EINVAL;
        n.pair_kernel = t->pair_kernel;
    }
    if (n.stage_density < 32 || n.stage_force < 32) return SPH_EINVAL;
    if (n.stage_density > 65535 || n.stage_force > 65535) return SPH_EINVAL;
    if (density_smem_bytes(n.block_threads, n.stage_density, (c->ws_flags & SPH_WS_LEVELS) != 0) > c->smem_optin)
        return SPH_EINVAL;
    if (force_smem_bytes(n.block_threads_force, n.stage_force) > c->smem_optin) return SPH_EINVAL;
    c->tuning = n;
    return SPH_OK;
}

sph_status sph_get_tuning(const sph_ctx *c, sph_tuning *out)
{
    if (!c || !out) return SPH_EINVAL;
    *out = c->tuning;
    return SPH_OK;
}

sph_status sph_describe(const sph_ctx *c, sph_desc *out)
{
    if (!c || !out) return SPH_EINVAL;
    std::memset(out, 0, sizeof(*out));
    out->n = c->n;
    for (int k = 0; k < 3; ++k) {
        out->ncell[k] = c->nc[k];
        out->cell_edge[k] = c->edge[k];
    }
    auto rel = [&](const void *p) { return p ? (int64_t)((const uint8_t *)p - c->ws) : (int64_t)-1; };
    out->off_perm = rel(c->perm());
    out->off_cell_of_slot = rel(c->slot_cell());
    out->off_cell_start = rel(c->cell_start);
    out->off_nngb = rel(c->nngb);
    out->off_nngb_force = rel(c->nngb_force);
    for (int f = 0; f < SPH_NFIELDS; ++f) {
        out->prec[f] = c->prec[f];
        for (int k = 0; k < 3; ++k) out->off_soa[f][k] = k < ncomp(f) ? rel(c->soa[f][k]) : -1;
    }
    out->valid = c->valid;
    out->subcells = c->sub;
    out->off_level = rel(c->level);
    out->off_density_flags = rel(c->dflags);
    return SPH_OK;
}

sph_status sph_aos_upload(sph_ctx *c, const void *host, size_t bytes)
{
    if (!c || !host || bytes > (size_t)c->n * (size_t)c->layout.record_bytes) return SPH_EINVAL;
    c->drift_keys = false;
    if (cudaMemcpyAsync(c->aos, host, bytes, cudaMemcpyDefault, c->stream) != cudaSuccess)
        return SPH_ECUDA;
    return SPH_OK;
}

sph_status sph_aos_download(sph_ctx *c, void *host, size_t bytes)
{
    if (!c || !host || bytes > (size_t)c->n * (size_t)c->layout.record_bytes) return SPH_EINVAL;
    if (cudaMemcpyAsync(host, c->aos, bytes, cudaMemcpyDefault, c->stream) != cudaSuccess)
        return SPH_ECUDA;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return SPH_ECUDA;
    return SPH_OK;
}

void sph_destroy(sph_ctx *c) { delete c; }

const char *sph_status_str(sph_status s)
{
    switch (s) {
    case SPH_OK: return "ok";
    case SPH_EINVAL: return "invalid argument";
    case SPH_ENOSPACE: return "workspace or cell capacity too small";
    case SPH_ECUDA: return "CUDA error";
    case SPH_ESTATE: return "call out of order: an input is not current";
    case SPH_ECAPACITY: return "cell grid unusable (fewer than 3 cells on an axis)";
    case SPH_ETIMEOUT: return "bounded device wait gave up";
    case SPH_ENUMERIC: return "device recorded a numerical condition";
    default: return "unknown status";
    }
}

}  // extern "C"
