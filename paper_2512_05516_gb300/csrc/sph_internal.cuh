// Internal declarations of libsph: the context, the workspace plan, the
// storage-format codecs used by every kernel, and the launch wrappers.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cstring>

#include "sph.h"

namespace sph {

constexpr int kRadixThreads = 256;
constexpr int kRadixItems = 8;
constexpr int kRadixTile = kRadixThreads * kRadixItems;   // keys per block per pass
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;      // elements per scan block
constexpr int kItemTile = 32;                              // i-particles per pair-kernel work item (one warp)
constexpr int kMaxSub = 2;                                 // sub-cells per cell edge, at most
constexpr int kMaxBlock = 256;
constexpr int kItemClasses = 32;                           // power-of-two cost classes of work items
constexpr int kMaxCellsPerAxis = 4096;                     // the binning caps n_c per axis here
constexpr float kSigma = 0.318309886183790671538f;        // 1/pi, 3D M4 normalisation
constexpr int kLevelMin = SPH_LEVEL_MIN;                   // coarsest level allowed (4 cells per axis)
constexpr int kLevelMax = SPH_LEVEL_MAX;                   // finest level: 3 x 10 key bits

// Morton (Z-order) keys of 10-bit cell coordinates: bit b of x, y, z goes to
// bit 3b, 3b + 1, 3b + 2.  Spreading by shifted masks (each step doubles the
// gap between the bit groups) is the usual bit-interleave construction.
__host__ __device__ __forceinline__ uint32_t morton_spread(uint32_t v)
{
    v &= 0x3FFu;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}
__host__ __device__ __forceinline__ uint32_t morton_compact(uint32_t v)
{
    v &= 0x09249249u;
    v = (v | (v >> 2)) & 0x030C30C3u;
    v = (v | (v >> 4)) & 0x0300F00Fu;
    v = (v | (v >> 8)) & 0x030000FFu;
    v = (v | (v >> 16)) & 0x3FFu;
    return v;
}
__host__ __device__ __forceinline__ uint32_t morton_key(uint32_t x, uint32_t y, uint32_t z)
{
    return morton_spread(x) | (morton_spread(y) << 1) | (morton_spread(z) << 2);
}

inline int ncomp(int f) { return (f == SPH_F_X || f == SPH_F_V || f == SPH_F_A) ? 3 : 1; }

// Device-resident counters and queue heads (lives in the workspace).
struct DevStats {
    unsigned long long pairs_density;
    unsigned long long pairs_force;
    unsigned long long tests_density;
    unsigned long long tests_force;
    unsigned long long hcap_clamps;
    unsigned int error_bits;
    unsigned int queue;          // persistent work-queue head (zeroed before each launch)
    int nitems;                  // pair-kernel work items of the current binning
    int max_occ;                 // particles in the fullest cell
    unsigned int defer_n;        // level hierarchy: targets gathered one by one, and their queue head
    unsigned int defer_q;
    unsigned int heavy_n;        // ... and those of them sent on to the block-wide pass
    unsigned int heavy_q;
    int pad[2];
    // level hierarchy: per level, the particles computed there (final) and
    // those moved from it to the next coarser level
    unsigned long long lvl_done[kLevelMax + 1];
    unsigned long long lvl_promoted[kLevelMax + 1];
};

// Byte offsets of every workspace array.
struct Plan {
    size_t keys[2], vals[2];
    size_t cell_count, cell_start, scan_part, ghist;
    size_t item_cell, item_first, item_count, item_tmp, item_sorted, item_class, class_hist;
    size_t nngb, nngb_force, dflags, stage, aos_tmp, stats, key_hmax, origin, pack, buf_origin;
    size_t level, level_tmp, tlist, tcode, tscan, iscan, lstart, lpack;   // level hierarchy (SPH_WS_LEVELS)
    size_t cidx;                 // level hierarchy: coarse indexes of the sorted keys
    int32_t cidx_lc;             // ... over the cells of this level (8^cidx_lc of them)
    size_t soa[SPH_NFIELDS][3];
    size_t total;
    int64_t item_max, nblk_radix;
};

bool make_plan(const sph_aos_layout &L, int64_t n, int64_t ncell_max, uint32_t ws_flags, Plan *p);

// Launch shape of a persistent kernel, computed once per tuning so that no
// attribute or occupancy query runs while a stream is being captured.
struct LaunchCache {
    size_t smem = 0;
    int block = 0;
    int per_sm_req = -1;
    int grid = 0;
};

// Per-field view handed to kernels: the SoA arrays, the storage format and
// the decode factor 2^-e of the field's power-of-two storage scale.
struct FieldRef {
    void *p[3];
    int fmt;
    float dec;
};

// ---------------------------------------------------------------------------
// storage-format codecs (Table 2 and bfloat16).  All formats decode to FP32.
// ---------------------------------------------------------------------------
// truncated FP32 with n mantissa bits at any width (SPH_P_FP32_TRUNC(n))
__host__ __device__ inline bool fmt_trunc_any(int fmt)
{
    return fmt >= SPH_P_FP32_TRUNC(SPH_P_FP32_TRUNC_MIN) && fmt <= SPH_P_FP32_TRUNC(SPH_P_FP32_TRUNC_MAX);
}
__host__ __device__ inline int fmt_bits(int fmt)
{
    if (fmt_trunc_any(fmt)) return 9 + (fmt - 100);
    switch (fmt) {
    case SPH_P_BF16: case SPH_P_FP16: return 16;
    case SPH_P_FP32_M16: return 25;
    case SPH_P_FP32_M10: return 19;
    default: return 32;
    }
}
__host__ __device__ inline bool fmt_packed(int fmt)
{
    return fmt == SPH_P_FP32_M16 || fmt == SPH_P_FP32_M10 || fmt_trunc_any(fmt);
}

// bit casts usable on both sides (the host-side conversion shares the encoders)
__host__ __device__ __forceinline__ uint32_t f32_bits(float f)
{
#ifdef __CUDA_ARCH__
    return __float_as_uint(f);
#else
    uint32_t u;
    std::memcpy(&u, &f, sizeof(u));
    return u;
#endif
}
__host__ __device__ __forceinline__ float f32_from_bits(uint32_t u)
{
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float f;
    std::memcpy(&f, &u, sizeof(f));
    return f;
#endif
}

__host__ __device__ __forceinline__ float dec_bf16(uint16_t b) { return f32_from_bits((uint32_t)b << 16); }

// round to nearest, ties to even, on the upper 16 bits; NaN stays a quiet NaN
__host__ __device__ __forceinline__ uint16_t enc_bf16(float f)
{
    uint32_t u = f32_bits(f);
    if ((u & 0x7F800000u) == 0x7F800000u && (u & 0x7FFFFFu)) return (uint16_t)((u >> 16) | 0x40u);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

// truncated single: keep the top B bits (sign, exponent, B-9 mantissa bits)
__host__ __device__ __forceinline__ uint32_t enc_trunc(float f, int B)
{
    uint32_t u = f32_bits(f);
    if ((u & 0x7F800000u) == 0x7F800000u && (u & 0x7FFFFFu)) u |= 0x400000u;
    return u >> (32 - B);
}

__device__ __forceinline__ float ld_packed(const uint32_t *__restrict__ w, int64_t k, int B)
{
    int64_t bit = k * (int64_t)B;
    int64_t wi = bit >> 5;
    int sh = (int)(bit & 31);
    uint32_t lo = __ldg(w + wi);
    uint32_t hi = (sh + B > 32) ? __ldg(w + wi + 1) : 0u;
    uint32_t code = __funnelshift_r(lo, hi, sh) & ((1u << B) - 1u);
    return __uint_as_float(code << (32 - B));
}

__device__ __forceinline__ float ld_val(const void *p, int fmt, int64_t k)
{
    switch (fmt) {
    case SPH_P_BF16: return dec_bf16(__ldg((const unsigned short *)p + k));
    case SPH_P_FP16: return __half2float(__ushort_as_half(__ldg((const unsigned short *)p + k)));
    case SPH_P_FP32_M16: return ld_packed((const uint32_t *)p, k, 25);
    case SPH_P_FP32_M10: return ld_packed((const uint32_t *)p, k, 19);
    default:
        if (fmt_trunc_any(fmt)) return ld_packed((const uint32_t *)p, k, fmt_bits(fmt));
        return __ldg((const float *)p + k);
    }
}

// element store for the non-packed formats
__device__ __forceinline__ void st_val(void *p, int fmt, int64_t k, float v)
{
    switch (fmt) {
    case SPH_P_BF16: ((uint16_t *)p)[k] = enc_bf16(v); break;
    case SPH_P_FP16: ((__half *)p)[k] = __float2half_rn(v); break;
    default: ((float *)p)[k] = v; break;
    }
}

// Warp-cooperative store into a packed stream.  All 32 lanes must call it
// together with consecutive k whose warp base (k - lane) is a multiple of 32;
// lanes with valid == false contribute zero bits.  The 32 codes of the warp
// fill exactly B words starting at word (base/32)*B; words at or beyond
// `nwords` are not written.
__device__ __forceinline__ void st_packed_warp(uint32_t *w, int64_t k, float v, bool valid,
                                               int B, int64_t nwords)
{
    const int lane = threadIdx.x & 31;
    const int64_t base = k - lane;
    uint32_t code = valid ? enc_trunc(v, B) : 0u;
    const int j = lane;                  // word j of this warp's B-word block
    const int v0 = (32 * j) / B;
    const int v1 = (32 * j + 31) / B;
    uint32_t word = 0u;
    // a word holds parts of at most floor(31 / B) + 2 values (5 at B = 10);
    // the bound is warp-uniform, so every lane runs the same shuffles
    const int nt = 31 / B + 2;
#pragma unroll
    for (int t = 0; t < 5; ++t) {
        if (t >= nt) break;
        int src = v0 + t;
        uint32_t cv = __shfl_sync(0xffffffffu, code, src < 32 ? src : 31);
        if (j < B && src <= v1 && src < 32) {
            int pos = src * B - 32 * j;  // bit position of value src inside word j
            word |= pos >= 0 ? (cv << pos) : (cv >> (-pos));
        }
    }
    int64_t wi = (base >> 5) * B + j;
    if (j < B && wi < nwords) w[wi] = word;
}

__device__ __forceinline__ void st_any(void *p, int fmt, int64_t k, float v, bool valid,
                                       int64_t n)
{
    if (fmt_packed(fmt)) {
        const int B = fmt_bits(fmt);
        st_packed_warp((uint32_t *)p, k, v, valid, B, (n * B + 31) / 32);
    } else if (valid) {
        st_val(p, fmt, k, v);
    }
}

__device__ __forceinline__ void set_error(DevStats *s, unsigned bits) { atomicOr(&s->error_bits, bits); }

// ---------------------------------------------------------------------------
// FP64 <-> FP32 conversions on the integer pipes.  On this GPU FP64
// instructions (conversions included) issue at a small fraction of the FP32
// rate, and the memory-bound kernels would be bound by them.  These follow
// the IEEE 754 definitions: binary32 -> binary64 is exact (re-bias the
// exponent, widen the mantissa); binary64 -> binary32 rounds to nearest,
// ties to even.  Values outside the normal binary32 range (zeros excepted)
// take the hardware conversion: they are rare.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double f2d_bits(float f)
{
    const uint32_t u = __float_as_uint(f);
    const uint32_t e = (u >> 23) & 0xFFu;
    const uint32_t s = u & 0x80000000u;
    if (e - 1u > 253u) {                                   // zero, subnormal, inf, nan
        if ((u & 0x7FFFFFFFu) == 0u) return __hiloint2double((int)s, 0);
        if (e == 0u) return (double)f;                     // subnormal: rare
        return __hiloint2double((int)(s | 0x7FF00000u | ((u & 0x7FFFFFu) >> 3)), (int)(u << 29));
    }
    // re-bias the exponent (+896) and widen the mantissa: 32-bit halves only
    const uint32_t hi = s | (((u & 0x7FFFFFFFu) >> 3) + (896u << 20));
    return __hiloint2double((int)hi, (int)(u << 29));
}

__device__ __forceinline__ float d2f_bits_rn(double d)
{
    const uint32_t lo = (uint32_t)__double2loint(d);
    const uint32_t hi = (uint32_t)__double2hiint(d);
    const uint32_t e = (hi >> 20) & 0x7FFu;
    if (e - 897u > 253u) {                                 // not a normal float
        if (((hi & 0x7FFFFFFFu) | lo) == 0u) return __uint_as_float(hi & 0x80000000u);     // +-0
        return __double2float_rn(d);                       // rare
    }
    // bits 31..23 of w: the exponent's low 9 bits; 22..0: the top 23 mantissa
    // bits; e - 896 = (low 9 bits - 0x180) mod 512 lies in [1, 254]
    const uint32_t w = __funnelshift_l(lo, hi, 3);
    uint32_t r = (w - (0x180u << 23)) | (hi & 0x80000000u);
    // round half to even on the 29 dropped bits; a carry moves into the
    // exponent (up to infinity)
    r += ((lo & 0x1FFFFFFFu) + 0x0FFFFFFFu + (r & 1u)) >> 29;
    return __uint_as_float(r);
}

}  // namespace sph

// ---------------------------------------------------------------------------
// The context (host side).
// ---------------------------------------------------------------------------
struct sph_ctx {
    sph_aos_layout layout;
    sph_params params;
    int64_t n = 0, ncell_max = 0;
    uint32_t ws_flags = 0;
    uint8_t *aos = nullptr;
    bool aos_device = false;      // the records are in device memory (not host-mapped)
    uint8_t *ws = nullptr;
    size_t ws_bytes = 0;
    cudaStream_t stream = nullptr;
    int device = 0, sm_count = 0;
    size_t smem_optin = 0;
    sph_tuning tuning{};
    sph::Plan plan{};

    // cell grid of the last binning
    int32_t nc[3] = {0, 0, 0};
    double edge[3] = {0, 0, 0};
    double inv[3] = {0, 0, 0};
    int64_t ncell = 0;
    int sub = 1;                  // sub-cells per cell edge of the last binning
    bool binned = false;
    // keys[0] holds the cell key of every record's position as the last
    // kick/drift wrote it, on the grid dk_nc / dk_sub (sph_bin_cells may
    // use them when the caller asks)
    bool drift_keys = false;
    int32_t dk_nc[3] = {0, 0, 0};
    int32_t dk_sub = 0;
    int32_t buffer = 0;           // buffer mode: records taken in buffers of this size (0: cell lists)
    bool levels = false;          // level mode: Morton order over a hierarchy of grids
    bool levels_fixed = false;    // level mode: the density fixed the levels (every h within its cap)
    int32_t lvl_min = 0, lvl_max = 0;
    sph::LaunchCache lc_density, lc_force;   // launch shapes of the persistent pair kernels
    sph::LaunchCache lc_density_lv, lc_density_one, lc_force_lv, lc_force_one;   // ... and over the level hierarchy
    sph::LaunchCache lc_density_blk, lc_force_blk;   // ... the block-wide per-target passes
    int sorted_buf = 0;          // which ping-pong buffer holds the sorted keys/values

    // workspace arrays
    int32_t *keys[2] = {nullptr, nullptr};
    int32_t *vals[2] = {nullptr, nullptr};
    int32_t *cell_count = nullptr, *cell_start = nullptr, *scan_part = nullptr;
    uint32_t *ghist = nullptr;
    int32_t *item_cell = nullptr, *item_first = nullptr, *item_count = nullptr, *item_tmp = nullptr;
    int32_t *item_sorted = nullptr;   // 3 x item_max: the items in queue order, while sorting
    int32_t *item_class = nullptr;    // cost class of every item
    int32_t *class_hist = nullptr;    // per class: count, start (kItemClasses + 1), cursor
    bool items_by_class = false;      // the last binning grouped the items by cost class
    int32_t *nngb = nullptr, *nngb_force = nullptr;
    uint8_t *dflags = nullptr;    // per-slot flags of the last density call (SPH_PFLAG_*)
    float *stage = nullptr;
    float *key_hmax = nullptr;    // largest h of every sub-cell (force pruning)
    double *origin = nullptr;     // cell origins k * (L_d / nc_d), kMaxCellsPerAxis per axis
    double *buf_origin = nullptr; // buffer mode: first position of every buffer, 3 x nbuf, axis-major
    float4 *pack = nullptr;       // 3 x n: the force's packed FP32 inputs per slot
    uint8_t *aos_tmp = nullptr;
    // level hierarchy: level of every slot, of every particle before the
    // sort, and one level's target slots, their cell codes and two scans
    int8_t *level = nullptr, *level_tmp = nullptr;
    int32_t *tlist = nullptr, *tcode = nullptr, *tscan = nullptr, *iscan = nullptr;
    int32_t *lstart = nullptr;    // start of every level's list (force), kLevelMax + 2 entries
    float4 *lpack = nullptr;      // 3 x n: the force's pack arrays in the order of the level lists
    // coarse indexes of sorted finest-cell keys: entry q of a table is the
    // first index whose key lies in coarse cell q or later (8^cs_lc + 1
    // entries, a table every cs_stride): table 0 over all slots (after
    // sph_bin_levels), table 1 + j over the force's list of level
    // lvl_min + j.  They bound the binary searches of the level kernels.
    int32_t *cidx = nullptr;
    int32_t cs_lc = 0;            // coarse level of the slots' table (<= the plan's, <= lvl_max)
    int32_t cl_lc = 0;            // ... of the force lists' tables (at most 6: they are rebuilt every force)
    int64_t cs_stride = 0;
    sph::DevStats *dstats = nullptr;
    void *soa[SPH_NFIELDS][3] = {};
    int prec[SPH_NFIELDS] = {};
    int32_t scale_exp[SPH_NFIELDS] = {};   // storage scale 2^e of every field
    uint32_t valid = 0;
    uint64_t launches = 0;        // kernels launched through this context
    cudaEvent_t kev[2][2] = {};   // timing hooks around the density and force pair kernels

    int32_t *perm() const { return vals[sorted_buf]; }
    float enc(int f) const { return ldexpf(1.0f, scale_exp[f]); }     // value -> stored
    float dec(int f) const { return ldexpf(1.0f, -scale_exp[f]); }    // stored -> value
    int32_t *slot_cell() const { return keys[sorted_buf]; }
};

namespace sph {
// launch wrappers (each returns the first CUDA error, or cudaSuccess)
cudaError_t run_binning(sph_ctx *c, int reorder, bool drift_keys);
cudaError_t run_items(sph_ctx *c);
cudaError_t run_aos_to_soa(sph_ctx *c, uint32_t fields);
cudaError_t run_soa_to_aos(sph_ctx *c, uint32_t fields);
cudaError_t run_density(sph_ctx *c, int newton_steps);
cudaError_t run_force(sph_ctx *c);
cudaError_t run_kick_drift(sph_ctx *c, double dt_kick, double dt_drift, uint32_t wb_fields);
// level hierarchy (k_bin.cu, k_pairs.cu)
cudaError_t run_bin_levels(sph_ctx *c, double grow);
cudaError_t run_level_items(sph_ctx *c, int level);
cudaError_t run_level_lists(sph_ctx *c, int32_t *plist, int32_t *pkey);
// coarse index tables (sph_ctx::cidx) of `nlist` sorted key lists over the
// 8^lc cells of level lc: with bounds == null one list [0, n); else list j
// is [bounds[j], bounds[j + 1])
cudaError_t run_coarse_index(sph_ctx *c, const int32_t *keys, const int32_t *bounds, int nlist, int lc,
                             int32_t *tables);
cudaError_t run_force_levels(sph_ctx *c);
cudaError_t run_density_levels(sph_ctx *c, int newton_steps);
// host-side conversion (host_convert.cu)
size_t host_stage_bytes(const sph_ctx *c);
cudaError_t run_aos_to_soa_host(sph_ctx *c, const uint8_t *host_aos, uint32_t fields, uint8_t *stage,
                                int32_t nthreads);
cudaError_t run_soa_to_aos_host(sph_ctx *c, uint8_t *host_aos, uint32_t fields, uint8_t *stage, int32_t nthreads);
// buffer mode (k_buffers.cu)
cudaError_t run_bin_buffers(sph_ctx *c);
cudaError_t run_buffer_density(sph_ctx *c, int source);
cudaError_t run_buffer_force(sph_ctx *c, int source);
cudaError_t run_buffer_kick(sph_ctx *c, int source, double dt);
cudaError_t run_buffer_drift(sph_ctx *c, int source, double dt);
cudaError_t scan_exclusive(const int32_t *in, int32_t *out, int64_t len, int32_t *part,
                           cudaStream_t s, uint64_t *launches);
int max_dynamic_smem(const sph_ctx *c);
// binning over explicit buffers (used by the allocation-free entry point)
struct BinRaw {
    const uint8_t *aos;
    int64_t n;
    int32_t stride, xoff;
    double inv[3], box[3];
    int32_t nc[3];
    int64_t ncell;
    int32_t *keys[2], *vals[2];
    int32_t *count, *scan_part;
    uint32_t *ghist;
    DevStats *st;
    int32_t *out_perm, *out_cell, *out_start;
};
cudaError_t bin_raw(const BinRaw &b, cudaStream_t s);
size_t density_smem_bytes(int block_threads, int stage_cap, bool levels = false);
size_t force_smem_bytes(int block_threads, int stage_cap);
}  // namespace sph
