// S3-S5: the quadratic SPH kernels (the paper's Density and Force, Section 6),
// as persistent CUDA-core kernels over a work queue of warp-sized items.
//
// Work item = (cell, first slot, count <= 32): a tile of one cell, one lane
// per i-particle.  Inside a cell the particles are ordered by sub-cell, so a
// tile is spatially compact.  Warps are independent: each pops its own item,
// lists the sub-cells of the 27 neighbour cells (periodic) whose box comes
// within reach of the bounding box of its lanes, stages the particles of
// those sub-cells that are themselves within reach into its own shared-memory
// region (converted to FP32 and shifted into the cell's frame: positions are
// cell-relative, so the shift is the neighbour's cell offset times the cell
// edge), and runs the pair loop.  No block-wide barrier is ever taken.  A
// neighbourhood that does not fit the stage is streamed through it in chunks.
//
// Density (Eq. 6, gather form): rho_i = sum_j m_j W(r_ij, h_i), M4 cubic
// spline W = sigma/h^3 w(r/h), support 2h, compensated FP32 sum (Kahan);
// `newton_steps` Newton steps on f(h) = rho(h) - m_i (eta/h)^3 clamped to
// [h/2, 2h] and h_max, then a final sum; EOS P = (gamma-1) rho u,
// c = sqrt(gamma P / rho).  Each lane keeps the list of staged candidates
// within 2 h (1 + skin); the passes walk only that list, and it is rebuilt
// when h outgrows the skin.
//
// Force (Eq. 7 + Monaghan viscosity, Eq. 5 for du/dt), pairs r < h_i + h_j:
//   a_i    -= m_j (P_i/rho_i^2 + P_j/rho_j^2 + Pi_ij) gradW(r_ij, hbar)
//   du_i/dt += m_j (P_i/rho_i^2 + Pi_ij/2) v_ij . gradW
// Each lane first lists its pairs among the staged candidates, then
// evaluates them with every lane busy.
//
// Summation order: every lane accumulates its pairs in staged order
// (stencil cell, sub-cell, slot), whatever the chunking, list or launch
// shape, so results do not depend on the tuning.
#include "k_pair_math.cuh"

namespace sph {
cudaError_t run_pack(sph_ctx *c, const float *src, int f);

namespace {

constexpr unsigned FULL = 0xffffffffu;
#ifndef SPH_FORCE_CAP
#define SPH_FORCE_CAP 128
#endif
constexpr int kForceCap = SPH_FORCE_CAP;                     // force: per-lane pair list entries
constexpr int kForceSlots = kForceCap + 1;                   // plus one scratch slot per lane
#ifndef SPH_DENS_CAP
#define SPH_DENS_CAP 96
#endif
constexpr int kDensCapUni = SPH_DENS_CAP;                    // density: list entries r
constexpr int kDensCapPair = SPH_DENS_CAP / 2;               // density: list entries (r, m)
constexpr int kDensSlots = SPH_DENS_CAP + 2;                 // words per lane, scratch entry included
static_assert(kDensCapUni < kDensSlots && 2 * kDensCapPair + 1 < kDensSlots, "density list scratch entry");
#ifndef SPH_LIST_SKIN
#define SPH_LIST_SKIN 0.01f
#endif
constexpr float kSkin = SPH_LIST_SKIN;                       // list radius = 2 h (1 + skin)
constexpr float kStageSkin = 0.12f;                          // stage radius = 2 max h (1 + skin)
constexpr float kSkinTight = 0.0f;                           // list skin of a lane whose list overflowed
constexpr int kMaxEnt = 27 * kMaxSub * kMaxSub * kMaxSub;    // stencil sub-cells
constexpr int kEntPerLane = (kMaxEnt + 31) / 32;
constexpr int kStageUnroll = 4;                              // 32-candidate batches in flight

struct Common {
    int64_t n;
    int32_t nc[3];
    float edge[3];
    float4 shift[27];                // offset of stencil cell t in the item cell's frame (from edge)
    int sub, s3;                     // sub-cells per cell edge, per cell
    int lg_sub, lg_s3;               // their base-2 logarithms (sub is 1 or 2)
    const int32_t *cell_start;       // indexed by key = cell * s3 + sub-cell
    const int32_t *icell, *ifirst, *icount;
    const int32_t *range;            // [first, last) item of this launch in device memory, or null: all
    DevStats *st;
    FieldRef x, m, h;
    int cap;                         // staged candidates per warp (one streaming round)
    int defer_cap;                   // level density: staged candidates beyond which an item is deferred
    // level hierarchy: cells of one level, particles in Morton order of
    // their finest cell, positions offsets from that cell's origin
    const int32_t *tslot;            // item entry -> slot (null: entry = slot)
    const int32_t *mkey;             // finest-cell Morton key of every slot (null: dense cells)
    int lvl_dn;                      // levels from this one to the finest
    int lvl_n;                       // cells per axis at this level
    int fine_n;                      // cells per axis at the finest level
    float fine_edge[3];
    int32_t *defer;                  // slots of the targets gathered one by one (k_density_one)
    // the per-target passes run twice: one warp per target over `defer`,
    // sending a target whose stream holds more than heavy_at candidates on
    // to `heavy` (phase 0); then a block of warps per target over `heavy`
    // (phase 1)
    int32_t *heavy;
    int heavy_at;
    int one_phase;
    // level force: the finest-cell keys of the per-level lists (every
    // level's slots in Morton order, one list after the other: level l at
    // [lstart[l], lstart[l+1])), and the largest h of each level's particles
    const int32_t *pkey, *lstart;
    int lvl_min, lvl_max;
    // coarse indexes of the sorted keys (cs[q]: the first index in coarse
    // cell q or later, q in [0, cs_C]), for the slots and for each level's
    // force list (table lp - lvl_min), cs_stride apart
    const int32_t *cs_slot, *cs_list;
    int cs_shift, cs_C;              // the slots' table
    int cl_shift, cl_C;              // the lists' tables
    int64_t cs_stride;
    float lcap[kLevelMax + 1];
};

struct DensityArgs {
    Common c;
    FieldRef u;
    bool has_u;
    int npass;                       // newton_steps + 1
    float eta3, h_cap, gm1, gamma;
    bool plain_sum;
    void *rho_out; int rho_fmt;
    void *h_out; int h_fmt;          // h_out may be the FP32 stage when H is packed
    bool write_h;
    void *P_out; int P_fmt;
    void *cs_out; int cs_fmt;
    float rho_enc, h_enc, P_enc, cs_enc;   // storage scales of the outputs
    const float4 *pD;                // every slot's (x, y, z, m) in FP32, from the pack pass
    int32_t *nngb;
    uint8_t *pflags;                 // per-slot SPH_PFLAG_* of this call
    // level hierarchy: this level, and whether a clamped particle moves up
    int8_t *level;
    int lvl;
    bool promote;
};

struct ForceArgs {
    Common c;
    FieldRef v, rho, P, cs;
    const float *key_hmax;           // largest h of every sub-cell
    float alpha, beta, eps, h_cap;
    float *a[3];
    float *dudt;
    int32_t *nngb;
    // every slot's force inputs decoded to FP32 by the pack pass:
    const float4 *pA;                // (x, y, z, h), positions cell-relative
    const float4 *pB;                // (vx, vy, vz, m)
    const float4 *pC;                // (P / rho^2, rho, c, 0)
    // level force: the same three arrays in the order of the per-level
    // lists (entry i holds slot plist[i]; lC's w is that slot), so that a
    // candidate run is read contiguously
    const float4 *lA, *lB, *lC;
    int lvl;                         // level force: the level of this launch's items
};

// The candidate stream of one warp: the kept (non-empty, within reach)
// stencil sub-cells, compacted in stencil order (neighbour cell t, then
// sub-cell), as prefix sums in shared memory.  Stream position g lies in the
// first entry e with incl[e] > g, at slot base[e] + g; t[e] is the entry's
// neighbour cell (for the shift into the item's cell frame).
struct __align__(16) Tab {
    int incl[kMaxEnt];
    int base[kMaxEnt];
    uint8_t t[kMaxEnt];
    int nk;                          // kept entries
};
// Each warp's shared-memory region is stage | lists | table; the next warp's
// float4 stage starts right after, so every part keeps 16-byte multiples.
static_assert(sizeof(Tab) % 16 == 0, "stencil table size must keep 16-byte alignment");
static_assert((32 * kForceSlots * sizeof(uint8_t)) % 16 == 0, "list size must keep 16-byte alignment");
static_assert(kForceCap <= 256, "force list entries are byte offsets into a range of kForceCap candidates");
// staged force candidates are followed by kForcePad far-away entries, so the
// pair tests run whole batches of 8 without bounds checks
constexpr int kForcePad = 8;
static_assert((32 * kDensSlots * sizeof(float)) % 16 == 0, "list size must keep 16-byte alignment");
// level force: an item whose candidate stream is longer than this many
// stages (8192 candidates at the default stage of 128) is gathered target by
// target (k_force_one)
constexpr int kForceDeferStages = 64;
// the level kernel adds the 27 x 9 run boundaries of its item's stencil
constexpr size_t kBndBytes = (27 * 9 * sizeof(int) + 15) / 16 * 16;
// warps per block of the level hierarchy's per-target passes (one target per
// block), fewer when their stages do not fit the shared memory
#ifndef SPH_ONE_WARPS
#define SPH_ONE_WARPS 4
#endif
constexpr int kOneWarps = SPH_ONE_WARPS;
// a target goes from the one-warp pass to the block-wide one when its stream
// holds more candidates than one warp's stage (density) or than this many
// force stages
#ifndef SPH_FORCE_HEAVY_STAGES
#define SPH_FORCE_HEAVY_STAGES 64
#endif
constexpr int kForceHeavyStages = SPH_FORCE_HEAVY_STAGES;
static_assert(kOneWarps >= 1 && kOneWarps * 32 <= kMaxBlock, "per-target block");

__device__ __forceinline__ int pop_item(DevStats *st, int lane)
{
    int it = 0;
    if (lane == 0) it = (int)atomicAdd(&st->queue, 1u);
    return __shfl_sync(FULL, it, 0);
}

__device__ __forceinline__ float warp_max(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(FULL, v, o));
    return v;
}
__device__ __forceinline__ float warp_min(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(FULL, v, o));
    return v;
}
__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

struct Box { float lo[3], hi[3]; };

__device__ __forceinline__ Box warp_box(bool ok, float x, float y, float z)
{
    Box b;
    b.lo[0] = warp_min(ok ? x : 3.0e38f);
    b.lo[1] = warp_min(ok ? y : 3.0e38f);
    b.lo[2] = warp_min(ok ? z : 3.0e38f);
    b.hi[0] = warp_max(ok ? x : -3.0e38f);
    b.hi[1] = warp_max(ok ? y : -3.0e38f);
    b.hi[2] = warp_max(ok ? z : -3.0e38f);
    return b;
}

__device__ __forceinline__ float box_dist2(const Box &b, float x, float y, float z)
{
    float dx = fmaxf(0.0f, fmaxf(b.lo[0] - x, x - b.hi[0]));
    float dy = fmaxf(0.0f, fmaxf(b.lo[1] - y, y - b.hi[1]));
    float dz = fmaxf(0.0f, fmaxf(b.lo[2] - z, z - b.hi[2]));
    return fmaf(dx, dx, fmaf(dy, dy, dz * dz));
}

// offset of stencil cell t (0..26) in the item cell's frame
__device__ __forceinline__ void stencil_shift(const Common &c, int t, float &sx, float &sy, float &sz)
{
    const float4 v = c.shift[t];
    sx = v.x;
    sy = v.y;
    sz = v.z;
}

// List the stencil sub-cells of `cell` whose box comes within reach of the
// warp box (every particle of a sub-cell sits inside its box: positions are
// cell-relative offsets, widened here by a rounding margin).  The reach is
// sqrt(R2), or, with `key_hmax`, hw + the largest h of the sub-cell.  Returns
// the number of candidates in the stream (warp-uniform).
__device__ int build_stream(const Common &c, int cell, const Box &box, float R2, Tab &tab, int lane,
                            const float *key_hmax = nullptr, float hw = 0.0f)
{
    const int nent = 27 * c.s3;
    const int E = (nent + 31) / 32;            // entries per lane, lane-blocked
    const int kx = cell % c.nc[0];
    const int ky = (cell / c.nc[0]) % c.nc[1];
    const int kz = cell / (c.nc[0] * c.nc[1]);
    int cnt[kEntPerLane], st[kEntPerLane];
    int local = 0;
#pragma unroll
    for (int i = 0; i < kEntPerLane; ++i) {
        cnt[i] = 0;
        st[i] = 0;
        const int e = lane * E + i;
        if (i < E && e < nent) {
            const int t = e >> c.lg_s3, q = e & (c.s3 - 1);
            const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
            int nx = kx + dx, ny = ky + dy, nz = kz + dz;      // periodic wrap, |d| <= 1
            nx += nx < 0 ? c.nc[0] : (nx >= c.nc[0] ? -c.nc[0] : 0);
            ny += ny < 0 ? c.nc[1] : (ny >= c.nc[1] ? -c.nc[1] : 0);
            nz += nz < 0 ? c.nc[2] : (nz >= c.nc[2] ? -c.nc[2] : 0);
            const int key = ((nx + c.nc[0] * (ny + c.nc[1] * nz)) << c.lg_s3) + q;
            const int s0 = c.cell_start[key];
            const int n0 = c.cell_start[key + 1] - s0;
            st[i] = s0;
            if (n0 > 0) {
                const int m1 = c.sub - 1;
                const int qa[3] = {q & m1, (q >> c.lg_sub) & m1, q >> (2 * c.lg_sub)};
                const int da[3] = {dx, dy, dz};
                float d2 = 0.0f;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const float se = c.edge[a] / (float)c.sub;
                    const float margin = c.edge[a] * (1.0f / 512.0f);
                    const float lo = (float)da[a] * c.edge[a] + (float)qa[a] * se - margin;
                    const float hi = lo + se + 2.0f * margin;
                    const float g = fmaxf(0.0f, fmaxf(lo - box.hi[a], box.lo[a] - hi));
                    d2 = fmaf(g, g, d2);
                }
                float reach2 = R2;
                if (key_hmax) {
                    const float rr = hw + key_hmax[key];
                    reach2 = rr * rr;
                }
                if (d2 < reach2) cnt[i] = n0;
            }
        }
        local += cnt[i];
    }
    // prefix sums over the lanes: candidates, and kept entries (compaction)
    int kept = 0;
#pragma unroll
    for (int i = 0; i < kEntPerLane; ++i) kept += cnt[i] > 0 ? 1 : 0;
    int inc = local, kinc = kept;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(FULL, inc, o);
        const int w = __shfl_up_sync(FULL, kinc, o);
        if (lane >= o) {
            inc += v;
            kinc += w;
        }
    }
    int run = inc - local, pos = kinc - kept;
#pragma unroll
    for (int i = 0; i < kEntPerLane; ++i) {
        const int e = lane * E + i;
        if (i < E && e < nent && cnt[i] > 0) {
            run += cnt[i];
            tab.incl[pos] = run;
            tab.base[pos] = st[i] - (run - cnt[i]);
            tab.t[pos] = (uint8_t)(e >> c.lg_s3);
            ++pos;
        }
    }
    if (lane == 31) tab.nk = kinc;
    __syncwarp();
    return __shfl_sync(FULL, inc, 31);
}

// Walk forward from kept entry e to the entry holding stream position g
// (g < total).
__device__ __forceinline__ int advance(const Tab &tab, int nk, int e, int g)
{
    while (e < nk - 1 && tab.incl[e] <= g) ++e;
    return e;
}

// ---------------------------------------------------------------------------
// Level hierarchy: a candidate's position in the item cell's frame, and the
// candidate stream of the 27 cells of the item's level
// ---------------------------------------------------------------------------

// Slot position p (offset from its finest cell, FP32) moved into the frame
// whose origin is the finest cell `org`: + (periodic cell difference) x
// finest edge, one rounding per axis.  Every stencil particle lies within
// [-2^dn, 2^(dn+1)) finest cells of the origin (level >= 2), inside the
// wrap window [-F/2, F/2).
__device__ __forceinline__ float4 lvl_frame(const Common &c, uint32_t key, int3 org, float4 p)
{
    const int hf = c.fine_n >> 1, m = c.fine_n - 1;
    const int dx = (((int)morton_compact(key) - org.x + hf) & m) - hf;
    const int dy = (((int)morton_compact(key >> 1) - org.y + hf) & m) - hf;
    const int dz = (((int)morton_compact(key >> 2) - org.z + hf) & m) - hf;
    return make_float4(__fmaf_rn((float)dx, c.fine_edge[0], p.x), __fmaf_rn((float)dy, c.fine_edge[1], p.y),
                       __fmaf_rn((float)dz, c.fine_edge[2], p.z), p.w);
}

// first slot in [lo, hi) whose key is >= v (keys ascend)
__device__ __forceinline__ int key_lower_bound(const int32_t *key, int lo, int hi, int32_t v)
{
    while (lo < hi) {
        const int mid = lo + ((hi - lo) >> 1);
        if (__ldg(key + mid) < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// The same, within a sub-range [lo, hi) of a sorted list whose coarse index
// is cs: the answer over the whole list lies in [cs[q], cs[q + 1]] for v's
// coarse cell q, so the search runs over that bracket only (none at all when
// v opens a coarse cell) and the answer is then clamped to [lo, hi).
__device__ __forceinline__ int key_lower_bound_cs(const int32_t *key, int lo, int hi, int32_t v, const int32_t *cs,
                                                  int shift, int C)
{
    const int q = min(C, (int)((uint32_t)v >> shift));
    const int A = __ldg(cs + q), B = __ldg(cs + min(q + 1, C));
    const int a = max(A, lo), b = min(B, hi);
    if (a >= b) return min(max(A, lo), hi);
    return key_lower_bound(key, a, b, v);
}

// Slot runs of the 27 cells of the item's level around `cell` (its Morton
// code at that level), periodic, and of their 8 children at the next level:
// a cell of level l is the run of keys with its code as prefix, found by
// binary search; its children are sub-runs found inside it.  Lane t < 27
// writes the 9 boundaries of stencil cell t to bnd[9t .. 9t+8] (children
// 0..7 span [bnd[9t+q], bnd[9t+q+1])).  At the finest level there are no
// children: child 0 is the whole cell and 1..7 are empty.  Computed once
// per work item; the candidate tables below only prune them.
__device__ void lvl_bounds(const Common &c, int cell, int *bnd, int lane)
{
    if (lane < 27) {
        const int da[3] = {lane % 3 - 1, (lane / 3) % 3 - 1, lane / 9 - 1};
        const uint32_t m = (uint32_t)c.lvl_n - 1u, cc = (uint32_t)cell;
        const uint32_t nx = (morton_compact(cc) + (uint32_t)da[0]) & m;
        const uint32_t ny = (morton_compact(cc >> 1) + (uint32_t)da[1]) & m;
        const uint32_t nz = (morton_compact(cc >> 2) + (uint32_t)da[2]) & m;
        const int sh = 3 * c.lvl_dn;
        const int32_t code = (int32_t)morton_key(nx, ny, nz);
        const int s0 = key_lower_bound_cs(c.mkey, 0, (int)c.n, code << sh, c.cs_slot, c.cs_shift, c.cs_C);
        const int e0 = key_lower_bound_cs(c.mkey, s0, (int)c.n, (code + 1) << sh, c.cs_slot, c.cs_shift, c.cs_C);
        int *b = bnd + 9 * lane;
        b[0] = s0;
        b[8] = e0;
        int lo = s0;
#pragma unroll
        for (int q = 1; q < 8; ++q) {
            if (c.lvl_dn > 0 && lo < e0)
                lo = key_lower_bound_cs(c.mkey, lo, e0, ((code << 3) + q) << (sh - 3), c.cs_slot, c.cs_shift, c.cs_C);
            else lo = c.lvl_dn > 0 ? lo : e0;
            b[q] = lo;
        }
    }
    __syncwarp();
}

// As build_stream, from the runs of lvl_bounds: the children (or, at the
// finest level, the cells) whose box comes within reach sqrt(R2) of `box`,
// compacted in (stencil cell, child) order.  Returns the candidate count.
__device__ int lvl_table(const Common &c, const int *bnd, const Box &box, float R2, Tab &tab, int lane)
{
    int cnt[8], st[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        cnt[q] = 0;
        st[q] = 0;
    }
    if (lane < 27) {
        const int da[3] = {lane % 3 - 1, (lane / 3) % 3 - 1, lane / 9 - 1};
        const bool kids = c.lvl_dn > 0;
        float lo[3];
        float d2 = 0.0f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float margin = c.edge[a] * (1.0f / 512.0f);
            lo[a] = (float)da[a] * c.edge[a] - margin;
            const float g = fmaxf(0.0f, fmaxf(lo[a] - box.hi[a], box.lo[a] - (lo[a] + c.edge[a] + 2.0f * margin)));
            d2 = fmaf(g, g, d2);
        }
        if (d2 < R2) {
            const int *b = bnd + 9 * lane;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int s0 = b[q], e0 = b[q + 1];
                if (e0 <= s0) continue;
                float g2 = 0.0f;
                if (kids) {
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        const float half = 0.5f * c.edge[a], margin = c.edge[a] * (1.0f / 512.0f);
                        const float l0 = lo[a] + (float)((q >> a) & 1) * half;
                        const float g = fmaxf(0.0f, fmaxf(l0 - box.hi[a], box.lo[a] - (l0 + half + 2.0f * margin)));
                        g2 = fmaf(g, g, g2);
                    }
                }
                if (g2 < R2) {
                    cnt[q] = e0 - s0;
                    st[q] = s0;
                }
            }
        }
    }
    int local = 0, kept = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        local += cnt[q];
        kept += cnt[q] > 0 ? 1 : 0;
    }
    int inc = local, kinc = kept;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(FULL, inc, o);
        const int w = __shfl_up_sync(FULL, kinc, o);
        if (lane >= o) {
            inc += v;
            kinc += w;
        }
    }
    int run = inc - local, pos = kinc - kept;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        if (cnt[q] > 0) {
            run += cnt[q];
            tab.incl[pos] = run;
            tab.base[pos] = st[q] - (run - cnt[q]);
            tab.t[pos] = (uint8_t)lane;
            ++pos;
        }
    }
    if (lane == 31) tab.nk = kinc;
    __syncwarp();
    return __shfl_sync(FULL, inc, 31);
}

// ---------------------------------------------------------------------------
// Density
// ---------------------------------------------------------------------------

// density pass accumulators of one lane
struct DAcc {
    float s, c;      // compensated sum of m w (s - c)
    float d;         // sum of m (3w + q w') / 3
    float n;         // pairs with r < 2h, self included (exact: far below 2^24)
};

// The separation of a candidate from (xi, yi, zi), as every density path
// forms it: r = r^2 rsqrt(r^2), 0 for the self pair.
__device__ __forceinline__ float pair_r(float xi, float yi, float zi, const float4 q)
{
    const float dx = xi - q.x, dy = yi - q.y, dz = zi - q.z;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    return r2 * rsqrt_normal(r2 + 1.0e-30f);
}

// One pair of a density pass from its separation r: the spline at q = r/h,
// m_j w into the (compensated) sum, on Newton passes the dh term
// m_j (3w + q w') / 3 = m_j (w + q (u^2 - p^2)), and the neighbour count
// (q < 2, i.e. p > 0: the pairs the spline gives weight; sat(p 2^100) is 1
// for every p > 0, as p >= 2^-24 then).  With one mass for every pair (mj = 1
// here and the sums scaled by m afterwards) the multiplications by m fold
// away.
template <bool kPlain, bool kDeriv>
__device__ __forceinline__ void dens_acc(DAcc &a, float r, float hinv, float mj)
{
    const float qq = r * hinv;
    const SplineTerms t = spline_terms(qq);
    const float w = fmaf(t.p2 + t.p2, t.p, -(t.u2 * t.u));
    const float mw = mj * w;
    if (kPlain) a.s += mw;
    else kahan_add(a.s, a.c, mw);
    if (kDeriv) a.d = fmaf(mj, fmaf(qq, t.u2 - t.p2, w), a.d);
    a.n += __saturatef(t.p * 1.2676506e30f);
}

__device__ __forceinline__ void dens_acc_rt(DAcc &a, float r, float hinv, float mj, bool plain, bool deriv)
{
    if (plain) {
        if (deriv) dens_acc<true, true>(a, r, hinv, mj);
        else dens_acc<true, false>(a, r, hinv, mj);
    } else {
        if (deriv) dens_acc<false, true>(a, r, hinv, mj);
        else dens_acc<false, false>(a, r, hinv, mj);
    }
}

// A position in the candidate stream and the table entry holding it.
struct Cursor {
    int g, e;
};

// The density's stage holds its candidates in pairs: candidate e's (x, y, z,
// m) are the floats 8 (e / 2) + (e % 2) + {0, 2, 4, 6}, so that candidates 2k
// and 2k + 1 load as packed pairs (x0, x1, y0, y1), (z0, z1, m0, m1) with two
// 16-byte loads.  A stage of cap float4 holds cap candidates (cap even).
__device__ __forceinline__ void stage_put(float4 *sj, int e, float4 v)
{
    float *f = reinterpret_cast<float *>(sj) + 8 * (e >> 1) + (e & 1);
    f[0] = v.x;
    f[2] = v.y;
    f[4] = v.z;
    f[6] = v.w;
}

__device__ __forceinline__ float4 stage_get(const float4 *sj, int e)
{
    const float *f = reinterpret_cast<const float *>(sj) + 8 * (e >> 1) + (e & 1);
    return make_float4(f[0], f[2], f[4], f[6]);
}

// Stage the stream's candidates within distance sqrt(R2) of the warp box, in
// stream order, starting at `cur`, until the stage is full or the stream ends.
// Returns how many were staged (<= cap) and moves `cur` to the first batch
// not staged (cur.g == total when the stream is exhausted).  A chunk always
// stages at least one batch, since a batch holds at most 32 <= cap.
template <bool kLvl, int kU = kStageUnroll>
__device__ int stage_density(const Common &c, const float4 *pD, const Tab &tab, int total, const Box &box,
                             float R2, float4 *sj, int cap, Cursor &cur, int lane, int3 org, float mref = 0.0f,
                             bool *mixed = nullptr)
{
    const unsigned lt = (1u << lane) - 1u;
    const int nk = tab.nk;
    cap &= ~1;                       // the paired layout holds an even count
    int found = 0;
    int ecur = cur.e;
    for (int g0 = cur.g; g0 < total; g0 += 32 * kU) {
        float4 q[kU];
        int eu[kU];
        int e = ecur;
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int g = g0 + u * 32 + lane;
            q[u] = make_float4(3.0e38f, 3.0e38f, 3.0e38f, 0.0f);
            if (g < total) {
                e = advance(tab, nk, e, g);
                const int64_t j = (int64_t)tab.base[e] + g;
                const float4 p = __ldg(pD + j);
                if (kLvl) {
                    q[u] = lvl_frame(c, (uint32_t)__ldg(c.mkey + j), org, p);
                } else {
                    float sx, sy, sz;
                    stencil_shift(c, tab.t[e], sx, sy, sz);
                    q[u] = make_float4(p.x + sx, p.y + sy, p.z + sz, p.w);
                }
            }
            eu[u] = e;
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const bool keep = box_dist2(box, q[u].x, q[u].y, q[u].z) < R2;
            const unsigned b = __ballot_sync(FULL, keep);
            const int nb = __popc(b);
            if (found + nb > cap) {     // stage full: resume at this batch
                cur.g = g0 + u * 32;
                cur.e = __shfl_sync(FULL, eu[u], 0);
                __syncwarp();
                return found;
            }
            if (keep) {
                stage_put(sj, found + __popc(b & lt), q[u]);
                if (mixed && q[u].w != mref) *mixed = true;
            }
            found += nb;
        }
        ecur = __shfl_sync(FULL, e, 31);
    }
    cur.g = total;
    cur.e = ecur;
    __syncwarp();
    return found;
}

// The density's pack pass: every slot's (x, y, z, m) decoded from their
// storage formats into one FP32 float4, so that staging loads a candidate
// with one 16-byte load.
__global__ void __launch_bounds__(256) k_density_pack(Common c, float4 *pD)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= c.n) return;
    pD[k] = make_float4(ld_val(c.x.p[0], c.x.fmt, k) * c.x.dec, ld_val(c.x.p[1], c.x.fmt, k) * c.x.dec,
                        ld_val(c.x.p[2], c.x.fmt, k) * c.x.dec, ld_val(c.m.p[0], c.m.fmt, k) * c.m.dec);
}

// Shared memory of one density warp: the streaming stage (cap candidates),
// the per-lane lists of separations and the stencil table (plus, in level
// mode, the run boundaries of the item's stencil).
__host__ __device__ inline size_t density_warp_bytes(int cap, bool levels)
{
    return (size_t)cap * sizeof(float4) + (size_t)32 * kDensSlots * sizeof(float) + sizeof(Tab) +
           (levels ? kBndBytes : 0);
}

// A lane's list of separations.  With one mass for every staged candidate
// (`uni`) entry e is r at lr[e * 32 + lane], up to kDensCapUni entries;
// otherwise entry e is the pair (r, m_j) at lr[2e * 32 + lane],
// lr[(2e + 1) * 32 + lane], up to kDensCapPair.  Appends past the capacity
// land in the scratch entry (the count keeps growing, so an overflow is seen).

// One candidate onto a lane's list (branch-free: a candidate that is not
// kept is written to the next entry and overwritten by the next append).
template <bool kUni>
__device__ __forceinline__ void append_one(float *lr, int &n, float r, float m, bool keep, int lane)
{
    constexpr int lcap = kUni ? kDensCapUni : kDensCapPair;
    const int s = min(n, lcap);
    if (kUni) {
        lr[s * 32 + lane] = r;
    } else {
        lr[(2 * s) * 32 + lane] = r;
        lr[(2 * s + 1) * 32 + lane] = m;
    }
    n += keep ? 1 : 0;
}

// Append the staged candidates 0..len-1 with r^2 < R2l to a lane's list, in
// stage order.  Two candidates at a time: their separations in packed FP32
// pairs, each component rounding as pair_r does.
template <bool kUni>
__device__ __forceinline__ int append_list(const float4 *sj, int len, float xi, float yi, float zi, float R2l,
                                           float *lr, int n, int lane)
{
    const float2 XI = make_float2(xi, xi), YI = make_float2(yi, yi), ZI = make_float2(zi, zi);
    int e0 = 0;
    for (; e0 + 4 <= len; e0 += 4) {
        float4 a[2], b[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            a[u] = sj[e0 + 2 * u];          // (x, x', y, y') of candidates e0 + 2u, e0 + 2u + 1
            b[u] = sj[e0 + 2 * u + 1];      // (z, z', m, m')
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const float2 dx = __fadd2_rn(XI, make_float2(-a[u].x, -a[u].y));
            const float2 dy = __fadd2_rn(YI, make_float2(-a[u].z, -a[u].w));
            const float2 dz = __fadd2_rn(ZI, make_float2(-b[u].x, -b[u].y));
            const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
            const float2 t = __fadd2_rn(r2, make_float2(1.0e-30f, 1.0e-30f));
            const float2 r = __fmul2_rn(r2, make_float2(rsqrt_normal(t.x), rsqrt_normal(t.y)));
            append_one<kUni>(lr, n, r.x, b[u].z, r2.x < R2l, lane);
            append_one<kUni>(lr, n, r.y, b[u].w, r2.y < R2l, lane);
        }
    }
    for (; e0 < len; ++e0) {
        const float4 q = stage_get(sj, e0);
        const float r = pair_r(xi, yi, zi, q);
        const float dx = xi - q.x, dy = yi - q.y, dz = zi - q.z;
        append_one<kUni>(lr, n, r, q.w, fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < R2l, lane);
    }
    return n;
}

// Stream the item's candidates within 2 h_list of the lanes with `bld` and
// append each of those lanes' candidates with r < 2 h_list to its list, in
// stream order.  `box` and R2s (the squared reach of the building lanes)
// prune the stream.  `mixed` is set when a staged candidate's mass differs
// from mref (then the lists cannot share one mass).  Returns the staged
// candidate count of the warp, or -1 in level mode once it exceeds
// `defer_at` (the item is deferred).  `stop_at` ends the stream early once
// every building lane has found more entries than that (their lists
// overflow whatever follows).
template <bool kLvl>
__device__ int build_lists(const Common &c, const float4 *pD, Tab &tab, const int *bnd, int cell, const Box &box,
                           float R2s, float4 *sj, int cap, float *lr, bool uni, bool bld, float xi, float yi, float zi,
                           float mref, float R2l, int &n, bool &mixed, int stop_at, int defer_at,
                           unsigned long long &tests, int lane, int3 org)
{
    const int total = kLvl ? lvl_table(c, bnd, box, R2s, tab, lane) : build_stream(c, cell, box, R2s, tab, lane);
    if (bld) n = 0;
    bool mix = false;
    int staged = 0;
    Cursor cur{0, 0};
    do {
        const int len = stage_density<kLvl>(c, pD, tab, total, box, R2s, sj, cap, cur, lane, org, mref, &mix);
        staged += len;
        if (kLvl && staged > defer_at) return -1;
        if (bld) {
            tests += (unsigned long long)len;
            n = uni ? append_list<true>(sj, len, xi, yi, zi, R2l, lr, n, lane)
                    : append_list<false>(sj, len, xi, yi, zi, R2l, lr, n, lane);
        }
        __syncwarp();
        if (__all_sync(FULL, !bld || n > stop_at)) break;
    } while (cur.g < total);
    mixed = __any_sync(FULL, mix);
    return staged;
}

// Two consecutive list entries of a density pass, their spline terms in
// packed FP32 pairs (one instruction for both entries; each component rounds
// as the scalar code does), then accumulated one after the other, entry e
// before e + 1, exactly as two calls of dens_acc would.
template <bool kPlain, bool kDeriv, bool kUni>
__device__ __forceinline__ void dens_acc2(DAcc &a, float2 r, float2 hinv, float2 mj)
{
    const float2 qq = __fmul2_rn(r, hinv);
    const float2 p = make_float2(__saturatef(fmaf(qq.x, -0.5f, 1.0f)), __saturatef(fmaf(qq.y, -0.5f, 1.0f)));
    const float2 u = make_float2(__saturatef(1.0f - qq.x), __saturatef(1.0f - qq.y));
    const float2 p2 = __fmul2_rn(p, p), u2 = __fmul2_rn(u, u);
    const float2 nu3 = __fmul2_rn(u2, make_float2(-u.x, -u.y));           // -(u^2 u), exactly
    const float2 w = __ffma2_rn(__fadd2_rn(p2, p2), p, nu3);
    const float2 mw = kUni ? w : __fmul2_rn(mj, w);
    if (kPlain) {
        a.s += mw.x;
        a.s += mw.y;
    } else {
        kahan_add(a.s, a.c, mw.x);
        kahan_add(a.s, a.c, mw.y);
    }
    if (kDeriv) {
        const float2 g = __ffma2_rn(qq, __fadd2_rn(u2, make_float2(-p2.x, -p2.y)), w);
        if (kUni) {
            a.d = a.d + g.x;
            a.d = a.d + g.y;
        } else {
            a.d = fmaf(mj.x, g.x, a.d);
            a.d = fmaf(mj.y, g.y, a.d);
        }
    }
    a.n += __saturatef(p.x * 1.2676506e30f);
    a.n += __saturatef(p.y * 1.2676506e30f);
}

// One pass over a lane's list, two entries at a time.
template <bool kPlain, bool kDeriv, bool kUni>
__device__ __forceinline__ void list_pass(DAcc &acc, const float *lr, int n, float hinv, int lane)
{
    const float2 hv = make_float2(hinv, hinv);
    int e = 0;
    if (kUni) {
#pragma unroll 2
        for (; e + 2 <= n; e += 2)
            dens_acc2<kPlain, kDeriv, true>(acc, make_float2(lr[e * 32 + lane], lr[(e + 1) * 32 + lane]), hv,
                                            make_float2(1.0f, 1.0f));
        if (e < n) dens_acc<kPlain, kDeriv>(acc, lr[e * 32 + lane], hinv, 1.0f);
    } else {
#pragma unroll 2
        for (; e + 2 <= n; e += 2)
            dens_acc2<kPlain, kDeriv, false>(acc, make_float2(lr[(2 * e) * 32 + lane], lr[(2 * e + 2) * 32 + lane]),
                                             hv, make_float2(lr[(2 * e + 1) * 32 + lane], lr[(2 * e + 3) * 32 + lane]));
        if (e < n) dens_acc<kPlain, kDeriv>(acc, lr[(2 * e) * 32 + lane], hinv, lr[(2 * e + 1) * 32 + lane]);
    }
}

__device__ __forceinline__ void list_pass_rt(DAcc &acc, const float *lr, int n, float hinv, bool plain, bool deriv,
                                             bool uni, int lane)
{
    if (uni) {
        if (plain) {
            if (deriv) list_pass<true, true, true>(acc, lr, n, hinv, lane);
            else list_pass<true, false, true>(acc, lr, n, hinv, lane);
        } else {
            if (deriv) list_pass<false, true, true>(acc, lr, n, hinv, lane);
            else list_pass<false, false, true>(acc, lr, n, hinv, lane);
        }
    } else {
        if (plain) {
            if (deriv) list_pass<true, true, false>(acc, lr, n, hinv, lane);
            else list_pass<true, false, false>(acc, lr, n, hinv, lane);
        } else {
            if (deriv) list_pass<false, true, false>(acc, lr, n, hinv, lane);
            else list_pass<false, false, false>(acc, lr, n, hinv, lane);
        }
    }
}

// Density over the warp work items.  Per item, every lane keeps the list of
// its candidates within 2 h (1 + skin) as separations r (the passes need
// nothing else: the positions do not move during the Newton steps), built by
// streaming the stencil's candidates through a small stage; a lane rebuilds
// its list only when its h outgrows the list radius.  While every listed
// candidate of the item has the mass of the lane that lists it (`uni`, the
// usual case) the lists hold r alone and the sums are scaled by that mass;
// otherwise the item's lists hold (r, m_j) pairs at half the capacity.  A
// lane whose list overflows even at the tight skin sums every pass straight
// from the stream.  Level mode defers an item whose box gathers more than
// `defer_at` staged candidates to the per-target pass (k_density_one).
template <bool kLvl>
__global__ void __launch_bounds__(kMaxBlock, 1) k_density(DensityArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const Common &c = a.c;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float4 *sj = reinterpret_cast<float4 *>(smem + warp * density_warp_bytes(c.cap, kLvl));
    float *lr = reinterpret_cast<float *>(sj + c.cap);
    Tab &tab = *reinterpret_cast<Tab *>(lr + 32 * kDensSlots);
    int *bnd = reinterpret_cast<int *>(&tab + 1);          // level kernel: the item's stencil runs

    unsigned long long my_pairs = 0, my_tests = 0, my_done = 0, my_prom = 0;
    unsigned my_err = 0;
    const int lo = c.range ? c.range[0] : 0;
    const int hi = c.range ? c.range[1] : c.st->nitems;

    for (int it = lo + pop_item(c.st, lane); it < hi; it = lo + pop_item(c.st, lane)) {
        const int cell = c.icell[it];
        const int first = c.ifirst[it];
        const int count = c.icount[it];
        const bool ok = lane < count;
        int64_t k = (int64_t)first + lane;
        int3 org = make_int3(0, 0, 0);       // level mode: the item cell's origin in finest cells
        if (kLvl) {
            k = ok ? (int64_t)__ldg(c.tslot + first + lane) : 0;
            const uint32_t cc = (uint32_t)cell;
            org = make_int3((int)(morton_compact(cc) << c.lvl_dn), (int)(morton_compact(cc >> 1) << c.lvl_dn),
                            (int)(morton_compact(cc >> 2) << c.lvl_dn));
            lvl_bounds(c, cell, bnd, lane);
        }
        bool clamped = false;
        unsigned lf = 0;           // this particle's SPH_PFLAG_* bits
        float xi = 0.f, yi = 0.f, zi = 0.f, mi = 0.f, hi = 0.f, ui = 0.f;
        if (ok) {
            float4 p = __ldg(a.pD + k);
            if (kLvl) p = lvl_frame(c, (uint32_t)__ldg(c.mkey + k), org, p);
            xi = p.x;
            yi = p.y;
            zi = p.z;
            mi = p.w;
            hi = ld_val(c.h.p[0], c.h.fmt, k) * c.h.dec;
            if (a.has_u) ui = ld_val(a.u.p[0], a.u.fmt, k) * a.u.dec;
            if (!(hi > 0.0f) || !isfinite(hi)) { hi = a.h_cap; lf |= SPH_PFLAG_NONFINITE; }
            if (hi > a.h_cap) { hi = a.h_cap; clamped = true; }
        }

        float h_list = 0.0f;       // this lane's list holds every candidate within 2 h_list
        int nl = 0;                // entries in this lane's list (may exceed the capacity)
        bool direct = false;       // list overflowed: every pass sums straight from the stream
        bool uni = true;           // warp-uniform list layout (see build_lists)
        bool per_target = false;
        const float mref = __shfl_sync(FULL, mi, 0);
        float rho = 0.f, drdh = 0.f;
        int cnt = 0;
        unsigned long long lane_pairs = 0;
        for (int pass = 0; pass < a.npass; ++pass) {
            const float hinv = 1.0f / hi;
            const bool deriv = pass + 1 < a.npass;     // the last pass needs no dh term
            // (re)build the lists of the lanes whose h outgrew their list radius
            bool need = ok && !direct && hi > h_list;
            if (__any_sync(FULL, need)) {
                if (need) h_list = fminf(hi * (1.0f + kSkin), a.h_cap);
                for (int round = 0; round < 2; ++round) {
                    const Box bb = warp_box(need, xi, yi, zi);
                    const float hb = 2.0f * warp_max(need ? h_list : 0.0f);
                    const int lc = uni ? kDensCapUni : kDensCapPair;
                    bool mixed = false;
                    const int st = build_lists<kLvl>(c, a.pD, tab, bnd, cell, bb, hb * hb, sj, c.cap, lr, uni, need, xi,
                                                     yi, zi, mref, 4.0f * h_list * h_list, nl, mixed, lc + lc / 4,
                                                     c.defer_cap, my_tests, lane, org);
                    if (kLvl && st < 0) {
                        per_target = true;
                        break;
                    }
                    // a staged candidate of another mass: every list of the
                    // item is rebuilt as (r, m) pairs
                    if (uni && mixed) {
                        uni = false;
                        need = ok && !direct;
                        continue;
                    }
                    break;
                }
                if (per_target) break;
                // overflowing lists: once more with the tight skin, then the stream
                const int lcap = uni ? kDensCapUni : kDensCapPair;
                const bool over = need && nl > lcap;
                if (__any_sync(FULL, over)) {
                    // far above the capacity the tight skin cannot help
                    const bool retry = over && nl <= lcap + lcap / 4;
                    if (over && !retry) direct = true;
                    if (__any_sync(FULL, retry)) {
                        if (retry) h_list = fminf(hi * (1.0f + kSkinTight), a.h_cap);
                        const Box bb = warp_box(retry, xi, yi, zi);
                        const float hb = 2.0f * warp_max(retry ? h_list : 0.0f);
                        bool mixed = false;
                        const int st = build_lists<kLvl>(c, a.pD, tab, bnd, cell, bb, hb * hb, sj, c.cap, lr, uni, retry,
                                                         xi, yi, zi, mref, 4.0f * h_list * h_list, nl, mixed, lcap,
                                                         c.defer_cap, my_tests, lane, org);
                        if (kLvl && st < 0) {
                            per_target = true;
                            break;
                        }
                        if (retry && nl > lcap) direct = true;
                    }
                    // level mode: a lane that would stream every pass (its
                    // frames cost a Morton decode per candidate) sends the
                    // item to the per-target pass instead
                    if (kLvl && __any_sync(FULL, direct)) {
                        per_target = true;
                        break;
                    }
                }
            }
            DAcc acc{0.f, 0.f, 0.f, 0.f};
            if (ok && !direct) {
                my_tests += (unsigned long long)nl;
                list_pass_rt(acc, lr, nl, hinv, a.plain_sum, deriv, uni, lane);
            }
            const bool dl = ok && direct;
            if (__any_sync(FULL, dl)) {
                // lists that overflow: stream the candidates within reach of
                // those lanes through the stage, every pass
                const Box bb = warp_box(dl, xi, yi, zi);
                const float hw = 2.0f * warp_max(dl ? hi : 0.0f);
                const float R2 = hw * hw;
                const int tot = kLvl ? lvl_table(c, bnd, bb, R2, tab, lane) : build_stream(c, cell, bb, R2, tab, lane);
                Cursor sc{0, 0};
                do {
                    const int len = stage_density<kLvl>(c, a.pD, tab, tot, bb, R2, sj, c.cap, sc, lane, org);
                    if (dl) {
                        my_tests += (unsigned long long)len;
                        for (int e = 0; e < len; ++e) {
                            const float4 q = stage_get(sj, e);
                            dens_acc_rt(acc, pair_r(xi, yi, zi, q), hinv, q.w, a.plain_sum, deriv);
                        }
                    }
                    __syncwarp();
                } while (sc.g < tot);
            }
            if (ok) {
                const float h3inv = hinv * hinv * hinv;
                const float ms = (uni && !direct) ? mi : 1.0f;    // the lists' common mass
                rho = kSigma * h3inv * ((acc.s - acc.c) * ms);
                drdh = -3.0f * kSigma * h3inv * hinv * (acc.d * ms);
                cnt = (int)acc.n - 1;      // the self term is in rho, not in the count
                lane_pairs += (unsigned long long)cnt;
                if (pass + 1 < a.npass) {
                    // Newton step on f(h) = rho(h) - m (eta/h)^3
                    const float f = rho - mi * a.eta3 * h3inv;
                    const float fp = drdh + 3.0f * mi * a.eta3 * h3inv * hinv;
                    float hn = hi;
                    if (fp > 0.0f && isfinite(f) && isfinite(fp)) hn = hi - f / fp;
                    else lf |= SPH_PFLAG_NEWTON;
                    hn = fminf(fmaxf(hn, 0.5f * hi), 2.0f * hi);
                    if (hn > a.h_cap) { hn = a.h_cap; clamped = true; }
                    hi = hn;
                }
            }
        }
        if (kLvl && per_target) {
            // The item's box gathers (or, as h grows, comes to gather) more
            // candidates than defer_at: coarse-level targets spread over their
            // cell next to a dense cluster, or started from an h far too large
            // for what surrounds them.  Its targets go to the per-target list
            // and are gathered one by one, each by a warp (a block of warps
            // when its stream outgrows a warp's stage), in the launches that
            // follow (k_density_one); nothing is written here.
            const unsigned bal = __ballot_sync(FULL, ok);
            unsigned base = 0;
            if (lane == 0) base = atomicAdd(&c.st->defer_n, (unsigned)__popc(bal));
            base = __shfl_sync(FULL, base, 0);
            if (ok) c.defer[base + __popc(bal & ((1u << lane) - 1u))] = (int32_t)k;
            continue;
        }

        if (kLvl && ok && clamped && a.promote) {
            // h met this level's cap: the particle moves one level up and is
            // computed again there from its original h (nothing written)
            a.level[k] = (int8_t)(a.lvl - 1);
            ++my_prom;
        } else if (ok) {
            my_pairs += lane_pairs;
            if (kLvl) ++my_done;
            if (!isfinite(rho)) lf |= SPH_PFLAG_NONFINITE;
            if (clamped) lf |= SPH_PFLAG_HCAP;
            a.pflags[k] = (uint8_t)lf;
            if (lf & SPH_PFLAG_NONFINITE) my_err |= SPH_ERR_NONFINITE;
            if (lf & SPH_PFLAG_NEWTON) my_err |= SPH_ERR_NEWTON;
            st_val(a.rho_out, a.rho_fmt, k, rho * a.rho_enc);
            if (a.write_h) st_val(a.h_out, a.h_fmt, k, hi * a.h_enc);
            a.nngb[k] = cnt;
            if (a.has_u) {
                const float P = a.gm1 * rho * ui;
                st_val(a.P_out, a.P_fmt, k, P * a.P_enc);
                st_val(a.cs_out, a.cs_fmt, k, __fsqrt_rn(a.gamma * P / rho) * a.cs_enc);
            }
            if (clamped) {   // each clamped particle counted once per call
                atomicAdd(&c.st->hcap_clamps, 1ull);
                my_err |= SPH_ERR_HCAP;
            }
        }
    }
    my_pairs = warp_sum_u64(my_pairs);
    my_tests = warp_sum_u64(my_tests);
    if (kLvl) {
        my_done = warp_sum_u64(my_done);
        my_prom = warp_sum_u64(my_prom);
    }
    if (lane == 0) {
        if (my_pairs) atomicAdd(&c.st->pairs_density, my_pairs);
        if (my_tests) atomicAdd(&c.st->tests_density, my_tests);
        if (kLvl && my_done) atomicAdd(&c.st->lvl_done[a.lvl], my_done);
        if (kLvl && my_prom) atomicAdd(&c.st->lvl_promoted[a.lvl], my_prom);
    }
    if (my_err) set_error(c.st, my_err);
}

// A warp's share of a candidate stream of `total` positions when the W warps
// of a block split it: [g0, g1), contiguous, in stream order.
__device__ __forceinline__ void stream_slice(int total, int warp, int W, int &g0, int &g1)
{
    g0 = (int)(((long long)total * warp) / W);
    g1 = (int)(((long long)total * (warp + 1)) / W);
}

// Sum of the W warps' partials v[w] (in w order, so every thread gets the
// same bits); `red` is block-shared scratch of kMaxBlock / 32 entries.
__device__ __forceinline__ float block_sum_ordered(float v, float *red, int warp, int lane, int W)
{
    if (lane == 0) red[warp] = v;
    __syncthreads();
    float t = 0.0f;
    for (int w = 0; w < W; ++w) t += red[w];
    __syncthreads();
    return t;
}

// The level kernel's per-target pass: every target of the per-target list
// (k_density deferred it) is gathered by one whole block of W warps.  Its
// stream is pruned to its own reach with the children of the stencil cells
// and split into W contiguous slices, one per warp; a warp's lanes take its
// slice's candidates in turn, the lanes' partial sums meet in a butterfly and
// the warps' in stream order, so every thread holds the same bits and runs
// the same Newton steps.  Heavy targets (thousands of candidates: coarse
// particles next to a cluster) are what this pass gathers, and few are left
// at its end, so each gets W warps.  Staging keeps 8 batches of 32
// candidates in flight (4 in k_density).  Persistent blocks pop targets from
// the list; the outputs, promotion and counters follow k_density's epilogue.
__global__ void __launch_bounds__(kMaxBlock, 1) k_density_one(DensityArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ float red[kMaxBlock / 32];
    __shared__ unsigned next;
    const Common &c = a.c;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
    float4 *sj = reinterpret_cast<float4 *>(smem + warp * density_warp_bytes(c.cap, true));
    // no per-lane lists here: the stage extends over their space
    const int cap1 = c.cap + 32 * kDensSlots * (int)sizeof(float) / (int)sizeof(float4);
    Tab &tab = *reinterpret_cast<Tab *>(sj + cap1);
    int *bnd = reinterpret_cast<int *>(&tab + 1);
    unsigned long long my_pairs = 0, my_tests = 0, my_done = 0, my_prom = 0;
    unsigned my_err = 0;
    const int32_t *list = c.one_phase ? c.heavy : c.defer;
    unsigned *head = c.one_phase ? &c.st->heavy_q : &c.st->defer_q;
    const unsigned nd = c.one_phase ? c.st->heavy_n : c.st->defer_n;
    for (;;) {
        if (threadIdx.x == 0) next = atomicAdd(head, 1u);
        __syncthreads();
        const unsigned j = next;
        __syncthreads();
        if (j >= nd) break;
        const int64_t k = list[j];
        const uint32_t key = (uint32_t)__ldg(c.mkey + k);
        const int cell = (int)(key >> (3 * c.lvl_dn));
        const int3 org = make_int3((int)(morton_compact((uint32_t)cell) << c.lvl_dn),
                                   (int)(morton_compact((uint32_t)cell >> 1) << c.lvl_dn),
                                   (int)(morton_compact((uint32_t)cell >> 2) << c.lvl_dn));
        lvl_bounds(c, cell, bnd, lane);
        const float4 p = lvl_frame(c, key, org, __ldg(a.pD + k));
        const float xt = p.x, yt = p.y, zt = p.z, mt = p.w;
        float ht = ld_val(c.h.p[0], c.h.fmt, k) * c.h.dec;
        bool clamped = false;
        unsigned lf = 0;           // the target's SPH_PFLAG_* bits (the same in every thread)
        if (!(ht > 0.0f) || !isfinite(ht)) {
            ht = a.h_cap;
            lf |= SPH_PFLAG_NONFINITE;
        }
        if (ht > a.h_cap) {
            ht = a.h_cap;
            clamped = true;
        }
        const Box pb{{xt, yt, zt}, {xt, yt, zt}};
        float hs = 0.0f, rt = 0.0f, dt = 0.0f;
        int Tt = 0, nt = 0;
        bool fit_t = false;        // every warp's slice of the stream sits in its stage
        bool sent = false;         // passed on to the block-wide pass
        unsigned long long pt = 0;
        for (int pass = 0; pass < a.npass; ++pass) {
            if (pass == 0 || (fit_t && ht > hs)) {
                hs = fminf(ht * (1.0f + kStageSkin), a.h_cap);
                const float R2p = 4.0f * hs * hs;
                const int tot = lvl_table(c, bnd, pb, R2p, tab, lane);
                if (pass == 0 && c.heavy_at > 0 && tot > c.heavy_at) {
                    if (threadIdx.x == 0) c.heavy[atomicAdd(&c.st->heavy_n, 1u)] = (int32_t)k;
                    sent = true;
                    break;
                }
                int g0, g1;
                stream_slice(tot, warp, W, g0, g1);
                Cursor pc{g0, g0 < g1 ? advance(tab, tab.nk, 0, g0) : 0};
                Tt = stage_density<true, 8>(c, a.pD, tab, g1, pb, R2p, sj, cap1, pc, lane, org);
                fit_t = __syncthreads_and(pc.g >= g1) != 0;
            }
            const float h2x4 = 4.0f * ht * ht;
            const float hinv = 1.0f / ht;
            const bool deriv = pass + 1 < a.npass;
            DAcc acc{0.f, 0.f, 0.f, 0.f};
            if (fit_t) {
                for (int e = lane; e < Tt; e += 32) {
                    const float4 q = stage_get(sj, e);
                    dens_acc_rt(acc, pair_r(xt, yt, zt, q), hinv, q.w, a.plain_sum, deriv);
                }
                my_tests += (unsigned long long)max(0, (Tt - lane + 31) >> 5);
            } else {
                // more than the stages within the target's own reach: stream it
                const int tot = lvl_table(c, bnd, pb, h2x4, tab, lane);
                int g0, g1;
                stream_slice(tot, warp, W, g0, g1);
                Cursor sc{g0, g0 < g1 ? advance(tab, tab.nk, 0, g0) : 0};
                while (sc.g < g1) {
                    const int len = stage_density<true, 8>(c, a.pD, tab, g1, pb, h2x4, sj, cap1, sc, lane, org);
                    for (int e = lane; e < len; e += 32) {
                        const float4 q = stage_get(sj, e);
                        dens_acc_rt(acc, pair_r(xt, yt, zt, q), hinv, q.w, a.plain_sum, deriv);
                    }
                    my_tests += (unsigned long long)max(0, (len - lane + 31) >> 5);
                    __syncwarp();
                }
            }
            float sum = acc.s - acc.c, dsum = acc.d;
            int nn = (int)acc.n;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                sum += __shfl_xor_sync(FULL, sum, o);
                dsum += __shfl_xor_sync(FULL, dsum, o);
                nn += __shfl_xor_sync(FULL, nn, o);
            }
            if (W > 1) {
                sum = block_sum_ordered(sum, red, warp, lane, W);
                dsum = block_sum_ordered(dsum, red, warp, lane, W);
                nn = (int)block_sum_ordered((float)nn, red, warp, lane, W);   // exact: far below 2^24
            }
            const float h3inv = hinv * hinv * hinv;
            rt = kSigma * h3inv * sum;
            dt = -3.0f * kSigma * h3inv * hinv * dsum;
            nt = nn - 1;
            pt += (unsigned long long)nt;
            if (pass + 1 < a.npass) {
                // Newton step on f(h) = rho(h) - m (eta/h)^3, as in k_density
                const float f = rt - mt * a.eta3 * h3inv;
                const float fp = dt + 3.0f * mt * a.eta3 * h3inv * hinv;
                float hn = ht;
                if (fp > 0.0f && isfinite(f) && isfinite(fp)) hn = ht - f / fp;
                else lf |= SPH_PFLAG_NEWTON;
                hn = fminf(fmaxf(hn, 0.5f * ht), 2.0f * ht);
                if (hn > a.h_cap) {
                    hn = a.h_cap;
                    clamped = true;
                }
                ht = hn;
            }
        }
        if (sent || threadIdx.x != 0) continue;
        if (clamped && a.promote) {
            a.level[k] = (int8_t)(a.lvl - 1);
            ++my_prom;
            continue;
        }
        my_pairs += pt;
        ++my_done;
        if (!isfinite(rt)) lf |= SPH_PFLAG_NONFINITE;
        if (clamped) lf |= SPH_PFLAG_HCAP;
        a.pflags[k] = (uint8_t)lf;
        if (lf & SPH_PFLAG_NONFINITE) my_err |= SPH_ERR_NONFINITE;
        if (lf & SPH_PFLAG_NEWTON) my_err |= SPH_ERR_NEWTON;
        st_val(a.rho_out, a.rho_fmt, k, rt * a.rho_enc);
        if (a.write_h) st_val(a.h_out, a.h_fmt, k, ht * a.h_enc);
        a.nngb[k] = nt;
        if (a.has_u) {
            const float ui = ld_val(a.u.p[0], a.u.fmt, k) * a.u.dec;
            const float P = a.gm1 * rt * ui;
            st_val(a.P_out, a.P_fmt, k, P * a.P_enc);
            st_val(a.cs_out, a.cs_fmt, k, __fsqrt_rn(a.gamma * P / rt) * a.cs_enc);
        }
        if (clamped) {
            atomicAdd(&c.st->hcap_clamps, 1ull);
            my_err |= SPH_ERR_HCAP;
        }
    }
    my_tests = warp_sum_u64(my_tests);
    if (lane == 0) {
        if (my_pairs) atomicAdd(&c.st->pairs_density, my_pairs);
        if (my_tests) atomicAdd(&c.st->tests_density, my_tests);
        if (my_done) atomicAdd(&c.st->lvl_done[a.lvl], my_done);
        if (my_prom) atomicAdd(&c.st->lvl_promoted[a.lvl], my_prom);
    }
    if (my_err) set_error(c.st, my_err);
}

// ---------------------------------------------------------------------------
// Force
// ---------------------------------------------------------------------------

// The force's pack pass: every slot's inputs decoded from their storage
// formats into three FP32 float4 arrays (so the pair kernel loads a
// candidate with one 16-byte load per array), and the largest h of every
// sub-cell for the stencil pruning.  Slots are sorted by key, so the lanes of
// a warp share few keys; each key group reduces in the warp and its leader
// does one atomic max (h > 0, so the float order is the unsigned order).
__global__ void __launch_bounds__(256) k_force_pack(ForceArgs a, const int32_t *slot_key, float *key_hmax,
                                                    float4 *pA, float4 *pB, float4 *pC)
{
    const Common &c = a.c;
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool ok = k < c.n;
    const int key = ok ? slot_key[k] : -1;
    float hv = 0.0f;
    if (ok) {
        hv = ld_val(c.h.p[0], c.h.fmt, k) * c.h.dec;
        pA[k] = make_float4(ld_val(c.x.p[0], c.x.fmt, k) * c.x.dec, ld_val(c.x.p[1], c.x.fmt, k) * c.x.dec,
                            ld_val(c.x.p[2], c.x.fmt, k) * c.x.dec, hv);
        pB[k] = make_float4(ld_val(a.v.p[0], a.v.fmt, k) * a.v.dec, ld_val(a.v.p[1], a.v.fmt, k) * a.v.dec,
                            ld_val(a.v.p[2], a.v.fmt, k) * a.v.dec, ld_val(c.m.p[0], c.m.fmt, k) * c.m.dec);
        const float rho = ld_val(a.rho.p[0], a.rho.fmt, k) * a.rho.dec;
        const float P = ld_val(a.P.p[0], a.P.fmt, k) * a.P.dec;
        pC[k] = make_float4(P / (rho * rho), rho, ld_val(a.cs.p[0], a.cs.fmt, k) * a.cs.dec, 0.0f);
        if (!(hv > 0.0f && hv <= 3.0e38f)) hv = a.h_cap;       // NaN / non-positive: assume h_max
    }
    if (!key_hmax) return;           // level mode: no sub-cell table
    const unsigned peers = __match_any_sync(FULL, key);
    const unsigned mx = __reduce_max_sync(peers, __float_as_uint(hv));
    if (ok && (threadIdx.x & 31) == __ffs(peers) - 1)
        atomicMax(reinterpret_cast<unsigned *>(key_hmax) + key, mx);
}

// The level force's pack arrays copied into the order of the per-level lists
// (every slot appears once in them), each entry's slot in lC's w.
__global__ void __launch_bounds__(256) k_lvl_gather_pack(const int32_t *plist, int64_t n, const float4 *pA,
                                                         const float4 *pB, const float4 *pC, float4 *lA, float4 *lB,
                                                         float4 *lC)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int j = __ldg(plist + i);
    lA[i] = __ldg(pA + j);
    lB[i] = __ldg(pB + j);
    float4 q = __ldg(pC + j);
    q.w = __int_as_float(j);
    lC[i] = q;
}

// The level force's candidate streams for an item of level `lvl` whose cell
// has Morton code `cell` at that level and finest-cell origin `org`: one per
// level l' of the hierarchy, over the list of level-l' particles.  Pairs need
// r < h_i + h_j; h_j <= h_l' and h_i <= h_lvl, so a partner of a finer or
// equal level lies in the 27 cells of level lvl around the item's cell, and
// one of a coarser level in the 27 cells of its own level l' around the
// item's level-l' cell: stencil level s = min(l', lvl).  Entry (l', t) is
// stencil cell t at level s, kept when its box comes within hw + h_l' of the
// warp box; its run in list l' is found by binary search on the keys.
// Entries go in (l', t) order, at most 8 x 27.
__device__ int lvl_force_table(const Common &c, int cell, int lvl, int3 org, const Box &box, float hw, Tab &tab,
                               int lane)
{
    const int K = c.lvl_max - c.lvl_min + 1;
    const int nent = 27 * K;
    const int E = (nent + 31) / 32;
    constexpr int kE = (27 * 8 + 31) / 32;
    int cnt[kE], st[kE];
    int local = 0, kept = 0;
#pragma unroll
    for (int i = 0; i < kE; ++i) {
        cnt[i] = 0;
        st[i] = 0;
        const int e = lane * E + i;
        if (i < E && e < nent) {
            const int lp = c.lvl_min + e / 27, t = e % 27;
            const int sl = min(lp, lvl);                       // stencil level
            const int dn = c.lvl_max - sl;                     // its cells in finest cells: 2^dn
            const uint32_t cs = (uint32_t)cell >> (3 * (lvl - sl));
            const int da[3] = {t % 3 - 1, (t / 3) % 3 - 1, t / 9 - 1};
            const int oc[3] = {(int)morton_compact(cs), (int)morton_compact(cs >> 1), (int)morton_compact(cs >> 2)};
            const int og[3] = {org.x, org.y, org.z};
            const float reach = hw + c.lcap[lp];
            float d2 = 0.0f;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                // the stencil cell's box in the item frame, in finest cells:
                // (coordinate + d) 2^dn - org, one level-sl edge wide
                const float fe = c.fine_edge[a];
                const float lo = (float)((oc[a] + da[a]) * (1 << dn) - og[a]) * fe - fe * (1.0f / 512.0f);
                const float hi = lo + (float)(1 << dn) * fe + fe * (1.0f / 256.0f);
                const float g = fmaxf(0.0f, fmaxf(lo - box.hi[a], box.lo[a] - hi));
                d2 = fmaf(g, g, d2);
            }
            if (d2 < reach * reach) {
                const uint32_t m = (1u << sl) - 1u;
                const int32_t code = (int32_t)morton_key((uint32_t)(oc[0] + da[0]) & m, (uint32_t)(oc[1] + da[1]) & m,
                                                         (uint32_t)(oc[2] + da[2]) & m);
                const int l0 = __ldg(c.lstart + lp), l1 = __ldg(c.lstart + lp + 1);
                const int32_t *cs = c.cs_list + (lp - c.lvl_min) * c.cs_stride;
                const int s0 = key_lower_bound_cs(c.pkey, l0, l1, code << (3 * dn), cs, c.cl_shift, c.cl_C);
                cnt[i] = key_lower_bound_cs(c.pkey, s0, l1, (code + 1) << (3 * dn), cs, c.cl_shift, c.cl_C) - s0;
                st[i] = s0;
            }
        }
        local += cnt[i];
        kept += cnt[i] > 0 ? 1 : 0;
    }
    int inc = local, kinc = kept;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(FULL, inc, o);
        const int w = __shfl_up_sync(FULL, kinc, o);
        if (lane >= o) {
            inc += v;
            kinc += w;
        }
    }
    int run = inc - local, pos = kinc - kept;
#pragma unroll
    for (int i = 0; i < kE; ++i) {
        if (cnt[i] > 0) {
            run += cnt[i];
            tab.incl[pos] = run;
            tab.base[pos] = st[i] - (run - cnt[i]);
            tab.t[pos] = 0;
            ++pos;
        }
    }
    if (lane == 31) tab.nk = kinc;
    __syncwarp();
    return __shfl_sync(FULL, inc, 31);
}

// Stage the force candidates (those within h_max(warp) + h_j of the warp box)
// from `cur` on, until the stage is full or the stream ends: their packed
// inputs (one 16-byte load per array, issued for every batch in flight before
// anything is stored), positions shifted into the item's cell frame, and the
// slot in sC.w.  Returns how many were staged and moves `cur` (as
// stage_density).  The 27-cell grid covers pairs up to 2 h_max only; a
// candidate with a larger h sets the h-cap error bit.
template <bool kLvl>
__device__ int stage_force(const ForceArgs &a, const Tab &tab, int total, const Box &box, float hw, float4 *sA,
                           float4 *sB, float4 *sC, int cap, Cursor &cur, int lane, unsigned &err, int3 org)
{
    const Common &c = a.c;
    const unsigned lt = (1u << lane) - 1u;
    const int nk = tab.nk;
    int found = 0;
    int ecur = cur.e;
    for (int g0 = cur.g; g0 < total; g0 += 32 * kStageUnroll) {
        float4 qa[kStageUnroll], qb[kStageUnroll], qc[kStageUnroll];
        int eu[kStageUnroll];
        int e = ecur;
#pragma unroll
        for (int u = 0; u < kStageUnroll; ++u) {
            const int g = g0 + u * 32 + lane;
            qa[u] = make_float4(3.0e38f, 3.0e38f, 3.0e38f, 0.0f);
            qb[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            qc[u] = make_float4(0.f, 1.f, 0.f, 0.f);
            if (g < total) {
                e = advance(tab, nk, e, g);
                const int j = tab.base[e] + g;      // level mode: an entry of the level lists
                if (kLvl) {
                    qa[u] = lvl_frame(c, (uint32_t)__ldg(c.pkey + j), org, __ldg(a.lA + j));
                    qb[u] = __ldg(a.lB + j);
                    qc[u] = __ldg(a.lC + j);
                } else {
                    const float4 p = __ldg(a.pA + j);
                    float sx, sy, sz;
                    stencil_shift(c, tab.t[e], sx, sy, sz);
                    qa[u] = make_float4(p.x + sx, p.y + sy, p.z + sz, p.w);
                    qb[u] = __ldg(a.pB + j);
                    qc[u] = __ldg(a.pC + j);
                    qc[u].w = __int_as_float(j);
                }
            }
            eu[u] = e;
        }
#pragma unroll
        for (int u = 0; u < kStageUnroll; ++u) {
            if (qa[u].w > a.h_cap) err |= SPH_ERR_HCAP;
            const float rr = hw + qa[u].w;
            const bool keep = box_dist2(box, qa[u].x, qa[u].y, qa[u].z) < rr * rr;
            const unsigned b = __ballot_sync(FULL, keep);
            const int nb = __popc(b);
            if (found + nb > cap) {     // stage full: resume at this batch
                cur.g = g0 + u * 32;
                cur.e = __shfl_sync(FULL, eu[u], 0);
                __syncwarp();
                return found;
            }
            if (keep) {
                const int pos = found + __popc(b & lt);
                sA[pos] = qa[u];
                sB[pos] = qb[u];
                sC[pos] = qc[u];
            }
            found += nb;
        }
        ecur = __shfl_sync(FULL, e, 31);
    }
    cur.g = total;
    cur.e = ecur;
    __syncwarp();
    return found;
}

// shared memory of one force warp: the staged (x, y, z, h), (v, m),
// (P/rho^2, rho, c, slot), the per-lane pair lists and the stencil table
__host__ __device__ inline size_t force_warp_bytes(int cap)
{
    return (size_t)(cap + kForcePad) * 3 * sizeof(float4) + (size_t)32 * kForceSlots * sizeof(uint8_t) + sizeof(Tab);
}

template <bool kLvl>
__global__ void __launch_bounds__(kMaxBlock, 1) k_force(ForceArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const Common &c = a.c;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float4 *sA = reinterpret_cast<float4 *>(smem + warp * force_warp_bytes(c.cap));   // x, y, z, h
    float4 *sB = sA + c.cap + kForcePad;                                                 // vx, vy, vz, m
    float4 *sC = sB + c.cap + kForcePad;                                                 // P/rho^2, rho, c, slot
    uint8_t *lst = reinterpret_cast<uint8_t *>(sC + c.cap + kForcePad);                  // per-lane pair lists
    Tab &tab = *reinterpret_cast<Tab *>(lst + 32 * kForceSlots);
    unsigned long long my_pairs = 0, my_tests = 0;
    unsigned my_err = 0;
    const int lo = c.range ? c.range[0] : 0;
    const int hi_item = c.range ? c.range[1] : c.st->nitems;

    for (int it = lo + pop_item(c.st, lane); it < hi_item; it = lo + pop_item(c.st, lane)) {
        const int cell = c.icell[it];
        const int first = c.ifirst[it];
        const int count = c.icount[it];
        const bool ok = lane < count;
        int k = first + lane;
        int3 org = make_int3(0, 0, 0);       // level mode: the item cell's origin in finest cells
        if (kLvl) {
            k = ok ? __ldg(c.tslot + first + lane) : 0;
            const uint32_t cc = (uint32_t)cell;
            org = make_int3((int)(morton_compact(cc) << c.lvl_dn), (int)(morton_compact(cc >> 1) << c.lvl_dn),
                            (int)(morton_compact(cc >> 2) << c.lvl_dn));
        }
        float xi = 0.f, yi = 0.f, zi = 0.f, hi = 0.f, vxi = 0.f, vyi = 0.f, vzi = 0.f;
        float rhoi = 1.f, Pr2i = 0.f, ci = 0.f;
        if (ok) {
            float4 qa = __ldg(a.pA + k);
            const float4 qb = __ldg(a.pB + k), qc = __ldg(a.pC + k);
            if (kLvl) qa = lvl_frame(c, (uint32_t)__ldg(c.mkey + k), org, qa);
            xi = qa.x;
            yi = qa.y;
            zi = qa.z;
            hi = qa.w;
            vxi = qb.x;
            vyi = qb.y;
            vzi = qb.z;
            Pr2i = qc.x;
            rhoi = qc.y;
            ci = qc.z;
        }
        const Box box = warp_box(ok, xi, yi, zi);
        const float hw = warp_max(ok ? hi : 0.0f);
        const int total = kLvl ? lvl_force_table(c, cell, a.lvl, org, box, hw, tab, lane)
                               : build_stream(c, cell, box, 0.0f, tab, lane, a.key_hmax, hw);
        if (kLvl && total > kForceDeferStages * c.cap) {
            // A long stream: coarse targets spread over their cell next to a
            // dense cluster, whose box takes in the cluster's fine lists.
            // Each target goes to the per-target list instead and is gathered
            // with its own reach by a warp, or by a block of warps when its
            // stream is long (k_force_one).
            const unsigned bal = __ballot_sync(FULL, ok);
            unsigned base = 0;
            if (lane == 0) base = atomicAdd(&c.st->defer_n, (unsigned)__popc(bal));
            base = __shfl_sync(FULL, base, 0);
            if (ok) c.defer[base + __popc(bal & ((1u << lane) - 1u))] = k;
            continue;
        }
        float ax = 0.f, ay = 0.f, az = 0.f, du = 0.f;
        int cnt = 0;
        if (hi > a.h_cap) my_err |= SPH_ERR_HCAP;
        Cursor cur{0, 0};
        do {
            const int len = stage_force<kLvl>(a, tab, total, box, hw, sA, sB, sC, c.cap, cur, lane, my_err, org);
            if (lane < kForcePad) sA[len + lane] = make_float4(3.0e38f, 3.0e38f, 3.0e38f, 0.0f);   // far away
            __syncwarp();
            if (ok) {
                my_tests += (unsigned long long)len;
                // phase 1 collects this lane's pairs among up to kForceCap
                // staged candidates into its list (branch-free appends in
                // batches of 8: loads first, then the stores; the far-away
                // entries after the stage fail every test; a range of
                // kForceCap candidates cannot overflow the list), phase 2
                // evaluates them; repeated over the stage
                for (int s0 = 0; s0 < len; s0 += kForceCap) {
                    const int s1 = min(s0 + kForceCap, len);
                    uint8_t *lp = lst + lane;
                    constexpr int LB = 8;
                    static_assert(kForceCap % LB == 0 && LB <= kForcePad, "force test batches");
                    for (int e0 = s0; e0 < s1; e0 += LB) {
                        bool in[LB];
#pragma unroll
                        for (int u = 0; u < LB; ++u) {
                            const float4 q = sA[e0 + u];
                            const float dx = xi - q.x, dy = yi - q.y, dz = zi - q.z;
                            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                            const float hs = hi + q.w;
                            in[u] = r2 < hs * hs;
                        }
#pragma unroll
                        for (int u = 0; u < LB; ++u) {
                            // a range of kForceCap candidates advances lp at
                            // most kForceCap rows: row kForceCap is scratch
                            *lp = (uint8_t)(e0 + u - s0);
                            lp += in[u] ? 32 : 0;
                        }
                    }
                    const int nl = (int)(lp - (lst + lane)) >> 5;
                    // every listed pair is evaluated: the self pair and
                    // coincident pairs (r = 0) contribute exactly zero (the
                    // spline derivative vanishes at q = 0 and v_ij . d = 0), so
                    // only the count excludes the particle itself
#pragma unroll 2
                    for (int l = 0; l < nl; ++l) {
                        const int p = s0 + lst[l * 32 + lane];
                        const float4 qc = sC[p];
                        const float4 q = sA[p];
                        const float dx = xi - q.x, dy = yi - q.y, dz = zi - q.z;
                        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                        cnt += __float_as_int(qc.w) != k ? 1 : 0;
                        force_pair(ax, ay, az, du, vxi, vyi, vzi, rhoi, Pr2i, ci, dx, dy, dz, r2, hi + q.w, sB[p], qc,
                                   a.alpha, a.beta, a.eps);
                    }
                }
            }
            __syncwarp();
        } while (cur.g < total);
        if (ok) {
            if (!isfinite(ax) || !isfinite(ay) || !isfinite(az) || !isfinite(du)) my_err |= SPH_ERR_NONFINITE;
            a.a[0][k] = ax;
            a.a[1][k] = ay;
            a.a[2][k] = az;
            a.dudt[k] = du;
            a.nngb[k] = cnt;
            my_pairs += (unsigned long long)cnt;
        }
    }
    my_pairs = warp_sum_u64(my_pairs);
    my_tests = warp_sum_u64(my_tests);
    if (lane == 0) {
        if (my_pairs) atomicAdd(&c.st->pairs_force, my_pairs);
        if (my_tests) atomicAdd(&c.st->tests_force, my_tests);
    }
    if (my_err) set_error(c.st, my_err);
}

// The level force's per-target pass: every target that k_force<true>
// deferred is gathered by one whole block of W warps.  Its K level streams
// are pruned to its own reach (h_i + h_l') and split into W contiguous
// slices, one per warp; a warp's lanes evaluate its slice's staged
// candidates in turn, the lanes' partial sums meet in a butterfly and the
// warps' in stream order.  Thread 0 writes.
__global__ void __launch_bounds__(kMaxBlock, 1) k_force_one(ForceArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ float red[kMaxBlock / 32];
    __shared__ unsigned next;
    const Common &c = a.c;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
    float4 *sA = reinterpret_cast<float4 *>(smem + warp * force_warp_bytes(c.cap));
    float4 *sB = sA + c.cap + kForcePad;
    float4 *sC = sB + c.cap + kForcePad;
    uint8_t *lst = reinterpret_cast<uint8_t *>(sC + c.cap + kForcePad);
    Tab &tab = *reinterpret_cast<Tab *>(lst + 32 * kForceSlots);
    unsigned long long my_pairs = 0, my_tests = 0;
    unsigned my_err = 0;
    const int32_t *list = c.one_phase ? c.heavy : c.defer;
    unsigned *head = c.one_phase ? &c.st->heavy_q : &c.st->defer_q;
    const unsigned nd = c.one_phase ? c.st->heavy_n : c.st->defer_n;
    for (;;) {
        if (threadIdx.x == 0) next = atomicAdd(head, 1u);
        __syncthreads();
        const unsigned j = next;
        __syncthreads();
        if (j >= nd) break;
        const int k = list[j];
        const uint32_t key = (uint32_t)__ldg(c.mkey + k);
        const int cell = (int)(key >> (3 * c.lvl_dn));
        const int3 org = make_int3((int)(morton_compact((uint32_t)cell) << c.lvl_dn),
                                   (int)(morton_compact((uint32_t)cell >> 1) << c.lvl_dn),
                                   (int)(morton_compact((uint32_t)cell >> 2) << c.lvl_dn));
        const float4 qa = lvl_frame(c, key, org, __ldg(a.pA + k));
        const float4 qb = __ldg(a.pB + k), qcv = __ldg(a.pC + k);
        const float xi = qa.x, yi = qa.y, zi = qa.z, hi = qa.w;
        const Box pb{{xi, yi, zi}, {xi, yi, zi}};
        const int total = lvl_force_table(c, cell, a.lvl, org, pb, hi, tab, lane);
        if (c.heavy_at > 0 && total > c.heavy_at) {
            if (threadIdx.x == 0) c.heavy[atomicAdd(&c.st->heavy_n, 1u)] = k;
            continue;
        }
        if (hi > a.h_cap && threadIdx.x == 0) my_err |= SPH_ERR_HCAP;
        int g0, g1;
        stream_slice(total, warp, W, g0, g1);
        float ax = 0.f, ay = 0.f, az = 0.f, du = 0.f;
        int cnt = 0;
        Cursor cur{g0, g0 < g1 ? advance(tab, tab.nk, 0, g0) : 0};
        while (cur.g < g1) {
            const int len = stage_force<true>(a, tab, g1, pb, hi, sA, sB, sC, c.cap, cur, lane, my_err, org);
            my_tests += (unsigned long long)max(0, (len - lane + 31) >> 5);
            for (int p = lane; p < len; p += 32) {
                const float4 qc = sC[p];
                const float4 q = sA[p];
                const float dx = xi - q.x, dy = yi - q.y, dz = zi - q.z;
                const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                const float hs = hi + q.w;
                if (__float_as_int(qc.w) != k && r2 < hs * hs) {
                    ++cnt;
                    if (r2 > 0.0f)
                        force_pair(ax, ay, az, du, qb.x, qb.y, qb.z, qcv.y, qcv.x, qcv.z, dx, dy, dz, r2, hs, sB[p], qc,
                                   a.alpha, a.beta, a.eps);
                }
            }
            __syncwarp();
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ax += __shfl_xor_sync(FULL, ax, o);
            ay += __shfl_xor_sync(FULL, ay, o);
            az += __shfl_xor_sync(FULL, az, o);
            du += __shfl_xor_sync(FULL, du, o);
            cnt += __shfl_xor_sync(FULL, cnt, o);
        }
        if (W > 1) {
            ax = block_sum_ordered(ax, red, warp, lane, W);
            ay = block_sum_ordered(ay, red, warp, lane, W);
            az = block_sum_ordered(az, red, warp, lane, W);
            du = block_sum_ordered(du, red, warp, lane, W);
            cnt = (int)block_sum_ordered((float)cnt, red, warp, lane, W);   // exact: far below 2^24
        }
        if (threadIdx.x == 0) {
            if (!isfinite(ax) || !isfinite(ay) || !isfinite(az) || !isfinite(du)) my_err |= SPH_ERR_NONFINITE;
            a.a[0][k] = ax;
            a.a[1][k] = ay;
            a.a[2][k] = az;
            a.dudt[k] = du;
            a.nngb[k] = cnt;
            my_pairs += (unsigned long long)cnt;
        }
    }
    my_tests = warp_sum_u64(my_tests);
    if (lane == 0) {
        if (my_pairs) atomicAdd(&c.st->pairs_force, my_pairs);
        if (my_tests) atomicAdd(&c.st->tests_force, my_tests);
    }
    if (my_err) set_error(c.st, my_err);
}

// ---------------------------------------------------------------------------
// The plain form: one thread per particle, looping over the particles of the
// 27 neighbour cells straight from the SoA (no work items, no staging, no
// pruning).  The same arithmetic as the batched kernels, kept as the
// baseline that batching and staging are measured against.
// ---------------------------------------------------------------------------

__device__ __forceinline__ void cell_of_key(const Common &c, int key, int &kx, int &ky, int &kz)
{
    const int cell = key >> c.lg_s3;
    kx = cell % c.nc[0];
    ky = (cell / c.nc[0]) % c.nc[1];
    kz = cell / (c.nc[0] * c.nc[1]);
}

// first key of neighbour cell t (0..26) of cell (kx, ky, kz), periodic
__device__ __forceinline__ int neighbour_key(const Common &c, int kx, int ky, int kz, int t)
{
    int nx = kx + t % 3 - 1, ny = ky + (t / 3) % 3 - 1, nz = kz + t / 9 - 1;
    nx += nx < 0 ? c.nc[0] : (nx >= c.nc[0] ? -c.nc[0] : 0);
    ny += ny < 0 ? c.nc[1] : (ny >= c.nc[1] ? -c.nc[1] : 0);
    nz += nz < 0 ? c.nc[2] : (nz >= c.nc[2] ? -c.nc[2] : 0);
    return (nx + c.nc[0] * (ny + c.nc[1] * nz)) << c.lg_s3;
}

__global__ void __launch_bounds__(128) k_density_plain(DensityArgs a, const int32_t *slot_key)
{
    const Common &c = a.c;
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= c.n) return;
    int kx, ky, kz;
    cell_of_key(c, slot_key[k], kx, ky, kz);
    const float xi = ld_val(c.x.p[0], c.x.fmt, k) * c.x.dec;
    const float yi = ld_val(c.x.p[1], c.x.fmt, k) * c.x.dec;
    const float zi = ld_val(c.x.p[2], c.x.fmt, k) * c.x.dec;
    const float mi = ld_val(c.m.p[0], c.m.fmt, k) * c.m.dec;
    float hi = ld_val(c.h.p[0], c.h.fmt, k) * c.h.dec;
    const float ui = a.has_u ? ld_val(a.u.p[0], a.u.fmt, k) * a.u.dec : 0.0f;
    unsigned err = 0, lf = 0;
    bool clamped = false;
    if (!(hi > 0.0f) || !isfinite(hi)) { hi = a.h_cap; lf |= SPH_PFLAG_NONFINITE; }
    if (hi > a.h_cap) { hi = a.h_cap; clamped = true; }
    float rho = 0.f;
    int cnt = 0;
    unsigned long long tests = 0, pairs = 0;
    for (int pass = 0; pass < a.npass; ++pass) {
        const float hinv = 1.0f / hi;
        const bool deriv = pass + 1 < a.npass;
        DAcc acc{0.f, 0.f, 0.f, 0.f};
        for (int t = 0; t < 27; ++t) {
            float sx, sy, sz;
            stencil_shift(c, t, sx, sy, sz);
            const int key0 = neighbour_key(c, kx, ky, kz, t);
            const int j0 = c.cell_start[key0], j1 = c.cell_start[key0 + c.s3];
            tests += (unsigned long long)(j1 - j0);
            for (int j = j0; j < j1; ++j) {
                const float4 q = make_float4(fmaf(ld_val(c.x.p[0], c.x.fmt, j), c.x.dec, sx),
                                             fmaf(ld_val(c.x.p[1], c.x.fmt, j), c.x.dec, sy),
                                             fmaf(ld_val(c.x.p[2], c.x.fmt, j), c.x.dec, sz),
                                             ld_val(c.m.p[0], c.m.fmt, j) * c.m.dec);
                dens_acc_rt(acc, pair_r(xi, yi, zi, q), hinv, q.w, a.plain_sum, deriv);
            }
        }
        const float h3inv = hinv * hinv * hinv;
        rho = kSigma * h3inv * (acc.s - acc.c);
        const float drdh = -3.0f * kSigma * h3inv * hinv * acc.d;
        cnt = (int)acc.n - 1;
        pairs += (unsigned long long)cnt;      // every pass's pairs, as the batched kernel counts them
        if (pass + 1 < a.npass) {
            const float f = rho - mi * a.eta3 * h3inv;
            const float fp = drdh + 3.0f * mi * a.eta3 * h3inv * hinv;
            float hn = hi;
            if (fp > 0.0f && isfinite(f) && isfinite(fp)) hn = hi - f / fp;
            else lf |= SPH_PFLAG_NEWTON;
            hn = fminf(fmaxf(hn, 0.5f * hi), 2.0f * hi);
            if (hn > a.h_cap) { hn = a.h_cap; clamped = true; }
            hi = hn;
        }
    }
    if (!isfinite(rho)) lf |= SPH_PFLAG_NONFINITE;
    if (clamped) lf |= SPH_PFLAG_HCAP;
    a.pflags[k] = (uint8_t)lf;
    if (lf & SPH_PFLAG_NONFINITE) err |= SPH_ERR_NONFINITE;
    if (lf & SPH_PFLAG_NEWTON) err |= SPH_ERR_NEWTON;
    st_val(a.rho_out, a.rho_fmt, k, rho * a.rho_enc);
    if (a.write_h) st_val(a.h_out, a.h_fmt, k, hi * a.h_enc);
    a.nngb[k] = cnt;
    if (a.has_u) {
        const float P = a.gm1 * rho * ui;
        st_val(a.P_out, a.P_fmt, k, P * a.P_enc);
        st_val(a.cs_out, a.cs_fmt, k, __fsqrt_rn(a.gamma * P / rho) * a.cs_enc);
    }
    if (clamped) {
        atomicAdd(&c.st->hcap_clamps, 1ull);
        err |= SPH_ERR_HCAP;
    }
    if (err) set_error(c.st, err);
    atomicAdd(&c.st->pairs_density, pairs);
    atomicAdd(&c.st->tests_density, tests);
}

__global__ void __launch_bounds__(128) k_force_plain(ForceArgs a, const int32_t *slot_key)
{
    const Common &c = a.c;
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= c.n) return;
    int kx, ky, kz;
    cell_of_key(c, slot_key[k], kx, ky, kz);
    const float xi = ld_val(c.x.p[0], c.x.fmt, k) * c.x.dec;
    const float yi = ld_val(c.x.p[1], c.x.fmt, k) * c.x.dec;
    const float zi = ld_val(c.x.p[2], c.x.fmt, k) * c.x.dec;
    const float hi = ld_val(c.h.p[0], c.h.fmt, k) * c.h.dec;
    const float vxi = ld_val(a.v.p[0], a.v.fmt, k) * a.v.dec;
    const float vyi = ld_val(a.v.p[1], a.v.fmt, k) * a.v.dec;
    const float vzi = ld_val(a.v.p[2], a.v.fmt, k) * a.v.dec;
    const float rhoi = ld_val(a.rho.p[0], a.rho.fmt, k) * a.rho.dec;
    const float Pr2i = ld_val(a.P.p[0], a.P.fmt, k) * a.P.dec / (rhoi * rhoi);
    const float ci = ld_val(a.cs.p[0], a.cs.fmt, k) * a.cs.dec;
    unsigned err = hi > a.h_cap ? SPH_ERR_HCAP : 0u;
    float ax = 0.f, ay = 0.f, az = 0.f, du = 0.f;
    int cnt = 0;
    unsigned long long tests = 0;
    for (int t = 0; t < 27; ++t) {
        float sx, sy, sz;
        stencil_shift(c, t, sx, sy, sz);
        const int key0 = neighbour_key(c, kx, ky, kz, t);
        const int j0 = c.cell_start[key0], j1 = c.cell_start[key0 + c.s3];
        tests += (unsigned long long)(j1 - j0);
        for (int j = j0; j < j1; ++j) {
            const float dx = xi - fmaf(ld_val(c.x.p[0], c.x.fmt, j), c.x.dec, sx);
            const float dy = yi - fmaf(ld_val(c.x.p[1], c.x.fmt, j), c.x.dec, sy);
            const float dz = zi - fmaf(ld_val(c.x.p[2], c.x.fmt, j), c.x.dec, sz);
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            const float hj = ld_val(c.h.p[0], c.h.fmt, j) * c.h.dec;
            const float hs = hi + hj;
            if (hj > a.h_cap) err |= SPH_ERR_HCAP;
            if (!(r2 < hs * hs) || j == k) continue;
            ++cnt;
            if (r2 > 0.0f) {
                const float rj = ld_val(a.rho.p[0], a.rho.fmt, j) * a.rho.dec;
                const float4 qb = make_float4(ld_val(a.v.p[0], a.v.fmt, j) * a.v.dec,
                                              ld_val(a.v.p[1], a.v.fmt, j) * a.v.dec,
                                              ld_val(a.v.p[2], a.v.fmt, j) * a.v.dec,
                                              ld_val(c.m.p[0], c.m.fmt, j) * c.m.dec);
                const float4 qc = make_float4(ld_val(a.P.p[0], a.P.fmt, j) * a.P.dec / (rj * rj), rj,
                                              ld_val(a.cs.p[0], a.cs.fmt, j) * a.cs.dec, 0.0f);
                force_pair(ax, ay, az, du, vxi, vyi, vzi, rhoi, Pr2i, ci, dx, dy, dz, r2, hs, qb, qc, a.alpha,
                           a.beta, a.eps);
            }
        }
    }
    if (!isfinite(ax) || !isfinite(ay) || !isfinite(az) || !isfinite(du)) err |= SPH_ERR_NONFINITE;
    a.a[0][k] = ax;
    a.a[1][k] = ay;
    a.a[2][k] = az;
    a.dudt[k] = du;
    a.nngb[k] = cnt;
    if (err) set_error(c.st, err);
    atomicAdd(&c.st->pairs_force, (unsigned long long)cnt);
    atomicAdd(&c.st->tests_force, tests);
}

Common make_common(sph_ctx *c, int cap)
{
    Common m;
    m.n = c->n;
    for (int k = 0; k < 3; ++k) {
        m.nc[k] = c->nc[k];
        m.edge[k] = (float)c->edge[k];
    }
    for (int t = 0; t < 27; ++t)
        m.shift[t] = make_float4((float)(t % 3 - 1) * m.edge[0], (float)((t / 3) % 3 - 1) * m.edge[1],
                                 (float)(t / 9 - 1) * m.edge[2], 0.0f);
    m.sub = c->sub;
    m.s3 = c->sub * c->sub * c->sub;
    m.lg_sub = c->sub == 2 ? 1 : 0;
    m.lg_s3 = 3 * m.lg_sub;
    m.cell_start = c->cell_start;
    m.icell = c->item_cell;
    m.ifirst = c->item_first;
    m.icount = c->item_count;
    m.range = nullptr;
    m.tslot = nullptr;
    m.mkey = nullptr;
    m.lvl_dn = 0;
    m.lvl_n = 0;
    m.fine_n = 0;
    for (int k = 0; k < 3; ++k) m.fine_edge[k] = 0.0f;
    m.defer = nullptr;
    m.pkey = m.lstart = nullptr;
    m.cs_slot = m.cs_list = nullptr;
    m.cs_shift = m.cl_shift = 0;
    m.cs_C = m.cl_C = 0;
    m.cs_stride = 0;
    if (c->cidx) {
        m.cs_slot = c->cidx;
        m.cs_list = c->cidx + c->cs_stride;
        m.cs_shift = 3 * (c->lvl_max - c->cs_lc);
        m.cs_C = 1 << (3 * c->cs_lc);
        m.cl_shift = 3 * (c->lvl_max - c->cl_lc);
        m.cl_C = 1 << (3 * c->cl_lc);
        m.cs_stride = c->cs_stride;
    }
    m.heavy = nullptr;
    m.heavy_at = 0;
    m.one_phase = 0;
    m.lvl_min = m.lvl_max = 0;
    for (int l = 0; l <= kLevelMax; ++l) m.lcap[l] = 0.0f;
    m.st = c->dstats;
    auto ref = [&](int f) {
        FieldRef r;
        for (int k = 0; k < 3; ++k) r.p[k] = c->soa[f][k];
        r.fmt = c->prec[f];
        r.dec = c->dec(f);
        return r;
    };
    m.x = ref(SPH_F_X);
    m.m = ref(SPH_F_M);
    m.h = ref(SPH_F_H);
    m.cap = cap;
    m.defer_cap = 8 * cap;
    return m;
}

template <typename K, typename A>
cudaError_t launch_persistent(sph_ctx *c, K kernel, const A &args, size_t smem, LaunchCache &lc, int block)
{
    cudaError_t e;
    if (lc.smem != smem || lc.block != block || lc.per_sm_req != c->tuning.ctas_per_sm) {
        if ((e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
            return e;
        int per_sm = c->tuning.ctas_per_sm;
        if (per_sm <= 0) {
            if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem)) != cudaSuccess)
                return e;
            if (per_sm < 1) per_sm = 1;
        }
        lc.smem = smem;
        lc.block = block;
        lc.per_sm_req = c->tuning.ctas_per_sm;
        lc.grid = c->sm_count * per_sm;
    }
    if (c->tuning.class_launches && c->items_by_class) {
        // one launch per cost class, over that class's items
        const int32_t *start = c->class_hist + kItemClasses;
        for (int k = 0; k < kItemClasses; ++k) {
            A per = args;
            per.c.range = start + k;
            if ((e = cudaMemsetAsync(&c->dstats->queue, 0, sizeof(unsigned), c->stream)) != cudaSuccess) return e;
            kernel<<<(unsigned)lc.grid, block, smem, c->stream>>>(per);
            c->launches += 1;
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    if ((e = cudaMemsetAsync(&c->dstats->queue, 0, sizeof(unsigned), c->stream)) != cudaSuccess) return e;
    kernel<<<(unsigned)lc.grid, block, smem, c->stream>>>(args);
    c->launches += 1;
    return cudaGetLastError();
}

// The level hierarchy's per-target passes of one level: one warp per target
// over the deferred list, passing targets whose stream holds more than
// heavy_at candidates on to a block of w warps per target.
template <typename K, typename A>
cudaError_t run_per_target(sph_ctx *c, K kernel, const A &args, size_t smem_1, size_t smem_w, int w, int heavy_at,
                           LaunchCache &lc_1, LaunchCache &lc_w)
{
    A a = args;
    a.c.heavy = c->tscan;      // scan scratch, free while a level's kernels run
    a.c.one_phase = 0;
    a.c.heavy_at = w > 1 ? heavy_at : 0;
    cudaError_t e = launch_persistent(c, kernel, a, smem_1, lc_1, 32);
    if (e != cudaSuccess || w == 1) return e;
    a.c.one_phase = 1;
    a.c.heavy_at = 0;
    return launch_persistent(c, kernel, a, smem_w, lc_w, 32 * w);
}

}  // namespace

size_t density_smem_bytes(int block_threads, int cap, bool levels)
{
    return (size_t)(block_threads / 32) * density_warp_bytes(cap, levels);
}

size_t force_smem_bytes(int block_threads, int cap)
{
    return (size_t)(block_threads / 32) * force_warp_bytes(cap);
}

namespace {

DensityArgs density_args(sph_ctx *c, int newton_steps)
{
    DensityArgs a;
    a.c = make_common(c, c->tuning.stage_density);
    a.has_u = (c->valid & SPH_BIT(SPH_F_U)) != 0;
    for (int k = 0; k < 3; ++k) a.u.p[k] = c->soa[SPH_F_U][0];
    a.u.fmt = c->prec[SPH_F_U];
    a.u.dec = c->dec(SPH_F_U);
    a.npass = newton_steps + 1;
    const double eta = c->params.eta;
    a.eta3 = (float)(eta * eta * eta);
    a.h_cap = (float)c->params.h_max;
    a.gamma = (float)c->params.gamma;
    a.gm1 = (float)(c->params.gamma - 1.0);
    a.plain_sum = (c->params.flags & SPH_FLAG_PLAIN_SUM) != 0;
    a.rho_out = c->soa[SPH_F_RHO][0];
    a.rho_fmt = c->prec[SPH_F_RHO];
    const bool h_packed = fmt_packed(c->prec[SPH_F_H]);
    a.write_h = newton_steps > 0;
    a.h_out = h_packed ? (void *)c->stage : c->soa[SPH_F_H][0];
    a.h_fmt = h_packed ? SPH_P_FP32 : c->prec[SPH_F_H];
    a.P_out = c->soa[SPH_F_P][0];
    a.P_fmt = c->prec[SPH_F_P];
    a.cs_out = c->soa[SPH_F_CS][0];
    a.cs_fmt = c->prec[SPH_F_CS];
    a.rho_enc = c->enc(SPH_F_RHO);
    a.h_enc = c->enc(SPH_F_H);
    a.P_enc = c->enc(SPH_F_P);
    a.cs_enc = c->enc(SPH_F_CS);
    a.nngb = c->nngb;
    a.pflags = c->dflags;
    a.level = nullptr;
    a.lvl = 0;
    a.promote = false;
    a.pD = c->pack;
    return a;
}

}  // namespace

cudaError_t run_density(sph_ctx *c, int newton_steps)
{
    if (c->n == 0) return cudaSuccess;
    DensityArgs a = density_args(c, newton_steps);
    const bool h_packed = fmt_packed(c->prec[SPH_F_H]);
    if (c->tuning.pair_kernel == 1) {
        k_density_plain<<<(unsigned)((c->n + 127) / 128), 128, 0, c->stream>>>(a, c->slot_cell());
        c->launches += 1;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        if (a.write_h && h_packed) return run_pack(c, c->stage, SPH_F_H);
        return cudaSuccess;
    }
    // the pack pass (the force's pack arrays are free until the force runs)
    k_density_pack<<<(unsigned)((c->n + 255) / 256), 256, 0, c->stream>>>(a.c, c->pack);
    c->launches += 1;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = density_smem_bytes(c->tuning.block_threads, a.c.cap);
    if (c->kev[SPH_KEV_DENSITY][0] && (e = cudaEventRecord(c->kev[SPH_KEV_DENSITY][0], c->stream)) != cudaSuccess)
        return e;
    if ((e = launch_persistent(c, k_density<false>, a, smem, c->lc_density, c->tuning.block_threads)) != cudaSuccess) return e;
    if (c->kev[SPH_KEV_DENSITY][1] && (e = cudaEventRecord(c->kev[SPH_KEV_DENSITY][1], c->stream)) != cudaSuccess)
        return e;
    if (a.write_h && h_packed) return run_pack(c, c->stage, SPH_F_H);
    return cudaSuccess;
}

// The density over the level hierarchy: one pack pass (offsets from the
// finest cells), then the levels from the finest to the coarsest, each with
// its own work items and h cap; particles promoted at a level are in the
// next level's items.
cudaError_t run_density_levels(sph_ctx *c, int newton_steps)
{
    if (c->n == 0) return cudaSuccess;
    DensityArgs a = density_args(c, newton_steps);
    const bool h_packed = fmt_packed(c->prec[SPH_F_H]);
    a.c.mkey = c->slot_cell();
    a.c.tslot = c->tlist;
    a.c.fine_n = 1 << c->lvl_max;
    for (int k = 0; k < 3; ++k) a.c.fine_edge[k] = (float)c->edge[k];
    a.level = c->level;
    a.c.defer = c->tcode;     // free while the level's kernels run (its items are built)
    // h is written even without Newton steps: an input h above its level's cap
    // is clamped, and the level force relies on every h being within its cap
    a.write_h = true;
    k_density_pack<<<(unsigned)((c->n + 255) / 256), 256, 0, c->stream>>>(a.c, c->pack);
    c->launches += 1;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = density_smem_bytes(c->tuning.block_threads, a.c.cap, true);
    int w_one = kOneWarps;
    while (w_one > 1 && density_smem_bytes(32 * w_one, a.c.cap, true) + 256 > c->smem_optin) --w_one;
    const size_t smem_one = density_smem_bytes(32 * w_one, a.c.cap, true);
    const size_t smem_1 = density_smem_bytes(32, a.c.cap, true);
    // one warp's stage holds cap + the per-lane list space (k_density_one)
    const int heavy_dens = a.c.cap + 32 * kDensSlots * (int)sizeof(float) / (int)sizeof(float4);
    for (int l = c->lvl_max; l >= c->lvl_min; --l) {
        if ((e = run_level_items(c, l)) != cudaSuccess) return e;
        double cap = std::ldexp(c->params.box[0], -l);
        for (int k = 0; k < 3; ++k) {
            const double e_l = std::ldexp(c->params.box[k], -l);
            a.c.edge[k] = (float)e_l;
            cap = std::fmin(cap, e_l);
        }
        cap = std::fmin(0.5 * cap, c->params.h_max);
        a.c.lvl_dn = c->lvl_max - l;
        a.c.lvl_n = 1 << l;
        a.h_cap = (float)cap;
        a.lvl = l;
        a.promote = l > c->lvl_min;
        if ((e = cudaMemsetAsync(&c->dstats->defer_n, 0, 4 * sizeof(unsigned), c->stream)) != cudaSuccess) return e;
        if ((e = launch_persistent(c, k_density<true>, a, smem, c->lc_density_lv, c->tuning.block_threads)) != cudaSuccess) return e;
        if ((e = run_per_target(c, k_density_one, a, smem_1, smem_one, w_one, heavy_dens, c->lc_density_one,
                                c->lc_density_blk)) != cudaSuccess)
            return e;
    }
    if (a.write_h && h_packed) return run_pack(c, c->stage, SPH_F_H);
    return cudaSuccess;
}

namespace {

ForceArgs force_args(sph_ctx *c)
{
    ForceArgs a;
    a.c = make_common(c, c->tuning.stage_force);
    auto ref = [&](int f) {
        FieldRef r;
        for (int k = 0; k < 3; ++k) r.p[k] = c->soa[f][k];
        r.fmt = c->prec[f];
        r.dec = c->dec(f);
        return r;
    };
    a.v = ref(SPH_F_V);
    a.rho = ref(SPH_F_RHO);
    a.P = ref(SPH_F_P);
    a.cs = ref(SPH_F_CS);
    a.alpha = (float)c->params.alpha_av;
    a.beta = (float)c->params.beta_av;
    a.eps = (float)c->params.eps_av;
    a.h_cap = (float)c->params.h_max;
    for (int k = 0; k < 3; ++k) a.a[k] = (float *)c->soa[SPH_F_A][k];
    a.dudt = (float *)c->soa[SPH_F_DUDT][0];
    a.nngb = c->nngb_force;
    a.pA = c->pack;
    a.pB = c->pack + c->n;
    a.pC = c->pack + 2 * c->n;
    a.key_hmax = nullptr;
    a.lA = a.lB = a.lC = nullptr;
    a.lvl = 0;
    return a;
}

}  // namespace

cudaError_t run_force(sph_ctx *c)
{
    if (c->n == 0) return cudaSuccess;
    ForceArgs a = force_args(c);
    // the pack pass: FP32 inputs per slot, and the reach of every sub-cell
    // from the h the force will read
    cudaError_t e;
    const int64_t nkeys = c->ncell * c->sub * c->sub * c->sub;
    if ((e = cudaMemsetAsync(c->key_hmax, 0, sizeof(float) * nkeys, c->stream)) != cudaSuccess) return e;
    k_force_pack<<<(unsigned)((c->n + 255) / 256), 256, 0, c->stream>>>(a, c->slot_cell(), c->key_hmax, c->pack,
                                                                       c->pack + c->n, c->pack + 2 * c->n);
    c->launches += 1;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    a.key_hmax = c->key_hmax;
    if (c->tuning.pair_kernel == 1) {
        k_force_plain<<<(unsigned)((c->n + 127) / 128), 128, 0, c->stream>>>(a, c->slot_cell());
        c->launches += 1;
        return cudaGetLastError();
    }
    // the pair kernel reads only the packed FP32 arrays: one instantiation
    const size_t smem = force_smem_bytes(c->tuning.block_threads_force, a.c.cap);
    if (c->kev[SPH_KEV_FORCE][0] && (e = cudaEventRecord(c->kev[SPH_KEV_FORCE][0], c->stream)) != cudaSuccess)
        return e;
    if ((e = launch_persistent(c, k_force<false>, a, smem, c->lc_force, c->tuning.block_threads_force)) != cudaSuccess)
        return e;
    if (c->kev[SPH_KEV_FORCE][1]) return cudaEventRecord(c->kev[SPH_KEV_FORCE][1], c->stream);
    return cudaSuccess;
}

// The force over the level hierarchy: one pack pass, the per-level lists,
// then one launch per level over that level's work items.
cudaError_t run_force_levels(sph_ctx *c)
{
    if (c->n == 0) return cudaSuccess;
    ForceArgs a = force_args(c);
    a.c.mkey = c->slot_cell();
    a.c.tslot = c->tlist;
    a.c.fine_n = 1 << c->lvl_max;
    for (int k = 0; k < 3; ++k) a.c.fine_edge[k] = (float)c->edge[k];
    int32_t *plist = c->keys[c->sorted_buf ^ 1], *pkey = c->vals[c->sorted_buf ^ 1];   // free after the sort
    a.c.pkey = pkey;
    a.c.lstart = c->lstart;
    a.c.lvl_min = c->lvl_min;
    a.c.lvl_max = c->lvl_max;
    a.c.defer = c->tcode;     // free while the level's kernels run (its items are built)
    for (int l = 0; l <= kLevelMax; ++l) {
        double e_l = std::ldexp(c->params.box[0], -l);
        for (int k = 1; k < 3; ++k) e_l = std::fmin(e_l, std::ldexp(c->params.box[k], -l));
        a.c.lcap[l] = (float)std::fmin(0.5 * e_l, c->params.h_max);
    }
    cudaError_t e;
    k_force_pack<<<(unsigned)((c->n + 255) / 256), 256, 0, c->stream>>>(a, c->slot_cell(), nullptr, c->pack,
                                                                       c->pack + c->n, c->pack + 2 * c->n);
    c->launches += 1;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = run_level_lists(c, plist, pkey)) != cudaSuccess) return e;
    if ((e = run_coarse_index(c, pkey, c->lstart + c->lvl_min, c->lvl_max - c->lvl_min + 1, c->cl_lc,
                              c->cidx + c->cs_stride)) != cudaSuccess)
        return e;
    a.lA = c->lpack;
    a.lB = c->lpack + c->n;
    a.lC = c->lpack + 2 * c->n;
    k_lvl_gather_pack<<<(unsigned)((c->n + 255) / 256), 256, 0, c->stream>>>(plist, c->n, a.pA, a.pB, a.pC,
                                                                             c->lpack, c->lpack + c->n,
                                                                             c->lpack + 2 * c->n);
    c->launches += 1;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const size_t smem = force_smem_bytes(c->tuning.block_threads_force, a.c.cap);
    int w_one = kOneWarps;
    while (w_one > 1 && force_smem_bytes(32 * w_one, a.c.cap) + 256 > c->smem_optin) --w_one;
    const size_t smem_one = force_smem_bytes(32 * w_one, a.c.cap);
    const size_t smem_1 = force_smem_bytes(32, a.c.cap);
    for (int l = c->lvl_max; l >= c->lvl_min; --l) {
        if ((e = run_level_items(c, l)) != cudaSuccess) return e;
        for (int k = 0; k < 3; ++k) a.c.edge[k] = (float)std::ldexp(c->params.box[k], -l);
        a.c.lvl_dn = c->lvl_max - l;
        a.c.lvl_n = 1 << l;
        a.lvl = l;
        if ((e = cudaMemsetAsync(&c->dstats->defer_n, 0, 4 * sizeof(unsigned), c->stream)) != cudaSuccess) return e;
        if ((e = launch_persistent(c, k_force<true>, a, smem, c->lc_force_lv, c->tuning.block_threads_force)) != cudaSuccess) return e;
        if ((e = run_per_target(c, k_force_one, a, smem_1, smem_one, w_one, kForceHeavyStages * a.c.cap,
                                c->lc_force_one, c->lc_force_blk)) != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

}  // namespace sph
