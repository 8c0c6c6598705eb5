// S1 cell binning: FP64 cell index per particle, cell histogram, exclusive
// scan, then the particles placed cell by cell in ascending original index
// (the result of a stable sort by cell): on the uniform grid by counting
// placement and an ordering pass over each cell's range, for the level
// hierarchy and the allocation-free entry point by a stable LSD radix sort of
// (key, particle index) pairs.  Also builds the pair-kernel work items (cell,
// first slot, count) and optionally rewrites the AoS records in cell order.
#include "k_cellkey.cuh"

namespace sph {
namespace {

// ---------------------------------------------------------------------------
// cell id of every particle: k_d = clamp(floor(x_d * (nc_d / L_d)), 0, nc_d-1)
// ---------------------------------------------------------------------------
struct CellArgs {
    const uint8_t *aos;
    int64_t n;
    int32_t stride, xoff;
    double box[3];
    CellGrid g;
    int32_t *keys, *vals, *count;
    DevStats *st;
};

// x in [0, L) compared on bit patterns (FP64 compares are slow on this GPU):
// non-negative doubles order like their bits; -0 counts as inside
__device__ __forceinline__ bool in_box(double x, double L)
{
    const long long b = __double_as_longlong(x);
    return (b >= 0 && b < __double_as_longlong(L)) || b == (long long)0x8000000000000000ull;
}

// Each thread takes kBinU particles, kBinThreads apart, their loads issued
// together (a thread per particle leaves too few loads in flight).
constexpr int kBinThreads = 256;
constexpr int kBinU = 4;

__global__ void __launch_bounds__(kBinThreads) k_cell_ids(CellArgs a)
{
    const int64_t i0 = (int64_t)blockIdx.x * (kBinThreads * kBinU) + threadIdx.x;
    double x[kBinU][3];
#pragma unroll
    for (int u = 0; u < kBinU; ++u) {
        const int64_t i = i0 + u * kBinThreads;
        if (i < a.n) {
            const double *p = (const double *)(a.aos + i * a.stride + a.xoff);
            x[u][0] = p[0];
            x[u][1] = p[1];
            x[u][2] = p[2];
        }
    }
#pragma unroll
    for (int u = 0; u < kBinU; ++u) {
        const int64_t i = i0 + u * kBinThreads;
        const bool ok = i < a.n;
        int32_t c = -1;
        if (ok) {
            const double x0 = x[u][0], x1 = x[u][1], x2 = x[u][2];
            const bool outside = !(in_box(x0, a.box[0]) && in_box(x1, a.box[1]) && in_box(x2, a.box[2]));
            if (outside)
                set_error(a.st, SPH_ERR_OUTSIDE |
                                    ((isfinite(x0) && isfinite(x1) && isfinite(x2)) ? 0u : SPH_ERR_NONFINITE));
            c = cell_key(a.g, x0, x1, x2);
            a.keys[i] = c;
            if (a.vals) a.vals[i] = (int32_t)i;
        }
        // one atomic per key present in the warp (neighbouring records often
        // share their cell)
        const unsigned peers = __match_any_sync(0xffffffffu, c);
        if (ok && (int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&a.count[c], __popc(peers));
    }
}

// The histogram alone, over the keys the drift computed for the positions it
// wrote (k_kick_drift), when the caller vouches that the records have not
// changed since.
__global__ void __launch_bounds__(kBinThreads) k_key_hist(const int32_t *keys, int64_t n, int32_t *count)
{
    const int64_t i0 = (int64_t)blockIdx.x * (kBinThreads * kBinU) + threadIdx.x;
    int32_t c[kBinU];
#pragma unroll
    for (int u = 0; u < kBinU; ++u) {
        const int64_t i = i0 + u * kBinThreads;
        c[u] = i < n ? keys[i] : -1;
    }
#pragma unroll
    for (int u = 0; u < kBinU; ++u) {
        const unsigned peers = __match_any_sync(0xffffffffu, c[u]);
        if (c[u] >= 0 && (int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&count[c[u]], __popc(peers));
    }
}

// ---------------------------------------------------------------------------
// counting placement (the context's binning): the histogram and its scan
// give every key its range of slots; each particle takes a slot in its
// key's range, and k_seg_order then puts every range in ascending particle
// index, which makes the result that of a stable sort by key
// ---------------------------------------------------------------------------
// cursor[K] holds K's count on entry and 0 on exit.  A warp claims, per key
// present in it, the next block of its range (one atomic), its lanes in
// index order.  Blocks of different warps follow the order of their atomics.
__global__ void __launch_bounds__(kBinThreads) k_place(const int32_t *key, int64_t n, const int32_t *start,
                                                     int32_t *cursor, int32_t *perm, int32_t *skey)
{
    const int64_t i0 = (int64_t)blockIdx.x * (kBinThreads * kBinU) + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    int32_t K[kBinU], s0[kBinU], s1[kBinU], left[kBinU];
    unsigned peers[kBinU];
#pragma unroll
    for (int u = 0; u < kBinU; ++u) {
        const int64_t i = i0 + u * kBinThreads;
        K[u] = i < n ? key[i] : -1;
    }
#pragma unroll
    for (int u = 0; u < kBinU; ++u) {
        s0[u] = K[u] >= 0 ? start[K[u]] : 0;
        s1[u] = K[u] >= 0 ? start[K[u] + 1] : 0;
        peers[u] = __match_any_sync(0xffffffffu, K[u]);
        left[u] = 0;
        if (K[u] >= 0 && lane == __ffs(peers[u]) - 1) left[u] = atomicSub(&cursor[K[u]], __popc(peers[u]));
    }
#pragma unroll
    for (int u = 0; u < kBinU; ++u) {
        const int64_t i = i0 + u * kBinThreads;
        const int l = __shfl_sync(0xffffffffu, left[u], __ffs(peers[u]) - 1);
        if (i < n) {
            const int32_t pos = s0[u] + (s1[u] - s0[u] - l) + __popc(peers[u] & lt);
            perm[pos] = (int32_t)i;
            skey[pos] = K[u];
        }
    }
}

// A slot whose successor in the same key range holds a smaller particle
// index marks that key (plain stores: every writer stores 1).  mark[] is zero
// on entry (the cursors after k_place).  A thread checks four slots, loaded
// as one 16-byte vector per array.
__global__ void __launch_bounds__(kBinThreads) k_inversions(const int32_t *perm, const int32_t *skey, int64_t n,
                                                          int32_t *mark)
{
    const int64_t p = 4 * ((int64_t)blockIdx.x * kBinThreads + threadIdx.x);
    if (p + 1 >= n) return;
    int32_t pv[5], kv[5];
    int m;
    if (p + 4 < n) {
        const int4 a = *reinterpret_cast<const int4 *>(perm + p);
        const int4 b = *reinterpret_cast<const int4 *>(skey + p);
        pv[0] = a.x, pv[1] = a.y, pv[2] = a.z, pv[3] = a.w, pv[4] = perm[p + 4];
        kv[0] = b.x, kv[1] = b.y, kv[2] = b.z, kv[3] = b.w, kv[4] = skey[p + 4];
        m = 4;
    } else {
        m = (int)(n - 1 - p);
        for (int j = 0; j <= m; ++j) {
            pv[j] = perm[p + j];
            kv[j] = skey[p + j];
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j)
        if (j < m && kv[j] == kv[j + 1] && pv[j] > pv[j + 1]) mark[kv[j]] = 1;
}

// ascending bitonic sort of one value per lane
__device__ __forceinline__ int32_t warp_bitonic32(int32_t v, int lane)
{
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1)
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const int32_t o = __shfl_xor_sync(0xffffffffu, v, j);
            const bool up = (lane & k) == 0;          // this block of k lanes ascends
            const bool low = (lane & j) == 0;         // this lane keeps the smaller of the pair
            v = (low == up) ? min(v, o) : max(v, o);
        }
    return v;
}

constexpr int kSegSmem = 1024;        // particle indices one warp sorts in shared memory
constexpr int kSegWarps = 8;          // warps per k_seg_order block

// One key range put in ascending order by one warp: up to 32 indices in
// registers, up to kSegSmem by a bitonic network in shared memory, longer
// ranges by a stable LSD radix sort on the index bits (8 per pass) through
// the same range of `scratch`.
__device__ void warp_order_range(int32_t *seg, int32_t *scratch, int32_t len, int64_t n, int32_t *buf, int lane)
{
    const unsigned lt = (1u << lane) - 1u;
    if (len <= 32) {
        const int32_t v = warp_bitonic32(lane < len ? seg[lane] : INT32_MAX, lane);
        if (lane < len) seg[lane] = v;
        return;
    }
    if (len <= kSegSmem) {
        int P = 64;
        while (P < len) P <<= 1;
        for (int i = lane; i < P; i += 32) buf[i] = i < len ? seg[i] : INT32_MAX;
        __syncwarp();
        for (int k = 2; k <= P; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = lane; i < P; i += 32) {
                    const int l = i ^ j;
                    if (l > i) {
                        const int32_t x = buf[i], y = buf[l];
                        if ((x > y) == ((i & k) == 0)) {
                            buf[i] = y;
                            buf[l] = x;
                        }
                    }
                }
                __syncwarp();
            }
        for (int i = lane; i < len; i += 32) seg[i] = buf[i];
        __syncwarp();
        return;
    }
    int bits = 1;
    while (bits < 31 && ((int64_t)1 << bits) < n) ++bits;
    int32_t *src = seg, *dst = scratch;
    for (int shift = 0; shift < bits; shift += 8) {
        for (int d = lane; d < 256; d += 32) buf[d] = 0;
        __syncwarp();
        for (int i = lane; i < len; i += 32) atomicAdd(&buf[((uint32_t)src[i] >> shift) & 255u], 1);
        __syncwarp();
        {   // exclusive scan of the 256 digit counts, 8 per lane
            int32_t cnt[8], sum = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                cnt[q] = buf[lane * 8 + q];
                sum += cnt[q];
            }
            int32_t inc = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            int32_t e = inc - sum;
            __syncwarp();
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                buf[lane * 8 + q] = e;
                e += cnt[q];
            }
        }
        __syncwarp();
        // stable scatter, 32 indices per round in index order
        for (int b0 = 0; b0 < len; b0 += 32) {
            const int i = b0 + lane;
            const bool ok = i < len;
            const int32_t v = ok ? src[i] : 0;
            const uint32_t d = ok ? (((uint32_t)v >> shift) & 255u) : 256u;
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            const int r = __popc(peers & lt);
            if (ok) dst[buf[d] + r] = v;
            __syncwarp();
            if (ok && r == 0) buf[d] += __popc(peers);
            __syncwarp();
        }
        int32_t *tmp = src;
        src = dst;
        dst = tmp;
    }
    if (src != seg)
        for (int i = lane; i < len; i += 32) seg[i] = src[i];
    __syncwarp();
}

// Every marked key range put in ascending order.  A warp task is 32
// consecutive keys.  Its marked ranges of up to 32 indices are sorted four at
// a time in registers (four independent loads and bitonic networks keep the
// warp busy while one range waits on memory), longer ones one by one.
__global__ void __launch_bounds__(32 * kSegWarps) k_seg_order(const int32_t *start, const int32_t *mark, int64_t nkeys,
                                                             int32_t *perm, int32_t *scratch, int64_t n)
{
    __shared__ int32_t sm[kSegWarps][kSegSmem];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t nw = (int64_t)gridDim.x * kSegWarps;
    for (int64_t t = (int64_t)blockIdx.x * kSegWarps + w; t * 32 < nkeys; t += nw) {
        const int64_t k0 = t * 32;
        const bool in = k0 + lane < nkeys && mark[k0 + lane] != 0;
        const int32_t my_s = in ? start[k0 + lane] : 0;
        const int32_t my_len = in ? start[k0 + lane + 1] - my_s : 0;
        unsigned small = __ballot_sync(0xffffffffu, in && my_len <= 32);
        unsigned big = __ballot_sync(0xffffffffu, in && my_len > 32);
        while (small) {
            int32_t v[4], sq[4], lq[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int src = small ? __ffs(small) - 1 : 0;
                lq[q] = small ? __shfl_sync(0xffffffffu, my_len, src) : 0;
                sq[q] = __shfl_sync(0xffffffffu, my_s, src);
                small &= small - 1;
                v[q] = lane < lq[q] ? perm[sq[q] + lane] : INT32_MAX;
            }
#pragma unroll
            for (int k = 2; k <= 32; k <<= 1)
#pragma unroll
                for (int j = k >> 1; j > 0; j >>= 1) {
                    const bool keep_min = ((lane & j) == 0) == ((lane & k) == 0);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int32_t o = __shfl_xor_sync(0xffffffffu, v[q], j);
                        v[q] = keep_min ? min(v[q], o) : max(v[q], o);
                    }
                }
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (lane < lq[q]) perm[sq[q] + lane] = v[q];
        }
        while (big) {
            const int src = __ffs(big) - 1;
            big &= big - 1;
            const int32_t s0 = __shfl_sync(0xffffffffu, my_s, src), len = __shfl_sync(0xffffffffu, my_len, src);
            warp_order_range(perm + s0, scratch + s0, len, n, sm[w], lane);
        }
    }
}

// ---------------------------------------------------------------------------
// device-wide exclusive scan (reduce / scan partials / downsweep)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int32_t warp_incl_scan(int32_t v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// exclusive scan of one value per thread across a 1024-thread block; returns
// the block total in *total
__device__ int32_t block_excl_scan(int32_t v, int32_t *smem32, int32_t *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t inc = warp_incl_scan(v);
    if (lane == 31) smem32[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int32_t w = lane < (int)(blockDim.x >> 5) ? smem32[lane] : 0;
        int32_t wi = warp_incl_scan(w);
        smem32[lane] = wi - w;
        if (lane == 31) smem32[32] = wi;
    }
    __syncthreads();
    int32_t r = inc - v + smem32[warp];
    *total = smem32[32];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const int32_t *in, int64_t len, int32_t *part)
{
    __shared__ int32_t s[33];
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int32_t sum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < len) sum += in[base + k];
    int32_t tot;
    block_excl_scan(sum, s, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// exclusive scan of part[0..nb) in place by one block; writes the grand total
// to part[nb] and to out[len]
__global__ void __launch_bounds__(kScanThreads) k_scan_partials(int32_t *part, int64_t nb, int32_t *out, int64_t len)
{
    __shared__ int32_t s[33];
    int32_t carry = 0;
    for (int64_t c0 = 0; c0 < nb; c0 += kScanThreads) {
        int64_t i = c0 + threadIdx.x;
        int32_t v = i < nb ? part[i] : 0;
        int32_t tot;
        int32_t e = block_excl_scan(v, s, &tot);
        if (i < nb) part[i] = e + carry;
        carry += tot;
    }
    if (threadIdx.x == 0) {
        part[nb] = carry;
        out[len] = carry;
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_down(const int32_t *in, int32_t *out, int64_t len, const int32_t *part)
{
    __shared__ int32_t s[33];
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int32_t v[kScanItems];
    int32_t sum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = base + k < len ? in[base + k] : 0;
        sum += v[k];
    }
    int32_t tot;
    int32_t e = block_excl_scan(sum, s, &tot) + part[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < len) out[base + k] = e;
        e += v[k];
    }
}

// ---------------------------------------------------------------------------
// stable LSD radix sort, 8-bit digits
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kRadixThreads) k_radix_hist(const int32_t *keys, int64_t n, int shift, uint32_t *ghist, int64_t nblk)
{
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kRadixTile;
#pragma unroll
    for (int r = 0; r < kRadixItems; ++r) {
        int64_t i = base + r * kRadixThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[((uint32_t)keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    ghist[(int64_t)threadIdx.x * nblk + blockIdx.x] = h[threadIdx.x];
}

// Scatter one tile.  Keys are ranked in tile order (round by round, then
// warp, then lane), so equal digits keep their input order: the sort is
// stable.  ghist holds the exclusive scan over (digit, block).
__global__ void __launch_bounds__(kRadixThreads) k_radix_scatter(const int32_t *kin, const int32_t *vin, int32_t *kout,
                                                                 int32_t *vout, int64_t n, int shift,
                                                                 const uint32_t *ghist, int64_t nblk)
{
    constexpr int W = kRadixThreads / 32;
    __shared__ uint32_t s_base[256];
    __shared__ uint32_t s_run[256];
    __shared__ uint32_t s_cnt[W][256];
    __shared__ uint32_t s_pre[W][256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    s_base[tid] = ghist[(int64_t)tid * nblk + blockIdx.x];
    s_run[tid] = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) s_cnt[w][tid] = 0;
    __syncthreads();
    const uint32_t lt = (1u << lane) - 1u;
    int64_t base = (int64_t)blockIdx.x * kRadixTile;
    for (int r = 0; r < kRadixItems; ++r) {
        int64_t i = base + r * kRadixThreads + tid;
        bool ok = i < n;
        int32_t key = ok ? kin[i] : 0;
        int32_t val = ok ? vin[i] : 0;
        uint32_t d = ok ? (((uint32_t)key >> shift) & 255u) : 256u;
        uint32_t peers = __match_any_sync(0xffffffffu, d);
        uint32_t rank = __popc(peers & lt);
        if (ok && rank == 0) s_cnt[warp][d] = __popc(peers);
        __syncthreads();
        {   // per digit: exclusive prefix over warps, carried across rounds
            uint32_t run = s_run[tid];
#pragma unroll
            for (int w = 0; w < W; ++w) {
                uint32_t c = s_cnt[w][tid];
                s_pre[w][tid] = run;
                s_cnt[w][tid] = 0;
                run += c;
            }
            s_run[tid] = run;
        }
        __syncthreads();
        if (ok) {
            uint32_t pos = s_base[d] + s_pre[warp][d] + rank;
            kout[pos] = key;
            vout[pos] = val;
        }
    }
}

// ---------------------------------------------------------------------------
// work items: each cell is split into tiles of `block` slots
// ---------------------------------------------------------------------------
// cell_start is indexed by sub-cell key; cell c spans keys [c s3, (c+1) s3)
__global__ void k_items_count(const int32_t *cell_start, int64_t ncell, int s3, int block, int32_t *tmp,
                              DevStats *st)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int32_t cnt = 0;
    if (c < ncell) {
        cnt = cell_start[(c + 1) * s3] - cell_start[c * s3];
        tmp[c] = (cnt + block - 1) / block;
    }
    // one atomic per block
    __shared__ int32_t wmax[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt = max(cnt, __shfl_xor_sync(0xffffffffu, cnt, o));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) cnt = max(cnt, wmax[w]);
        if (cnt > 0) atomicMax(&st->max_occ, cnt);
    }
}

__global__ void k_items_fill(const int32_t *cell_start, const int32_t *item_off, int64_t ncell, int s3, int block,
                             int32_t *icell, int32_t *ifirst, int32_t *icount, DevStats *st)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c == 0) st->nitems = item_off[ncell];
    if (c >= ncell) return;
    int32_t s = cell_start[c * s3], e = cell_start[(c + 1) * s3];
    int32_t o = item_off[c];
    for (int32_t f = s; f < e; f += block, ++o) {
        icell[o] = (int32_t)c;
        ifirst[o] = f;
        icount[o] = min(block, e - f);
    }
}

// ---------------------------------------------------------------------------
// optional queue order: work items grouped by cost class, costliest first
// ---------------------------------------------------------------------------

__device__ __forceinline__ int item_class_key(const int32_t *cell_start, int cell, int count, int3 nc, int s3)
{
    const int kx = cell % nc.x, t = cell / nc.x, ky = t % nc.y, kz = t / nc.y;
    long long occ = 0;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const int x = (kx + dx + nc.x) % nc.x, y = (ky + dy + nc.y) % nc.y, z = (kz + dz + nc.z) % nc.z;
                const long long cid = x + (long long)nc.x * (y + (long long)nc.y * z);
                occ += cell_start[(cid + 1) * s3] - cell_start[cid * s3];
            }
    const long long cost = (long long)count * occ;
    const int lg = cost > 0 ? min(63 - __clzll(cost), kItemClasses - 1) : 0;
    return kItemClasses - 1 - lg;
}

// class key of every item: the power of two of (its particle count x the
// particles of the 27 cells around its cell), stored as
// kItemClasses - 1 - log2 so that ascending keys put the costliest first
__global__ void k_item_class(const int32_t *cell_start, const int32_t *icell, const int32_t *icount, int3 nc,
                             int s3, const DevStats *st, int32_t *key, int32_t *hist)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool ok = i < st->nitems;
    int kk = -1;
    if (ok) kk = item_class_key(cell_start, icell[i], icount[i], nc, s3);
    if (ok) key[i] = kk;
    // few distinct classes: one atomic per class present in the warp
    const unsigned peers = __match_any_sync(0xffffffffu, kk);
    if (ok && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&hist[kk], __popc(peers));
}

// one warp: class starts (kItemClasses + 1 entries) and scatter cursors
__global__ void k_class_scan(int32_t *hist)
{
    const int lane = threadIdx.x;
    const int32_t v = hist[lane];
    int32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    int32_t *start = hist + kItemClasses, *cursor = hist + 2 * kItemClasses + 1;
    start[lane] = inc - v;
    cursor[lane] = inc - v;
    if (lane == 31) start[kItemClasses] = inc;
}

__global__ void k_item_scatter(const int32_t *icell, const int32_t *ifirst, const int32_t *icount,
                               const int32_t *key, int32_t *cursor, int32_t *sorted, int64_t item_max,
                               const DevStats *st)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const bool ok = i < st->nitems;
    const int kk = ok ? key[i] : -1;
    // one atomic per class present in the warp; the lanes of a class take
    // consecutive positions from it
    const unsigned peers = __match_any_sync(0xffffffffu, kk);
    const int leader = __ffs(peers) - 1;
    int base = 0;
    if (ok && lane == leader) base = atomicAdd(&cursor[kk], __popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (!ok) return;
    const int pos = base + __popc(peers & ((1u << lane) - 1u));
    sorted[pos] = icell[i];
    sorted[item_max + pos] = ifirst[i];
    sorted[2 * item_max + pos] = icount[i];
}

// ---------------------------------------------------------------------------
// optional AoS reordering
// ---------------------------------------------------------------------------
__global__ void k_gather_records(const uint8_t *aos, uint8_t *dst, const int32_t *perm, int64_t n, int32_t stride)
{
    // one warp per record, 8-byte words
    int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (warp >= n) return;
    const uint64_t *src = (const uint64_t *)(aos + (int64_t)perm[warp] * stride);
    uint64_t *d = (uint64_t *)(dst + warp * stride);
    for (int w = lane; w < stride / 8; w += 32) d[w] = src[w];
}

// cell origins k * edge_d per axis (FP64 product, as the conversion's
// cell-relative offsets define them), kMaxCellsPerAxis entries per axis
__global__ void k_origins(double *origin, int3 nc, double3 edge)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= kMaxCellsPerAxis) return;
    origin[k] = k < nc.x ? __dmul_rn((double)k, edge.x) : 0.0;
    origin[kMaxCellsPerAxis + k] = k < nc.y ? __dmul_rn((double)k, edge.y) : 0.0;
    origin[2 * kMaxCellsPerAxis + k] = k < nc.z ? __dmul_rn((double)k, edge.z) : 0.0;
}

__global__ void k_iota(int32_t *p, int64_t n)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = (int32_t)i;
}

// ---------------------------------------------------------------------------
// level hierarchy: Morton key of the finest cell and the level of every
// particle
// ---------------------------------------------------------------------------
struct LevelArgs {
    const uint8_t *aos;
    int64_t n;
    int32_t stride, xoff, hoff;
    bool h64;                    // h stored as FP64 in the record (else FP32)
    double inv[3], box[3];       // inv = 2^lmax / L per axis
    int32_t F;                   // 2^lmax cells per axis
    int32_t lmin, lmax;
    double grow;                 // 1 + margin
    double cap[kLevelMax + 1];   // h_l = min_d (L_d / 2^l) / 2
    int32_t *keys, *vals;
    int8_t *lvl;
    DevStats *st;
};

__global__ void k_level_keys(LevelArgs a)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const uint8_t *rec = a.aos + i * a.stride;
    const double *x = (const double *)(rec + a.xoff);
    const double x0 = x[0], x1 = x[1], x2 = x[2];
    const bool outside = !(in_box(x0, a.box[0]) && in_box(x1, a.box[1]) && in_box(x2, a.box[2]));
    if (outside) set_error(a.st, SPH_ERR_OUTSIDE | ((isfinite(x0) && isfinite(x1) && isfinite(x2)) ? 0u : SPH_ERR_NONFINITE));
    const uint32_t fx = (uint32_t)cell_coord(x0, a.inv[0], a.F);
    const uint32_t fy = (uint32_t)cell_coord(x1, a.inv[1], a.F);
    const uint32_t fz = (uint32_t)cell_coord(x2, a.inv[2], a.F);
    a.keys[i] = (int32_t)morton_key(fx, fy, fz);
    a.vals[i] = (int32_t)i;
    const double h = a.h64 ? *(const double *)(rec + a.hoff) : (double)*(const float *)(rec + a.hoff);
    int lv = a.lmin;
    if (h > 0.0 && isfinite(h)) {
        // the finest level whose cap holds h (1 + margin); caps shrink with l
        const double t = __dmul_rn(h, a.grow);
        for (int l = a.lmax; l > a.lmin; --l)
            if (t <= a.cap[l]) {
                lv = l;
                break;
            }
    }
    a.lvl[i] = (int8_t)lv;
}

__global__ void k_level_permute(const int8_t *lvl_in, const int32_t *perm, int64_t n, int8_t *lvl_out)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) lvl_out[k] = lvl_in[perm[k]];
}

// ---------------------------------------------------------------------------
// work items of one level: the level's particles in slot order, split into
// tiles of <= 32 that share a cell of the level
// ---------------------------------------------------------------------------
__global__ void k_lvl_flags(const int8_t *level, int64_t n, int l, int32_t *flag)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) flag[k] = level[k] == l ? 1 : 0;
}

// pos: exclusive scan of the flags; the level's slots and their cell codes
// at the level (key >> sh) in slot order
__global__ void k_lvl_compact(const int8_t *level, const int32_t *pos, const int32_t *key, int64_t n, int l, int sh,
                              int32_t *tlist, int32_t *tcode)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n || level[k] != l) return;
    const int32_t j = pos[k];
    tlist[j] = (int32_t)k;
    tcode[j] = key[k] >> sh;
}

// first index in [lo, hi) whose code is >= v (codes ascend)
__device__ __forceinline__ int32_t code_lower_bound(const int32_t *code, int32_t lo, int32_t hi, int32_t v)
{
    while (lo < hi) {
        const int32_t mid = lo + ((hi - lo) >> 1);
        if (code[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// entry j opens a work item when its rank inside its cell's run is a
// multiple of 32; *M (the scan total) is the level's particle count
__global__ void k_lvl_starts(const int32_t *tcode, const int32_t *M, int64_t n, int32_t *start)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    if (j >= *M) {
        start[j] = 0;
        return;
    }
    const int32_t head = code_lower_bound(tcode, 0, (int32_t)j, tcode[j]);
    start[j] = (((int32_t)j - head) & (kItemTile - 1)) == 0 ? 1 : 0;
}

// iscan: exclusive scan of the start flags (iscan[n] = items)
__global__ void k_lvl_items(const int32_t *tcode, const int32_t *M, const int32_t *iscan, int64_t n, int64_t item_max,
                            int32_t *icell, int32_t *ifirst, int32_t *icount, DevStats *st)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j == 0) st->nitems = (int)min((int64_t)iscan[n], item_max);
    if (j >= n) return;
    const int32_t m = *M;
    if (j >= m || iscan[j + 1] == iscan[j]) return;
    const int32_t o = iscan[j];
    if (o >= item_max) return;     // cannot happen: item_max >= n/32 + n + 1
    const int32_t code = tcode[j];
    const int32_t end = code_lower_bound(tcode, (int32_t)j, m, code + 1);
    icell[o] = code;
    ifirst[o] = (int32_t)j;
    icount[o] = min(kItemTile, end - (int32_t)j);
}

// per-level lists: level l's slots in slot (Morton) order at
// [lstart[l], lstart[l+1]) of plist, with their keys
__global__ void k_lvl_list(const int8_t *level, const int32_t *pos, const int32_t *key, int64_t n, int l,
                           const int32_t *lstart, int32_t *plist, int32_t *pkey)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n || level[k] != l) return;
    const int32_t j = lstart[l] + pos[k];
    plist[j] = (int32_t)k;
    pkey[j] = key[k];
}

__global__ void k_lvl_list_next(int32_t *lstart, int l, const int32_t *M)
{
    if (threadIdx.x == 0) lstart[l + 1] = lstart[l] + *M;
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t scan_exclusive(const int32_t *in, int32_t *out, int64_t len, int32_t *part, cudaStream_t s,
                           uint64_t *launches)
{
    if (len <= 0) {
        return cudaMemsetAsync(out, 0, sizeof(int32_t), s);
    }
    *launches += 3;
    int64_t nb = (len + kScanTile - 1) / kScanTile;
    k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, s>>>(in, len, part);
    k_scan_partials<<<1, kScanThreads, 0, s>>>(part, nb, out, len);
    k_scan_down<<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, len, part);
    return cudaGetLastError();
}

namespace {

// stable LSD radix sort of the (keys[0], vals[0]) pairs on their low `bits`
// bits, 8 per pass; sorted_buf names the buffer that holds the result
cudaError_t radix_sort(sph_ctx *c, int bits)
{
    cudaStream_t s = c->stream;
    cudaError_t e;
    const int64_t n = c->n;
    const int64_t nblk = c->plan.nblk_radix;
    int cur = 0;
    for (int shift = 0; shift < bits; shift += 8) {
        k_radix_hist<<<(unsigned)nblk, kRadixThreads, 0, s>>>(c->keys[cur], n, shift, c->ghist, nblk);
        c->launches += 2;   // histogram and scatter
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = scan_exclusive((const int32_t *)c->ghist, (int32_t *)c->ghist, 256 * nblk, c->scan_part, s,
                                &c->launches)) != cudaSuccess)
            return e;
        k_radix_scatter<<<(unsigned)nblk, kRadixThreads, 0, s>>>(c->keys[cur], c->vals[cur], c->keys[cur ^ 1],
                                                                 c->vals[cur ^ 1], n, shift, c->ghist, nblk);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        cur ^= 1;
    }
    c->sorted_buf = cur;
    return cudaSuccess;
}

}  // namespace

cudaError_t run_binning(sph_ctx *c, int reorder, bool drift_keys)
{
    cudaStream_t s = c->stream;
    cudaError_t e;
    const int64_t n = c->n;
    const int S = c->sub;
    const int64_t nkeys = c->ncell * S * S * S;     // sub-cells
    if ((e = cudaMemsetAsync(c->cell_count, 0, sizeof(int32_t) * nkeys, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(&c->dstats->max_occ, 0, sizeof(int), s)) != cudaSuccess) return e;
    c->sorted_buf = 0;
    k_origins<<<kMaxCellsPerAxis / 256, 256, 0, s>>>(c->origin, make_int3(c->nc[0], c->nc[1], c->nc[2]),
                                                     make_double3(c->edge[0], c->edge[1], c->edge[2]));
    c->launches += 1;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (n > 0 && drift_keys) {
        // keys[0] holds the keys of the drifted positions
        k_key_hist<<<blocks_for(n, kBinThreads * kBinU), kBinThreads, 0, s>>>(c->keys[0], n, c->cell_count);
        c->launches += 1;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    } else if (n > 0) {
        CellArgs a;
        a.aos = c->aos;
        a.n = n;
        a.stride = c->layout.record_bytes;
        a.xoff = c->layout.offset[SPH_F_X];
        a.g = cell_grid(c->nc, S, c->params.box);
        for (int k = 0; k < 3; ++k) a.box[k] = c->params.box[k];
        a.keys = c->keys[0];
        a.vals = nullptr;
        a.count = c->cell_count;
        a.st = c->dstats;
        k_cell_ids<<<blocks_for(n, kBinThreads * kBinU), kBinThreads, 0, s>>>(a);
        c->launches += 1;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if ((e = scan_exclusive(c->cell_count, c->cell_start, nkeys, c->scan_part, s, &c->launches)) != cudaSuccess) return e;
    if (n > 0) {
        // keys[0] (the particles' keys) -> keys[1] / vals[1] (sorted keys and
        // permutation); cell_count (the cursors, zero after k_place) marks the
        // ranges to order and vals[0] is the radix scratch of long ranges
        k_place<<<blocks_for(n, kBinThreads * kBinU), kBinThreads, 0, s>>>(c->keys[0], n, c->cell_start, c->cell_count, c->vals[1],
                                                   c->keys[1]);
        k_inversions<<<blocks_for((n + 3) / 4, kBinThreads), kBinThreads, 0, s>>>(c->vals[1], c->keys[1], n, c->cell_count);
        k_seg_order<<<(unsigned)(c->sm_count * 4), 32 * kSegWarps, 0, s>>>(c->cell_start, c->cell_count, nkeys,
                                                                          c->vals[1], c->vals[0], n);
        c->launches += 3;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        c->sorted_buf = 1;
        if (reorder) {
            k_gather_records<<<blocks_for(n * 32, 256), 256, 0, s>>>(c->aos, c->aos_tmp, c->perm(), n,
                                                                     c->layout.record_bytes);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            // (cudaMemcpyDefault: the records may live in host memory the
            // device maps, the streaming layout)
            if ((e = cudaMemcpyAsync(c->aos, c->aos_tmp, (size_t)n * c->layout.record_bytes,
                                     cudaMemcpyDefault, s)) != cudaSuccess)
                return e;
            k_iota<<<blocks_for(n, 256), 256, 0, s>>>(c->perm(), n);
            c->launches += 2;   // gather and iota
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

// Binning over caller-supplied buffers (no context): the same kernels as
// run_binning, driven with explicit pointers.  Results go to out_perm,
// out_cell and out_start.
cudaError_t bin_raw(const BinRaw &b, cudaStream_t s)
{
    cudaError_t e;
    if ((e = cudaMemsetAsync(b.count, 0, sizeof(int32_t) * (size_t)b.ncell, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(b.st, 0, sizeof(DevStats), s)) != cudaSuccess) return e;
    uint64_t launches = 0;
    if (b.n > 0) {
        CellArgs a;
        a.aos = b.aos;
        a.n = b.n;
        a.stride = b.stride;
        a.xoff = b.xoff;
        a.g.sub = 1;                 // plain cells: b.ncell keys
        for (int k = 0; k < 3; ++k) {
            a.g.inv[k] = b.inv[k];
            a.g.invh[k] = (float)b.inv[k];
            a.g.invl[k] = (float)(b.inv[k] - (double)a.g.invh[k]);
            a.g.nc[k] = b.nc[k];
            a.box[k] = b.box[k];
        }
        a.keys = b.keys[0];
        a.vals = b.vals[0];
        a.count = b.count;
        a.st = b.st;
        k_cell_ids<<<blocks_for(b.n, kBinThreads * kBinU), kBinThreads, 0, s>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if ((e = scan_exclusive(b.count, b.out_start, b.ncell, b.scan_part, s, &launches)) != cudaSuccess) return e;
    if (b.n == 0) return cudaSuccess;
    int bits = 0;
    while (bits < 31 && ((int64_t)1 << bits) < b.ncell) ++bits;
    const int64_t nblk = (b.n + kRadixTile - 1) / kRadixTile;
    int cur = 0;
    for (int shift = 0; shift < bits; shift += 8) {
        k_radix_hist<<<(unsigned)nblk, kRadixThreads, 0, s>>>(b.keys[cur], b.n, shift, b.ghist, nblk);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = scan_exclusive((const int32_t *)b.ghist, (int32_t *)b.ghist, 256 * nblk, b.scan_part, s,
                                &launches)) != cudaSuccess)
            return e;
        k_radix_scatter<<<(unsigned)nblk, kRadixThreads, 0, s>>>(b.keys[cur], b.vals[cur], b.keys[cur ^ 1],
                                                                 b.vals[cur ^ 1], b.n, shift, b.ghist, nblk);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        cur ^= 1;
    }
    const size_t bytes = sizeof(int32_t) * (size_t)b.n;
    if ((e = cudaMemcpyAsync(b.out_perm, b.vals[cur], bytes, cudaMemcpyDeviceToDevice, s)) != cudaSuccess) return e;
    return cudaMemcpyAsync(b.out_cell, b.keys[cur], bytes, cudaMemcpyDeviceToDevice, s);
}

cudaError_t run_bin_levels(sph_ctx *c, double grow)
{
    cudaStream_t s = c->stream;
    cudaError_t e;
    const int64_t n = c->n;
    if ((e = cudaMemsetAsync(&c->dstats->max_occ, 0, sizeof(int), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(&c->dstats->nitems, 0, sizeof(int), s)) != cudaSuccess) return e;
    c->sorted_buf = 0;
    // origins of the finest cells, for the conversion's offsets
    k_origins<<<kMaxCellsPerAxis / 256, 256, 0, s>>>(c->origin, make_int3(c->nc[0], c->nc[1], c->nc[2]),
                                                     make_double3(c->edge[0], c->edge[1], c->edge[2]));
    c->launches += 1;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (n == 0) return cudaSuccess;
    LevelArgs a;
    a.aos = c->aos;
    a.n = n;
    a.stride = c->layout.record_bytes;
    a.xoff = c->layout.offset[SPH_F_X];
    a.hoff = c->layout.offset[SPH_F_H];
    a.h64 = c->layout.type[SPH_F_H] == SPH_AOS_F64;
    a.F = c->nc[0];
    for (int k = 0; k < 3; ++k) {
        a.inv[k] = c->inv[k];
        a.box[k] = c->params.box[k];
    }
    a.lmin = c->lvl_min;
    a.lmax = c->lvl_max;
    a.grow = grow;
    for (int l = 0; l <= kLevelMax; ++l) {
        double e_l = std::ldexp(c->params.box[0], -l);
        for (int k = 1; k < 3; ++k) e_l = std::fmin(e_l, std::ldexp(c->params.box[k], -l));
        a.cap[l] = 0.5 * e_l;
    }
    a.keys = c->keys[0];
    a.vals = c->vals[0];
    a.lvl = c->level_tmp;
    a.st = c->dstats;
    k_level_keys<<<blocks_for(n, 256), 256, 0, s>>>(a);
    c->launches += 1;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = radix_sort(c, 3 * c->lvl_max)) != cudaSuccess) return e;
    k_level_permute<<<blocks_for(n, 256), 256, 0, s>>>(c->level_tmp, c->perm(), n, c->level);
    c->launches += 1;
    return cudaGetLastError();
}

// Coarse index of the sorted keys of list j (blockIdx.y): entry q of its
// table is the first index of the list whose key >> shift is >= q, for q in
// [0, C]; one thread per entry, each a binary search over the list.
__global__ void k_coarse_index(const int32_t *keys, const int32_t *bounds, int64_t n, int shift, int C,
                               int64_t stride, int32_t *tables)
{
    const int j = blockIdx.y;
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q > C) return;
    int64_t lo = bounds ? bounds[j] : 0, hi = bounds ? bounds[j + 1] : n;
    const int64_t v = q << shift;           // keys are below 2^31, so v never wraps them
    while (lo < hi) {
        const int64_t mid = lo + ((hi - lo) >> 1);
        if ((int64_t)__ldg(keys + mid) < v) lo = mid + 1;
        else hi = mid;
    }
    tables[j * stride + q] = (int32_t)lo;
}

cudaError_t run_coarse_index(sph_ctx *c, const int32_t *keys, const int32_t *bounds, int nlist, int lc,
                             int32_t *tables)
{
    if (nlist <= 0) return cudaSuccess;
    const int shift = 3 * (c->lvl_max - lc);
    const int C = 1 << (3 * lc);
    const dim3 grid(blocks_for((int64_t)C + 1, 256), (unsigned)nlist);
    k_coarse_index<<<grid, 256, 0, c->stream>>>(keys, bounds, c->n, shift, C, c->cs_stride, tables);
    c->launches += 1;
    return cudaGetLastError();
}

cudaError_t run_level_items(sph_ctx *c, int l)
{
    cudaStream_t s = c->stream;
    cudaError_t e;
    const int64_t n = c->n;
    const unsigned g = blocks_for(n, 256);
    k_lvl_flags<<<g, 256, 0, s>>>(c->level, n, l, c->tscan);
    c->launches += 1;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = scan_exclusive(c->tscan, c->tscan, n, c->scan_part, s, &c->launches)) != cudaSuccess) return e;
    k_lvl_compact<<<g, 256, 0, s>>>(c->level, c->tscan, c->slot_cell(), n, l, 3 * (c->lvl_max - l), c->tlist,
                                    c->tcode);
    k_lvl_starts<<<g, 256, 0, s>>>(c->tcode, c->tscan + n, n, c->iscan);
    c->launches += 2;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = scan_exclusive(c->iscan, c->iscan, n, c->scan_part, s, &c->launches)) != cudaSuccess) return e;
    k_lvl_items<<<g, 256, 0, s>>>(c->tcode, c->tscan + n, c->iscan, n, c->plan.item_max, c->item_cell,
                                  c->item_first, c->item_count, c->dstats);
    c->launches += 1;
    return cudaGetLastError();
}

cudaError_t run_level_lists(sph_ctx *c, int32_t *plist, int32_t *pkey)
{
    cudaStream_t s = c->stream;
    cudaError_t e;
    const int64_t n = c->n;
    const unsigned g = blocks_for(n, 256);
    if ((e = cudaMemsetAsync(c->lstart, 0, sizeof(int32_t) * (kLevelMax + 2), s)) != cudaSuccess) return e;
    for (int l = c->lvl_min; l <= c->lvl_max; ++l) {
        k_lvl_flags<<<g, 256, 0, s>>>(c->level, n, l, c->tscan);
        c->launches += 1;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = scan_exclusive(c->tscan, c->tscan, n, c->scan_part, s, &c->launches)) != cudaSuccess) return e;
        k_lvl_list<<<g, 256, 0, s>>>(c->level, c->tscan, c->slot_cell(), n, l, c->lstart, plist, pkey);
        k_lvl_list_next<<<1, 32, 0, s>>>(c->lstart, l, c->tscan + n);
        c->launches += 2;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t run_items(sph_ctx *c)
{
    cudaStream_t s = c->stream;
    cudaError_t e;
    const int block = kItemTile;    // one warp per work item
    const int s3 = c->sub * c->sub * c->sub;
    k_items_count<<<blocks_for(c->ncell, 256), 256, 0, s>>>(c->cell_start, c->ncell, s3, block, c->item_tmp,
                                                            c->dstats);
    c->launches += 2;   // count and fill
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = scan_exclusive(c->item_tmp, c->item_tmp, c->ncell, c->scan_part, s, &c->launches)) != cudaSuccess) return e;
    k_items_fill<<<blocks_for(c->ncell, 256), 256, 0, s>>>(c->cell_start, c->item_tmp, c->ncell, s3, block,
                                                           c->item_cell, c->item_first, c->item_count, c->dstats);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    c->items_by_class = false;
    if (c->tuning.item_order == 1) {
        const int64_t im = c->plan.item_max;
        const unsigned g = blocks_for(im, 256);
        if ((e = cudaMemsetAsync(c->class_hist, 0, sizeof(int32_t) * kItemClasses, s)) != cudaSuccess) return e;
        k_item_class<<<g, 256, 0, s>>>(c->cell_start, c->item_cell, c->item_count,
                                       make_int3(c->nc[0], c->nc[1], c->nc[2]), s3, c->dstats, c->item_class,
                                       c->class_hist);
        k_class_scan<<<1, 32, 0, s>>>(c->class_hist);
        k_item_scatter<<<g, 256, 0, s>>>(c->item_cell, c->item_first, c->item_count, c->item_class,
                                         c->class_hist + 2 * kItemClasses + 1, c->item_sorted, im, c->dstats);
        c->launches += 3;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        int32_t *dst[3] = {c->item_cell, c->item_first, c->item_count};
        for (int a = 0; a < 3; ++a)
            if ((e = cudaMemcpyAsync(dst[a], c->item_sorted + a * im, sizeof(int32_t) * im, cudaMemcpyDeviceToDevice,
                                     s)) != cudaSuccess)
                return e;
        c->items_by_class = true;
    }
    return cudaSuccess;
}

}  // namespace sph
