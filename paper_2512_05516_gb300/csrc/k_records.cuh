// Moving whole AoS records between global and shared memory, one warp at a
// time, and the exact cell-relative position offset.  Shared by the
// conversion kernels (k_convert.cu) and the fused kick/drift + write-back
// (k_kick_drift.cu).
//
// A warp handles 32 sorted slots; lane l's record is o_l = perm[slot] (or -1).
// The records are cut into chunks of sizeof(T) bytes (16 when the record
// size allows, else 8) and the warp moves chunk c = 32 b + lane of its
// record block (record c / U, chunk c % U) per instruction, so consecutive
// lanes touch consecutive bytes of a record and one instruction covers
// several whole records.  In shared memory record r's chunks sit at
// rec[r * Up + q] (Up >= U, odd where that helps the bank layout).
#pragma once

#include <cstring>

#include "sph_internal.cuh"

namespace sph {

struct RecGeom {
    int32_t U;            // chunks per record
    int32_t Up;           // chunk stride of a record in shared memory
    uint32_t magic;       // chunk_magic(U)
};

// chunk c of a warp's record block -> record index (clamped to a lane id);
// magic = ceil(2^32 / n) for n chunks per record, 0 for n = 1 (2^32 does not
// fit: the record index is c itself)
__device__ __forceinline__ int rec_of_chunk(uint32_t c, uint32_t magic)
{
    return min(magic ? (int)__umulhi(c, magic) : (int)c, 31);
}

inline uint32_t chunk_magic(uint32_t n) { return n > 1 ? (uint32_t)(0xFFFFFFFFu / n) + 1u : 0u; }

// chunk loads in flight per lane: 64 bytes
template <typename T>
__host__ __device__ constexpr int chunk_batch() { return 64 / (int)sizeof(T); }

// A run of chunks [q0, q0 + nq) of every record, of which those in `cmask`
// (bit q) are loaded; chunk c of the warp's run block belongs to record
// c / nq (magic = ceil(2^32 / nq)).
struct ChunkRun {
    int32_t q0, nq;
    uint32_t magic;
    uint64_t cmask;
};

// the chunks (of `chunk` bytes) holding any unit of a 4-byte unit mask
inline uint64_t chunks_of_units(const uint64_t umask[2], int chunk)
{
    const int K = chunk / 4;
    uint64_t m = 0;
    for (int u = 0; u < 128; ++u)
        if ((umask[u >> 6] >> (u & 63)) & 1ull) m |= 1ull << (u / K);
    return m;
}

// the chunks (of `chunk` bytes) all of whose units are in a unit mask
inline uint64_t full_chunks_of_units(const uint64_t umask[2], int chunk)
{
    const int K = chunk / 4;
    uint64_t m = 0;
    for (int q = 0; q < 128 / K && q < 64; ++q) {
        bool all = true;
        for (int u = q * K; u < (q + 1) * K; ++u) all = all && ((umask[u >> 6] >> (u & 63)) & 1ull);
        if (all) m |= 1ull << q;
    }
    return m;
}

inline ChunkRun chunk_run(uint64_t cmask)
{
    ChunkRun r;
    r.cmask = cmask;
    r.q0 = 0;
    while (cmask && !((cmask >> r.q0) & 1ull)) ++r.q0;
    int q1 = r.q0;
    for (int q = r.q0; q < 64; ++q)
        if ((cmask >> q) & 1ull) q1 = q;
    r.nq = cmask ? q1 - r.q0 + 1 : 0;
    r.magic = chunk_magic((uint32_t)r.nq);
    return r;
}

// Copy the chunks of `run` of the warp's 32 records into shared memory.
// Every lane calls it (shuffles inside).
template <typename T>
__device__ __forceinline__ void load_chunks(const T *__restrict__ aos, T *rec, int64_t o, const RecGeom g,
                                            const ChunkRun run, int lane)
{
    constexpr int B = chunk_batch<T>();
    const uint32_t total = 32u * (uint32_t)run.nq;
    for (uint32_t c0 = 0; c0 < total; c0 += 32u * B) {
        T buf[B];
        int dst[B];
#pragma unroll
        for (int b = 0; b < B; ++b) {
            dst[b] = -1;
            if (c0 + 32u * b >= total) continue;      // warp-uniform: total is a multiple of 32
            const uint32_t c = c0 + 32u * b + (uint32_t)lane;
            const int r = rec_of_chunk(c, run.magic);
            const int q = run.q0 + (int)c - r * run.nq;
            const int64_t orr = __shfl_sync(0xffffffffu, o, r);
            if (orr >= 0 && ((run.cmask >> q) & 1ull)) {
                buf[b] = __ldg(aos + orr * g.U + q);
                dst[b] = r * g.Up + q;
            }
        }
#pragma unroll
        for (int b = 0; b < B; ++b)
            if (dst[b] >= 0) rec[dst[b]] = buf[b];
    }
    __syncwarp();
}

// 4-byte units of chunk q in a unit mask (bit u = bytes [4u, 4u + 4))
template <typename T>
__device__ __forceinline__ uint32_t chunk_units(const uint64_t umask[2], int q)
{
    constexpr int K = sizeof(T) / 4;
    const int u0 = q * K;
    return (uint32_t)(umask[u0 >> 6] >> (u0 & 63)) & ((1u << K) - 1u);
}

// Store the 4-byte units in `umask` of the warp's 32 records from shared
// memory, over the chunks of `run` (those holding any written unit): whole
// chunks where every unit is written, else 8- and 4-byte pieces.  Every lane
// calls it.
template <typename T>
__device__ __forceinline__ void store_chunks(T *__restrict__ aos, const T *rec, int64_t o, const RecGeom g,
                                             const ChunkRun run, const uint64_t umask[2], int lane)
{
    constexpr int K = sizeof(T) / 4;
    constexpr uint32_t ALL = (1u << K) - 1u;
    __syncwarp();
    const uint32_t total = 32u * (uint32_t)run.nq;
    for (uint32_t c = (uint32_t)lane; c < total; c += 32u) {      // total = 32 nq: same trip count in every lane
        const int r = rec_of_chunk(c, run.magic);
        const int q = run.q0 + (int)c - r * run.nq;
        const int64_t orr = __shfl_sync(0xffffffffu, o, r);
        if (orr < 0) continue;
        const uint32_t m = chunk_units<T>(umask, q);
        if (m == 0u) continue;
        T *dst = aos + orr * g.U + q;
        const T *src = rec + r * g.Up + q;
        if (m == ALL) {
            *dst = *src;
        } else {
            uint32_t *d32 = reinterpret_cast<uint32_t *>(dst);
            const uint32_t *s32 = reinterpret_cast<const uint32_t *>(src);
#pragma unroll
            for (int h = 0; h < K; h += 2) {
                const uint32_t mm = (m >> h) & 3u;
                if (mm == 3u) {
                    *reinterpret_cast<uint2 *>(d32 + h) = *reinterpret_cast<const uint2 *>(s32 + h);
                } else {
                    if (mm & 1u) d32[h] = s32[h];
                    if (mm & 2u) d32[h + 1] = s32[h + 1];
                }
            }
        }
    }
}

// x - o rounded once to FP32 (nearest, ties to even), for the cell-relative
// position offsets.  The origin o is 0 or, for cells k >= 1, satisfies
// o/2 <= x <= 2o, so the FP64 difference is exact (Sterbenz) and the only
// rounding is the final one.  One FP64 subtraction per component; the
// rounding to FP32 runs on the integer pipes (d2f_bits_rn).  Outside that
// frame the result is the FP64 difference rounded to FP32.
__device__ __forceinline__ float cell_offset_f32(double x, double o) { return d2f_bits_rn(__dsub_rn(x, o)); }

// x - o moved to the nearest periodic image, rounded once to FP32: positions
// relative to a buffer's first particle.  FP64: the difference, then - L when
// it is >= L/2 or + L when it is < -L/2.
__device__ __forceinline__ float buffer_offset_f32(double x, double o, double L)
{
    double d = __dsub_rn(x, o);
    if (d >= 0.5 * L) d = __dsub_rn(d, L);
    else if (d < -0.5 * L) d = __dadd_rn(d, L);
    return d2f_bits_rn(d);
}

// ---------------------------------------------------------------------------
// Bulk asynchronous copies (the non-tensor form of TMA) of record runs.
// In cell-ordered records (the usual case once they have been reordered) a
// warp's 32 records form one run of consecutive records, or a few runs where
// particles changed cells since the reorder (a few more per warp every step
// in a flow).  The warp moves its records with one cp.async.bulk per run,
// completion counted in bytes on a per-warp mbarrier, and stores them back
// the same way.  Fully scattered records (one run per lane) move as fast
// this way as by per-lane chunk loads, and their write-back faster.  Every
// wait is bounded: a copy that has not landed after kBulkPolls polls sets
// SPH_ERR_TIMEOUT (bulk_wait says what follows).
constexpr uint32_t kBulkPolls = 1u << 22;

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// arrive on `bar` and add `bytes` to the transaction count its phase waits for
__device__ __forceinline__ void mbar_arrive_expect(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// global -> shared, `bytes` (a multiple of 16, both addresses 16-byte aligned)
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t polls)
{
    for (uint32_t i = 0; i < polls; ++i) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(smem_addr(bar)), "r"(parity)
                     : "memory");
        if (done) return true;
    }
    return false;
}

// shared -> global from one lane, returning once the shared source has been
// read (the global writes complete asynchronously, before the kernel ends)
__device__ __forceinline__ void bulk_s2g_wait(void *dst, const void *src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_addr(src)),
                 "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

// What a kernel moves by bulk copies.
struct BulkPlan {
    int32_t load;                // load whole records, one copy per run
    int32_t store;               // store whole records, one copy per run (after a whole-record load)
};

// The warp's records as runs of consecutive records.  Lane l starts a run
// when it holds a record and lane l-1 holds none or not record o_l - 1; a run
// ends at the next start or the next lane without a record.  Warp-uniform
// fields; `len` (lanes in the run) is meaningful in start lanes only.
struct WarpRuns {
    int nvalid;                  // lanes holding a record
    bool start;
    int len;
};

__device__ __forceinline__ WarpRuns warp_runs(int64_t o, bool ok, int lane)
{
    WarpRuns w;
    const int64_t prev = __shfl_up_sync(0xffffffffu, o, 1);
    const unsigned valid = __ballot_sync(0xffffffffu, ok);
    w.start = ok && (lane == 0 || !((valid >> (lane - 1)) & 1u) || prev + 1 != o);
    const unsigned starts = __ballot_sync(0xffffffffu, w.start);
    const unsigned after = ~((2u << lane) - 1u);                // lanes above this one (none for lane 31)
    const unsigned stop = (starts | ~valid) & after;
    w.len = (stop ? __ffs((int)stop) - 1 : 32) - lane;
    w.nvalid = __popc(valid);
    return w;
}

// Start bulk loads of the warp's record runs (rb bytes per record) into its
// image rec (lane l's record at chunk l * U).  Every lane calls it.
__device__ __forceinline__ void bulk_issue_runs(const uint8_t *aos, int64_t o, const WarpRuns &w, int rb,
                                                uint4 *rec, int U, uint64_t *bar, int lane)
{
    if (lane == 0) {
        mbar_init(bar, 1);
        mbar_arrive_expect(bar, (uint32_t)w.nvalid * (uint32_t)rb);
    }
    __syncwarp();
    if (w.start) bulk_g2s(rec + lane * U, aos + o * rb, (uint32_t)w.len * (uint32_t)rb, bar);
}

// Wait for them.  Every lane calls it.  A copy that has not landed within
// the first bound sets SPH_ERR_TIMEOUT; then the whole warp keeps waiting,
// up to kBulkFinal times as long, so that its shared memory (and with it the
// CTA) stays allocated while the copy may still be landing there.  Returns
// whether the copy landed: if it did in that second wait, the records are
// processed as usual (the error bit still reports the slow copy); if not,
// the caller skips its records and exits without issuing another copy into
// that memory.
constexpr uint32_t kBulkFinal = 16u;

__device__ __forceinline__ bool bulk_wait(uint64_t *bar, unsigned int *err, int lane)
{
    if (__all_sync(0xffffffffu, mbar_wait(bar, 0, kBulkPolls))) return true;
    if (lane == 0) atomicOr(err, (unsigned)SPH_ERR_TIMEOUT);
    bool landed = false;
    for (uint32_t r = 0; r < kBulkFinal && !landed; ++r)
        landed = __all_sync(0xffffffffu, mbar_wait(bar, 0, kBulkPolls));
    return landed;
}

__device__ __forceinline__ bool bulk_load_runs(const uint8_t *aos, int64_t o, const WarpRuns &w, int rb,
                                               uint4 *rec, int U, uint64_t *bar, unsigned int *err, int lane)
{
    bulk_issue_runs(aos, o, w, rb, rec, U, bar, lane);
    return bulk_wait(bar, err, lane);
}

// Store the warp's record runs back from its image with one bulk copy per
// run.  The image must hold every byte of those records.  Every lane calls it.
__device__ __forceinline__ void bulk_store_runs(uint8_t *aos, int64_t o, const WarpRuns &w, int rb,
                                                const uint4 *rec, int U, int lane)
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic writes -> async proxy
    __syncwarp();
    if (w.start) bulk_s2g_wait(aos + o * rb, rec + lane * U, (uint32_t)w.len * (uint32_t)rb);
    __syncwarp();
}

// Host: the bulk plan of a kernel.  `can`: 16-byte chunks, records packed in
// shared memory as in global memory (Up == U), device-resident records.
// need: chunks a gather reads; written: 4-byte units a write-back writes
// (null for a gather).  A gather loads whole records when it reads at least
// 3/4 of each.  A write-back loads and stores whole records when its written
// chunks make up at least 3/4 of the record: the sectors it leaves partly
// written would be read from DRAM anyway, and below that share whole-record
// stores move more bytes than partial stores.
inline BulkPlan bulk_plan(bool can, int U, uint64_t need, const uint64_t *written)
{
    BulkPlan p;
    std::memset(&p, 0, sizeof(p));
    if (!can) return p;
    const uint64_t all = U >= 64 ? ~0ull : (1ull << U) - 1ull;
    const uint64_t mask = written ? chunks_of_units(written, 16) & all : need & all;
    if (__builtin_popcountll(mask) * 4 < U * 3) return p;
    p.load = 1;
    p.store = written ? 1 : 0;
    return p;
}

// Chunk size of a record layout: 16 bytes when the record size allows it.
inline int record_chunk_bytes(int record_bytes) { return record_bytes % 16 == 0 ? 16 : 8; }

// Record geometry for chunks of `chunk` bytes (16 or 8).
inline RecGeom rec_geom(int record_bytes, int chunk)
{
    RecGeom g;
    g.U = record_bytes / chunk;
    g.Up = (g.U % 2 == 0) ? g.U + 1 : g.U;
    g.magic = chunk_magic((uint32_t)g.U);
    return g;
}

// ceil(2^64 / d): n / d == umul64hi(n, m) for 0 <= n < 2^32, 2 <= d < 2^20
inline uint64_t magic64(uint32_t d) { return ~0ull / d + 1ull; }

__device__ __forceinline__ uint32_t div_magic(uint32_t n, uint64_t m) { return (uint32_t)__umul64hi(n, m); }

}  // namespace sph
