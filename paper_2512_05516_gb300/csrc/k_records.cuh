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
// rounding is the final one; the integer form below subtracts the aligned
// significands exactly and rounds that to 24 bits, keeping the work off the
// FP64 pipe.  Anything outside that frame (signs, subnormals, exponents more
// than one apart, results outside the normal FP32 range) takes the hardware
// FP64 subtraction and conversion.
__device__ __forceinline__ float cell_offset_f32(double x, double o)
{
    const uint64_t bx = (uint64_t)__double_as_longlong(x);
    const uint64_t bo = (uint64_t)__double_as_longlong(o);
    if (bo == 0u) return d2f_bits_rn(x);
    const int ex = (int)(bx >> 52), eo = (int)(bo >> 52);      // sign bit included: negative -> > 0x7FF
    const bool plain = ex >= 1 && ex <= 0x7FE && eo >= 1 && eo <= 0x7FE && ex - eo <= 1 && eo - ex <= 1;
    if (plain) {
        const int e = min(ex, eo);
        const uint64_t hid = 1ull << 52, frac = hid - 1u;
        const int64_t mx = (int64_t)(((bx & frac) | hid) << (ex - e));
        const int64_t mo = (int64_t)(((bo & frac) | hid) << (eo - e));
        const int64_t D = mx - mo;                               // x - o = D * 2^(e - 1075), exactly
        if (D == 0) return 0.0f;
        const uint32_t s = D < 0 ? 0x80000000u : 0u;
        const uint64_t A = D < 0 ? (uint64_t)(-D) : (uint64_t)D;
        const int msb = 63 - __clzll((long long)A);
        int E = msb + e - 1075 + 127;                            // biased FP32 exponent
        if (A < (1ull << 53) && E >= 1 && E <= 253) {
            uint32_t m;
            if (msb > 23) {
                const int sh = msb - 23;
                m = (uint32_t)(A >> sh);
                const uint64_t rem = A & ((1ull << sh) - 1u);
                const uint64_t half = 1ull << (sh - 1);
                if (rem > half || (rem == half && (m & 1u))) {
                    ++m;
                    if (m == (1u << 24)) {
                        m >>= 1;
                        ++E;
                    }
                }
            } else {
                m = (uint32_t)(A << (23 - msb));
            }
            return __uint_as_float(s | ((uint32_t)E << 23) | (m & 0x7FFFFFu));
        }
    }
    return __double2float_rn(__dsub_rn(x, o));
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
