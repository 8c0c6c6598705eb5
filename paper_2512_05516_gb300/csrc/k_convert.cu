// S2 and S7: the paper's conversion operators (Section 4).
//   U o N o C      gather the narrowed field set from the FP64 AoS records in
//                  cell order, round to the storage format, write SoA
//   C^T N^T U^T    decode SoA values, widen to the AoS element type, scatter
//                  to the particle's record
// One thread per sorted slot.  A warp moves the records of its 32 slots
// through shared memory: with bulk copies (TMA) when the 32 records are
// consecutive in memory, else in 16-byte chunks (8-byte ones when the record
// size is not a multiple of 16), lane-contiguous, so each load or store
// instruction covers whole records; each lane then reads (or writes) its own
// record's fields there.  The bulk write-back loads the whole block, places
// the fields in it and stores it whole, so every DRAM sector is written
// whole.  The fields a call moves are unrolled on the host into a table of
// scalar components.  All 32 lanes stay alive so that packed formats can be
// written warp-cooperatively.  Widening and narrowing work on the bit
// patterns (integer pipes); the cell-relative offsets of the positions take
// one FP64 subtraction per component, exact, before that rounding.
#include <cstring>

#include "k_records.cuh"

namespace sph {
namespace {

constexpr int kConvThreads = 128;
constexpr int kMaxComp = 3 * SPH_NFIELDS;

// one scalar component a call moves
struct Comp {
    int32_t off;                 // byte offset in the record
    int32_t kind;                // 0: FP64 value, 1: FP32 value, 2 + a: FP64 position, axis a
    int32_t fmt;                 // storage format
    float scl;                   // 2^e on the way in, 2^-e on the way out
    void *soa;
};

struct ConvArgs {
    uint8_t *aos;
    int64_t n;
    RecGeom g;
    ChunkRun run;                // chunks the gather reads / the write-back writes
    uint64_t umask[2];           // 4-byte units the write-back writes
    const int32_t *perm;
    const int32_t *slot_cell;    // key = cell * s^3 + sub-cell
    int32_t lg_s3;
    bool morton;                 // level mode: the key is the Morton code of the finest cell
    uint64_t m_nc0, m_nc1;       // magic divisors for nc_x, nc_y
    int32_t nc0, nc1;
    const double *origin[3];     // cell origin k * (L / nc) per axis
    const double *bufo;          // buffer mode: buffer origins, 3 x nbuf, axis-major (else null)
    int64_t nbuf;
    int32_t lgB;                 // buffer size 2^lgB
    double box[3];
    bool has_x;
    BulkPlan bulk;               // bulk copies of consecutive record blocks
    int32_t rb;                  // record bytes
    unsigned int *err;           // sticky error bits
    int ncomp;
    Comp comp[kMaxComp];
};

template <typename T>
__global__ void __launch_bounds__(kConvThreads, 12) k_aos_to_soa(ConvArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *smem = reinterpret_cast<T *>(smem_raw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T *rec = smem + (size_t)warp * 32 * a.g.Up;
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool ok = k < a.n;
    const int64_t o = ok ? a.perm[k] : -1;
    double org0 = 0.0, org1 = 0.0, org2 = 0.0;
    if (a.has_x && ok && a.bufo) {
        // buffer mode: slot k is record k, in buffer k / B
        const int64_t b = k >> a.lgB;
        org0 = __ldg(a.bufo + b);
        org1 = __ldg(a.bufo + a.nbuf + b);
        org2 = __ldg(a.bufo + 2 * a.nbuf + b);
    } else if (a.has_x && ok && a.morton) {
        const uint32_t key = (uint32_t)a.slot_cell[k];
        org0 = __ldg(a.origin[0] + morton_compact(key));
        org1 = __ldg(a.origin[1] + morton_compact(key >> 1));
        org2 = __ldg(a.origin[2] + morton_compact(key >> 2));
    } else if (a.has_x && ok) {
        // the cell's coordinates from its key, then its origin (tables)
        const uint32_t cell = (uint32_t)a.slot_cell[k] >> a.lg_s3;
        const uint32_t t = div_magic(cell, a.m_nc0);
        const uint32_t kx = cell - t * (uint32_t)a.nc0;
        const uint32_t kz = div_magic(t, a.m_nc1);
        const uint32_t ky = t - kz * (uint32_t)a.nc1;
        org0 = __ldg(a.origin[0] + kx);
        org1 = __ldg(a.origin[1] + ky);
        org2 = __ldg(a.origin[2] + kz);
    }
    const WarpRuns w = warp_runs(o, ok, lane);
    if (sizeof(T) == 16 && a.bulk.load) {
        uint64_t *bar = reinterpret_cast<uint64_t *>(smem + (size_t)(blockDim.x >> 5) * 32 * a.g.Up) + warp;
        if (!bulk_load_runs(a.aos, o, w, a.rb, reinterpret_cast<uint4 *>(smem + (size_t)warp * 32 * a.g.Up), a.g.U,
                            bar, a.err, lane))
            return;
    } else {
        load_chunks<T>(reinterpret_cast<const T *>(a.aos), rec, o, a.g, a.run, lane);
    }
    const unsigned char *mine = reinterpret_cast<const unsigned char *>(rec + lane * a.g.Up);
    for (int i = 0; i < a.ncomp; ++i) {
        const Comp cp = a.comp[i];
        float v = 0.0f;
        if (ok) {
            if (cp.kind == 1) {
                v = *reinterpret_cast<const float *>(mine + cp.off);
            } else {
                const double d = *reinterpret_cast<const double *>(mine + cp.off);
                if (cp.kind >= 2) {
                    const double og = cp.kind == 2 ? org0 : (cp.kind == 3 ? org1 : org2);
                    v = a.bufo ? buffer_offset_f32(d, og, a.box[cp.kind - 2]) : cell_offset_f32(d, og);
                } else {
                    v = d2f_bits_rn(d);
                }
            }
        }
        st_any(cp.soa, cp.fmt, k, v * cp.scl, ok, a.n);
    }
}

// kPos: positions are among the fields (buffer mode only)
template <typename T, bool kPos>
__global__ void __launch_bounds__(kConvThreads, 12) k_soa_to_aos(ConvArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *smem = reinterpret_cast<T *>(smem_raw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T *rec = smem + (size_t)warp * 32 * a.g.Up;
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool ok = k < a.n;
    const int64_t o = ok ? a.perm[k] : -1;
    // the first SoA values are loaded before anything waits: they depend on
    // neither the permutation nor the records
    constexpr int W = 8;
    float pre[W];
#pragma unroll
    for (int i = 0; i < W; ++i)
        if (ok && i < a.ncomp) pre[i] = ld_val(a.comp[i].soa, a.comp[i].fmt, k);
    unsigned char *mine = reinterpret_cast<unsigned char *>(rec + lane * a.g.Up);
    const WarpRuns w = warp_runs(o, ok, lane);
    const bool bulk = sizeof(T) == 16 && a.bulk.store;
    uint4 *img = reinterpret_cast<uint4 *>(smem + (size_t)warp * 32 * a.g.Up);
    if (bulk) {
        // whole records, so that the image holds every byte it stores
        uint64_t *bar = reinterpret_cast<uint64_t *>(smem + (size_t)(blockDim.x >> 5) * 32 * a.g.Up) + warp;
        if (!bulk_load_runs(a.aos, o, w, a.rb, img, a.g.U, bar, a.err, lane)) return;
    }
    if (ok) {
        for (int i = 0; i < a.ncomp; ++i) {
            const Comp cp = a.comp[i];
            float v = 0.0f;
#pragma unroll
            for (int j = 0; j < W; ++j)
                if (j == i) v = pre[j];
            if (i >= W) v = ld_val(cp.soa, cp.fmt, k);
            v *= cp.scl;
            if (cp.kind == 1) {
                *reinterpret_cast<float *>(mine + cp.off) = v;
            } else if (kPos && cp.kind >= 2) {
                // buffer mode: position = buffer origin + offset, wrapped into [0, L)
                const int ax = cp.kind - 2;
                const double L = a.box[ax];
                double y = __dadd_rn(__ldg(a.bufo + ax * a.nbuf + (k >> a.lgB)), f2d_bits(v));
                if (y < 0.0 || y >= L) {
                    y = __dsub_rn(y, __dmul_rn(L, floor(y / L)));
                    if (y >= L) y = 0.0;                         // rounding onto L
                }
                *reinterpret_cast<double *>(mine + cp.off) = y;
            } else {
                *reinterpret_cast<double *>(mine + cp.off) = f2d_bits(v);
            }
        }
    }
    if (bulk) bulk_store_runs(a.aos, o, w, a.rb, img, a.g.U, lane);
    else store_chunks<T>(reinterpret_cast<T *>(a.aos), rec, o, a.g, a.run, a.umask, lane);
}

__global__ void __launch_bounds__(256) k_pack(const float *src, void *dst, int fmt, int64_t n)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool ok = k < n;
    st_any(dst, fmt, k, ok ? src[k] : 0.0f, ok, n);
}

ConvArgs make_args(sph_ctx *c, uint32_t fields, bool to_soa)
{
    ConvArgs a;
    std::memset(&a, 0, sizeof(a));
    a.aos = c->aos;
    a.n = c->n;
    const int cb = record_chunk_bytes(c->layout.record_bytes);
    a.g = rec_geom(c->layout.record_bytes, cb);
    a.perm = c->perm();
    a.slot_cell = c->slot_cell();
    a.lg_s3 = c->sub == 2 ? 3 : 0;
    a.morton = c->levels;
    a.nc0 = c->nc[0];
    a.nc1 = c->nc[1];
    a.m_nc0 = magic64((uint32_t)c->nc[0]);
    a.m_nc1 = magic64((uint32_t)c->nc[1]);
    for (int d = 0; d < 3; ++d) a.origin[d] = c->origin + d * kMaxCellsPerAxis;
    for (int d = 0; d < 3; ++d) a.box[d] = c->params.box[d];
    if (c->buffer) {
        a.bufo = c->buf_origin;
        a.lgB = 31 - __builtin_clz((unsigned)c->buffer);
        a.nbuf = (c->n + c->buffer - 1) / c->buffer;
    }
    a.has_x = false;
    a.ncomp = 0;
    uint64_t cmask = 0;
    for (int f = 0; f < SPH_NFIELDS; ++f) {
        if (!(fields & SPH_BIT(f))) continue;
        const bool f64 = c->layout.type[f] == SPH_AOS_F64;
        const int es = f64 ? 8 : 4;
        for (int comp = 0; comp < ncomp(f); ++comp) {
            Comp &cp = a.comp[a.ncomp++];
            cp.off = c->layout.offset[f] + es * comp;
            cp.kind = !f64 ? 1 : (f == SPH_F_X ? 2 + comp : 0);
            cp.fmt = c->prec[f];
            cp.scl = to_soa ? c->enc(f) : c->dec(f);
            cp.soa = c->soa[f][comp];
        }
        if (f == SPH_F_X) a.has_x = true;
        const int b0 = c->layout.offset[f], b1 = b0 + es * ncomp(f);     // byte range [b0, b1)
        for (int q = b0 / cb; q <= (b1 - 1) / cb; ++q) cmask |= 1ull << q;
        for (int u = b0 / 4; u <= (b1 - 1) / 4; ++u) a.umask[u >> 6] |= 1ull << (u & 63);
    }
    a.run = chunk_run(to_soa ? cmask : chunks_of_units(a.umask, cb));
    a.rb = c->layout.record_bytes;
    a.err = &c->dstats->error_bits;
    const bool can = cb == 16 && a.g.Up == a.g.U && c->aos_device;
    a.bulk = to_soa ? bulk_plan(can, a.g.U, cmask, nullptr) : bulk_plan(can, a.g.U, 0, a.umask);
    return a;
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

template <typename T>
cudaError_t launch_conv(sph_ctx *c, const ConvArgs &a, bool to_soa)
{
    const size_t smem = (size_t)(kConvThreads / 32) * 32 * a.g.Up * sizeof(T) + (kConvThreads / 32) * sizeof(uint64_t);
    cudaError_t e;
    auto kern = to_soa ? k_aos_to_soa<T> : (a.has_x ? k_soa_to_aos<T, true> : k_soa_to_aos<T, false>);
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return e;
    kern<<<blocks_for(c->n, kConvThreads), kConvThreads, smem, c->stream>>>(a);
    c->launches += 1;
    return cudaGetLastError();
}

}  // namespace

cudaError_t run_aos_to_soa(sph_ctx *c, uint32_t fields)
{
    if (c->n == 0) return cudaSuccess;
    const ConvArgs a = make_args(c, fields, true);
    return record_chunk_bytes(c->layout.record_bytes) == 16 ? launch_conv<uint4>(c, a, true)
                                                            : launch_conv<uint2>(c, a, true);
}

cudaError_t run_soa_to_aos(sph_ctx *c, uint32_t fields)
{
    if (c->n == 0) return cudaSuccess;
    const ConvArgs a = make_args(c, fields, false);
    return record_chunk_bytes(c->layout.record_bytes) == 16 ? launch_conv<uint4>(c, a, false)
                                                            : launch_conv<uint2>(c, a, false);
}

// pack an FP32 staging array into field f's packed stream
cudaError_t run_pack(sph_ctx *c, const float *src, int f)
{
    if (c->n == 0) return cudaSuccess;
    k_pack<<<blocks_for(c->n, 256), 256, 0, c->stream>>>(src, c->soa[f][0], c->prec[f], c->n);
    c->launches += 1;
    return cudaGetLastError();
}

}  // namespace sph
