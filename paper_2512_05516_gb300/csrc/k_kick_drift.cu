// S6: the paper's linear kernels Kick and Drift (Section 6), fused, and
// optionally fused with S7, the write-back of the step's results.
//   v += a dt_kick, u += du/dt dt_kick       FP32 (storage format of v and u
//                                            applied to the result)
//   x += v dt_drift, wrapped into [0, L)      FP64, in the AoS record
// One thread per sorted slot.  The warp's 32 records move through shared
// memory in 16-byte chunks (k_records.cuh): the chunks holding x are loaded,
// the new x (and, with a write-back, every written field) is placed in the
// record image, and the written 4-byte units go back lane-contiguously.
// When the write-back covers most of the record and the warp's records are
// consecutive in memory, the whole block moves by bulk copies instead: one
// load, the new values placed in the image, one store.
// With the write-back, x and the fields share one pass over the records, so
// the sectors they cover are written whole instead of being merged twice.
#include <algorithm>
#include <cstring>

#include "k_cellkey.cuh"
#include "k_records.cuh"

namespace sph {
namespace {

constexpr int kKDThreads = 128;
constexpr int kMaxWb = 3 * SPH_NFIELDS;

// one written-back scalar component
struct WbComp {
    int32_t off;                 // byte offset in the record
    int32_t f64;                 // AoS element is FP64
    int32_t src;                 // 0: the SoA value; 1 + c: kicked v_c; 4: kicked u
    int32_t fmt;                 // storage format of the SoA value
    float dec;                   // 2^-e
    const void *soa;
};

struct KDArgs {
    uint8_t *aos;
    int64_t n;
    RecGeom g;
    ChunkRun xrun;               // the chunks holding x
    ChunkRun wrun;               // the chunks holding any written unit
    int32_t xoff;                // byte offset of x in the record
    uint64_t umask[2];           // units written: x, plus the write-back fields
    const int32_t *perm;
    double box[3];
    float dtk;
    double dtd;
    void *v[3];
    int vfmt;
    float vdec, venc;            // storage scale of v: stored = v * venc
    const float *a[3];
    void *u;
    int ufmt;
    float udec, uenc;
    const float *dudt;
    bool write_soa;              // store the kicked v, u in the SoA
    BulkPlan bulk;               // bulk copies of consecutive record blocks
    int32_t rb;                  // record bytes
    int nwb;
    WbComp wb[kMaxWb];
    int32_t *keys_out;           // the next binning's cell key of every record (by record index), or null
    CellGrid kg;                 // ... on this grid
    DevStats *st;
};

// the value a store in `fmt` followed by a load returns
__device__ __forceinline__ float quantize_fmt(float x, int fmt)
{
    switch (fmt) {
    case SPH_P_BF16: return dec_bf16(enc_bf16(x));
    case SPH_P_FP16: return __half2float(__float2half_rn(x));
    case SPH_P_FP32_M16: return __uint_as_float(enc_trunc(x, 25) << 7);
    case SPH_P_FP32_M10: return __uint_as_float(enc_trunc(x, 19) << 13);
    default:
        if (fmt_trunc_any(fmt)) {
            const int B = fmt_bits(fmt);
            return __uint_as_float(enc_trunc(x, B) << (32 - B));
        }
        return x;
    }
}

template <typename T>
__global__ void __launch_bounds__(kKDThreads, 10) k_kick_drift(KDArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *smem = reinterpret_cast<T *>(smem_raw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T *rec = smem + (size_t)warp * 32 * a.g.Up;
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool ok = k < a.n;
    const int64_t o = ok ? a.perm[k] : -1;
    // kick first: its loads do not wait for the permutation
    float vn[3] = {0.f, 0.f, 0.f};
    float un = 0.f;
    if (ok) {
        for (int c = 0; c < 3; ++c) vn[c] = fmaf(a.a[c][k], a.dtk, ld_val(a.v[c], a.vfmt, k) * a.vdec);
        un = fmaf(a.dudt[k], a.dtk, ld_val(a.u, a.ufmt, k) * a.udec);
    }
    // the write-back values read from the SoA: issued before the record
    // loads (a fixed unrolled window keeps them in flight together)
    constexpr int W = 8;
    float pre[W];
#pragma unroll
    for (int i = 0; i < W; ++i)
        if (ok && i < a.nwb && a.wb[i].src == 0) pre[i] = ld_val(a.wb[i].soa, a.wb[i].fmt, k);
    const WarpRuns w = warp_runs(o, ok, lane);
    const bool bulk = sizeof(T) == 16 && a.bulk.store;
    uint4 *img = reinterpret_cast<uint4 *>(smem + (size_t)warp * 32 * a.g.Up);
    if (bulk) {
        uint64_t *bar = reinterpret_cast<uint64_t *>(smem + (size_t)(blockDim.x >> 5) * 32 * a.g.Up) + warp;
        if (!bulk_load_runs(a.aos, o, w, a.rb, img, a.g.U, bar, &a.st->error_bits, lane)) return;
    } else {
        load_chunks<T>(reinterpret_cast<const T *>(a.aos), rec, o, a.g, a.xrun, lane);
    }
    unsigned char *mine = reinterpret_cast<unsigned char *>(rec + lane * a.g.Up);
    if (ok) {
        double *xs = reinterpret_cast<double *>(mine + a.xoff);
        bool bad = false;
        for (int c = 0; c < 3; ++c) {
            // x += v dt in FP64 (one FMA, the FP64 arithmetic the step
            // needs); a position already in [0, L) -- tested on the bit
            // patterns, since non-negative doubles order like their bits --
            // needs no wrap; the few that left the box take the periodic
            // wrap x - L floor(x / L)
            double y = fma(f2d_bits(vn[c]), a.dtd, xs[c]);
            const long long yb = __double_as_longlong(y);
            if (yb < 0 || yb >= __double_as_longlong(a.box[c])) {
                if ((yb & 0x7FF0000000000000ll) == 0x7FF0000000000000ll) {
                    bad = true;                        // inf or nan
                } else {
                    y = __dsub_rn(y, __dmul_rn(a.box[c], floor(y / a.box[c])));
                    if (y >= a.box[c]) y = 0.0;        // rounding onto L
                }
            }
            xs[c] = y;
        }
        if (bad || !isfinite(un)) set_error(a.st, SPH_ERR_NONFINITE);
        // the cell key of the new position, as the next binning computes it
        // from the record (a non-finite position: outside the box, as there)
        if (a.keys_out) {
            a.keys_out[o] = cell_key(a.kg, xs[0], xs[1], xs[2]);
            if (bad) set_error(a.st, SPH_ERR_OUTSIDE);
        }
        // the write-back: v and u as the storage format holds them after the
        // kick, the other fields as stored
#pragma unroll
        for (int i = 0; i < W; ++i) {
            if (i >= a.nwb) break;
            const WbComp w = a.wb[i];
            float val;
            if (w.src == 0) val = pre[i] * w.dec;
            else if (w.src == 4) val = quantize_fmt(un * a.uenc, a.ufmt) * a.udec;
            else val = quantize_fmt((w.src == 1 ? vn[0] : (w.src == 2 ? vn[1] : vn[2])) * a.venc, a.vfmt) * a.vdec;
            if (w.f64) *reinterpret_cast<double *>(mine + w.off) = f2d_bits(val);
            else *reinterpret_cast<float *>(mine + w.off) = val;
        }
        for (int i = W; i < a.nwb; ++i) {
            const WbComp w = a.wb[i];
            float val;
            if (w.src == 0) val = ld_val(w.soa, w.fmt, k) * w.dec;
            else if (w.src == 4) val = quantize_fmt(un * a.uenc, a.ufmt) * a.udec;
            else val = quantize_fmt((w.src == 1 ? vn[0] : (w.src == 2 ? vn[1] : vn[2])) * a.venc, a.vfmt) * a.vdec;
            if (w.f64) *reinterpret_cast<double *>(mine + w.off) = f2d_bits(val);
            else *reinterpret_cast<float *>(mine + w.off) = val;
        }
    }
    if (bulk) bulk_store_runs(a.aos, o, w, a.rb, img, a.g.U, lane);
    else store_chunks<T>(reinterpret_cast<T *>(a.aos), rec, o, a.g, a.wrun, a.umask, lane);
    if (a.write_soa) {
        for (int c = 0; c < 3; ++c) st_any(a.v[c], a.vfmt, k, vn[c] * a.venc, ok, a.n);
        st_any(a.u, a.ufmt, k, un * a.uenc, ok, a.n);
    }
}

inline void add_units(uint64_t umask[2], int b0, int b1)
{
    for (int u = b0 / 4; u <= (b1 - 1) / 4; ++u) umask[u >> 6] |= 1ull << (u & 63);
}

template <typename T>
cudaError_t launch_kd(sph_ctx *c, const KDArgs &a)
{
    const size_t smem = (size_t)(kKDThreads / 32) * 32 * a.g.Up * sizeof(T) + (kKDThreads / 32) * sizeof(uint64_t);
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_kick_drift<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
        cudaSuccess)
        return e;
    const unsigned grid = (unsigned)((c->n + kKDThreads - 1) / kKDThreads);
    k_kick_drift<T><<<grid, kKDThreads, smem, c->stream>>>(a);
    c->launches += 1;
    return cudaGetLastError();
}

}  // namespace

// wb_fields == 0: kick/drift alone (v, u stored back in the SoA); otherwise
// kick/drift fused with the write-back of wb_fields (v, u not stored in SoA)
cudaError_t run_kick_drift(sph_ctx *c, double dt_kick, double dt_drift, uint32_t wb_fields)
{
    if (c->n == 0) return cudaSuccess;
    KDArgs a;
    std::memset(&a, 0, sizeof(a));
    a.aos = c->aos;
    a.n = c->n;
    const int cb = record_chunk_bytes(c->layout.record_bytes);
    a.g = rec_geom(c->layout.record_bytes, cb);
    a.xoff = c->layout.offset[SPH_F_X];
    uint64_t xm = 0;
    for (int q = a.xoff / cb; q <= (a.xoff + 23) / cb; ++q) xm |= 1ull << q;
    a.xrun = chunk_run(xm);
    add_units(a.umask, a.xoff, a.xoff + 24);
    a.perm = c->perm();
    for (int k = 0; k < 3; ++k) {
        a.box[k] = c->params.box[k];
        a.v[k] = c->soa[SPH_F_V][k];
        a.a[k] = (const float *)c->soa[SPH_F_A][k];
    }
    a.dtk = (float)dt_kick;
    a.dtd = dt_drift;
    a.vfmt = c->prec[SPH_F_V];
    a.vdec = c->dec(SPH_F_V);
    a.venc = c->enc(SPH_F_V);
    a.u = c->soa[SPH_F_U][0];
    a.ufmt = c->prec[SPH_F_U];
    a.udec = c->dec(SPH_F_U);
    a.uenc = c->enc(SPH_F_U);
    a.dudt = (const float *)c->soa[SPH_F_DUDT][0];
    a.write_soa = wb_fields == 0;
    a.nwb = 0;
    for (int f = 0; f < SPH_NFIELDS; ++f) {
        if (!(wb_fields & SPH_BIT(f))) continue;
        const bool f64 = c->layout.type[f] == SPH_AOS_F64;
        const int es = f64 ? 8 : 4;
        for (int comp = 0; comp < ncomp(f); ++comp) {
            WbComp &w = a.wb[a.nwb++];
            w.off = c->layout.offset[f] + es * comp;
            w.f64 = f64 ? 1 : 0;
            w.src = f == SPH_F_V ? 1 + comp : (f == SPH_F_U ? 4 : 0);
            w.fmt = c->prec[f];
            w.dec = c->dec(f);
            w.soa = c->soa[f][comp];
        }
        add_units(a.umask, c->layout.offset[f], c->layout.offset[f] + es * ncomp(f));
    }
    // SoA-sourced components first: the kernel preloads the first ones
    std::stable_partition(a.wb, a.wb + a.nwb, [](const WbComp &w) { return w.src == 0; });
    a.wrun = chunk_run(chunks_of_units(a.umask, cb));
    a.rb = c->layout.record_bytes;
    a.bulk = bulk_plan(cb == 16 && a.g.Up == a.g.U && c->aos_device, a.g.U, xm, a.umask);
    if (c->binned && !c->levels && c->buffer == 0) {
        a.keys_out = c->keys[0];     // free between binnings on the cell grid
        a.kg = cell_grid(c->nc, c->sub, c->params.box);
    }
    a.st = c->dstats;
    return cb == 16 ? launch_kd<uint4>(c, a) : launch_kd<uint2>(c, a);
}

}  // namespace sph
