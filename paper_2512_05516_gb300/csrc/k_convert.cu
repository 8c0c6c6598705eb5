// S2 and S7: the paper's conversion operators (Section 4).
//   U o N o C      gather the narrowed field set from the FP64 AoS records in
//                  cell order, round to the storage format, write SoA
//   C^T N^T U^T    decode SoA values, widen to the AoS element type, scatter
//                  to the particle's record
// One thread per sorted slot.  A warp moves the records of its 32 slots
// through shared memory: lane-contiguous loads (or stores) of the 8-byte
// words (4-byte units) a call touches, so each instruction covers whole
// records instead of one word of 32 records; each lane then reads (or
// writes) its own record's fields there.  All 32 lanes stay alive so that
// packed formats can be written warp-cooperatively.
#include "sph_internal.cuh"

namespace sph {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kConvThreads = 128;

struct ConvArgs {
    uint8_t *aos;
    int64_t n;
    int32_t W;                   // record words (record_bytes / 8)
    int32_t Wp;                  // words per record in shared memory (odd: fewer bank conflicts)
    uint64_t wmask;              // record words the call reads
    uint64_t umask[2];           // 4-byte units the call writes (write-back)
    const int32_t *perm;
    const int32_t *slot_cell;
    int32_t nc[3];
    int32_t s3;                  // sub-cells per cell
    double edge[3];
    int nf;
    int fid[SPH_NFIELDS];
    int off[SPH_NFIELDS];
    int type[SPH_NFIELDS];
    int fmt[SPH_NFIELDS];
    float scl[SPH_NFIELDS];      // storage scale: 2^e on the way in, 2^-e on the way out
    int nco[SPH_NFIELDS];
    void *soa[SPH_NFIELDS][3];
};

constexpr int kLoadBatch = 8;    // record words in flight per lane

// Copy the words in `wmask` of the warp's 32 records (record index o of each
// lane, -1 for none) into rec[r * Wp + w], kLoadBatch loads in flight per lane.
__device__ __forceinline__ void load_records(const uint64_t *aos64, uint64_t *rec, int64_t o, int W, int Wp,
                                             uint64_t wmask, int lane)
{
    int r = 0, w = lane;
    while (w >= W) { w -= W; ++r; }
    for (int idx0 = 0; idx0 < 32 * W; idx0 += 32 * kLoadBatch) {
        uint64_t buf[kLoadBatch];
        int dst[kLoadBatch];
#pragma unroll
        for (int b = 0; b < kLoadBatch; ++b) {
            const int idx = idx0 + 32 * b + lane;
            dst[b] = -1;
            const int64_t orr = __shfl_sync(FULL, o, r < 32 ? r : 31);
            if (idx < 32 * W && orr >= 0 && ((wmask >> w) & 1ull)) {
                buf[b] = aos64[orr * W + w];
                dst[b] = r * Wp + w;
            }
            w += 32;
            while (w >= W) { w -= W; ++r; }
        }
#pragma unroll
        for (int b = 0; b < kLoadBatch; ++b)
            if (dst[b] >= 0) rec[dst[b]] = buf[b];
    }
    __syncwarp();
}

// Store the 4-byte units in `umask` of the warp's 32 records from shared memory.
__device__ __forceinline__ void store_records(uint32_t *aos32, const uint32_t *rec32, int64_t o, int W, int Wp,
                                              const uint64_t umask[2], int lane)
{
    __syncwarp();
    const int U = 2 * W, Up = 2 * Wp;
    int r = 0, u = lane;
    while (u >= U) { u -= U; ++r; }
    for (int idx = lane; idx < 32 * U; idx += 32) {
        const int64_t orr = __shfl_sync(FULL, o, r);
        if (orr >= 0 && ((umask[u >> 6] >> (u & 63)) & 1ull)) aos32[orr * U + u] = rec32[r * Up + u];
        u += 32;
        while (u >= U) { u -= U; ++r; }
    }
}

__global__ void __launch_bounds__(kConvThreads) k_aos_to_soa(ConvArgs a)
{
    extern __shared__ uint64_t smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t *rec = smem + (size_t)warp * 32 * a.Wp;
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool ok = k < a.n;
    const int64_t o = ok ? a.perm[k] : -1;
    const int32_t key = ok ? a.slot_cell[k] : 0;     // issued before the record loads
    load_records((const uint64_t *)a.aos, rec, o, a.W, a.Wp, a.wmask, lane);
    const uint8_t *mine = (const uint8_t *)(rec + lane * a.Wp);
    for (int j = 0; j < a.nf; ++j) {
        const int f = a.fid[j];
        double org[3] = {0.0, 0.0, 0.0};
        if (f == SPH_F_X && ok) {
            // cell-relative positions: offset from k_d * (L_d / nc_d), in FP64
            int32_t cid = key / a.s3;                // key = cell * s^3 + sub-cell
            int32_t kx = cid % a.nc[0];
            int32_t t = cid / a.nc[0];
            int32_t ky = t % a.nc[1];
            int32_t kz = t / a.nc[1];
            org[0] = (double)kx * a.edge[0];
            org[1] = (double)ky * a.edge[1];
            org[2] = (double)kz * a.edge[2];
        }
        for (int c = 0; c < a.nco[j]; ++c) {
            float v = 0.0f;
            if (ok) {
                if (a.type[j] == SPH_AOS_F64) {
                    double d = *(const double *)(mine + a.off[j] + 8 * c);
                    if (f == SPH_F_X) d = __dsub_rn(d, org[c]);     // the only FP64 arithmetic here
                    v = d2f_bits_rn(d);
                } else {
                    v = *(const float *)(mine + a.off[j] + 4 * c);
                }
            }
            st_any(a.soa[j][c], a.fmt[j], k, v * a.scl[j], ok, a.n);
        }
    }
}

__global__ void __launch_bounds__(kConvThreads) k_soa_to_aos(ConvArgs a)
{
    extern __shared__ uint64_t smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t *rec = smem + (size_t)warp * 32 * a.Wp;
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool ok = k < a.n;
    const int64_t o = ok ? a.perm[k] : -1;
    uint8_t *mine = (uint8_t *)(rec + lane * a.Wp);
    if (ok) {
        for (int j = 0; j < a.nf; ++j) {
            for (int c = 0; c < a.nco[j]; ++c) {
                const float v = ld_val(a.soa[j][c], a.fmt[j], k) * a.scl[j];
                if (a.type[j] == SPH_AOS_F64) *(double *)(mine + a.off[j] + 8 * c) = f2d_bits(v);
                else *(float *)(mine + a.off[j] + 4 * c) = v;
            }
        }
    }
    store_records((uint32_t *)a.aos, (const uint32_t *)rec, o, a.W, a.Wp, a.umask, lane);
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
    a.aos = c->aos;
    a.n = c->n;
    a.W = c->layout.record_bytes / 8;
    a.Wp = a.W | 1;
    a.wmask = 0;
    a.umask[0] = a.umask[1] = 0;
    a.perm = c->perm();
    a.slot_cell = c->slot_cell();
    a.s3 = c->sub * c->sub * c->sub;
    for (int k = 0; k < 3; ++k) {
        a.nc[k] = c->nc[k];
        a.edge[k] = c->edge[k];
    }
    a.nf = 0;
    for (int f = 0; f < SPH_NFIELDS; ++f) {
        if (!(fields & SPH_BIT(f))) continue;
        int j = a.nf++;
        a.fid[j] = f;
        a.off[j] = c->layout.offset[f];
        a.type[j] = c->layout.type[f];
        a.fmt[j] = c->prec[f];
        a.scl[j] = to_soa ? c->enc(f) : c->dec(f);
        a.nco[j] = ncomp(f);
        for (int k = 0; k < 3; ++k) a.soa[j][k] = c->soa[f][k];
        const int es = a.type[j] == SPH_AOS_F64 ? 8 : 4;
        const int b0 = a.off[j], b1 = a.off[j] + es * a.nco[j];     // byte range [b0, b1)
        for (int w = b0 / 8; w <= (b1 - 1) / 8; ++w) a.wmask |= 1ull << w;
        for (int u = b0 / 4; u <= (b1 - 1) / 4; ++u) a.umask[u >> 6] |= 1ull << (u & 63);
    }
    return a;
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

inline size_t conv_smem(const ConvArgs &a) { return (size_t)(kConvThreads / 32) * 32 * a.Wp * sizeof(uint64_t); }

}  // namespace

cudaError_t run_aos_to_soa(sph_ctx *c, uint32_t fields)
{
    if (c->n == 0) return cudaSuccess;
    ConvArgs a = make_args(c, fields, true);
    const size_t smem = conv_smem(a);
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_aos_to_soa, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return e;
    k_aos_to_soa<<<blocks_for(c->n, kConvThreads), kConvThreads, smem, c->stream>>>(a);
    c->launches += 1;
    return cudaGetLastError();
}

cudaError_t run_soa_to_aos(sph_ctx *c, uint32_t fields)
{
    if (c->n == 0) return cudaSuccess;
    ConvArgs a = make_args(c, fields, false);
    const size_t smem = conv_smem(a);
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_soa_to_aos, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return e;
    k_soa_to_aos<<<blocks_for(c->n, kConvThreads), kConvThreads, smem, c->stream>>>(a);
    c->launches += 1;
    return cudaGetLastError();
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
