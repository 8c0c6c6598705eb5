// S2 and S7: the paper's conversion operators (Section 4).
//   U o N o C      gather the narrowed field set from the FP64 AoS records in
//                  cell order, round to the storage format, write SoA
//   C^T N^T U^T    decode SoA values, widen to the AoS element type, scatter
//                  to the particle's record
// One thread per sorted slot; all 32 lanes of a warp stay alive so that the
// packed formats can be written warp-cooperatively.
#include "sph_internal.cuh"

namespace sph {
namespace {

struct ConvArgs {
    uint8_t *aos;
    int64_t n;
    int32_t stride;
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
    int nco[SPH_NFIELDS];
    void *soa[SPH_NFIELDS][3];
};

__global__ void __launch_bounds__(256) k_aos_to_soa(ConvArgs a)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool ok = k < a.n;
    const int64_t o = ok ? a.perm[k] : 0;
    const uint8_t *rec = a.aos + o * a.stride;
    for (int j = 0; j < a.nf; ++j) {
        const int f = a.fid[j];
        double org[3] = {0.0, 0.0, 0.0};
        if (f == SPH_F_X && ok) {
            // cell-relative positions: offset from k_d * (L_d / nc_d), in FP64
            int32_t cid = a.slot_cell[k] / a.s3;   // key = cell * s^3 + sub-cell
            int32_t kx = cid % a.nc[0];
            int32_t t = cid / a.nc[0];
            int32_t ky = t % a.nc[1];
            int32_t kz = t / a.nc[1];
            org[0] = (double)kx * a.edge[0];
            org[1] = (double)ky * a.edge[1];
            org[2] = (double)kz * a.edge[2];
        }
        for (int c = 0; c < a.nco[j]; ++c) {
            double d = 0.0;
            if (ok) {
                if (a.type[j] == SPH_AOS_F64) d = *(const double *)(rec + a.off[j] + 8 * c);
                else d = (double)*(const float *)(rec + a.off[j] + 4 * c);
                d = __dsub_rn(d, org[c]);
            }
            st_any(a.soa[j][c], a.fmt[j], k, __double2float_rn(d), ok, a.n);
        }
    }
}

__global__ void __launch_bounds__(256) k_soa_to_aos(ConvArgs a)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= a.n) return;
    const int64_t o = a.perm[k];
    uint8_t *rec = a.aos + o * a.stride;
    for (int j = 0; j < a.nf; ++j) {
        for (int c = 0; c < a.nco[j]; ++c) {
            float v = ld_val(a.soa[j][c], a.fmt[j], k);
            if (a.type[j] == SPH_AOS_F64) *(double *)(rec + a.off[j] + 8 * c) = (double)v;
            else *(float *)(rec + a.off[j] + 4 * c) = v;
        }
    }
}

__global__ void __launch_bounds__(256) k_pack(const float *src, void *dst, int fmt, int64_t n)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool ok = k < n;
    st_any(dst, fmt, k, ok ? src[k] : 0.0f, ok, n);
}

ConvArgs make_args(sph_ctx *c, uint32_t fields)
{
    ConvArgs a;
    a.aos = c->aos;
    a.n = c->n;
    a.stride = c->layout.record_bytes;
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
        a.nco[j] = ncomp(f);
        for (int k = 0; k < 3; ++k) a.soa[j][k] = c->soa[f][k];
    }
    return a;
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t run_aos_to_soa(sph_ctx *c, uint32_t fields)
{
    if (c->n == 0) return cudaSuccess;
    ConvArgs a = make_args(c, fields);
    k_aos_to_soa<<<blocks_for(c->n, 256), 256, 0, c->stream>>>(a);
    c->launches += 1;
    return cudaGetLastError();
}

cudaError_t run_soa_to_aos(sph_ctx *c, uint32_t fields)
{
    if (c->n == 0) return cudaSuccess;
    ConvArgs a = make_args(c, fields);
    k_soa_to_aos<<<blocks_for(c->n, 256), 256, 0, c->stream>>>(a);
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
