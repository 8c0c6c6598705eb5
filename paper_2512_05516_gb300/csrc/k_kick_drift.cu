// S6: the paper's linear kernels Kick and Drift (Section 6), fused.
//   v += a dt_kick, u += du/dt dt_kick       FP32, in the SoA (storage format
//                                            of v and u applied on the store)
//   x += v dt_drift, wrapped into [0, L)      FP64, in place in the AoS record
// One thread per sorted slot; warps stay whole for packed v/u stores.  The
// three FP64 position words of the warp's 32 records are loaded and stored
// lane-contiguously through shared memory.
#include "sph_internal.cuh"

namespace sph {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kKDThreads = 256;

struct KDArgs {
    uint8_t *aos;
    int64_t n;
    int32_t W;                   // record words
    int32_t xw;                  // first position word in the record
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
    DevStats *st;
};

__global__ void __launch_bounds__(kKDThreads) k_kick_drift(KDArgs a)
{
    __shared__ double sx[kKDThreads / 32][32 * 3 + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double *xs = sx[warp];
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
    double *aos64 = (double *)a.aos;
    // lane l moves word l % 3 of record l / 3 (then +32, +64)
    double xw[3];
#pragma unroll
    for (int t = 0; t < 3; ++t) {
        const int idx = lane + 32 * t;
        const int r = idx / 3, w = idx - 3 * r;
        const int64_t orr = __shfl_sync(FULL, o, r);
        xw[t] = orr >= 0 ? aos64[orr * a.W + a.xw + w] : 0.0;
    }
#pragma unroll
    for (int t = 0; t < 3; ++t) xs[lane + 32 * t] = xw[t];
    __syncwarp();
    if (ok) {
        bool bad = false;
        for (int c = 0; c < 3; ++c) {
            // x += v dt in FP64 (one FMA, the FP64 arithmetic the step
            // needs); a position already in [0, L) -- tested on the bit
            // patterns, since non-negative doubles order like their bits --
            // needs no wrap; the few that left the box take the periodic
            // wrap x - L floor(x / L)
            double y = fma(f2d_bits(vn[c]), a.dtd, xs[3 * lane + c]);
            const long long yb = __double_as_longlong(y);
            if (yb < 0 || yb >= __double_as_longlong(a.box[c])) {
                if ((yb & 0x7FF0000000000000ll) == 0x7FF0000000000000ll) {
                    bad = true;                        // inf or nan
                } else {
                    y = __dsub_rn(y, __dmul_rn(a.box[c], floor(y / a.box[c])));
                    if (y >= a.box[c]) y = 0.0;        // rounding onto L
                }
            }
            xs[3 * lane + c] = y;
        }
        if (bad || !isfinite(un)) set_error(a.st, SPH_ERR_NONFINITE);
    }
    __syncwarp();
#pragma unroll
    for (int t = 0; t < 3; ++t) {
        const int idx = lane + 32 * t;
        const int r = idx / 3, w = idx - 3 * r;
        const int64_t orr = __shfl_sync(FULL, o, r);
        if (orr >= 0) aos64[orr * a.W + a.xw + w] = xs[idx];
    }
    for (int c = 0; c < 3; ++c) st_any(a.v[c], a.vfmt, k, vn[c] * a.venc, ok, a.n);
    st_any(a.u, a.ufmt, k, un * a.uenc, ok, a.n);
}

}  // namespace

cudaError_t run_kick_drift(sph_ctx *c, double dt_kick, double dt_drift)
{
    if (c->n == 0) return cudaSuccess;
    KDArgs a;
    a.aos = c->aos;
    a.n = c->n;
    a.W = c->layout.record_bytes / 8;
    a.xw = c->layout.offset[SPH_F_X] / 8;
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
    a.st = c->dstats;
    k_kick_drift<<<(unsigned)((c->n + kKDThreads - 1) / kKDThreads), kKDThreads, 0, c->stream>>>(a);
    c->launches += 1;
    return cudaGetLastError();
}

}  // namespace sph
