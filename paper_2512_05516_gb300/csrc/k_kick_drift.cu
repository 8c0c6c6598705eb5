// S6: the paper's linear kernels Kick and Drift (Section 6), fused.
//   v += a dt_kick, u += du/dt dt_kick       FP32, in the SoA (storage format
//                                            of v and u applied on the store)
//   x += v dt_drift, wrapped into [0, L)      FP64, in place in the AoS record
// One thread per sorted slot; warps stay whole for packed v/u stores.
#include "sph_internal.cuh"

namespace sph {
namespace {

struct KDArgs {
    uint8_t *aos;
    int64_t n;
    int32_t stride, xoff;
    const int32_t *perm;
    double box[3];
    float dtk;
    double dtd;
    void *v[3];
    int vfmt;
    const float *a[3];
    void *u;
    int ufmt;
    const float *dudt;
    DevStats *st;
};

__global__ void __launch_bounds__(256) k_kick_drift(KDArgs a)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool ok = k < a.n;
    float vn[3] = {0.f, 0.f, 0.f};
    float un = 0.f;
    if (ok) {
        for (int c = 0; c < 3; ++c) vn[c] = fmaf(a.a[c][k], a.dtk, ld_val(a.v[c], a.vfmt, k));
        un = fmaf(a.dudt[k], a.dtk, ld_val(a.u, a.ufmt, k));
        const int64_t o = a.perm[k];
        double *x = (double *)(a.aos + o * a.stride + a.xoff);
        bool bad = false;
        for (int c = 0; c < 3; ++c) {
            double y = __dadd_rn(x[c], __dmul_rn((double)vn[c], a.dtd));
            y = __dsub_rn(y, __dmul_rn(a.box[c], floor(y / a.box[c])));
            if (y >= a.box[c]) y = 0.0;
            bad |= !isfinite(y);
            x[c] = y;
        }
        if (bad || !isfinite(un)) set_error(a.st, SPH_ERR_NONFINITE);
    }
    for (int c = 0; c < 3; ++c) st_any(a.v[c], a.vfmt, k, vn[c], ok, a.n);
    st_any(a.u, a.ufmt, k, un, ok, a.n);
}

}  // namespace

cudaError_t run_kick_drift(sph_ctx *c, double dt_kick, double dt_drift)
{
    if (c->n == 0) return cudaSuccess;
    KDArgs a;
    a.aos = c->aos;
    a.n = c->n;
    a.stride = c->layout.record_bytes;
    a.xoff = c->layout.offset[SPH_F_X];
    a.perm = c->perm();
    for (int k = 0; k < 3; ++k) {
        a.box[k] = c->params.box[k];
        a.v[k] = c->soa[SPH_F_V][k];
        a.a[k] = (const float *)c->soa[SPH_F_A][k];
    }
    a.dtk = (float)dt_kick;
    a.dtd = dt_drift;
    a.vfmt = c->prec[SPH_F_V];
    a.u = c->soa[SPH_F_U][0];
    a.ufmt = c->prec[SPH_F_U];
    a.dudt = (const float *)c->soa[SPH_F_DUDT][0];
    a.st = c->dstats;
    k_kick_drift<<<(unsigned)((c->n + 255) / 256), 256, 0, c->stream>>>(a);
    c->launches += 1;
    return cudaGetLastError();
}

}  // namespace sph
