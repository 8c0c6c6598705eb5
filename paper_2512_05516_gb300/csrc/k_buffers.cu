// The paper's benchmark grouping (Section 6): particles in contiguous buffers
// of B spatially co-located records; the quadratic kernels Density and Force
// evaluate every pair of a buffer (64 x 64 for B = 64), the linear kernels
// Kick and Drift every particle once.  Each kernel reads its inputs either
// from the AoS records directly (the paper's AoS baseline) or from the SoA
// arrays the conversion wrote, through one of two accessors, and otherwise
// runs the same code, so that the two layouts can be timed against each
// other (the paper's Fig. 2).
//
// A CTA of 256 threads holds 256 / B whole buffers, one thread per particle.
// Each thread loads its own particle -- from the records with the record
// stride, its position made relative to the buffer's first particle there
// (one FP64 subtraction per component); from the SoA coalesced, the relative
// position already stored.  Staged form (the default): each thread puts its
// particle in shared memory and the pair loop reads its partners there.
// Plain form (tuning pair_kernel = 1, the structure of the paper's kernels):
// the pair loop reads every partner through the accessor from global memory
// (the L1 cache serves the repeats), so that the record layout acts on every
// pair.  Both forms do the same arithmetic in the same order and give
// identical bits.  Arithmetic is FP32 (the cell-list kernels' per-pair code,
// k_pair_math.cuh); the drift of AoS positions is FP64.
#include <cstring>

#include "k_pair_math.cuh"
#include "k_records.cuh"

namespace sph {
namespace {

constexpr int kBufThreads = 256;

struct BufField {
    void *p[3];
    int fmt;
    float dec, enc;              // storage scale: value = stored * dec, stored = value * enc
};

struct BufArgs {
    int64_t n, nbuf;
    int lgB;                     // buffer size 2^lgB
    uint8_t *aos;
    int64_t rb;                  // record bytes
    int off[SPH_NFIELDS];        // byte offset of each field in the record (-1: absent)
    int f64[SPH_NFIELDS];        // the record holds the field as FP64
    BufField soa[SPH_NFIELDS];
    const double *origin;        // buffer origins, 3 x nbuf, axis-major
    double box[3];
    float gamma, alpha, beta, eps;
    float dt;
    double dtd;
    DevStats *st;
};

// ---- the two accessors ----------------------------------------------------
__device__ __forceinline__ float rec_get(const BufArgs &a, int64_t i, int f, int comp)
{
    const uint8_t *p = a.aos + i * a.rb + a.off[f];
    return a.f64[f] ? d2f_bits_rn(reinterpret_cast<const double *>(p)[comp])
                    : reinterpret_cast<const float *>(p)[comp];
}

__device__ __forceinline__ void rec_put(const BufArgs &a, int64_t i, int f, int comp, float v)
{
    uint8_t *p = a.aos + i * a.rb + a.off[f];
    if (a.f64[f]) reinterpret_cast<double *>(p)[comp] = f2d_bits(v);
    else reinterpret_cast<float *>(p)[comp] = v;
}

__device__ __forceinline__ float soa_get(const BufArgs &a, int64_t i, int f, int comp)
{
    const BufField &F = a.soa[f];
    return ld_val(F.p[comp], F.fmt, i) * F.dec;
}

// every thread of the warp calls it (packed formats store warp-cooperatively)
__device__ __forceinline__ void soa_put(const BufArgs &a, int64_t i, int f, int comp, float v, bool ok)
{
    const BufField &F = a.soa[f];
    st_any(F.p[comp], F.fmt, i, v * F.enc, ok, a.n);
}

template <bool kAos>
__device__ __forceinline__ float get(const BufArgs &a, int64_t i, int f, int comp = 0)
{
    return kAos ? rec_get(a, i, f, comp) : soa_get(a, i, f, comp);
}

// position relative to the buffer's first particle
template <bool kAos>
__device__ __forceinline__ float3 pos_rel(const BufArgs &a, int64_t i)
{
    if (kAos) {
        const int64_t b = i >> a.lgB;
        const double *x = reinterpret_cast<const double *>(a.aos + i * a.rb + a.off[SPH_F_X]);
        return make_float3(buffer_offset_f32(x[0], a.origin[b], a.box[0]),
                           buffer_offset_f32(x[1], a.origin[a.nbuf + b], a.box[1]),
                           buffer_offset_f32(x[2], a.origin[2 * a.nbuf + b], a.box[2]));
    }
    return make_float3(soa_get(a, i, SPH_F_X, 0), soa_get(a, i, SPH_F_X, 1), soa_get(a, i, SPH_F_X, 2));
}

__device__ __forceinline__ void count_pairs(unsigned long long *ctr, int k)
{
    const unsigned s = __reduce_add_sync(0xffffffffu, (unsigned)k);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(ctr, (unsigned long long)s);
}

// ---- Density: rho_i = sum over the buffer of m_j W(r_ij, h_i), self included;
//      then P = (gamma - 1) rho u and c = sqrt(gamma P / rho) ----------------
template <bool kAos>
__device__ __forceinline__ float4 partner_xm(const BufArgs &a, int64_t j)
{
    const float3 x = pos_rel<kAos>(a, j);
    return make_float4(x.x, x.y, x.z, get<kAos>(a, j, SPH_F_M));
}

template <bool kAos, bool kStaged>
__global__ void __launch_bounds__(kBufThreads) k_buf_density(BufArgs a)
{
    __shared__ float4 sj[kStaged ? kBufThreads : 1];   // (x, y, z, m), buffer-relative
    const int t = threadIdx.x;
    const int64_t i = (int64_t)blockIdx.x * kBufThreads + t;
    const bool ok = i < a.n;
    float3 xi = make_float3(0.f, 0.f, 0.f);
    float m = 0.f, h = 1.f, u = 0.f;
    if (ok) {
        xi = pos_rel<kAos>(a, i);
        m = get<kAos>(a, i, SPH_F_M);
        h = get<kAos>(a, i, SPH_F_H);
        u = get<kAos>(a, i, SPH_F_U);
    }
    if (kStaged) {
        sj[t] = make_float4(xi.x, xi.y, xi.z, m);
        __syncthreads();
    }
    const int B = 1 << a.lgB;
    const int me = t & (B - 1);
    const int t0 = t - me;
    const int64_t first = i - me;                        // the buffer's first record
    const int64_t cnt64 = a.n - first;
    const int cnt = ok ? (int)(cnt64 < B ? cnt64 : B) : 0;
    const float hinv = 1.0f / h, h2x4 = 4.0f * h * h;
    float s = 0.f, cs = 0.f;
    int k = 0;
    for (int j = 0; j < cnt; ++j) {
        const float4 q = kStaged ? sj[t0 + j] : partner_xm<kAos>(a, first + j);
        const float dx = xi.x - q.x, dy = xi.y - q.y, dz = xi.z - q.z;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const float r = r2 * rsqrtf(fmaxf(r2, 1.0e-30f));     // 0 for the self pair
        float w, dw;
        spline(r * hinv, w, dw);                              // 0 beyond the support
        kahan_add(s, cs, q.w * w);
        k += (r2 < h2x4 && j != me) ? 1 : 0;
    }
    const float h3inv = hinv * hinv * hinv;
    const float rho = kSigma * h3inv * (s - cs);
    const float P = (a.gamma - 1.0f) * rho * u;
    const float c = sqrtf(a.gamma * P / rho);
    if (ok && !(isfinite(rho) && isfinite(P))) set_error(a.st, SPH_ERR_NONFINITE);
    if (kAos) {
        if (ok) {
            rec_put(a, i, SPH_F_RHO, 0, rho);
            rec_put(a, i, SPH_F_P, 0, P);
            if (a.off[SPH_F_CS] >= 0) rec_put(a, i, SPH_F_CS, 0, c);
        }
    } else {
        soa_put(a, i, SPH_F_RHO, 0, rho, ok);
        soa_put(a, i, SPH_F_P, 0, P, ok);
        soa_put(a, i, SPH_F_CS, 0, c, ok);
    }
    count_pairs(&a.st->pairs_density, k);
}

// ---- Force: the symmetric pair force with Monaghan viscosity over the
//      buffer's pairs r < h_i + h_j (Eq. 7, Eq. 5); c from the EOS --------------
// a partner's force inputs: (x, y, z, h), (v, m), (P / rho^2, rho, c, -)
template <bool kAos>
__device__ __forceinline__ void partner_force(const BufArgs &a, int64_t j, float4 &qa, float4 &qb, float4 &qc)
{
    const float3 x = pos_rel<kAos>(a, j);
    qa = make_float4(x.x, x.y, x.z, get<kAos>(a, j, SPH_F_H));
    qb = make_float4(get<kAos>(a, j, SPH_F_V, 0), get<kAos>(a, j, SPH_F_V, 1), get<kAos>(a, j, SPH_F_V, 2),
                     get<kAos>(a, j, SPH_F_M));
    const float rho = get<kAos>(a, j, SPH_F_RHO), P = get<kAos>(a, j, SPH_F_P);
    qc = make_float4(P / (rho * rho), rho, sqrtf(a.gamma * P / rho), 0.f);
}

template <bool kAos, bool kStaged>
__global__ void __launch_bounds__(kBufThreads) k_buf_force(BufArgs a)
{
    constexpr int S = kStaged ? kBufThreads : 1;
    __shared__ float4 sA[S], sB[S], sC[S];
    const int t = threadIdx.x;
    const int64_t i = (int64_t)blockIdx.x * kBufThreads + t;
    const bool ok = i < a.n;
    float3 xi = make_float3(0.f, 0.f, 0.f), vi = make_float3(0.f, 0.f, 0.f);
    float m = 0.f, h = 0.f, rho = 1.f, P = 0.f;
    if (ok) {
        xi = pos_rel<kAos>(a, i);
        vi = make_float3(get<kAos>(a, i, SPH_F_V, 0), get<kAos>(a, i, SPH_F_V, 1), get<kAos>(a, i, SPH_F_V, 2));
        m = get<kAos>(a, i, SPH_F_M);
        h = get<kAos>(a, i, SPH_F_H);
        rho = get<kAos>(a, i, SPH_F_RHO);
        P = get<kAos>(a, i, SPH_F_P);
    }
    const float Pr2 = P / (rho * rho);
    const float c = sqrtf(a.gamma * P / rho);
    if (kStaged) {
        sA[t] = make_float4(xi.x, xi.y, xi.z, h);
        sB[t] = make_float4(vi.x, vi.y, vi.z, m);
        sC[t] = make_float4(Pr2, rho, c, 0.f);
        __syncthreads();
    }
    const int B = 1 << a.lgB;
    const int me = t & (B - 1);
    const int t0 = t - me;
    const int64_t first = i - me;
    const int64_t cnt64 = a.n - first;
    const int cnt = ok ? (int)(cnt64 < B ? cnt64 : B) : 0;
    float ax = 0.f, ay = 0.f, az = 0.f, du = 0.f;
    int k = 0;
    for (int j = 0; j < cnt; ++j) {
        if (j == me) continue;
        float4 qa, qb, qc;
        if (kStaged) {
            qa = sA[t0 + j];
            qb = sB[t0 + j];
            qc = sC[t0 + j];
        } else {
            partner_force<kAos>(a, first + j, qa, qb, qc);
        }
        const float dx = xi.x - qa.x, dy = xi.y - qa.y, dz = xi.z - qa.z;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const float hs = h + qa.w;
        if (!(r2 < hs * hs)) continue;
        ++k;
        if (r2 == 0.0f) continue;                             // coincident pair: grad W = 0
        force_pair(ax, ay, az, du, vi.x, vi.y, vi.z, rho, Pr2, c, dx, dy, dz, r2, hs, qb, qc, a.alpha, a.beta,
                   a.eps);
    }
    if (ok && !(isfinite(ax) && isfinite(ay) && isfinite(az) && isfinite(du))) set_error(a.st, SPH_ERR_NONFINITE);
    if (kAos) {
        if (ok) {
            rec_put(a, i, SPH_F_A, 0, ax);
            rec_put(a, i, SPH_F_A, 1, ay);
            rec_put(a, i, SPH_F_A, 2, az);
            rec_put(a, i, SPH_F_DUDT, 0, du);
        }
    } else {
        soa_put(a, i, SPH_F_A, 0, ax, ok);
        soa_put(a, i, SPH_F_A, 1, ay, ok);
        soa_put(a, i, SPH_F_A, 2, az, ok);
        soa_put(a, i, SPH_F_DUDT, 0, du, ok);
    }
    count_pairs(&a.st->pairs_force, k);
}

// ---- Kick: v += a dt, u += du/dt dt (FP32) ---------------------------------
template <bool kAos>
__global__ void __launch_bounds__(kBufThreads) k_buf_kick(BufArgs a)
{
    const int64_t i = (int64_t)blockIdx.x * kBufThreads + threadIdx.x;
    const bool ok = i < a.n;
    float v[3] = {0.f, 0.f, 0.f}, u = 0.f;
    if (ok) {
        for (int c = 0; c < 3; ++c) v[c] = fmaf(get<kAos>(a, i, SPH_F_A, c), a.dt, get<kAos>(a, i, SPH_F_V, c));
        u = fmaf(get<kAos>(a, i, SPH_F_DUDT), a.dt, get<kAos>(a, i, SPH_F_U));
        if (!(isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]) && isfinite(u))) set_error(a.st, SPH_ERR_NONFINITE);
    }
    if (kAos) {
        if (ok) {
            for (int c = 0; c < 3; ++c) rec_put(a, i, SPH_F_V, c, v[c]);
            rec_put(a, i, SPH_F_U, 0, u);
        }
    } else {
        for (int c = 0; c < 3; ++c) soa_put(a, i, SPH_F_V, c, v[c], ok);
        soa_put(a, i, SPH_F_U, 0, u, ok);
    }
}

// ---- Drift: x += v dt.  Records: FP64, wrapped into [0, L).  SoA: the FP32
//      offsets from the buffer origin (the write-back wraps them) ---------------
template <bool kAos>
__global__ void __launch_bounds__(kBufThreads) k_buf_drift(BufArgs a)
{
    const int64_t i = (int64_t)blockIdx.x * kBufThreads + threadIdx.x;
    const bool ok = i < a.n;
    if (kAos) {
        if (!ok) return;
        double *x = reinterpret_cast<double *>(a.aos + i * a.rb + a.off[SPH_F_X]);
        bool bad = false;
        for (int c = 0; c < 3; ++c) {
            double y = fma(f2d_bits(rec_get(a, i, SPH_F_V, c)), a.dtd, x[c]);
            if (!isfinite(y)) {
                bad = true;
            } else if (y < 0.0 || y >= a.box[c]) {
                y = __dsub_rn(y, __dmul_rn(a.box[c], floor(y / a.box[c])));
                if (y >= a.box[c]) y = 0.0;                   // rounding onto L
            }
            x[c] = y;
        }
        if (bad) set_error(a.st, SPH_ERR_NONFINITE);
    } else {
        float y[3] = {0.f, 0.f, 0.f};
        if (ok) {
            for (int c = 0; c < 3; ++c) y[c] = fmaf(soa_get(a, i, SPH_F_V, c), a.dt, soa_get(a, i, SPH_F_X, c));
            if (!(isfinite(y[0]) && isfinite(y[1]) && isfinite(y[2]))) set_error(a.st, SPH_ERR_NONFINITE);
        }
        for (int c = 0; c < 3; ++c) soa_put(a, i, SPH_F_X, c, y[c], ok);
    }
}

__global__ void k_buf_setup(int32_t *perm, double *origin, const uint8_t *aos, int64_t n, int64_t rb,
                            int xoff, int lgB, int64_t nbuf)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) perm[k] = (int32_t)k;
    if (k < nbuf) {
        const double *x = reinterpret_cast<const double *>(aos + (k << lgB) * rb + xoff);
        origin[k] = x[0];
        origin[nbuf + k] = x[1];
        origin[2 * nbuf + k] = x[2];
    }
}

BufArgs make_buf_args(sph_ctx *c)
{
    BufArgs a;
    std::memset(&a, 0, sizeof(a));
    a.n = c->n;
    a.lgB = 31 - __builtin_clz((unsigned)c->buffer);
    a.nbuf = (c->n + c->buffer - 1) / c->buffer;
    a.aos = c->aos;
    a.rb = c->layout.record_bytes;
    for (int f = 0; f < SPH_NFIELDS; ++f) {
        a.off[f] = c->layout.offset[f];
        a.f64[f] = c->layout.type[f] == SPH_AOS_F64 ? 1 : 0;
        for (int k = 0; k < 3; ++k) a.soa[f].p[k] = c->soa[f][k];
        a.soa[f].fmt = c->prec[f];
        a.soa[f].dec = c->dec(f);
        a.soa[f].enc = c->enc(f);
    }
    a.origin = c->buf_origin;
    for (int k = 0; k < 3; ++k) a.box[k] = c->params.box[k];
    a.gamma = (float)c->params.gamma;
    a.alpha = (float)c->params.alpha_av;
    a.beta = (float)c->params.beta_av;
    a.eps = (float)c->params.eps_av;
    a.st = c->dstats;
    return a;
}

template <typename K>
cudaError_t launch_buf(sph_ctx *c, K kern, const BufArgs &a)
{
    if (c->n == 0) return cudaSuccess;
    const unsigned grid = (unsigned)((c->n + kBufThreads - 1) / kBufThreads);
    kern<<<grid, kBufThreads, 0, c->stream>>>(a);
    c->launches += 1;
    return cudaGetLastError();
}

}  // namespace

cudaError_t run_bin_buffers(sph_ctx *c)
{
    if (c->n == 0) return cudaSuccess;
    const int lgB = 31 - __builtin_clz((unsigned)c->buffer);
    const int64_t nbuf = (c->n + c->buffer - 1) / c->buffer;
    c->sorted_buf = 0;
    k_buf_setup<<<(unsigned)((c->n + 255) / 256), 256, 0, c->stream>>>(
        c->vals[0], c->buf_origin, c->aos, c->n, c->layout.record_bytes, c->layout.offset[SPH_F_X], lgB, nbuf);
    c->launches += 1;
    return cudaGetLastError();
}

cudaError_t run_buffer_density(sph_ctx *c, int source)
{
    const BufArgs a = make_buf_args(c);
    const bool staged = c->tuning.pair_kernel != 1;
    if (source == SPH_SRC_AOS)
        return staged ? launch_buf(c, k_buf_density<true, true>, a) : launch_buf(c, k_buf_density<true, false>, a);
    return staged ? launch_buf(c, k_buf_density<false, true>, a) : launch_buf(c, k_buf_density<false, false>, a);
}

cudaError_t run_buffer_force(sph_ctx *c, int source)
{
    const BufArgs a = make_buf_args(c);
    const bool staged = c->tuning.pair_kernel != 1;
    if (source == SPH_SRC_AOS)
        return staged ? launch_buf(c, k_buf_force<true, true>, a) : launch_buf(c, k_buf_force<true, false>, a);
    return staged ? launch_buf(c, k_buf_force<false, true>, a) : launch_buf(c, k_buf_force<false, false>, a);
}

cudaError_t run_buffer_kick(sph_ctx *c, int source, double dt)
{
    BufArgs a = make_buf_args(c);
    a.dt = (float)dt;
    return source == SPH_SRC_AOS ? launch_buf(c, k_buf_kick<true>, a) : launch_buf(c, k_buf_kick<false>, a);
}

cudaError_t run_buffer_drift(sph_ctx *c, int source, double dt)
{
    BufArgs a = make_buf_args(c);
    a.dt = (float)dt;
    a.dtd = dt;
    return source == SPH_SRC_AOS ? launch_buf(c, k_buf_drift<true>, a) : launch_buf(c, k_buf_drift<false>, a);
}

}  // namespace sph
