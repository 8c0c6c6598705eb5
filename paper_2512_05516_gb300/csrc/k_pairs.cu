// S3-S5: the quadratic SPH kernels (the paper's Density and Force, Section 6),
// as persistent CUDA-core kernels over a work queue.
//
// Work item = (cell, first slot, count <= blockDim): the i-particles of one
// tile of one cell, one thread each.  Per item the CTA stages the particles of
// the 27 neighbour cells (periodic) into shared memory, converted to FP32 and
// shifted into the item cell's frame (positions are cell-relative, so the
// shift is just the neighbour's cell offset times the cell edge).  Each warp
// then filters the staged candidates against the bounding box of its own 32
// i-particles (ballot + compaction into a per-warp index list), and each lane
// runs the pair loop over that list.  Candidates outside the support of every
// lane of the warp are never visited by the per-lane loop.
//
// Density (Eq. 6, gather form): rho_i = sum_j m_j W(r_ij, h_i), M4 cubic
// spline W = sigma/h^3 w(r/h), support 2h, Neumaier-compensated FP32 sum;
// `newton_steps` Newton steps on f(h) = rho(h) - m_i (eta/h)^3 clamped to
// [h/2, 2h] and h_max, then a final sum; EOS P = (gamma-1) rho u,
// c = sqrt(gamma P / rho).
//
// Force (Eq. 7 + Monaghan viscosity, Eq. 5 for du/dt), pairs r < h_i + h_j:
//   a_i    -= m_j (P_i/rho_i^2 + P_j/rho_j^2 + Pi_ij) gradW(r_ij, hbar)
//   du_i/dt += m_j (P_i/rho_i^2 + Pi_ij/2) v_ij . gradW
#include "sph_internal.cuh"

namespace sph {
cudaError_t run_pack(sph_ctx *c, const float *src, int f);

namespace {

constexpr unsigned FULL = 0xffffffffu;

struct Common {
    int64_t n;
    int32_t nc[3];
    float edge[3];
    const int32_t *cell_start;
    const int32_t *icell, *ifirst, *icount;
    DevStats *st;
    FieldRef x, m, h;
    int stage_cap;
};

struct DensityArgs {
    Common c;
    FieldRef u;
    bool has_u;
    int npass;               // newton_steps + 1
    float eta3, h_cap, gm1, gamma;
    bool plain_sum;
    void *rho_out; int rho_fmt;
    void *h_out; int h_fmt;  // h_out may be the FP32 stage when H is packed
    bool write_h;
    void *P_out; int P_fmt;
    void *cs_out; int cs_fmt;
    int32_t *nngb;
};

struct ForceArgs {
    Common c;
    FieldRef v, rho, P, cs;
    float alpha, beta, eps;
    float *a[3];
    float *dudt;
    int32_t *nngb;
};

struct ItemShared {
    int item, cell, first, count;
    int start[27];
    int off[28];
    float shift[27][3];
};

// Pop the next work item and describe its 27 neighbour cells.  Returns false
// when the queue is exhausted.  Must be called by the whole CTA.
__device__ bool next_item(const Common &c, ItemShared &s)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        int it = (int)atomicAdd(&c.st->queue, 1u);
        s.item = it < c.st->nitems ? it : -1;
        if (s.item >= 0) {
            s.cell = c.icell[it];
            s.first = c.ifirst[it];
            s.count = c.icount[it];
        }
    }
    __syncthreads();
    if (s.item < 0) return false;
    if (threadIdx.x < 32) {
        const int t = threadIdx.x;
        int cnt = 0;
        if (t < 27) {
            const int cell = s.cell;
            const int kx = cell % c.nc[0];
            const int ky = (cell / c.nc[0]) % c.nc[1];
            const int kz = cell / (c.nc[0] * c.nc[1]);
            const int dx = t % 3 - 1, dy = (t / 3) % 3 - 1, dz = t / 9 - 1;
            const int nx = (kx + dx + c.nc[0]) % c.nc[0];
            const int ny = (ky + dy + c.nc[1]) % c.nc[1];
            const int nz = (kz + dz + c.nc[2]) % c.nc[2];
            const int nb = nx + c.nc[0] * (ny + c.nc[1] * nz);
            const int st = c.cell_start[nb];
            cnt = c.cell_start[nb + 1] - st;
            s.start[t] = st;
            s.shift[t][0] = (float)dx * c.edge[0];
            s.shift[t][1] = (float)dy * c.edge[1];
            s.shift[t][2] = (float)dz * c.edge[2];
        }
        int inc = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int v = __shfl_up_sync(FULL, inc, o);
            if (t >= o) inc += v;
        }
        if (t < 27) s.off[t + 1] = inc;
        if (t == 0) s.off[0] = 0;
    }
    __syncthreads();
    return true;
}

__device__ __forceinline__ float warp_max(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(FULL, v, o));
    return v;
}
__device__ __forceinline__ float warp_min(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(FULL, v, o));
    return v;
}
__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

struct Box { float lo[3], hi[3]; };

__device__ __forceinline__ Box warp_box(bool ok, float x, float y, float z)
{
    Box b;
    b.lo[0] = warp_min(ok ? x : 3.0e38f);
    b.lo[1] = warp_min(ok ? y : 3.0e38f);
    b.lo[2] = warp_min(ok ? z : 3.0e38f);
    b.hi[0] = warp_max(ok ? x : -3.0e38f);
    b.hi[1] = warp_max(ok ? y : -3.0e38f);
    b.hi[2] = warp_max(ok ? z : -3.0e38f);
    return b;
}

__device__ __forceinline__ float box_dist2(const Box &b, float x, float y, float z)
{
    float dx = fmaxf(0.0f, fmaxf(b.lo[0] - x, x - b.hi[0]));
    float dy = fmaxf(0.0f, fmaxf(b.lo[1] - y, y - b.hi[1]));
    float dz = fmaxf(0.0f, fmaxf(b.lo[2] - z, z - b.hi[2]));
    return fmaf(dx, dx, fmaf(dy, dy, dz * dz));
}

// the slot index of staged candidate g (global position in the 27-cell list)
__device__ __forceinline__ int staged_slot(const ItemShared &s, int g)
{
    int lo = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1)
        if (lo + step < 27 && s.off[lo + step] <= g) lo += step;
    return lo;
}

// ---------------------------------------------------------------------------
// density
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kMaxBlock) k_density(DensityArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ ItemShared s;
    const Common &c = a.c;
    float4 *sj = reinterpret_cast<float4 *>(smem);
    uint16_t *lists = reinterpret_cast<uint16_t *>(smem + (size_t)c.stage_cap * sizeof(float4));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint16_t *wl = lists + warp * kListCap;
    const unsigned lt = (1u << lane) - 1u;

    unsigned long long my_pairs = 0, my_tests = 0;
    unsigned my_err = 0;

    while (next_item(c, s)) {
        bool clamped = false;
        const int t = threadIdx.x;
        const bool ok = t < s.count;
        const int64_t k = (int64_t)s.first + t;
        float xi = 0.f, yi = 0.f, zi = 0.f, mi = 0.f, hi = 0.f, ui = 0.f;
        if (ok) {
            xi = ld_val(c.x.p[0], c.x.fmt, k);
            yi = ld_val(c.x.p[1], c.x.fmt, k);
            zi = ld_val(c.x.p[2], c.x.fmt, k);
            mi = ld_val(c.m.p[0], c.m.fmt, k);
            hi = ld_val(c.h.p[0], c.h.fmt, k);
            if (a.has_u) ui = ld_val(a.u.p[0], a.u.fmt, k);
            if (!(hi > 0.0f) || !isfinite(hi)) { hi = a.h_cap; my_err |= SPH_ERR_NONFINITE; }
            if (hi > a.h_cap) { hi = a.h_cap; clamped = true; }
        }
        const bool warp_live = __any_sync(FULL, ok);
        const Box bx = warp_box(ok, xi, yi, zi);
        const int total = s.off[27];
        const bool one_chunk = total <= c.stage_cap;
        float rho = 0.f, drdh = 0.f;
        int cnt = 0;
        for (int pass = 0; pass < a.npass; ++pass) {
            const float h2x4 = 4.0f * hi * hi;
            const float hinv = 1.0f / hi;
            const float hw = warp_max(ok ? hi : 0.0f);
            const float R2 = 4.0f * hw * hw;
            float sr = 0.f, sc = 0.f, sd = 0.f;
            cnt = 0;
            for (int c0 = 0; c0 < total; c0 += c.stage_cap) {
                const int len = min(c.stage_cap, total - c0);
                if (!one_chunk || pass == 0) {
                    __syncthreads();
                    for (int p = threadIdx.x; p < len; p += blockDim.x) {
                        const int g = c0 + p;
                        const int sl = staged_slot(s, g);
                        const int64_t j = (int64_t)s.start[sl] + (g - s.off[sl]);
                        float4 q;
                        q.x = ld_val(c.x.p[0], c.x.fmt, j) + s.shift[sl][0];
                        q.y = ld_val(c.x.p[1], c.x.fmt, j) + s.shift[sl][1];
                        q.z = ld_val(c.x.p[2], c.x.fmt, j) + s.shift[sl][2];
                        q.w = ld_val(c.m.p[0], c.m.fmt, j);
                        sj[p] = q;
                    }
                    __syncthreads();
                }
                if (!warp_live) continue;
                int p0 = 0;
                while (p0 < len) {
                    int nl = 0;
                    while (p0 < len && nl <= kListCap - 32) {
                        const int p = p0 + lane;
                        bool keep = false;
                        if (p < len) {
                            const float4 q = sj[p];
                            keep = box_dist2(bx, q.x, q.y, q.z) < R2;
                        }
                        const unsigned bal = __ballot_sync(FULL, keep);
                        if (keep) wl[nl + __popc(bal & lt)] = (uint16_t)p;
                        nl += __popc(bal);
                        p0 += 32;
                    }
                    __syncwarp();
                    if (ok) {
                        my_tests += (unsigned long long)nl;
                        for (int e = 0; e < nl; ++e) {
                            const float4 q = sj[wl[e]];
                            const float dx = xi - q.x, dy = yi - q.y, dz = zi - q.z;
                            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                            if (r2 < h2x4) {
                                const float r = r2 > 0.0f ? r2 * rsqrtf(r2) : 0.0f;
                                const float qq = r * hinv;
                                float w, dw;
                                if (qq < 1.0f) {
                                    w = fmaf(qq * qq, fmaf(0.75f, qq, -1.5f), 1.0f);
                                    dw = qq * fmaf(2.25f, qq, -3.0f);
                                } else {
                                    const float tt = 2.0f - qq;
                                    w = 0.25f * tt * tt * tt;
                                    dw = -0.75f * tt * tt;
                                }
                                const float term = q.w * w;
                                if (a.plain_sum) {
                                    sr += term;
                                } else {   // Neumaier compensated summation
                                    const float tsum = __fadd_rn(sr, term);
                                    if (fabsf(sr) >= fabsf(term)) sc += __fadd_rn(__fsub_rn(sr, tsum), term);
                                    else sc += __fadd_rn(__fsub_rn(term, tsum), sr);
                                    sr = tsum;
                                }
                                sd = fmaf(q.w, fmaf(qq, dw, 3.0f * w), sd);
                                ++cnt;
                            }
                        }
                    }
                    __syncwarp();
                }
            }
            if (ok) {
                const float h3inv = hinv * hinv * hinv;
                rho = kSigma * h3inv * (sr + sc);
                drdh = -kSigma * h3inv * hinv * sd;
                cnt -= 1;            // the self term is in rho, not in the count
                my_pairs += (unsigned long long)cnt;
                if (pass + 1 < a.npass) {
                    // Newton step on f(h) = rho(h) - m (eta/h)^3
                    const float f = rho - mi * a.eta3 * h3inv;
                    const float fp = drdh + 3.0f * mi * a.eta3 * h3inv * hinv;
                    float hn = hi;
                    if (fp > 0.0f && isfinite(f) && isfinite(fp)) hn = hi - f / fp;
                    else my_err |= SPH_ERR_NEWTON;
                    hn = fminf(fmaxf(hn, 0.5f * hi), 2.0f * hi);
                    if (hn > a.h_cap) { hn = a.h_cap; clamped = true; }
                    hi = hn;
                }
            }
        }
        if (ok) {
            if (!isfinite(rho)) my_err |= SPH_ERR_NONFINITE;
            st_val(a.rho_out, a.rho_fmt, k, rho);
            if (a.write_h) st_val(a.h_out, a.h_fmt, k, hi);
            a.nngb[k] = cnt;
            if (a.has_u) {
                const float P = a.gm1 * rho * ui;
                st_val(a.P_out, a.P_fmt, k, P);
                st_val(a.cs_out, a.cs_fmt, k, __fsqrt_rn(a.gamma * P / rho));
            }
        }
        if (clamped) {   // each clamped particle counted once per call
            atomicAdd(&c.st->hcap_clamps, 1ull);
            my_err |= SPH_ERR_HCAP;
        }
    }
    my_pairs = warp_sum_u64(my_pairs);
    my_tests = warp_sum_u64(my_tests);
    if (lane == 0) {
        if (my_pairs) atomicAdd(&c.st->pairs_density, my_pairs);
        if (my_tests) atomicAdd(&c.st->tests_density, my_tests);
    }
    if (my_err) set_error(c.st, my_err);
}

// ---------------------------------------------------------------------------
// force
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kMaxBlock) k_force(ForceArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ ItemShared s;
    const Common &c = a.c;
    float4 *sA = reinterpret_cast<float4 *>(smem);                 // x, y, z, h
    float4 *sB = sA + c.stage_cap;                                   // vx, vy, vz, m
    float4 *sC = sB + c.stage_cap;                                   // P/rho^2, rho, c, -
    uint16_t *lists = reinterpret_cast<uint16_t *>(sC + c.stage_cap);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint16_t *wl = lists + warp * kListCap;
    const unsigned lt = (1u << lane) - 1u;
    unsigned long long my_pairs = 0, my_tests = 0;
    unsigned my_err = 0;

    while (next_item(c, s)) {
        const int t = threadIdx.x;
        const bool ok = t < s.count;
        const int64_t k = (int64_t)s.first + t;
        float xi = 0.f, yi = 0.f, zi = 0.f, hi = 0.f, vxi = 0.f, vyi = 0.f, vzi = 0.f;
        float rhoi = 1.f, Pr2i = 0.f, ci = 0.f;
        if (ok) {
            xi = ld_val(c.x.p[0], c.x.fmt, k);
            yi = ld_val(c.x.p[1], c.x.fmt, k);
            zi = ld_val(c.x.p[2], c.x.fmt, k);
            hi = ld_val(c.h.p[0], c.h.fmt, k);
            vxi = ld_val(a.v.p[0], a.v.fmt, k);
            vyi = ld_val(a.v.p[1], a.v.fmt, k);
            vzi = ld_val(a.v.p[2], a.v.fmt, k);
            rhoi = ld_val(a.rho.p[0], a.rho.fmt, k);
            const float Pi = ld_val(a.P.p[0], a.P.fmt, k);
            Pr2i = Pi / (rhoi * rhoi);
            ci = ld_val(a.cs.p[0], a.cs.fmt, k);
        }
        const bool warp_live = __any_sync(FULL, ok);
        const Box bx = warp_box(ok, xi, yi, zi);
        const float hw = warp_max(ok ? hi : 0.0f);
        const int total = s.off[27];
        const int pself = s.off[13] + (int)(k - s.start[13]);
        float ax = 0.f, ay = 0.f, az = 0.f, du = 0.f;
        int cnt = 0;
        for (int c0 = 0; c0 < total; c0 += c.stage_cap) {
            const int len = min(c.stage_cap, total - c0);
            __syncthreads();
            for (int p = threadIdx.x; p < len; p += blockDim.x) {
                const int g = c0 + p;
                const int sl = staged_slot(s, g);
                const int64_t j = (int64_t)s.start[sl] + (g - s.off[sl]);
                const float rj = ld_val(a.rho.p[0], a.rho.fmt, j);
                const float Pj = ld_val(a.P.p[0], a.P.fmt, j);
                sA[p] = make_float4(ld_val(c.x.p[0], c.x.fmt, j) + s.shift[sl][0],
                                    ld_val(c.x.p[1], c.x.fmt, j) + s.shift[sl][1],
                                    ld_val(c.x.p[2], c.x.fmt, j) + s.shift[sl][2],
                                    ld_val(c.h.p[0], c.h.fmt, j));
                sB[p] = make_float4(ld_val(a.v.p[0], a.v.fmt, j), ld_val(a.v.p[1], a.v.fmt, j),
                                    ld_val(a.v.p[2], a.v.fmt, j), ld_val(c.m.p[0], c.m.fmt, j));
                sC[p] = make_float4(Pj / (rj * rj), rj, ld_val(a.cs.p[0], a.cs.fmt, j), 0.0f);
            }
            __syncthreads();
            if (!warp_live) continue;
            int p0 = 0;
            while (p0 < len) {
                int nl = 0;
                while (p0 < len && nl <= kListCap - 32) {
                    const int p = p0 + lane;
                    bool keep = false;
                    if (p < len) {
                        const float4 q = sA[p];
                        const float rr = hw + q.w;
                        keep = box_dist2(bx, q.x, q.y, q.z) < rr * rr;
                    }
                    const unsigned bal = __ballot_sync(FULL, keep);
                    if (keep) wl[nl + __popc(bal & lt)] = (uint16_t)p;
                    nl += __popc(bal);
                    p0 += 32;
                }
                __syncwarp();
                if (ok) {
                    my_tests += (unsigned long long)nl;
                    for (int e = 0; e < nl; ++e) {
                        const int p = wl[e];
                        const float4 q = sA[p];
                        const float dx = xi - q.x, dy = yi - q.y, dz = zi - q.z;
                        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                        const float hs = hi + q.w;
                        if (r2 < hs * hs && c0 + p != pself) {
                            ++cnt;
                            if (r2 > 0.0f) {
                                const float4 qb = sB[p];
                                const float4 qc = sC[p];
                                const float rinv = rsqrtf(r2);
                                const float r = r2 * rinv;
                                const float hb = 0.5f * hs;
                                const float hbinv = 2.0f / hs;
                                const float qq = r * hbinv;
                                float dw;
                                if (qq < 1.0f) dw = qq * fmaf(2.25f, qq, -3.0f);
                                else { const float tt = 2.0f - qq; dw = -0.75f * tt * tt; }
                                const float hb2 = hbinv * hbinv;
                                const float gw = kSigma * hb2 * hb2 * dw * rinv;   // grad_i W = d * gw
                                const float vx = vxi - qb.x, vy = vyi - qb.y, vz = vzi - qb.z;
                                const float vdotr = fmaf(vx, dx, fmaf(vy, dy, vz * dz));
                                float visc = 0.0f;
                                if (vdotr < 0.0f) {
                                    const float mu = hb * vdotr / fmaf(a.eps * hb, hb, r2);
                                    const float cbar = 0.5f * (ci + qc.z);
                                    const float rbar = 0.5f * (rhoi + qc.y);
                                    visc = fmaf(-a.alpha * cbar, mu, a.beta * mu * mu) / rbar;
                                }
                                const float fac = qb.w * (Pr2i + qc.x + visc) * gw;
                                ax = fmaf(-fac, dx, ax);
                                ay = fmaf(-fac, dy, ay);
                                az = fmaf(-fac, dz, az);
                                du = fmaf(qb.w * fmaf(0.5f, visc, Pr2i), vdotr * gw, du);
                            }
                        }
                    }
                }
                __syncwarp();
            }
        }
        if (ok) {
            if (!isfinite(ax) || !isfinite(ay) || !isfinite(az) || !isfinite(du)) my_err |= SPH_ERR_NONFINITE;
            a.a[0][k] = ax;
            a.a[1][k] = ay;
            a.a[2][k] = az;
            a.dudt[k] = du;
            a.nngb[k] = cnt;
            my_pairs += (unsigned long long)cnt;
        }
    }
    my_pairs = warp_sum_u64(my_pairs);
    my_tests = warp_sum_u64(my_tests);
    if (lane == 0) {
        if (my_pairs) atomicAdd(&c.st->pairs_force, my_pairs);
        if (my_tests) atomicAdd(&c.st->tests_force, my_tests);
    }
    if (my_err) set_error(c.st, my_err);
}

Common make_common(sph_ctx *c, int stage_cap)
{
    Common m;
    m.n = c->n;
    for (int k = 0; k < 3; ++k) {
        m.nc[k] = c->nc[k];
        m.edge[k] = (float)c->edge[k];
    }
    m.cell_start = c->cell_start;
    m.icell = c->item_cell;
    m.ifirst = c->item_first;
    m.icount = c->item_count;
    m.st = c->dstats;
    auto ref = [&](int f) {
        FieldRef r;
        for (int k = 0; k < 3; ++k) r.p[k] = c->soa[f][k];
        r.fmt = c->prec[f];
        return r;
    };
    m.x = ref(SPH_F_X);
    m.m = ref(SPH_F_M);
    m.h = ref(SPH_F_H);
    m.stage_cap = stage_cap;
    return m;
}

template <typename K, typename A>
cudaError_t launch_persistent(sph_ctx *c, K kernel, const A &args, size_t smem)
{
    cudaError_t e;
    const int block = c->tuning.block_threads;
    if ((e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return e;
    int per_sm = c->tuning.ctas_per_sm;
    if (per_sm <= 0) {
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem)) != cudaSuccess)
            return e;
        if (per_sm < 1) per_sm = 1;
    }
    if ((e = cudaMemsetAsync(&c->dstats->queue, 0, sizeof(unsigned), c->stream)) != cudaSuccess) return e;
    kernel<<<(unsigned)(c->sm_count * per_sm), block, smem, c->stream>>>(args);
    c->launches += 1;
    return cudaGetLastError();
}

}  // namespace

cudaError_t run_density(sph_ctx *c, int newton_steps)
{
    if (c->n == 0) return cudaSuccess;
    cudaError_t e;
    if (c->items_block != c->tuning.block_threads && (e = run_items(c)) != cudaSuccess) return e;
    DensityArgs a;
    a.c = make_common(c, c->tuning.stage_density);
    a.has_u = (c->valid & SPH_BIT(SPH_F_U)) != 0;
    for (int k = 0; k < 3; ++k) a.u.p[k] = c->soa[SPH_F_U][0];
    a.u.fmt = c->prec[SPH_F_U];
    a.npass = newton_steps + 1;
    const double eta = c->params.eta;
    a.eta3 = (float)(eta * eta * eta);
    a.h_cap = (float)c->params.h_max;
    a.gamma = (float)c->params.gamma;
    a.gm1 = (float)(c->params.gamma - 1.0);
    a.plain_sum = (c->params.flags & SPH_FLAG_PLAIN_SUM) != 0;
    a.rho_out = c->soa[SPH_F_RHO][0];
    a.rho_fmt = c->prec[SPH_F_RHO];
    const bool h_packed = fmt_packed(c->prec[SPH_F_H]);
    a.write_h = newton_steps > 0;
    a.h_out = h_packed ? (void *)c->stage : c->soa[SPH_F_H][0];
    a.h_fmt = h_packed ? SPH_P_FP32 : c->prec[SPH_F_H];
    a.P_out = c->soa[SPH_F_P][0];
    a.P_fmt = c->prec[SPH_F_P];
    a.cs_out = c->soa[SPH_F_CS][0];
    a.cs_fmt = c->prec[SPH_F_CS];
    a.nngb = c->nngb;
    const size_t smem = (size_t)a.c.stage_cap * sizeof(float4) +
                        (size_t)(c->tuning.block_threads / 32) * kListCap * sizeof(uint16_t);
    if ((e = launch_persistent(c, k_density, a, smem)) != cudaSuccess) return e;
    if (a.write_h && h_packed) return run_pack(c, c->stage, SPH_F_H);
    return cudaSuccess;
}

cudaError_t run_force(sph_ctx *c)
{
    if (c->n == 0) return cudaSuccess;
    cudaError_t e;
    if (c->items_block != c->tuning.block_threads && (e = run_items(c)) != cudaSuccess) return e;
    ForceArgs a;
    a.c = make_common(c, c->tuning.stage_force);
    auto ref = [&](int f) {
        FieldRef r;
        for (int k = 0; k < 3; ++k) r.p[k] = c->soa[f][k];
        r.fmt = c->prec[f];
        return r;
    };
    a.v = ref(SPH_F_V);
    a.rho = ref(SPH_F_RHO);
    a.P = ref(SPH_F_P);
    a.cs = ref(SPH_F_CS);
    a.alpha = (float)c->params.alpha_av;
    a.beta = (float)c->params.beta_av;
    a.eps = (float)c->params.eps_av;
    for (int k = 0; k < 3; ++k) a.a[k] = (float *)c->soa[SPH_F_A][k];
    a.dudt = (float *)c->soa[SPH_F_DUDT][0];
    a.nngb = c->nngb_force;
    const size_t smem = (size_t)a.c.stage_cap * 3 * sizeof(float4) +
                        (size_t)(c->tuning.block_threads / 32) * kListCap * sizeof(uint16_t);
    return launch_persistent(c, k_force, a, smem);
}

}  // namespace sph
