// S3-S5: the quadratic SPH kernels (the paper's Density and Force, Section 6),
// as persistent CUDA-core kernels over a work queue of warp-sized items.
//
// Work item = (cell, first slot, count <= 32): a tile of one cell, one lane
// per i-particle.  Warps are independent: each pops its own item, stages into
// its own shared-memory region only those particles of the 27 neighbour cells
// (periodic) that can reach the bounding box of its lanes, converted to FP32
// and shifted into the cell's frame (positions are cell-relative, so the
// shift is the neighbour's cell offset times the cell edge), then runs the
// pair loop.  No block-wide barrier is ever taken.  When a neighbourhood does
// not fit the stage, it is streamed through it in chunks.
//
// Density (Eq. 6, gather form): rho_i = sum_j m_j W(r_ij, h_i), M4 cubic
// spline W = sigma/h^3 w(r/h), support 2h, compensated FP32 sum (TwoSum);
// `newton_steps` Newton steps on f(h) = rho(h) - m_i (eta/h)^3 clamped to
// [h/2, 2h] and h_max, then a final sum; EOS P = (gamma-1) rho u,
// c = sqrt(gamma P / rho).  Pass 0 also builds, per lane, the list of staged
// candidates within 2 h (1 + skin); later passes walk only that list and
// rebuild it when h outgrows the skin.
//
// Force (Eq. 7 + Monaghan viscosity, Eq. 5 for du/dt), pairs r < h_i + h_j:
//   a_i    -= m_j (P_i/rho_i^2 + P_j/rho_j^2 + Pi_ij) gradW(r_ij, hbar)
//   du_i/dt += m_j (P_i/rho_i^2 + Pi_ij/2) v_ij . gradW
//
// Summation order: every lane accumulates its pairs in staged order (cell of
// the stencil, then slot), whatever the chunking, list or launch shape, so
// results do not depend on the tuning.
#include "sph_internal.cuh"

namespace sph {
cudaError_t run_pack(sph_ctx *c, const float *src, int f);

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kLaneCap = 96;        // per-lane neighbour list entries (density)
constexpr float kSkin = 0.12f;      // list / stage radius = 2 h (1 + skin)

struct Common {
    int64_t n;
    int32_t nc[3];
    float edge[3];
    const int32_t *cell_start;
    const int32_t *icell, *ifirst, *icount;
    DevStats *st;
    FieldRef x, m, h;
    int cap;                         // staged candidates per warp
};

struct DensityArgs {
    Common c;
    FieldRef u;
    bool has_u;
    int npass;                       // newton_steps + 1
    float eta3, h_cap, gm1, gamma;
    bool plain_sum;
    void *rho_out; int rho_fmt;
    void *h_out; int h_fmt;          // h_out may be the FP32 stage when H is packed
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

// the 27 neighbour cells of an item, one per lane (lanes 27..31 hold empty cells)
struct Stencil {
    int start, count;
    float sx, sy, sz;
};

__device__ __forceinline__ Stencil stencil_lane(const Common &c, int cell, int lane)
{
    Stencil s{0, 0, 0.f, 0.f, 0.f};
    if (lane < 27) {
        const int kx = cell % c.nc[0];
        const int ky = (cell / c.nc[0]) % c.nc[1];
        const int kz = cell / (c.nc[0] * c.nc[1]);
        const int dx = lane % 3 - 1, dy = (lane / 3) % 3 - 1, dz = lane / 9 - 1;
        const int nx = (kx + dx + c.nc[0]) % c.nc[0];
        const int ny = (ky + dy + c.nc[1]) % c.nc[1];
        const int nz = (kz + dz + c.nc[2]) % c.nc[2];
        const int nb = nx + c.nc[0] * (ny + c.nc[1] * nz);
        s.start = c.cell_start[nb];
        s.count = c.cell_start[nb + 1] - s.start;
        s.sx = (float)dx * c.edge[0];
        s.sy = (float)dy * c.edge[1];
        s.sz = (float)dz * c.edge[2];
    }
    return s;
}

__device__ __forceinline__ int pop_item(DevStats *st, int lane)
{
    int it = 0;
    if (lane == 0) it = (int)atomicAdd(&st->queue, 1u);
    return __shfl_sync(FULL, it, 0);
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

// M4 spline w(q) and w'(q), branch-free
__device__ __forceinline__ void spline(float q, float &w, float &dw)
{
    const float t = 2.0f - q;
    const float t2 = t * t;
    const float w_in = fmaf(q * q, fmaf(0.75f, q, -1.5f), 1.0f);
    const float dw_in = q * fmaf(2.25f, q, -3.0f);
    const bool inner = q < 1.0f;
    w = inner ? w_in : 0.25f * t2 * t;
    dw = inner ? dw_in : -0.75f * t2;
}

// compensated accumulation: s + c carries the running sum (Knuth's TwoSum)
__device__ __forceinline__ void two_sum_add(float &s, float &c, float x)
{
    const float t = __fadd_rn(s, x);
    const float bp = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(x, bp));
    c = __fadd_rn(c, err);
    s = t;
}

// ---------------------------------------------------------------------------
// Density
// ---------------------------------------------------------------------------

// density pass accumulators of one lane
struct DAcc {
    float s, c, d;   // compensated sum of m w, and sum of m (3w + q w')
    int n;           // pairs with r < 2h (self included)
};

__device__ __forceinline__ void dens_pair(DAcc &a, float xi, float yi, float zi, float h2x4,
                                          float hinv, bool plain, const float4 q)
{
    const float dx = xi - q.x, dy = yi - q.y, dz = zi - q.z;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const bool in = r2 < h2x4;
    const float r = r2 > 0.0f ? r2 * rsqrtf(r2) : 0.0f;
    const float qq = r * hinv;
    float w, dw;
    spline(qq, w, dw);
    const float mw = in ? q.w * w : 0.0f;
    if (plain) a.s += mw;
    else two_sum_add(a.s, a.c, mw);
    a.d = fmaf(in ? q.w : 0.0f, fmaf(qq, dw, 3.0f * w), a.d);
    a.n += in ? 1 : 0;
}

// Stage the candidates of the 27 cells within distance sqrt(R2) of the warp
// box, in stencil order, from stream position `skip` on (chunked streaming).
// Writes at most `cap` entries; returns how many candidates were found from
// `skip` on (may exceed cap).
__device__ int stage_density(const Common &c, const Stencil &st, const Box &box, float R2,
                             float4 *sj, int cap, int skip, int lane)
{
    const unsigned lt = (1u << lane) - 1u;
    int found = 0;
    for (int t = 0; t < 27; ++t) {
        const int start = __shfl_sync(FULL, st.start, t);
        const int cnt = __shfl_sync(FULL, st.count, t);
        const float sx = __shfl_sync(FULL, st.sx, t);
        const float sy = __shfl_sync(FULL, st.sy, t);
        const float sz = __shfl_sync(FULL, st.sz, t);
        for (int p0 = 0; p0 < cnt; p0 += 32) {
            const int p = p0 + lane;
            bool keep = false;
            float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
            int64_t j = 0;
            if (p < cnt) {
                j = (int64_t)start + p;
                q.x = ld_val(c.x.p[0], c.x.fmt, j) + sx;
                q.y = ld_val(c.x.p[1], c.x.fmt, j) + sy;
                q.z = ld_val(c.x.p[2], c.x.fmt, j) + sz;
                keep = box_dist2(box, q.x, q.y, q.z) < R2;
            }
            const unsigned b = __ballot_sync(FULL, keep);
            if (keep) {
                const int pos = found + __popc(b & lt) - skip;
                if (pos >= 0 && pos < cap) {
                    q.w = ld_val(c.m.p[0], c.m.fmt, j);
                    sj[pos] = q;
                }
            }
            found += __popc(b);
        }
    }
    __syncwarp();
    return found - skip;
}

__global__ void __launch_bounds__(kMaxBlock, 1) k_density(DensityArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const Common &c = a.c;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const size_t per_warp = (size_t)c.cap * sizeof(float4) + (size_t)32 * kLaneCap * sizeof(uint16_t);
    float4 *sj = reinterpret_cast<float4 *>(smem + warp * per_warp);
    uint16_t *lst = reinterpret_cast<uint16_t *>(sj + c.cap);

    unsigned long long my_pairs = 0, my_tests = 0;
    unsigned my_err = 0;
    const int nitems = c.st->nitems;

    for (int it = pop_item(c.st, lane); it < nitems; it = pop_item(c.st, lane)) {
        const int cell = c.icell[it];
        const int first = c.ifirst[it];
        const int count = c.icount[it];
        const bool ok = lane < count;
        const int64_t k = (int64_t)first + lane;
        bool clamped = false;
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
        const Stencil st = stencil_lane(c, cell, lane);
        const Box box = warp_box(ok, xi, yi, zi);

        // stage everything within 2 h_stage of the box, h_stage = max h (1 + skin)
        float h_stage = fminf(warp_max(ok ? hi : 0.0f) * (1.0f + kSkin), a.h_cap);
        int T = stage_density(c, st, box, 4.0f * h_stage * h_stage, sj, c.cap, 0, lane);
        bool fits = T <= c.cap;
        bool lists_ok = false;     // this lane's list holds every staged candidate within 2 h_list
        float h_list = 0.0f;
        int nlist = 0;

        float rho = 0.f, drdh = 0.f;
        int cnt = 0;
        for (int pass = 0; pass < a.npass; ++pass) {
            const float h2x4 = 4.0f * hi * hi;
            const float hinv = 1.0f / hi;
            DAcc acc{0.f, 0.f, 0.f, 0};
            if (fits && __any_sync(FULL, ok && hi > h_stage)) {
                // h outgrew the stage: re-stage with the current h
                h_stage = fminf(warp_max(ok ? hi : 0.0f) * (1.0f + kSkin), a.h_cap);
                T = stage_density(c, st, box, 4.0f * h_stage * h_stage, sj, c.cap, 0, lane);
                fits = T <= c.cap;
                h_list = 0.0f;
            }
            if (fits) {
                // rebuild when some lane's h outgrew its list radius (always on pass 0)
                const bool rebuild = __any_sync(FULL, ok && hi > h_list);
                if (rebuild) {
                    // walk every staged candidate and rebuild this lane's list
                    h_list = fminf(hi * (1.0f + kSkin), h_stage);
                    const float R2l = 4.0f * h_list * h_list;
                    nlist = 0;
                    if (ok) {
                        my_tests += (unsigned long long)T;
                        for (int e = 0; e < T; ++e) {
                            const float4 q = sj[e];
                            const float dx = xi - q.x, dy = yi - q.y, dz = zi - q.z;
                            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                            if (r2 < R2l) {
                                if (nlist < kLaneCap) lst[nlist * 32 + lane] = (uint16_t)e;
                                ++nlist;
                                dens_pair(acc, xi, yi, zi, h2x4, hinv, a.plain_sum, q);
                            }
                        }
                    }
                    lists_ok = nlist <= kLaneCap;
                    __syncwarp();
                } else if (ok) {
                    if (lists_ok) {
                        my_tests += (unsigned long long)nlist;
#pragma unroll 4
                        for (int e = 0; e < nlist; ++e)
                            dens_pair(acc, xi, yi, zi, h2x4, hinv, a.plain_sum, sj[lst[e * 32 + lane]]);
                    } else {
                        // this lane's list overflowed: walk the whole stage
                        my_tests += (unsigned long long)T;
                        for (int e = 0; e < T; ++e) dens_pair(acc, xi, yi, zi, h2x4, hinv, a.plain_sum, sj[e]);
                    }
                }
            } else {
                // the neighbourhood does not fit: stream it through the stage
                const float hw = warp_max(ok ? hi : 0.0f);
                const float R2 = 4.0f * hw * hw;
                for (int skip = 0;; skip += c.cap) {
                    const int got = stage_density(c, st, box, R2, sj, c.cap, skip, lane);
                    const int len = min(got, c.cap);
                    if (ok) {
                        my_tests += (unsigned long long)len;
                        for (int e = 0; e < len; ++e) dens_pair(acc, xi, yi, zi, h2x4, hinv, a.plain_sum, sj[e]);
                    }
                    __syncwarp();
                    if (got <= c.cap) break;
                }
            }
            if (ok) {
                const float h3inv = hinv * hinv * hinv;
                rho = kSigma * h3inv * (acc.s + acc.c);
                drdh = -kSigma * h3inv * hinv * acc.d;
                cnt = acc.n - 1;           // the self term is in rho, not in the count
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
            if (clamped) {   // each clamped particle counted once per call
                atomicAdd(&c.st->hcap_clamps, 1ull);
                my_err |= SPH_ERR_HCAP;
            }
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
// Force
// ---------------------------------------------------------------------------

// Stage the force candidates (those within h_max(warp) + h_j of the warp box)
// from stream position `skip` on; returns how many were found (may exceed cap).
__device__ int stage_force(const ForceArgs &a, const Stencil &st, const Box &box, float hw,
                           float4 *sA, float4 *sB, float4 *sC, int cap, int skip, int lane)
{
    const Common &c = a.c;
    const unsigned lt = (1u << lane) - 1u;
    int found = 0;
    for (int t = 0; t < 27; ++t) {
        const int start = __shfl_sync(FULL, st.start, t);
        const int cnt = __shfl_sync(FULL, st.count, t);
        const float sx = __shfl_sync(FULL, st.sx, t);
        const float sy = __shfl_sync(FULL, st.sy, t);
        const float sz = __shfl_sync(FULL, st.sz, t);
        for (int p0 = 0; p0 < cnt; p0 += 32) {
            const int p = p0 + lane;
            bool keep = false;
            float4 qa = make_float4(0.f, 0.f, 0.f, 0.f);
            int64_t j = 0;
            if (p < cnt) {
                j = (int64_t)start + p;
                qa.x = ld_val(c.x.p[0], c.x.fmt, j) + sx;
                qa.y = ld_val(c.x.p[1], c.x.fmt, j) + sy;
                qa.z = ld_val(c.x.p[2], c.x.fmt, j) + sz;
                qa.w = ld_val(c.h.p[0], c.h.fmt, j);
                const float rr = hw + qa.w;
                keep = box_dist2(box, qa.x, qa.y, qa.z) < rr * rr;
            }
            const unsigned b = __ballot_sync(FULL, keep);
            if (keep) {
                const int pos = found + __popc(b & lt) - skip;
                if (pos >= 0 && pos < cap) {
                    const float rj = ld_val(a.rho.p[0], a.rho.fmt, j);
                    const float Pj = ld_val(a.P.p[0], a.P.fmt, j);
                    sA[pos] = qa;
                    sB[pos] = make_float4(ld_val(a.v.p[0], a.v.fmt, j), ld_val(a.v.p[1], a.v.fmt, j),
                                          ld_val(a.v.p[2], a.v.fmt, j), ld_val(c.m.p[0], c.m.fmt, j));
                    sC[pos] = make_float4(Pj / (rj * rj), rj, ld_val(a.cs.p[0], a.cs.fmt, j),
                                          __int_as_float((int)j));
                }
            }
            found += __popc(b);
        }
    }
    __syncwarp();
    return found - skip;
}

__global__ void __launch_bounds__(kMaxBlock, 1) k_force(ForceArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const Common &c = a.c;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float4 *sA = reinterpret_cast<float4 *>(smem) + (size_t)warp * 3 * c.cap;   // x, y, z, h
    float4 *sB = sA + c.cap;                                                  // vx, vy, vz, m
    float4 *sC = sB + c.cap;                                                  // P/rho^2, rho, c, slot
    unsigned long long my_pairs = 0, my_tests = 0;
    unsigned my_err = 0;
    const int nitems = c.st->nitems;

    for (int it = pop_item(c.st, lane); it < nitems; it = pop_item(c.st, lane)) {
        const int cell = c.icell[it];
        const int first = c.ifirst[it];
        const int count = c.icount[it];
        const bool ok = lane < count;
        const int64_t k = (int64_t)first + lane;
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
        const Stencil st = stencil_lane(c, cell, lane);
        const Box box = warp_box(ok, xi, yi, zi);
        const float hw = warp_max(ok ? hi : 0.0f);
        const int kself = (int)k;
        float ax = 0.f, ay = 0.f, az = 0.f, du = 0.f;
        int cnt = 0;
        for (int skip = 0;; skip += c.cap) {
            const int got = stage_force(a, st, box, hw, sA, sB, sC, c.cap, skip, lane);
            const int len = min(got, c.cap);
            if (ok) {
                my_tests += (unsigned long long)len;
                for (int e = 0; e < len; ++e) {
                    const float4 q = sA[e];
                    const float dx = xi - q.x, dy = yi - q.y, dz = zi - q.z;
                    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    const float hs = hi + q.w;
                    if (r2 < hs * hs) {
                        const float4 qc = sC[e];
                        if (__float_as_int(qc.w) != kself) {
                            ++cnt;
                            if (r2 > 0.0f) {
                                const float4 qb = sB[e];
                                const float rinv = rsqrtf(r2);
                                const float r = r2 * rinv;
                                const float hb = 0.5f * hs;
                                const float hbinv = 2.0f / hs;
                                const float qq = r * hbinv;
                                float w, dw;
                                spline(qq, w, dw);
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
            }
            __syncwarp();
            if (got <= c.cap) break;
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

Common make_common(sph_ctx *c, int cap)
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
    m.cap = cap;
    return m;
}

template <typename K, typename A>
cudaError_t launch_persistent(sph_ctx *c, K kernel, const A &args, size_t smem, LaunchCache &lc)
{
    cudaError_t e;
    const int block = c->tuning.block_threads;
    if (lc.smem != smem || lc.block != block || lc.per_sm_req != c->tuning.ctas_per_sm) {
        if ((e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
            return e;
        int per_sm = c->tuning.ctas_per_sm;
        if (per_sm <= 0) {
            if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem)) != cudaSuccess)
                return e;
            if (per_sm < 1) per_sm = 1;
        }
        lc.smem = smem;
        lc.block = block;
        lc.per_sm_req = c->tuning.ctas_per_sm;
        lc.grid = c->sm_count * per_sm;
    }
    if ((e = cudaMemsetAsync(&c->dstats->queue, 0, sizeof(unsigned), c->stream)) != cudaSuccess) return e;
    kernel<<<(unsigned)lc.grid, block, smem, c->stream>>>(args);
    c->launches += 1;
    return cudaGetLastError();
}

}  // namespace

size_t density_smem_bytes(int block_threads, int cap)
{
    return (size_t)(block_threads / 32) * ((size_t)cap * sizeof(float4) + (size_t)32 * kLaneCap * sizeof(uint16_t));
}

size_t force_smem_bytes(int block_threads, int cap)
{
    return (size_t)(block_threads / 32) * (size_t)cap * 3 * sizeof(float4);
}

cudaError_t run_density(sph_ctx *c, int newton_steps)
{
    if (c->n == 0) return cudaSuccess;
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
    cudaError_t e = launch_persistent(c, k_density, a, density_smem_bytes(c->tuning.block_threads, a.c.cap),
                                      c->lc_density);
    if (e != cudaSuccess) return e;
    if (a.write_h && h_packed) return run_pack(c, c->stage, SPH_F_H);
    return cudaSuccess;
}

cudaError_t run_force(sph_ctx *c)
{
    if (c->n == 0) return cudaSuccess;
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
    return launch_persistent(c, k_force, a, force_smem_bytes(c->tuning.block_threads, a.c.cap), c->lc_force);
}

}  // namespace sph
