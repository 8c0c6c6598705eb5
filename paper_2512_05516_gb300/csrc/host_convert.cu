// The conversion operators on the host: the paper's CPU placement (Section
// 6.3, Eq. 13-14: U o N o C on the host, then M moves the SoA to the device;
// the write-back moves the SoA back and scatters it there).  The device
// kernels (k_convert.cu) are the GPU placement; both produce the same codes.
//
// Host threads split the sorted slots into ranges of whole 32-slot blocks,
// so that every packed word belongs to one thread.  Each thread walks its
// blocks: it reads every record of a block once, in permutation order (the
// records of a block several blocks ahead are prefetched, since the gather
// is the cost), rounds each component the way the device does (IEEE
// round-to-nearest-even FP64 -> FP32 by the C++ cast, then the shared
// encoders of sph_internal.cuh) and writes the block into the SoA image in a
// caller-provided staging buffer; the image then moves with one copy per
// component array.  The permutation (and the cell keys or buffer origins
// the positions need) come from the device first.
#include <algorithm>
#include <cstring>
#include <thread>
#include <vector>

#include "sph_internal.cuh"

namespace sph {
namespace {

struct StageLayout {
    size_t perm, keys, origin, soa[SPH_NFIELDS][3], total;
};

// perm (4 B per slot), cell keys (4 B per slot), buffer origins (3 doubles
// per 32 slots), then every SoA array at its device size
StageLayout stage_layout(const sph_ctx *c)
{
    StageLayout s;
    std::memset(&s, 0, sizeof(s));
    const size_t n = (size_t)c->n;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) & ~(size_t)255;
        return o;
    };
    s.perm = take(4 * n);
    s.keys = take(4 * n);
    s.origin = take(sizeof(double) * 3 * (n / 32 + 1));
    for (int f = 0; f < SPH_NFIELDS; ++f)
        for (int k = 0; k < ncomp(f); ++k) s.soa[f][k] = take(4 * n + 64);
    s.total = off;
    return s;
}

// bytes of one SoA component array in format fmt
size_t soa_bytes(int64_t n, int fmt)
{
    if (fmt_packed(fmt)) return (size_t)((n * fmt_bits(fmt) + 31) / 32) * 4;
    return (size_t)n * (fmt == SPH_P_BF16 || fmt == SPH_P_FP16 ? 2 : 4);
}

float decode(const void *p, int fmt, int64_t k)
{
    switch (fmt) {
    case SPH_P_BF16: return dec_bf16(static_cast<const uint16_t *>(p)[k]);
    case SPH_P_FP16: return __half2float(static_cast<const __half *>(p)[k]);
    case SPH_P_FP32: return static_cast<const float *>(p)[k];
    default: {
        const int B = fmt_bits(fmt);
        const uint32_t *w = static_cast<const uint32_t *>(p);
        const int64_t bit = k * (int64_t)B;
        const int64_t wi = bit >> 5;
        const int sh = (int)(bit & 31);
        uint64_t two = w[wi];
        if (sh + B > 32) two |= (uint64_t)w[wi + 1] << 32;
        const uint32_t code = (uint32_t)(two >> sh) & ((1u << B) - 1u);
        return f32_from_bits(code << (32 - B));
    }
    }
}

// the 32-slot block starting at b0 (a multiple of 32; slots >= n get code 0)
// of one component, values vals[0..31] already scaled, into the array at p
void encode_block(void *p, int fmt, int64_t b0, int64_t n, const float *vals)
{
    const int cnt = (int)std::min<int64_t>(32, n - b0);
    if (!fmt_packed(fmt)) {
        for (int j = 0; j < cnt; ++j) {
            const int64_t k = b0 + j;
            switch (fmt) {
            case SPH_P_BF16: static_cast<uint16_t *>(p)[k] = enc_bf16(vals[j]); break;
            case SPH_P_FP16: static_cast<__half *>(p)[k] = __float2half_rn(vals[j]); break;
            default: static_cast<float *>(p)[k] = vals[j]; break;
            }
        }
        return;
    }
    // packed: value k at bits [kB, (k+1)B); 32 values fill B whole words
    const int B = fmt_bits(fmt);
    uint32_t words[32] = {};
    for (int j = 0; j < 32; ++j) {
        const uint32_t code = j < cnt ? enc_trunc(vals[j], B) : 0u;
        const int bit = j * B;
        words[bit >> 5] |= code << (bit & 31);
        if ((bit & 31) + B > 32) words[(bit >> 5) + 1] |= code >> (32 - (bit & 31));
    }
    uint32_t *w = static_cast<uint32_t *>(p) + (b0 / 32) * B;
    const int nw = cnt == 32 ? B : (cnt * B + 31) / 32;
    for (int i = 0; i < nw; ++i) w[i] = words[i];
}

template <typename F>
void parallel_blocks(int64_t n, int nthreads, F body)
{
    const int64_t nblk = (n + 31) / 32;
    const int T = (int)std::max<int64_t>(1, std::min<int64_t>(nthreads, nblk));
    if (T == 1) {
        body((int64_t)0, n);
        return;
    }
    // no exception may cross the C ABI: a thread that cannot be started
    // leaves its range to the calling thread
    std::vector<std::thread> pool;
    try {
        pool.reserve((size_t)T);
    } catch (...) {
    }
    for (int t = 0; t < T; ++t) {
        const int64_t k0 = std::min(n, (nblk * t / T) * 32);
        const int64_t k1 = std::min(n, (nblk * (t + 1) / T) * 32);
        bool started = false;
        try {
            pool.emplace_back([=] { body(k0, k1); });
            started = true;
        } catch (...) {
        }
        if (!started) body(k0, k1);
    }
    for (auto &th : pool) th.join();
}

int default_threads(int32_t nthreads)
{
    if (nthreads > 0) return nthreads;
    const unsigned hw = std::thread::hardware_concurrency();
    return hw ? (int)hw : 1;
}

double rec_value(const uint8_t *rec, const sph_aos_layout &L, int f, int comp)
{
    const uint8_t *p = rec + L.offset[f];
    if (L.type[f] == SPH_AOS_F64) {
        double d;
        std::memcpy(&d, p + 8 * comp, 8);
        return d;
    }
    float x;
    std::memcpy(&x, p + 4 * comp, 4);
    return (double)x;
}

}  // namespace

size_t host_stage_bytes(const sph_ctx *c) { return stage_layout(c).total; }

cudaError_t run_aos_to_soa_host(sph_ctx *c, const uint8_t *host_aos, uint32_t fields, uint8_t *stage,
                                int32_t nthreads)
{
    if (c->n == 0) return cudaSuccess;
    const StageLayout S = stage_layout(c);
    const int64_t n = c->n;
    const bool want_x = (fields & SPH_BIT(SPH_F_X)) != 0;
    cudaError_t e;
    // the slot order (and what the position offsets need) from the device
    if ((e = cudaMemcpyAsync(stage + S.perm, c->perm(), 4 * (size_t)n, cudaMemcpyDeviceToHost, c->stream)) !=
        cudaSuccess)
        return e;
    const int64_t nbuf = c->buffer ? (n + c->buffer - 1) / c->buffer : 0;
    if (want_x && c->buffer) {
        if ((e = cudaMemcpyAsync(stage + S.origin, c->buf_origin, sizeof(double) * 3 * (size_t)nbuf,
                                 cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess)
            return e;
    } else if (want_x) {
        if ((e = cudaMemcpyAsync(stage + S.keys, c->slot_cell(), 4 * (size_t)n, cudaMemcpyDeviceToHost, c->stream)) !=
            cudaSuccess)
            return e;
    }
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return e;
    const int32_t *perm = reinterpret_cast<const int32_t *>(stage + S.perm);
    const int32_t *keys = reinterpret_cast<const int32_t *>(stage + S.keys);
    const double *bufo = reinterpret_cast<const double *>(stage + S.origin);
    const sph_aos_layout L = c->layout;
    const int64_t rb = L.record_bytes;
    const int lgB = c->buffer ? 31 - __builtin_clz((unsigned)c->buffer) : 0;
    const int s3 = c->sub * c->sub * c->sub;
    double edge[3];
    for (int d = 0; d < 3; ++d) edge[d] = c->edge[d];
    const int nc0 = c->nc[0], nc1 = c->nc[1];
    const double box[3] = {c->params.box[0], c->params.box[1], c->params.box[2]};

    // the components to convert: field, component
    int cf[3 * SPH_NFIELDS], cc[3 * SPH_NFIELDS], nc_tot = 0;
    float cenc[3 * SPH_NFIELDS];
    for (int f = 0; f < SPH_NFIELDS; ++f)
        if (fields & SPH_BIT(f))
            for (int comp = 0; comp < ncomp(f); ++comp) {
                cf[nc_tot] = f;
                cenc[nc_tot] = c->enc(f);
                cc[nc_tot++] = comp;
            }
    constexpr int kAhead = 4;      // blocks prefetched ahead of the one converted

    parallel_blocks(n, default_threads(nthreads), [&](int64_t k0, int64_t k1) {
        float vals[3 * SPH_NFIELDS][32];
        for (int64_t b0 = k0; b0 < k1; b0 += 32) {
            const int64_t pf0 = b0 + 32 * kAhead, pf1 = std::min(k1, pf0 + 32);
            for (int64_t k = pf0; k < pf1; ++k) {
                const uint8_t *r = host_aos + (int64_t)perm[k] * rb;
                __builtin_prefetch(r);
                __builtin_prefetch(r + rb - 1);
            }
            const int cnt = (int)std::min<int64_t>(32, k1 - b0);
            for (int j = 0; j < cnt; ++j) {
                const int64_t k = b0 + j;
                const uint8_t *rec = host_aos + (int64_t)perm[k] * rb;
                for (int i = 0; i < nc_tot; ++i) {
                    const int f = cf[i], comp = cc[i];
                    const double x = rec_value(rec, L, f, comp);
                    float v;
                    if (f != SPH_F_X) {
                        v = (float)x;                                  // round to nearest, ties to even
                    } else if (c->buffer) {
                        const double o = bufo[comp * nbuf + (k >> lgB)];
                        const double Lb = box[comp];
                        double d = x - o;
                        if (d >= 0.5 * Lb) d = d - Lb;
                        else if (d < -0.5 * Lb) d = d + Lb;
                        v = (float)d;
                    } else {
                        // the cell's coordinate on this axis from its key, origin k * edge
                        const int cell = keys[k] / s3;
                        const int kc = c->levels ? (int)morton_compact((uint32_t)keys[k] >> comp)
                                       : comp == 0 ? cell % nc0
                                       : (comp == 1 ? (cell / nc0) % nc1 : cell / (nc0 * nc1));
                        const double o = (double)kc * edge[comp];
                        v = (float)(x - o);
                    }
                    vals[i][j] = v * cenc[i];
                }
            }
            for (int i = 0; i < nc_tot; ++i)
                encode_block(stage + S.soa[cf[i]][cc[i]], c->prec[cf[i]], b0, k1, vals[i]);
        }
    });
    // move the SoA image: one copy per component array
    for (int f = 0; f < SPH_NFIELDS; ++f) {
        if (!(fields & SPH_BIT(f))) continue;
        for (int comp = 0; comp < ncomp(f); ++comp)
            if ((e = cudaMemcpyAsync(c->soa[f][comp], stage + S.soa[f][comp], soa_bytes(n, c->prec[f]),
                                     cudaMemcpyHostToDevice, c->stream)) != cudaSuccess)
                return e;
    }
    return cudaSuccess;
}

cudaError_t run_soa_to_aos_host(sph_ctx *c, uint8_t *host_aos, uint32_t fields, uint8_t *stage, int32_t nthreads)
{
    if (c->n == 0) return cudaSuccess;
    const StageLayout S = stage_layout(c);
    const int64_t n = c->n;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(stage + S.perm, c->perm(), 4 * (size_t)n, cudaMemcpyDeviceToHost, c->stream)) !=
        cudaSuccess)
        return e;
    const int64_t nbuf = c->buffer ? (n + c->buffer - 1) / c->buffer : 0;
    if ((fields & SPH_BIT(SPH_F_X)) &&
        (e = cudaMemcpyAsync(stage + S.origin, c->buf_origin, sizeof(double) * 3 * (size_t)nbuf,
                             cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess)
        return e;
    for (int f = 0; f < SPH_NFIELDS; ++f) {
        if (!(fields & SPH_BIT(f))) continue;
        for (int comp = 0; comp < ncomp(f); ++comp)
            if ((e = cudaMemcpyAsync(stage + S.soa[f][comp], c->soa[f][comp], soa_bytes(n, c->prec[f]),
                                     cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess)
                return e;
    }
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return e;
    const int32_t *perm = reinterpret_cast<const int32_t *>(stage + S.perm);
    const double *bufo = reinterpret_cast<const double *>(stage + S.origin);
    const sph_aos_layout L = c->layout;
    const int64_t rb = L.record_bytes;
    const int lgB = c->buffer ? 31 - __builtin_clz((unsigned)c->buffer) : 0;
    const double box[3] = {c->params.box[0], c->params.box[1], c->params.box[2]};

    parallel_blocks(n, default_threads(nthreads), [&](int64_t k0, int64_t k1) {
        for (int64_t k = k0; k < k1; ++k) {
            if (k + 128 < k1) {
                uint8_t *r = host_aos + (int64_t)perm[k + 128] * rb;
                __builtin_prefetch(r, 1);
                __builtin_prefetch(r + rb - 1, 1);
            }
            uint8_t *rec = host_aos + (int64_t)perm[k] * rb;
            for (int f = 0; f < SPH_NFIELDS; ++f) {
                if (!(fields & SPH_BIT(f))) continue;
                const float dec = c->dec(f);
                for (int comp = 0; comp < ncomp(f); ++comp) {
                    const float v = decode(stage + S.soa[f][comp], c->prec[f], k) * dec;
                    uint8_t *p = rec + L.offset[f];
                    if (L.type[f] != SPH_AOS_F64) {
                        std::memcpy(p + 4 * comp, &v, 4);
                    } else if (f == SPH_F_X) {
                        // buffer mode: origin + offset, wrapped into [0, L)
                        const double Lb = box[comp];
                        double y = bufo[comp * nbuf + (k >> lgB)] + (double)v;
                        if (y < 0.0 || y >= Lb) {
                            y = y - Lb * std::floor(y / Lb);
                            if (y >= Lb) y = 0.0;
                        }
                        std::memcpy(p + 8 * comp, &y, 8);
                    } else {
                        const double d = (double)v;                  // exact widening
                        std::memcpy(p + 8 * comp, &d, 8);
                    }
                }
            }
        }
    });
    return cudaSuccess;
}

}  // namespace sph
