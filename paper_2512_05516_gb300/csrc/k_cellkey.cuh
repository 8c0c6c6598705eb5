// Cell key of a position on the uniform grid of sub-cells (S1): the
// binning computes it from the AoS records, and the drift computes it for the
// positions it writes, so that the next binning can skip reading them.  Both
// use these functions, so the two keys are the same bit for bit.
#pragma once

#include "sph_internal.cuh"

namespace sph {

// The grid: s sub-cells per cell edge, nc cells per axis, inv = s nc / L per
// axis (FP64) and the same as an FP32 pair, inv = invh + invl to a relative
// 2^-48.
struct CellGrid {
    double inv[3];
    float invh[3], invl[3];
    int32_t nc[3];
    int32_t sub;
};

inline CellGrid cell_grid(const int32_t nc[3], int32_t sub, const double box[3])
{
    CellGrid g;
    for (int k = 0; k < 3; ++k) {
        g.inv[k] = (double)(nc[k] * sub) / box[k];
        g.invh[k] = (float)g.inv[k];
        g.invl[k] = (float)(g.inv[k] - (double)g.invh[k]);
        g.nc[k] = nc[k];
    }
    g.sub = sub;
    return g;
}

// floor(x * inv) clamped to [0, nc-1]: one FP64 multiply (the product must
// round exactly as the definition says) and one round-down conversion, which
// maps NaN to INT_MIN and overflows to INT_MAX, so the integer clamp gives
// 0 for NaN and negatives and nc-1 above the grid.
__device__ __forceinline__ int32_t cell_coord(double x, double inv, int32_t nc)
{
    const int f = __double2int_rd(__dmul_rn(x, inv));
    return min(max(f, 0), nc - 1);
}

// cell_coord's result computed on the FP32 pipe for almost every particle
// (the FP64 pipe of this GPU runs at a small fraction of the FP32 rate).  x is
// split from its bits into FP32 parts, x = hi + lo up to a relative 2^-47
// (hi: the leading 24 significant bits, lo: the other 29 rounded to 24), and
// the product x * inv is formed as the unevaluated FP32 pair p + t, where
// p + fma(hi, ih, -p) = hi * ih exactly; the pair is within 2^-44 of the
// exact product, relatively, so within 2^-31 absolutely below 8192.  The
// floor of the pair then equals the floor of the rounded FP64 product unless
// the pair's fractional part lies within 2^-20 of 0 or 1, and those
// particles (on or next to a face), like x outside [2^-74, 2^100), negative
// or not finite, take the FP64 product.
__device__ __forceinline__ int32_t cell_coord_fast(double x, float ih, float il, double inv, int32_t nc)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    if (b == 0ull) return 0;                                // +0
    const int e = (int)(b >> 52);                          // biased exponent (sign bit set: >= 2048)
    bool exact = e < 949 || e >= 1123;
    int32_t f = 0;
    if (!exact) {
        const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
        const float hi = __int_as_float(((e - 896) << 23) | (int)(m >> 29));
        const float lo = __uint2float_rn((unsigned)(m & 0x1FFFFFFFu)) * __int_as_float((e - 948) << 23);
        const float p = hi * ih;
        const float t = fmaf(hi, ih, -p) + fmaf(hi, il, lo * ih);
        float fl = floorf(p);
        float d = (p - fl) + t;
        if (d < 0.0f) {
            fl -= 1.0f;
            d += 1.0f;
        } else if (d >= 1.0f) {
            fl += 1.0f;
            d -= 1.0f;
        }
        exact = d < 0x1p-20f || d > 1.0f - 0x1p-20f;
        f = min(max(__float2int_rz(fl), 0), nc - 1);
    }
    if (exact) f = cell_coord(x, inv, nc);
    return f;
}

// The key of position (x0, x1, x2): fine coordinates f_d on the grid of
// sub-cells, cell f / s, sub-cell f % s, key cell s^3 + (s_x + s (s_y + s s_z)).
// s is 1 or 2, so the divisions are shifts.
static_assert(kMaxSub <= 2, "cell_key takes s = 1 or 2");
__device__ __forceinline__ int32_t cell_key(const CellGrid &g, double x0, double x1, double x2)
{
    const int32_t S = g.sub, lg = S - 1;
    const int32_t fx = cell_coord_fast(x0, g.invh[0], g.invl[0], g.inv[0], g.nc[0] * S);
    const int32_t fy = cell_coord_fast(x1, g.invh[1], g.invl[1], g.inv[1], g.nc[1] * S);
    const int32_t fz = cell_coord_fast(x2, g.invh[2], g.invl[2], g.inv[2], g.nc[2] * S);
    const int32_t cell = (fx >> lg) + g.nc[0] * ((fy >> lg) + g.nc[1] * (fz >> lg));
    return (cell << (3 * lg)) + ((fx & lg) + ((fy & lg) << lg) + ((fz & lg) << (2 * lg)));
}

}  // namespace sph
