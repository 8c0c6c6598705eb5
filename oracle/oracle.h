/*
 * FP64 CPU oracle for the SPH hot path -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
 * load this code.  The CUDA library never calls it and shares no code with it.
 *
 * Everything is plain FP64 C, written from the paper's equations:
 *   Eq. 6  density sum          rho_i = sum_j m_j W(r_ij, h)
 *   Eq. 7  momentum equation    dv_i/dt = -sum_j m_j (P_i/rho_i^2 + P_j/rho_j^2) grad W + f_visc
 *   Section 2 (governing equations): h adapted to keep the neighbour number constant
 *   Table 2  reduced-precision storage formats (IEEE single/half, truncated single)
 * The paper names the kernel family but gives no formula, EOS, viscosity or
 * integrator; the readings taken are listed at each function.
 */
#ifndef SPH_ORACLE_H
#define SPH_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* per-particle flag bits written by orc_density / orc_force */
#define ORC_FLAG_HCAP      1  /* h was clamped to the upper bound h_cap            */
#define ORC_FLAG_NEWTON    2  /* Newton derivative not positive: step skipped       */
#define ORC_FLAG_NONFINITE 4  /* a non-finite value was met                         */

/* storage formats of the quantisers (Table 2 plus bfloat16) */
#define ORC_FMT_FP32   0
#define ORC_FMT_BF16   1
#define ORC_FMT_FP16   2
#define ORC_FMT_M16    3   /* single with 16 mantissa bits: 25-bit code */
#define ORC_FMT_M10    4   /* single with 10 mantissa bits: 19-bit code */
#define ORC_FMT_TRUNC(n) (100 + (n))   /* single with n mantissa bits (1..22): (9+n)-bit code */

/* ---- smoothing kernel: M4 cubic spline, support 2h, sigma = 1/pi (3D) ---- */
double orc_w(double q);
double orc_dw(double q);
double orc_W(double r, double h);
double orc_dWdr(double r, double h);
double orc_dWdh(double r, double h);

/* ---- cell binning: FP64 cell index, stable counting sort ---- */
int orc_bin_sub(int64_t n, const double *x, const double *box, const int32_t *nc, int32_t sub,
                int32_t *cell_of, int64_t *perm, int64_t *cell_start);
int orc_bin(int64_t n, const double *x, const double *box, const int32_t *nc,
            int32_t *cell_of, int64_t *perm, int64_t *cell_start);

/* ---- level hierarchy for per-particle h: Morton keys of the finest cells,
 *      levels from h, stable order by key ---- */
int orc_levels(int64_t n, const double *x, const double *h, const double *box, int32_t level_min,
               int32_t level_max, double margin, int32_t *key, int8_t *level, int64_t *perm);

/* ---- density with Newton smoothing-length iteration (Eq. 6) ---- */
void orc_density(int64_t n, const double *x, const double *m, const double *h_in,
                 const double *box, double eta, double h_cap, int newton_steps,
                 int brute, int64_t ntarget, const int64_t *targets,
                 double *rho, double *h_out, double *drho_dh, int32_t *nngb,
                 int32_t *flags, int64_t *pairs_all);

/* ---- ideal-gas equation of state ---- */
void orc_eos(int64_t n, const double *rho, const double *u, double gamma,
             double *P, double *c);

/* ---- symmetric hydro force with Monaghan artificial viscosity (Eq. 7) ---- */
void orc_force(int64_t n, const double *x, const double *v, const double *m,
               const double *h, const double *rho, const double *P, const double *c,
               const double *box, double alpha, double beta, double eps,
               int brute, int64_t ntarget, const int64_t *targets,
               double *a, double *dudt, int32_t *nngb);

/* ---- buffers of B co-located particles (Section 6 benchmark): every pair of
 *      a buffer; density (h fixed, self included) + EOS, and force ---- */
void orc_buffer_density(int64_t n, int32_t B, const double *x, const double *m,
                        const double *h, const double *u, const double *box, double gamma,
                        double *rho, double *P, double *c, int32_t *nngb);
void orc_buffer_force(int64_t n, int32_t B, const double *x, const double *v, const double *m,
                      const double *h, const double *rho, const double *P, const double *c,
                      const double *box, double alpha, double beta, double eps,
                      double *a, double *dudt, int32_t *nngb);

/* ---- kick/drift (symplectic Euler, periodic wrap) ---- */
void orc_kick_drift(int64_t n, double *x, double *v, const double *a, double *u,
                    const double *dudt, double dt_kick, double dt_drift,
                    const double *box);

/* ---- ball query helper: mark every particle within `radius` of a target ---- */
int64_t orc_ball_mark(int64_t n, const double *x, const double *box, double radius,
                      int64_t ntarget, const int64_t *targets, uint8_t *mark);

/* ---- quantisers (Table 2; round-to-nearest-even or truncation) ---- */
uint32_t orc_f32_bits(double d);
double   orc_f32_value(uint32_t bits);
uint16_t orc_f16_from_f32(uint32_t fbits);
uint32_t orc_f32_from_f16(uint16_t hbits);
uint16_t orc_bf16_from_f32(uint32_t fbits);
uint32_t orc_f32_from_bf16(uint16_t bbits);
uint32_t orc_trunc_code(uint32_t fbits, int mant_bits);
void orc_trunc64(int64_t n, const double *in, int mant, double *out);
void orc_trunc_half(int64_t n, const double *in, int mant, double *out);
uint32_t orc_f32_from_trunc(uint32_t code, int mant_bits);
int      orc_fmt_bits(int fmt);
void     orc_quantize(int64_t n, const double *in, int fmt, double *value, uint32_t *code);
void     orc_pack_bits(int64_t n, const uint32_t *codes, int bits, uint32_t *words);
void     orc_unpack_bits(int64_t n, const uint32_t *words, int bits, uint32_t *codes);

#ifdef __cplusplus
}
#endif
#endif
