/*
 * libsph -- GB300 (sm_103a) SPH particle kernels over FP64 array-of-structs
 * particle data, with on-device AoS->SoA conversion and reduced-precision
 * storage (arXiv 2512.05516, "Compiler-supported reduced precision and
 * AoS-SoA transformations for heterogeneous hardware").
 *
 * The paper's operator algebra (Section 4) maps onto the calls below:
 *   N   narrowing to the fields a kernel reads     -> `fields` masks
 *   C   AoS -> SoA layout change                    -> sph_aos_to_soa (on the GPU) or
 *                                                      sph_aos_to_soa_host (on the CPU)
 *   U   unpack reduced precision / U^T pack         -> per-field `prec`
 *   f   the compute kernel                          -> sph_density, sph_force,
 *                                                      sph_kick_drift (cell
 *                                                      lists) or sph_buffer_*
 *                                                      (the paper's buffers)
 *   C^T N^T U^T  widen and scatter back to the AoS  -> sph_soa_to_aos (or fused
 *                                                      with the kick/drift:
 *                                                      sph_kick_drift_writeback)
 *   M   host <-> device move                        -> sph_aos_upload/download
 * The GPU-side variant of Eq. 12 (convert on the device, "in-place" in
 * Section 6.3) is what one time step of these calls performs.
 *
 * Conventions shared by every entry point
 *   - Pointers named d_* are CUDA device pointers; everything else is host.
 *   - The caller owns the AoS records and one workspace buffer; the library
 *     never allocates device memory.  The context itself is a small host
 *     allocation freed by sph_destroy.
 *   - Every call that launches work is asynchronous on the stream given to
 *     sph_create and makes no host synchronisation, except sph_get_stats and
 *     sph_aos_download, which synchronise that stream.
 *   - Argument errors are detected on the host before any launch and return a
 *     negative sph_status with no device work issued.  Conditions found on the
 *     device (non-finite values, positions outside the box, h clamped) are
 *     recorded in a sticky error word read by sph_get_stats.
 *   - A context is not thread-safe; distinct contexts are independent.
 */
#ifndef SPH_H
#define SPH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SPH_ABI_VERSION 1

typedef enum {
    SPH_OK = 0,
    SPH_EINVAL = -1,     /* bad argument: null pointer, bad layout, unsupported format */
    SPH_ENOSPACE = -2,   /* workspace or cell capacity too small for the request */
    SPH_ECUDA = -3,      /* a CUDA runtime call or kernel launch failed */
    SPH_ESTATE = -4,     /* call out of order (e.g. sph_density before sph_bin_cells) */
    SPH_ECAPACITY = -5,  /* cell grid unusable: < 3 cells on an axis or cells < 2 h_max */
    SPH_ETIMEOUT = -6,   /* a bounded device wait gave up (reserved; no call waits today) */
    SPH_ENUMERIC = -7    /* the device recorded a numerical condition (see error_bits) */
} sph_status;

/* Particle fields.  Bit (1u << field) selects a field in a `fields` mask. */
enum {
    SPH_F_X = 0,     /* position, 3 components (AoS: FP64 absolute; SoA: cell-relative) */
    SPH_F_V = 1,     /* velocity, 3 components */
    SPH_F_A = 2,     /* acceleration, 3 components (written by sph_force) */
    SPH_F_M = 3,     /* mass */
    SPH_F_H = 4,     /* smoothing length (support radius 2h) */
    SPH_F_RHO = 5,   /* density (written by sph_density) */
    SPH_F_U = 6,     /* specific internal energy */
    SPH_F_P = 7,     /* pressure (written by sph_density when u is present) */
    SPH_F_DUDT = 8,  /* du/dt (written by sph_force) */
    SPH_F_CS = 9,    /* sound speed (written by sph_density when u is present) */
    SPH_NFIELDS = 10
};
#define SPH_BIT(f) (1u << (f))
/* the narrowing N of each kernel (Section 6.1: "narrowing tailored to a kernel") */
#define SPH_FIELDS_DENSITY (SPH_BIT(SPH_F_X) | SPH_BIT(SPH_F_M) | SPH_BIT(SPH_F_H) | SPH_BIT(SPH_F_U))
#define SPH_FIELDS_FORCE   (SPH_FIELDS_DENSITY | SPH_BIT(SPH_F_V))
#define SPH_FIELDS_KICK    (SPH_BIT(SPH_F_V) | SPH_BIT(SPH_F_U))
#define SPH_FIELDS_OUTPUT  (SPH_BIT(SPH_F_V) | SPH_BIT(SPH_F_A) | SPH_BIT(SPH_F_H) | \
                            SPH_BIT(SPH_F_RHO) | SPH_BIT(SPH_F_U) | SPH_BIT(SPH_F_P))

/* SoA storage formats (Table 2 of the paper, plus bfloat16).  Storage only:
 * every kernel computes in FP32 (Section 3.2, "expanded to a form supported
 * natively by the hardware").  FP64 values are first rounded to FP32 (nearest
 * even); the 16-bit formats round that FP32 value to nearest even; the
 * truncated formats keep sign, 8 exponent bits and the top 16 or 10 mantissa
 * bits and store the 25- or 19-bit codes as a packed little-endian bitstream
 * (value k at bits [kB, (k+1)B) of 32-bit words). */
typedef enum {
    SPH_P_FP32 = 0,
    SPH_P_BF16 = 1,
    SPH_P_FP16 = 2,
    SPH_P_FP32_M16 = 3,  /* 25-bit code */
    SPH_P_FP32_M10 = 4   /* 19-bit code */
} sph_prec;
/* The truncated family at any width (Table 2's rows from 31 down to 10 total
 * bits): FP32 with the top n mantissa bits kept by truncation, n in [1, 22],
 * stored as a packed stream of (9 + n)-bit codes.  SPH_P_FP32_TRUNC(16) and
 * SPH_P_FP32_TRUNC(10) are SPH_P_FP32_M16 and SPH_P_FP32_M10 under other
 * codes.  Wider formats (FP64-based, 33..63 bits) would decode to values that
 * the FP32 arithmetic rounds to FP32 anyway, so FP32 storage covers them. */
#define SPH_P_FP32_TRUNC(n) (100 + (n))
#define SPH_P_FP32_TRUNC_MIN 1
#define SPH_P_FP32_TRUNC_MAX 22

/* element type of a field inside the caller's AoS record */
enum { SPH_AOS_F64 = 0, SPH_AOS_F32 = 1 };

/* AoS layout descriptor: one record per particle, `record_bytes` apart.
 * offset[f] is the byte offset of field f inside a record (-1: absent); a
 * vector field stores its 3 components contiguously.  type[f] is SPH_AOS_F64
 * or SPH_AOS_F32.  Positions must be present and FP64 (absolute positions are
 * drifted in FP64).  record_bytes must be a multiple of 8 and at most 512;
 * every offset a multiple of the field's element size; the AoS base pointer
 * 16-byte aligned. */
typedef struct {
    int32_t record_bytes;
    int32_t offset[SPH_NFIELDS];
    int32_t type[SPH_NFIELDS];
} sph_aos_layout;

/* Physical and numerical parameters.
 *   box       periodic box edge lengths; positions lie in [0, box)
 *   gamma     adiabatic index of the ideal-gas EOS P = (gamma-1) rho u
 *   alpha_av, beta_av, eps_av   Monaghan artificial viscosity
 *   eta       h = eta (m/rho)^(1/3) at the smoothing-length fixed point;
 *             eta = 1/2 (3 N_ngb / (4 pi))^(1/3) for N_ngb neighbours
 *   h_max     upper clamp of h; cells are at least 2 h_max wide
 *   flags     SPH_FLAG_* bits */
typedef struct {
    double box[3];
    double gamma;
    double alpha_av, beta_av, eps_av;
    double eta;
    double h_max;
    int32_t flags;
    int32_t reserved;
} sph_params;

#define SPH_FLAG_PLAIN_SUM 1   /* density sum without compensation (default: Neumaier) */

/* workspace options */
#define SPH_WS_REORDER 1       /* reserve room for sph_bin_cells(SPH_BIN_REORDER) */
#define SPH_WS_LEVELS 2        /* reserve room for the level hierarchy (sph_bin_levels) */

/* Counters accumulated on the device since creation or sph_reset_stats. */
typedef struct {
    uint64_t pairs_density;      /* ordered pairs j != i, r < 2 h_i, over every density pass */
    uint64_t pairs_force;        /* ordered pairs j != i, r < h_i + h_j */
    uint64_t tests_density;      /* candidate distance tests made by the density kernel */
    uint64_t tests_force;        /* candidate distance tests made by the force kernel */
    uint64_t hcap_clamps;        /* particles whose h was clamped at h_max */
    uint32_t error_bits;         /* SPH_ERR_* bits, sticky */
    int32_t ncell[3];            /* current cell grid */
    int64_t nitems;              /* work items of the pair kernels */
    int64_t max_occupancy;       /* particles in the fullest cell */
    uint64_t launches;           /* kernels this context has launched (host-side count) */
} sph_stats;

#define SPH_ERR_NONFINITE 1      /* a non-finite value was produced or read */
#define SPH_ERR_OUTSIDE   2      /* a position lay outside [0, box) at binning */
#define SPH_ERR_HCAP      4      /* some h was clamped at h_max */
#define SPH_ERR_NEWTON    8      /* a Newton step met a non-positive derivative */
/* Per-particle flags of a density call (sph_desc.off_density_flags, slot
 * order): which particles set the error word's HCAP, NEWTON and NONFINITE
 * bits.  The FP64 oracle reports the same three conditions per particle. */
#define SPH_PFLAG_HCAP      1    /* h was clamped at its cap */
#define SPH_PFLAG_NEWTON    2    /* a Newton step met f'(h) <= 0 or a non-finite f: h kept */
#define SPH_PFLAG_NONFINITE 4    /* the input h or the resulting density was not finite */
#define SPH_ERR_TIMEOUT   16     /* an asynchronous record copy did not complete within its first
                                    bounded wait; the warp waited once more, longer, and skipped
                                    its records only if the copy had still not landed */

/* Launch shapes of the pair kernels (an autotuner sets them; the defaults
 * after sph_create are block_threads 32, ctas_per_sm 0, stage_density 128,
 * stage_force 128, subcells 2, item_order 1, class_launches 0, pair_kernel 0,
 * block_threads_force 32). */
typedef struct {
    int32_t block_threads;       /* threads per CTA of the density kernels (32..256, multiple of 32), one
                                    warp per work item; sph_set_tuning also gives it to the force
                                    kernels unless block_threads_force is set */
    int32_t ctas_per_sm;         /* persistent CTAs per SM (0: occupancy maximum) */
    int32_t stage_density;       /* density kernel: candidates staged per warp in one round of the
                                    stream that fills the per-lane lists (>= 32); in level mode
                                    an item whose box gathers more than 8 x stage_density
                                    candidates is deferred to the per-target pass */
    int32_t stage_force;         /* neighbour candidates staged per warp, force kernel (>= 32); in
                                    level mode an item whose candidate streams hold more than
                                    64 x stage_force candidates is deferred to the per-target
                                    pass */
    int32_t subcells;            /* sub-cells per cell edge used to order particles, 1 or 2
                                    (default 2); takes effect at the next sph_bin_cells */
    int32_t item_order;          /* order of the pair-kernel work queue, set at sph_bin_cells:
                                    0 cell order, 1 costliest first (items grouped by
                                    the power-of-two class of count x stencil occupancy,
                                    classes in descending order); -1 keeps the current */
    int32_t class_launches;      /* 1: one pair-kernel launch per cost class (needs
                                    item_order 1), 0: one persistent launch over the
                                    whole queue; -1 keeps the current */
    int32_t pair_kernel;         /* 0: the batched kernels (warp work items, staged and
                                    pruned neighbourhoods); 1: the plain form, one thread
                                    per particle looping over the 27 neighbour cells
                                    straight from the SoA (a baseline).  For the buffer
                                    kernels, 0 stages each buffer in shared memory and
                                    1 reads every partner from global memory (the
                                    paper's kernel structure); -1 keeps the current */
    int32_t block_threads_force; /* threads per CTA of the force kernels (32..256, multiple of 32);
                                    0 in sph_set_tuning: block_threads if that is set, else
                                    the current */
} sph_tuning;

/* Where the library's arrays live inside the workspace (byte offsets from the
 * workspace base, -1 when absent), for inspection and testing. */
typedef struct {
    int64_t n;
    int32_t ncell[3];
    double cell_edge[3];
    int64_t off_perm;            /* int32[n]: sorted slot -> original particle index */
    int64_t off_cell_of_slot;    /* int32[n]: sorted slot -> key = cell * s^3 + sub-cell
                                    (after sph_bin_levels: the finest cell's Morton key) */
    int64_t off_cell_start;      /* int32[ncell s^3 + 1]: first slot of each key */
    int64_t off_nngb;            /* int32[n], neighbour counts of the last density call */
    int64_t off_nngb_force;      /* int32[n], neighbour counts of the last force call */
    int64_t off_soa[SPH_NFIELDS][3];
    int32_t prec[SPH_NFIELDS];   /* current storage format of each SoA field */
    uint32_t valid;              /* fields whose SoA copy is current */
    int32_t subcells;            /* s: sub-cells per cell edge of the last binning */
    int64_t off_level;           /* int8[n]: level of every slot (sph_bin_levels; -1 without
                                    SPH_WS_LEVELS); after sph_density_levels, the level each
                                    particle's density was computed at */
    int64_t off_density_flags;   /* uint8[n]: per-slot flags of the last density call,
                                    SPH_PFLAG_* bits */
} sph_desc;

typedef struct sph_ctx sph_ctx;

/* Bytes of workspace a context needs for n particles and at most ncell_max
 * cells; `ws_flags` is a mask of SPH_WS_* bits.  Returns 0 on a bad argument.
 * Pure host function. */
size_t sph_workspace_bytes(const sph_aos_layout *layout, int64_t n, int64_t ncell_max,
                           uint32_t ws_flags);

/* Create a context over n caller-owned AoS records at d_aos (records in
 * `layout`), using the caller-owned device workspace d_workspace of
 * workspace_bytes (at least sph_workspace_bytes(layout, n, ncell_max, ws_flags),
 * 256-byte aligned).  `stream` is a cudaStream_t (NULL: the legacy default
 * stream).  The CUDA device current at this call is used for all later calls.
 * d_aos is device memory (the paper's in-place variant, Section 6.3) or host
 * memory the device can address -- pinned with cudaHostAlloc / cudaMallocHost,
 * whose pointer is a device pointer under unified addressing.  In the second
 * case the kernels that touch the records (binning, conversion, kick/drift,
 * write-back) read and write them over the host link while the SoA and the
 * workspace stay in device memory: the paper's streaming variant without
 * staging copies.  Device-resident records whose size is a multiple of 16
 * bytes (and an odd number of 16-byte chunks) move by bulk asynchronous
 * copies where a warp's 32 records are consecutive; host-mapped records
 * always take per-lane loads.  d_aos must be 16-byte aligned (it may be NULL
 * when n = 0: every call is then a no-op).
 * Errors: SPH_EINVAL (layout, params or pointers), SPH_ENOSPACE (workspace),
 * SPH_ECUDA (device query).  On success *out receives the context. */
sph_status sph_create(const sph_aos_layout *layout, const sph_params *params, int64_t n,
                      int64_t ncell_max, uint32_t ws_flags, void *d_aos, void *d_workspace,
                      size_t workspace_bytes, void *stream, sph_ctx **out);

/* S1, cell binning (the paper works on 64-particle co-located buffers,
 * Section 6; this library generalises them to a uniform grid).  Cells per axis
 * nc_d = floor(box_d / max(cell_edge, 2 h_max)); each particle's cell is
 * k_d = clamp(floor(x_d * (nc_d / box_d)), 0, nc_d - 1) in FP64, linear id
 * kx + nc_x (ky + nc_y kz).  Each cell is split into s^3 sub-cells
 * (s = tuning.subcells): fine coordinate f_d = clamp(floor(x_d * (s nc_d /
 * box_d)), 0, s nc_d - 1), cell f_d / s, sub-cell f_d % s, key
 * cell s^3 + (s_x + s (s_y + s s_z)).  The permutation lists particles by key,
 * ascending original index among equal keys (a stable sort), so every cell
 * stays contiguous and spatially compact inside; the pair-kernel work items
 * are rebuilt.  flags (SPH_BIN_*, or-ed; 0 for neither):
 *   SPH_BIN_REORDER    also rewrite the AoS records in that order (the
 *                      permutation then becomes the identity); needs a
 *                      workspace created with SPH_WS_REORDER;
 *   SPH_BIN_DRIFT_KEYS the caller vouches that no position in the AoS changed
 *                      since this context's last sph_kick_drift or
 *                      sph_kick_drift_writeback: the keys that call computed
 *                      for the positions it wrote are used instead of reading
 *                      the records again (the same keys, bit for bit).  The
 *                      flag is ignored, and the records read, when there are
 *                      no such keys: no kick/drift since the last binning, a
 *                      binning on another grid (cell_edge, subcells), the
 *                      level hierarchy or buffers, or a call that wrote
 *                      positions since (sph_aos_upload; sph_soa_to_aos and
 *                      sph_soa_to_aos_host of X).  The library cannot see writes made
 *                      to the records by other code: a caller who moves
 *                      particles between the two calls must not set it.
 *                      A kick/drift that computes the keys reports a
 *                      non-finite position as SPH_ERR_OUTSIDE too, as the
 *                      binning would.
 * Invalidates every SoA field.
 * Errors: SPH_EINVAL (unknown flags), SPH_ECAPACITY (< 3 cells on an axis),
 * SPH_ENOSPACE (more than ncell_max cells, or reorder without room),
 * SPH_ECUDA. */
#define SPH_BIN_REORDER 1
#define SPH_BIN_DRIFT_KEYS 2
sph_status sph_bin_cells(sph_ctx *ctx, double cell_edge, int32_t flags);

/* S2, U o N o C (Section 4, Eq. 12): gather the fields in `fields` from the AoS
 * in cell order, round them to their storage formats and write them as SoA.
 * prec[f] (SPH_NFIELDS entries, NULL: FP32 everywhere) is the storage format
 * of field f.  Positions are stored as offsets from their cell origin
 * k_d * box_d / nc_d (computed in FP64, then rounded); they accept FP32 or
 * FP16.  RHO, P and CS accept FP32, BF16 and FP16; A and DUDT (written by
 * the force, read by kick/drift) FP32 only; V, M, H and U accept every
 * format.  Each value is multiplied by its field's storage scale 2^e
 * (sph_set_field_scale) before rounding.  Requires sph_bin_cells.  Errors:
 * SPH_EINVAL (field absent from the layout, or format not allowed for it),
 * SPH_ESTATE. */
sph_status sph_aos_to_soa(sph_ctx *ctx, uint32_t fields, const int32_t *prec);

/* Exact power-of-two storage scale per field (a reading of the paper's
 * storage formats, Section 3 and Table 2, which fix the bit layout but not the
 * range: the paper's own values stay inside FP32's).  A 16-bit format covers
 * a fixed window -- FP16 keeps 11 significant bits only for magnitudes in
 * [2^-14, 65504] -- so a particle mass of 5e-7 would be stored as a
 * subnormal with 4 significant bits.  With exp2[f] = e, field f is stored as
 * the code of value * 2^e and read back as decode(code) * 2^-e everywhere
 * (conversion, kernel outputs, kick/drift, write-back).  Multiplying by a
 * power of two is exact while the product stays a normal FP32 number, so the
 * scale moves the window without adding rounding: the stored value is the
 * unscaled format's rounding of value * 2^e.  exp2 holds SPH_NFIELDS entries
 * in [-SPH_SCALE_MAX_EXP, SPH_SCALE_MAX_EXP]; A and DUDT are always FP32
 * and take 0 only.  All scales are 0 after sph_create.  A field whose scale
 * changes loses its SoA contents (convert it again).  Host-only, no device
 * work.  Errors: SPH_EINVAL. */
#define SPH_SCALE_MAX_EXP 64
sph_status sph_set_field_scale(sph_ctx *ctx, const int32_t *exp2);
sph_status sph_get_field_scale(const sph_ctx *ctx, int32_t *exp2_out);

/* S3+S4, density (Eq. 6, gather form rho_i = sum_j m_j W(r_ij, h_i), M4 cubic
 * spline with support 2h, FP32 arithmetic, compensated sum) with
 * `newton_steps` Newton steps on f(h) = rho(h) - m_i (eta/h)^3 (each step
 * clamped to [h/2, 2h] and to h_max) and a final density sum at the last h.
 * Writes RHO, the neighbour counts (j != i, r < 2h), H when newton_steps > 0,
 * and P = (gamma-1) rho u and CS = sqrt(gamma P / rho) when U is current.
 * Reads X, M, H (and U).  Requires sph_aos_to_soa of X, M, H.
 * Errors: SPH_EINVAL (newton_steps < 0 or > 32), SPH_ESTATE, SPH_ECUDA. */
sph_status sph_density(sph_ctx *ctx, int32_t newton_steps);

/* S5, symmetric hydro force (Eq. 7 with Monaghan artificial viscosity and the
 * matching energy equation, Eq. 5): for pairs r < h_i + h_j,
 *   a_i    = -sum_j m_j (P_i/rho_i^2 + P_j/rho_j^2 + Pi_ij) grad_i W(r_ij, (h_i+h_j)/2)
 *   du_i/dt =  sum_j m_j (P_i/rho_i^2 + Pi_ij/2) v_ij . grad_i W
 * in FP32.  Reads X, V, M, H, RHO, P, CS; writes A and DUDT.
 * Errors: SPH_ESTATE (inputs not current), SPH_ECUDA. */
sph_status sph_force(sph_ctx *ctx);

/* S6, kick/drift (the paper's linear kernels Kick and Drift, Section 6):
 * v += a dt_kick and u += du/dt dt_kick in FP32 in the SoA, then
 * x += v dt_drift in FP64 directly in the AoS, wrapped into [0, box).
 * Reads A, DUDT, V, U; writes V, U (SoA) and X (AoS).  The SoA positions
 * become stale (re-bin before the next pair kernel).
 * Errors: SPH_ESTATE, SPH_ECUDA. */
sph_status sph_kick_drift(sph_ctx *ctx, double dt_kick, double dt_drift);

/* S7, C^T o N^T o U^T (Section 4, the write-back epilogue): widen the SoA
 * fields in `fields` to the AoS element type and scatter them to their
 * records.  Positions are not written after sph_bin_cells or sph_bin_levels
 * (the AoS keeps them in FP64; drift updates them in place).  After
 * sph_bin_buffers they may be: x = buffer origin + offset in FP64, wrapped
 * into [0, box).
 * Errors: SPH_EINVAL (X requested outside buffer mode, or field absent from
 * the layout), SPH_ESTATE (field not current), SPH_ECUDA. */
sph_status sph_soa_to_aos(sph_ctx *ctx, uint32_t fields);

/* ---- The conversion on the host: the paper's CPU placement --------------
 * Section 6.3 (Eq. 13-14) converts on the CPU and then moves the narrowed,
 * reduced-precision SoA to the device, or moves the AoS first and converts
 * on the GPU.  sph_aos_to_soa is the GPU placement; these two calls are the
 * CPU one, over records in host memory (any host memory; the staging buffer
 * should be pinned for the copies to run at full speed).  They produce the
 * same codes and record bytes as their device counterparts.  Both read the
 * permutation (and what positions need) from the device and synchronise the
 * context's stream first, convert with `nthreads` host threads (<= 0: one
 * per hardware thread), and move the data with one copy per SoA array.
 * host_stage is a caller-owned host buffer of at least
 * sph_host_stage_bytes(ctx) bytes; after sph_aos_to_soa_host returns, the
 * copies out of it may still be in flight on the stream, so it must not be
 * rewritten before the stream has passed them. */
size_t sph_host_stage_bytes(const sph_ctx *ctx);

/* As sph_aos_to_soa (same fields, formats, scales, slot order and position
 * offsets), reading the records at host_aos (n records in the context's
 * layout).  Errors: SPH_EINVAL (pointers, fields, formats), SPH_ENOSPACE
 * (stage too small), SPH_ESTATE (not binned), SPH_ECUDA. */
sph_status sph_aos_to_soa_host(sph_ctx *ctx, const void *host_aos, uint32_t fields, const int32_t *prec,
                               void *host_stage, size_t stage_bytes, int32_t nthreads);

/* As sph_soa_to_aos, writing the records at host_aos.  Returns once the
 * records are written.  Errors as sph_soa_to_aos, and SPH_ENOSPACE. */
sph_status sph_soa_to_aos_host(sph_ctx *ctx, void *host_aos, uint32_t fields, void *host_stage,
                               size_t stage_bytes, int32_t nthreads);

/* ---- Buffer kernels: the paper's benchmark grouping (Section 6) ----------
 * The paper keeps particles in contiguous buffers of 64 spatially co-located
 * particles; its quadratic kernels Density and Force evaluate every pair of
 * a buffer (64 x 64), its linear kernels Kick and Drift every particle once,
 * and it times them reading the AoS directly against reading the converted
 * SoA (Fig. 2).  These calls run the four kernels on such buffers, reading
 * either layout:
 *   source = SPH_SRC_AOS: the records directly (strided; positions made
 *            relative to the buffer origin inside the kernel); outputs go to
 *            the records, and their SoA copies become stale;
 *   source = SPH_SRC_SOA: the SoA arrays sph_aos_to_soa wrote (inputs must
 *            be current); outputs go to the SoA arrays in their storage
 *            formats, and the records keep their old values until
 *            sph_soa_to_aos.
 * Arithmetic is FP32 in both (the AoS drift is FP64). */
#define SPH_SRC_AOS 0
#define SPH_SRC_SOA 1
#define SPH_BUFFER_MIN 32
#define SPH_BUFFER_MAX 256

/* Switch the context to buffers: buffer b holds records
 * [b buffer_size, min((b+1) buffer_size, n)); buffer_size is a power of two
 * in [SPH_BUFFER_MIN, SPH_BUFFER_MAX] (the paper uses 64).  The caller groups
 * co-located particles into consecutive records; nothing is sorted (slot k is
 * record k).  Each buffer's origin is the position of its first record; SoA
 * positions (sph_aos_to_soa of X) are then offsets from it, moved to the
 * nearest periodic image (FP64 difference, -box when >= box/2, +box when
 * < -box/2), rounded to the storage format.  Invalidates every SoA field;
 * sph_density and sph_force need sph_bin_cells again (SPH_ESTATE before).
 * Errors: SPH_EINVAL (buffer_size), SPH_ECUDA. */
sph_status sph_bin_buffers(sph_ctx *ctx, int32_t buffer_size);

/* Density over the buffer, h fixed: rho_i = sum_j m_j W(r_ij, h_i) over the
 * particles j of i's buffer, self included (Eq. 6 restricted to the buffer),
 * then P = (gamma - 1) rho u and c = sqrt(gamma P / rho).  Reads X, M, H, U;
 * writes RHO, P and CS (CS in the records only when the layout has it).
 * pairs_density counts the pairs j != i with r < 2 h_i.  Errors: SPH_EINVAL
 * (source, or with SPH_SRC_AOS a field absent from the layout), SPH_ESTATE
 * (not in buffer mode, or SoA inputs not current), SPH_ECUDA. */
sph_status sph_buffer_density(sph_ctx *ctx, int32_t source);

/* Force over the buffer: the symmetric pair force with Monaghan viscosity
 * (Eq. 7, Eq. 5) over the pairs j != i of i's buffer with r < h_i + h_j,
 * c = sqrt(gamma P / rho).  Reads X, V, M, H, RHO, P; writes A and DUDT
 * (FP32 in the SoA).  pairs_force counts the pairs.  Errors as
 * sph_buffer_density. */
sph_status sph_buffer_force(sph_ctx *ctx, int32_t source);

/* Kick: v += a dt, u += du/dt dt (FP32).  Reads V, A, U, DUDT; writes V, U.
 * Errors as sph_buffer_density, and SPH_EINVAL for a non-finite dt. */
sph_status sph_buffer_kick(sph_ctx *ctx, int32_t source, double dt);

/* Drift: x += v dt.  SPH_SRC_AOS: FP64 in the records, wrapped into
 * [0, box).  SPH_SRC_SOA: the FP32 offsets from the buffer origin (wrapped
 * when written back).  Reads X, V; writes X.  Errors as sph_buffer_kick. */
sph_status sph_buffer_drift(sph_ctx *ctx, int32_t source, double dt);

/* ---- Adaptive smoothing lengths: a hierarchy of cell levels --------------
 * The density's Newton iteration (Eq. 6 with f(h) = rho(h) - m (eta/h)^3)
 * gives every particle its own h, and in a clustered set those differ by a
 * factor of 30 or more between the dense cores and the background.  One grid
 * whose cells hold the largest 2h then puts hundreds of thousands of
 * particles into a core cell, and every core particle tests all of them.
 * These calls keep one grid per level l = level_min..level_max with 2^l
 * cells per axis (edge e_l,d = box_d / 2^l), nested like an octree, and
 * compute each particle's density on the finest level whose cells hold its
 * support.
 *
 * Cell of a particle at level_max: f_d = clamp(floor(x_d * (2^level_max /
 * box_d)), 0, 2^level_max - 1) in FP64; its key is the Morton code of
 * (f_x, f_y, f_z) (bit b of f_x, f_y, f_z at bits 3b, 3b+1, 3b+2).  Slots are
 * ordered by key, ascending original index among equal keys, so the cell of
 * every level is one run of consecutive slots (its key prefix).  Positions
 * in the SoA (sph_aos_to_soa) are offsets from the level_max cell origin
 * f_d * box_d / 2^level_max.
 *
 * Level of a particle: the largest l in [level_min, level_max] with
 * h_i (1 + h_margin) <= h_l = min_d e_l,d / 2, evaluated in FP64 on the
 * record's h; level_min when there is none or h_i is not finite and
 * positive.  The margin leaves room for h to grow during the Newton steps. */
#define SPH_LEVEL_MIN 2
#define SPH_LEVEL_MAX 10
#define SPH_LEVELS_MAX 8       /* levels in one hierarchy, at most */

/* Bin for the hierarchy: keys, the stable sort, and every particle's level.
 * Needs a context created with SPH_WS_LEVELS; requires
 * SPH_LEVEL_MIN <= level_min <= level_max <= SPH_LEVEL_MAX,
 * level_max - level_min < SPH_LEVELS_MAX, h_margin >= 0
 * and h_max <= h_level_min (the coarsest cells hold the largest support).
 * Invalidates every SoA field; leaves cell and buffer mode (sph_density,
 * sph_force and the buffer calls return SPH_ESTATE until sph_bin_cells or
 * sph_bin_buffers).  Positions outside [0, box) or not finite set
 * SPH_ERR_OUTSIDE (and SPH_ERR_NONFINITE) in the error word, as in
 * sph_bin_cells, and land in the edge cells.  Errors: SPH_EINVAL (levels,
 * margin, or no H in the layout), SPH_ENOSPACE (workspace without
 * SPH_WS_LEVELS), SPH_ECAPACITY (h_max > h_level_min), SPH_ECUDA. */
sph_status sph_bin_levels(sph_ctx *ctx, int32_t level_min, int32_t level_max, double h_margin);

/* S3+S4 over the hierarchy: the density of sph_density (same Newton steps,
 * sums, EOS and outputs) with each particle's neighbours gathered from the
 * 27 cells of its level around its own cell (periodic).  Levels run from
 * level_max to level_min.  At level l the Newton steps clamp h at
 * min(h_max, h_l); a particle whose h met that clamp while l > level_min
 * moves to level l - 1 and is computed again there from its original h, so
 * that every particle's result is the one a single grid of cells >= 2 h_max
 * gives (up to the order of the sums).  hcap_clamps counts the particles
 * clamped at level_min.  Reads X, M, H (and U); writes RHO, H (always, even
 * with newton_steps = 0, so that an input h above the level_min cap reaches
 * the force clamped), P and CS (U current) and the neighbour counts.  Requires
 * sph_bin_levels and sph_aos_to_soa of X, M, H.  Errors: SPH_EINVAL
 * (newton_steps < 0 or > 32), SPH_ESTATE, SPH_ECUDA. */
sph_status sph_density_levels(sph_ctx *ctx, int32_t newton_steps);

/* S5 over the hierarchy: the force of sph_force (Eq. 7 with Monaghan
 * viscosity, Eq. 5; pairs r < h_i + h_j) with every particle's own h, after
 * sph_density_levels has fixed the levels.  A level-l particle's h is at
 * most h_l, so a partner of a finer or equal level lies in the 27 cells of
 * level l around it, and one of a coarser level l' in the 27 cells of level
 * l' around it: each particle searches, for every level l', the particles of
 * level l' in the cells of level min(l, l'), and finds each pair once.
 * The search relies on every h being within its level's cap, which
 * sph_density_levels guarantees: it must have run since the last
 * sph_bin_levels and since H was last converted from the records.
 * Reads X, V, M, H, RHO, P, CS; writes A and DUDT (FP32).  Errors:
 * SPH_ESTATE (not in level mode, no sph_density_levels since, or inputs not
 * current), SPH_ECUDA. */
sph_status sph_force_levels(sph_ctx *ctx);

/* Per level l (index l of both arrays, SPH_LEVEL_MAX + 1 entries each):
 * done[l] the particles whose density was computed at level l, promoted[l]
 * those moved from level l to l - 1, summed since creation or
 * sph_reset_stats.  Synchronises the context's stream.  Errors: SPH_EINVAL,
 * SPH_ECUDA. */
sph_status sph_level_counts(sph_ctx *ctx, int64_t *done, int64_t *promoted);

/* S6 + S7 in one pass over the records: the same results in the AoS as
 * sph_kick_drift(dt_kick, dt_drift) followed by sph_soa_to_aos(fields) --
 * bit for bit, v and u written as their storage format holds them after the
 * kick -- but each record is visited once, so the sectors that x and the
 * written fields share are written whole.  The kicked v and u go to the AoS
 * only: afterwards the SoA copies of X, V and U are stale (convert again
 * before reading them on the device).  `fields` as for sph_soa_to_aos.
 * Errors: SPH_EINVAL (fields empty, X requested or a field absent from the
 * layout, non-finite dt), SPH_ESTATE (A, DUDT, V, U or a requested field
 * not current), SPH_ECUDA. */
sph_status sph_kick_drift_writeback(sph_ctx *ctx, double dt_kick, double dt_drift, uint32_t fields);

/* Copy the device counters to *out.  Synchronises the context's stream.
 * Returns SPH_ENUMERIC when error_bits has SPH_ERR_NONFINITE, SPH_ERR_OUTSIDE
 * or SPH_ERR_TIMEOUT set (the counters are still filled in), else SPH_OK. */
sph_status sph_get_stats(sph_ctx *ctx, sph_stats *out);

/* Zero the device counters and the sticky error word (asynchronous). */
sph_status sph_reset_stats(sph_ctx *ctx);

/* Timing hooks around the pair kernels themselves (measurement only; the
 * paper has no counterpart).  With a pair set, sph_density records ev_begin
 * on the context's stream right before its pair kernel (after its pack
 * pass) and ev_end right after it; with SPH_KEV_FORCE, sph_force does the
 * same around its pair kernel.  ev_begin and ev_end are cudaEvent_t handles
 * owned by the caller, who must keep them alive while they are set; NULL
 * for both clears the hook.  Only the cell-list kernels record (not the
 * level hierarchy's or the plain form's).  Errors: SPH_EINVAL (unknown
 * `which`, or one handle NULL and the other not). */
#define SPH_KEV_DENSITY 0
#define SPH_KEV_FORCE   1
sph_status sph_set_kernel_events(sph_ctx *ctx, int32_t which, void *ev_begin, void *ev_end);

/* Set launch shapes; values <= 0 keep the defaults.  Takes effect at the next
 * pair-kernel call.  Errors: SPH_EINVAL (block_threads not a multiple of 32 in
 * [32, 256], or stage sizes outside [32, 65535] or above the shared-memory limit). */
sph_status sph_set_tuning(sph_ctx *ctx, const sph_tuning *tuning);
sph_status sph_get_tuning(const sph_ctx *ctx, sph_tuning *out);

/* Describe where the library's arrays live in the workspace. */
sph_status sph_describe(const sph_ctx *ctx, sph_desc *out);

/* M (Section 4): copy `bytes` bytes of AoS records between pinned or pageable
 * host memory and the context's AoS on its stream.  bytes must not exceed
 * n * record_bytes.  sph_aos_download synchronises the stream before it
 * returns.  Errors: SPH_EINVAL, SPH_ECUDA. */
sph_status sph_aos_upload(sph_ctx *ctx, const void *host, size_t bytes);
sph_status sph_aos_download(sph_ctx *ctx, void *host, size_t bytes);

/* Allocation-free cell binning.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory at all, such
 * as a plugin running inside a host application that owns the whole device
 * memory pool and offers plugins no allocation hook, or a latency-critical
 * path where cudaMalloc's implicit device-wide synchronisation is not
 * acceptable.  It computes exactly what sph_bin_cells computes with one
 * sub-cell per cell (tuning.subcells = 1: same cell rule, same stable order)
 * without a context or a workspace: its scratch
 * memory is a fixed array of SPH_NOALLOC_SCRATCH_BYTES inside libsph, which
 * every device that loads the library holds until the process exits.
 *
 *   d_aos           n device records in `layout` (positions FP64, 8-byte aligned)
 *   box, nc         host arrays of 3: box edges and cells per axis (each >= 1)
 *   d_perm          device int32[n]: sorted slot -> original particle index
 *   d_cell_of_slot  device int32[n]: sorted slot -> cell id kx + nc_x (ky + nc_y kz)
 *   d_cell_start    device int32[nc_x nc_y nc_z + 1]: first slot of each cell
 *   stream          cudaStream_t (NULL: legacy default stream)
 *
 * The call is asynchronous and allocates nothing: no cudaMalloc, cudaFree or
 * allocating library routine.  The first call on a device (the device current
 * at the call) looks up the array's device address once; make that first
 * call before any stream capture.  All calls on a device share the one
 * array, which keeps the last call's contents (every call clears what must
 * start at zero), so calls that overlap on the GPU -- on different streams,
 * or from different threads -- race and must be serialised by the caller.
 * Positions outside [0, box) are clamped into the edge cells; no error word
 * is kept.  Errors: SPH_ENOSPACE when n > SPH_NOALLOC_MAX_PARTICLES or the
 * grid has more than SPH_NOALLOC_MAX_CELLS cells (nothing is launched),
 * SPH_EINVAL for bad arguments, SPH_ECUDA for a failed CUDA call. */
#define SPH_NOALLOC_MAX_PARTICLES 262144
#define SPH_NOALLOC_MAX_CELLS 262144
#define SPH_NOALLOC_SCRATCH_BYTES 5636096
sph_status sph_bin_cells_noalloc(const void *d_aos, const sph_aos_layout *layout, int64_t n,
                                 const double *box, const int32_t *nc, int32_t *d_perm,
                                 int32_t *d_cell_of_slot, int32_t *d_cell_start, void *stream);

/* Free the host-side context (the caller's buffers are untouched). */
void sph_destroy(sph_ctx *ctx);

/* Static English text for a status code. */
const char *sph_status_str(sph_status status);

#ifdef __cplusplus
}
#endif
#endif /* SPH_H */
