/*
 * ants.h -- C ABI of libants, a GB300 (sm_103a) library for the statistical
 * position/energy reconstruction of Anger-camera type detectors described in
 * "ANTS2 package: simulation and experimental data processing for Anger
 * camera type detectors" (Morozov et al., arXiv:1602.07247).
 *
 * The library reconstructs, for every event, the source position (x, y[, z])
 * and energy E from the photosensor signals by maximum likelihood, with the
 * light response functions (LRFs) of the sensors parameterised by cubic
 * B-splines (Sec. 5.1.2, 5.1.2.2, 6, 6.1).
 *
 * Conventions for every entry point:
 *   - Plain pointers and sizes only.  Arguments named *_dev are device
 *     pointers (CUDA global memory of the context's device), *_host are host
 *     pointers.  All of them are owned by the caller, who keeps them alive
 *     until the work on `stream` has completed.
 *   - Handles (ants_ctx, ants_detector, ants_lrf) are owned by the library
 *     and released with the matching *_free / *_destroy call.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Calls that take a stream are asynchronous with respect to
 *     the host unless documented otherwise.
 *   - Every call returns an ants_status.  Argument errors are detected
 *     before any launch and leave outputs untouched.  ants_last_error()
 *     returns a message for the calling thread's last non-OK return.
 *   - Problems of individual events never fail a call; they are reported in
 *     the per-event status array (ants_evt_status).
 *   - Coordinates are in millimetres; signals are photo-electron counts (or
 *     proportional amplitudes), non-negative.
 */
#ifndef ANTS_H
#define ANTS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define ANTS_API __attribute__((visibility("default")))
#else
#define ANTS_API
#endif

/* Return codes. */
typedef enum {
    ANTS_OK = 0,
    ANTS_E_ARG = -1,           /* invalid argument (null pointer, bad size, bad enum) */
    ANTS_E_CUDA = -2,          /* a CUDA runtime call or kernel launch failed */
    ANTS_E_OOM = -3,           /* device or host allocation failed */
    ANTS_E_LRF = -4,           /* LRF fit failed (normal matrix singular even with ridge) */
    ANTS_E_SHAPE = -5,         /* sizes inconsistent with the LRF or detector */
    ANTS_E_TIMEOUT = -6,       /* a bounded device-side wait gave up */
    ANTS_E_INTERNAL = -7,      /* internal consistency check failed */
    ANTS_E_UNIMPLEMENTED = -8, /* method or option not available */
    ANTS_E_IO = -9             /* file could not be read or written, or bad format */
} ants_status;

/* LRF parameterisations (Sec. 6.1.1 "Axial" and "XY", Sec. 6.1 3D). */
typedef enum {
    ANTS_LRF_RADIAL = 1, /* eta_i(x,y) = g_i f(|(x,y) - (X_i,Y_i)|), f a cubic B-spline in r */
    ANTS_LRF_XY = 2,     /* eta_i(x,y) = sum_jk c_ijk B_j(x) B_k(y), one tensor spline per sensor */
    ANTS_LRF_XYZ = 3,    /* eta_i(x,y,z) = sum_jkl c_ijkl B_j(x) B_k(y) B_l(z) */
    /* ants_lrf_create_scheme / ants_lrf_fit_scheme: */
    ANTS_LRF_COMPOSITE = 4, /* Sec. 6.1.1: eta_i(x,y) = A_i(r_i) + X_i(x,y), an axial and an XY spline */
    ANTS_LRF_AXIAL_Z = 5,   /* Sec. 6.1.2: eta_i(x,y,z) = one spline of (r_i, z) */
    ANTS_LRF_SLICED = 6     /* Sec. 6.1.2: XY splines on z planes, linear in z between the two closest */
} ants_lrf_type;

/* Per-event status codes written by the reconstruction calls. */
typedef enum {
    ANTS_EVT_OK = 0,
    ANTS_EVT_FALLBACK = 1,      /* reserved: event re-run by a fallback search */
    ANTS_EVT_ZERO_SIGNAL = 2,   /* sum of signals <= 0: outputs NaN */
    ANTS_EVT_BAD_SIGNAL = 3,    /* a signal is negative, NaN or infinite: outputs NaN */
    ANTS_EVT_OUT_OF_DOMAIN = 4, /* the start position lies outside the LRF domain: outputs NaN */
    ANTS_EVT_LOW_LOGL = 5       /* reserved: logL below a threshold */
} ants_evt_status;

/* Reconstruction methods. */
typedef enum {
    ANTS_CGS_PLAIN = 0, /* contracting grids, FP32, all sensors (Sec. 5.1.2.2) */
    ANTS_GEMM_TOPK = 1, /* global-grid tensor-core scores, top-K, local contracting grids */
    ANTS_MLP_SEEDED = 2, /* network proposal + local contracting grids + plain fallback */
    ANTS_CGS_VARIANT = 3, /* contracting grids with another criterion, start or sensor selection */
    ANTS_MINIMIZE = 4     /* continuous minimisation of the match (Sec. 5.1.2.1) */
} ants_method;

/* Match criterion of ANTS_CGS_VARIANT (Sec. 5.1.2). */
typedef enum { ANTS_CRIT_ML = 0, ANTS_CRIT_LS = 1 } ants_criterion;

/* Start position of ANTS_CGS_VARIANT (Sec. 5.1.2.1, 5.1.2.2). */
typedef enum { ANTS_START_COG = 0, ANTS_START_MAX_SENSOR = 1 } ants_start_mode;

/* Signal element types. */
/* Element type of signal arrays: FP32, or FP16 (IEEE binary16; widened to
 * FP32 on the device before the search, exactly). */
typedef enum { ANTS_F32 = 0, ANTS_F16 = 1, ANTS_F64 = 2 } ants_dtype;

typedef struct ants_ctx ants_ctx;
typedef struct ants_detector ants_detector;
typedef struct ants_lrf ants_lrf;
typedef struct ants_mlp ants_mlp;
typedef struct ants_batch_plan ants_batch_plan;
typedef struct ants_logtable ants_logtable;

/* Parameters of the contracting-grid search (Sec. 5.1.2.2).
 * The grid has n_xy x n_xy (x n_z) nodes centred on the current centre with
 * spacing step_xy (step_z); flat node index k = (iz*n_xy + iy)*n_xy + ix.
 * After each of `iters` grids the best node (maximum likelihood, ties to
 * the lowest k) becomes the centre and the spacings are multiplied by
 * `shrink`.  The result is the best node of the last grid.
 * n_xy, n_z odd; n_xy in [3, 15], n_z in [1, 15] (n_z = 1 unless the LRF is
 * ANTS_LRF_XYZ); iters in [1, 32]; 0 < shrink < 1; step_xy > 0; z0 is the
 * start z for XYZ LRFs. */
typedef struct {
    int n_xy;
    int n_z;
    int iters;
    float shrink;
    float step_xy;
    float step_z;
    float z0;
} ants_cgs_params;

/* Learned proposal network (the neural-network reconstruction role of
 * Sec. 5.1.3): u = s / sum(s); h1 = GELU(W1 u + b1); h2 = GELU(W2 h1 + b2);
 * o = W3 h2 + b3, GELU(x) = x Phi(x).  Outputs: o0 = x / xy_scale,
 * o1 = y / xy_scale, o2 = (ln E - loge_mean) / loge_std. */
typedef struct {
    int n_hidden;    /* width of both hidden layers, 4..1024 */
    float xy_scale;  /* > 0 */
    float loge_mean;
    float loge_std;  /* > 0 */
} ants_mlp_config;

/* Training settings (Adam on FP32 master weights; Sec. 5.1.3: the last
 * monitor_frac of the events is held out and training stops when its error
 * has not improved by 0.1 % for `patience` epochs; the best weights are kept). */
typedef struct {
    int epochs;          /* maximum number of epochs */
    int batch;           /* events per step, 1..65536 */
    float lr, beta1, beta2, eps;
    float monitor_frac;  /* in (0, 1) */
    int patience;        /* >= 1 */
    int bf16;            /* 1: BF16 matrix-product operands, FP32 accumulation */
    uint64_t seed;       /* shuffling */
} ants_train_params;

typedef struct {
    int epochs_run;
    int best_epoch;
    float best_monitor_mse;
    float last_train_mse;
} ants_train_report;

/* Synthetic event source (ants_simulate_events). */
typedef struct {
    int region;      /* 0: disk of radius `extent`, 1: square of half-width `extent` */
    float extent;    /* mm, >= 0 */
    float cx, cy;    /* centre of the region */
    float z_lo, z_hi;/* source depth range (XYZ LRFs only) */
    float e0;        /* mean number of photons (> 0) */
    float e_spread;  /* E uniform in e0 (1 +- e_spread), 0 <= e_spread < 1 */
    float spe_sigma; /* relative width of the single photo-electron response (0: counts) */
} ants_sim_params;

/* Parameters of ANTS_GEMM_TOPK: every event is scored at every point of the
 * table's global grid with one BF16 tensor-core product (FP32 accumulation),
 * the top_k points (1..8) are kept, candidates within nms_cells grid cells
 * (Chebyshev distance) of a better one are dropped, each remaining one
 * starts the `refine` search, and the result with the largest logL wins. */
typedef struct {
    const ants_logtable *table;
    int top_k;
    float nms_cells;
    ants_cgs_params refine;
} ants_gemm_params;

/* Parameters of ANTS_CGS_VARIANT: the contracting grids of `grid` with
 *   criterion: ANTS_CRIT_ML, maximum likelihood (the score of ANTS_CGS_PLAIN
 *     over the sensors in the match), or ANTS_CRIT_LS, least squares read as
 *     Pearson's statistic sum (s_i - E eta_i)^2 / (E eta_i) with the node's
 *     energy ratio E = sum s / sum eta over the sensors in the match
 *     (smallest wins);
 *   start: ANTS_START_COG, the centroid of the non-passive sensors with the
 *     detector's relative gains, or ANTS_START_MAX_SENSOR, the position of the
 *     non-passive sensor with the largest s_i / g_i (ties: lowest index);
 *     clamped into the XY box of an XY / XYZ LRF;
 *   the sensors in the match: the non-passive ones (passive_host[i] != 0,
 *     Sec. 5.3: never read, not even for the status), without those whose
 *     signal is below min_signal (when > 0) or whose distance from the start
 *     exceeds max_distance (when > 0) (Sec. 5.1.2).
 * E is S / H and logL the full Poisson log-likelihood over the sensors in the
 * match.  Status: BAD_SIGNAL for a negative or non-finite non-passive
 * signal, ZERO_SIGNAL when the non-passive or the matched signals sum to 0,
 * OUT_OF_DOMAIN when an LRF in the match is undefined at the start.  At most
 * 1024 sensors; every LRF type; no start_xyz (the variant picks its start);
 * the trace is supported.  Every node is evaluated on its own (no separable
 * form), so variants run slower than ANTS_CGS_PLAIN. */
typedef struct {
    ants_cgs_params grid;
    int criterion;
    int start;
    float min_signal;
    float max_distance;
    const unsigned char *passive_host; /* nullable, [n_sensors], read during the call */
} ants_cgs_variant_params;

/* Parameters of ANTS_MINIMIZE (Sec. 5.1.2.1: the match is minimised over
 * the two or three coordinates by a gradient method, from the centroid or the
 * strongest sensor; the paper uses Minuit2's Migrad): damped Fisher scoring
 * (Levenberg-Marquardt) with the energy profiled out, E = S / H at every
 * position.  The criterion, the start and the sensors in the match are those
 * of ants_cgs_variant_params; start_xyz_dev, when given, starts every event
 * instead (e.g. from a contracting-grid result: a continuous refine).
 * Each trial at p solves (J + lambda diag J) delta = g, with J = E sum_A
 * (grad eta_i - eta_i grad H / H)(...)^T / eta_i the Fisher information of
 * the position and g = grad F (maximum likelihood) or -grad chi^2 / 2 (least
 * squares), over x, y and, for a 3D LRF with fit_z, z; q = p + delta is
 * moved onto the domain's box (XY box, z range) and accepted when every LRF
 * in the match is defined there and the match improves: by the sign of the
 * change when it exceeds tau = 2^-18 S, else by the sign of (g(p) + g(q)) .
 * (q - p).  An accepted trial divides lambda by 10 (floor 1e-12) and ends
 * the minimisation when |q - p| < tol; a rejected one multiplies lambda by
 * 10 and ends it above 1e8.  At most max_iter trials.
 * Outputs as for the other methods; trace_dev, when given, is [n_events][1]
 * int16: the trials used, negative when max_iter ran out first (0 for
 * events that were not minimised).  Status as for ANTS_CGS_VARIANT (with a
 * given start: OUT_OF_DOMAIN when an LRF in the match is undefined there).
 * Every LRF type; at most 1024 sensors. */
typedef struct {
    int criterion;           /* ANTS_CRIT_ML or ANTS_CRIT_LS */
    int start;               /* ANTS_START_COG or ANTS_START_MAX_SENSOR (no start_xyz_dev) */
    float z0;                /* start z of a 3D LRF (no start_xyz_dev) */
    int fit_z;               /* 3D LRFs: 1 = z is fitted, 0 = z stays at the start */
    int max_iter;            /* >= 1 trials */
    float tol;               /* > 0, mm */
    float lambda0;           /* >= 0, initial damping (e.g. 1e-3) */
    float min_signal;        /* as ants_cgs_variant_params */
    float max_distance;
    const unsigned char *passive_host; /* nullable, [n_sensors], read during the call */
} ants_minimize_params;

/* Parameters of ANTS_MLP_SEEDED: the network's (x, y), clamped into the LRF's
 * XY box, starts the `refine` search; events whose Poisson deviance
 * D = 2 sum_i [s_i ln(s_i/mu_i) - (s_i - mu_i)] exceeds deviance_max (> 0
 * enables the test), whose final refine node lies on the border of the last
 * grid (border_fallback = 1), or whose start is outside the domain, are
 * searched again with `fallback` from the centroid (status ANTS_EVT_FALLBACK).
 * The call waits for the count of flagged events before it launches the
 * fallback search.  XY and RADIAL LRFs. */
typedef struct {
    const ants_mlp *mlp;
    int bf16;                 /* network precision at inference */
    ants_cgs_params refine;   /* e.g. 5 x 5 nodes, 4 grids */
    ants_cgs_params fallback; /* e.g. the plain 11 x 11 x 8 search */
    float deviance_max;
    int border_fallback;
} ants_mlp_seeded_params;

/* Event cuts (Sec. 5.2: events are filtered on the reconstruction's
 * chi-squared, its energy, the sum of the signals and the position; Sec. 8:
 * the iterative procedure discards badly reconstructed events with them).
 * A cut is off when chi2_max <= 0, r_max <= 0, or a window's upper bound is
 * not above its lower bound.  Bounds are inclusive; comparisons are made in
 * FP64 on the FP32 values. */
typedef struct {
    double chi2_max;       /* chi2 <= chi2_max */
    double e_lo, e_hi;     /* e_lo <= E <= e_hi */
    double sum_lo, sum_hi; /* sum_lo <= sum of the signals <= sum_hi */
    double r_max, cx, cy;  /* (x - cx)^2 + (y - cy)^2 <= r_max^2 */
} ants_event_cuts;

/* LRF refit from reconstructed events (ants_lrf_refit). */
typedef struct {
    int shared;          /* RADIAL: 1 one group (a profile times per-sensor gains, Sec. 6.2), 0 per sensor */
    int refit_gains;     /* RADIAL group: refit the gains with the new profile fixed (Sec. 6.3) */
    double shift_sigma;  /* > 0: add normal offsets of this standard deviation (mm) to x and y (Sec. 8) */
    uint64_t seed;       /* Philox key of the offsets */
    int cycle;           /* counter word of the offsets (the cycle number of an iteration) */
    double ridge;        /* as ants_lrf_fit */
} ants_refit_params;

/* Iterative LRF reconstruction (ants_lrf_iterate, Sec. 8). */
typedef struct {
    ants_cgs_params cgs;   /* the reconstruction of every cycle (plain contracting grids) */
    int cycles;            /* >= 1 */
    ants_event_cuts cuts;
    int refit_gains;       /* RADIAL group: refit the gains every cycle */
    double shift_sigma;    /* random shift (mm) of the kept positions ... */
    int shift_cycles;      /* ... during the first shift_cycles cycles */
    uint64_t seed;
    double ridge;
    int method;                    /* the reconstruction of every cycle: ANTS_CGS_PLAIN (cgs) or ANTS_MINIMIZE */
    ants_minimize_params minimize; /* with ANTS_MINIMIZE (from its own start, no start_xyz) */
} ants_iter_params;

/* Per-cycle record of ants_lrf_iterate. */
typedef struct {
    long n_kept;            /* events that passed the cuts and entered the refit */
    double mean_chi2;       /* their mean chi-squared (under the cycle's input LRFs) */
    double mean_E;          /* their mean energy */
    double rel_change;      /* relative RMS change of the LRFs where the data are:
                               sqrt(sum (eta_new - eta_old)^2 / sum eta_old^2) over the kept
                               events (at their reconstructed positions) and all sensors */
} ants_iter_stats;

/* ------------------------------------------------------------------------ */
/* Library and context                                                        */
/* ------------------------------------------------------------------------ */

/* Message for the calling thread's last non-OK return ("" if none).  The
 * string stays valid until the thread's next ants_* call. */
ANTS_API const char *ants_last_error(void);

/* ABI version of this header (increases on incompatible changes). */
ANTS_API int ants_version(void);

/* Create a context on CUDA device `device` (makes it current for the
 * calling thread).  *out receives the handle.  Errors: ANTS_E_ARG (null
 * out, bad device), ANTS_E_CUDA. */
ANTS_API int ants_ctx_create(int device, ants_ctx **out);

/* Release a context and the device buffers it owns (NULL is a no-op).  The
 * caller must have synchronised all streams that used it. */
ANTS_API void ants_ctx_destroy(ants_ctx *ctx);

/* Read and clear the context's device fault word (no counterpart in the
 * paper; robustness of the tensor-core kernels).  Synchronises the device,
 * stores 1 in *fault if a kernel launched through this context gave up a
 * bounded device-side wait since the last call (its outputs are then
 * undefined) and returns ANTS_E_TIMEOUT; otherwise stores 0, returns ANTS_OK. */
ANTS_API int ants_ctx_fault(ants_ctx *ctx, int *fault);

/* Self-test of that mechanism (no counterpart in the paper): launches a small
 * tensor-core top-K product whose TMA producer is held back, so that its MMA
 * thread's wait runs out after 1 s; the kernel must stop, drain, free its
 * tensor memory and set the fault word, and a normal launch on the same
 * context must then give the right answer.  Synchronous (about 1 s); faults,
 * traps and hangs nothing.  Returns ANTS_OK when all of that holds,
 * ANTS_E_INTERNAL otherwise; it clears the fault word. */
ANTS_API int ants_selftest_stalled_product(ants_ctx *ctx);

/* Build options of the loaded library (no counterpart in the paper):
 * ANTS_BUILD_DEBUG_BOUNDS set when it was compiled with ANTS_DEBUG_BOUNDS. */
#define ANTS_BUILD_DEBUG_BOUNDS 1
ANTS_API int ants_build_flags(void);

/* Index checks of the ANTS_DEBUG_BOUNDS build (no counterpart in the paper;
 * it stands in for a memory checker).  In that build the search kernels
 * (separable XY team kernel, small-grid patch kernel) and the tensor-core
 * product check their shared-memory, tensor-memory and global indices against
 * the buffers' extents; an index out of range is not accessed, and the number
 * of the first failing check site goes to a per-context device word, after
 * which ants_reconstruct, ants_logtable_topk and ants_mlp_train return
 * ANTS_E_INTERNAL (they synchronise in that build).  This call synchronises
 * the device, stores the recorded site in *site (0: none; always 0 in the
 * normal build) and clears it.  Errors: ANTS_E_ARG, ANTS_E_CUDA. */
ANTS_API int ants_debug_bounds_site(ants_ctx *ctx, int *site);

/* Self-test of the index checks (no counterpart in the paper): one thread
 * checks the index 7 against an extent of 5 at site 9999 and performs no
 * access.  The debug build must then report site 9999 through
 * ants_debug_bounds_site; the normal build reports 0.  Synchronous. */
ANTS_API int ants_selftest_bounds(ants_ctx *ctx);

/* ------------------------------------------------------------------------ */
/* Detector definition (Sec. 2 "detector definitions"; Sec. 5.1.1 gains)      */
/* ------------------------------------------------------------------------ */

/* Describe a planar sensor array: sensor_xy_host[n_sensors][2] sensor
 * centres (mm, row-major), rel_gain_host[n_sensors] the relative gains g_i
 * used by the centroid x = sum X_i S_i/g_i / sum S_i/g_i (Sec. 5.1.1,
 * centroid equation); NULL means g_i = 1.  Gains must be > 0.  Data are
 * copied.  n_sensors in [1, 1024].  Errors: ANTS_E_ARG. */
ANTS_API int ants_detector_create(int n_sensors, const double *sensor_xy_host,
                                  const double *rel_gain_host, ants_detector **out);
ANTS_API void ants_detector_free(ants_detector *det);

/* ------------------------------------------------------------------------ */
/* Light response functions (Sec. 6, 6.1, 6.2)                               */
/* ------------------------------------------------------------------------ */

/* Build an LRF set from FP64 B-spline coefficients.
 * type: ants_lrf_type.  Axis a (a < dims; dims = 1 radial, 2 XY, 3 XYZ) has
 * n_int[a] uniform intervals on [lo[a], hi[a]] and n_int[a] + 3 cubic
 * B-spline coefficients (knots lo + (j-3)h, j = 0..n+6).  For RADIAL, axis 0
 * is r = distance in the sensor plane, with lo[0] = 0.
 * coef_host: [n_sets][n_coef] with n_coef = prod_a (n_int[a] + 3), x index
 * fastest, then y, then z; n_sets = 1 when `shared` (one group, Sec. 6.2:
 * one LRF for all sensors times gain_host[i]) else n_sensors.  shared is
 * allowed for RADIAL only.  gain_host (RADIAL only, nullable = 1) scales
 * sensor i's LRF.  n_int[a] in [1, 256]; lo < hi.
 * The coefficients are kept in FP64 on the host and uploaded as FP32.
 * Errors: ANTS_E_ARG, ANTS_E_OOM, ANTS_E_CUDA. */
ANTS_API int ants_lrf_create(ants_ctx *ctx, const ants_detector *det, int type, const int *n_int,
                             const double *lo, const double *hi, int shared,
                             const double *coef_host, const double *gain_host, ants_lrf **out);

/* Fit an LRF set by FP64 least squares on the device and return it as
 * ants_lrf_create would (Sec. 6: LRFs are computed from datasets of source
 * positions and sensor signals; Sec. 6.2: one group shares one LRF).
 * pts_host [n_pts][dims] FP64 sample positions (RADIAL: r; XY: x, y; XYZ:
 * x, y, z), vals_host [n_pts][n_sets] FP64 values, n_sets = 1 when `shared`
 * else n_sensors.  Grid arguments as in ants_lrf_create.  Solves
 * (B^T B + ridge I) c = B^T v per value set with a square-root-free
 * Cholesky (L D L^T) factorisation of the banded normal matrix; when it is
 * not positive definite (a region without samples) the solve is retried
 * once with ridge = 1e-10 trace(B^T B) / n_coef.  *ridge_used (nullable)
 * receives the ridge applied.  Samples outside the domain are ignored.
 * Synchronous; the result is bitwise reproducible.
 * Errors: ANTS_E_ARG, ANTS_E_LRF (still singular), ANTS_E_OOM, ANTS_E_CUDA. */
ANTS_API int ants_lrf_fit(ants_ctx *ctx, const ants_detector *det, int type, const int *n_int,
                          const double *lo, const double *hi, int shared, long n_pts,
                          const double *pts_host, const double *vals_host, double ridge,
                          double *ridge_used, ants_lrf **out);

/* A grouped RADIAL LRF set (Sec. 6.2: sensors of a group share one LRF
 * profile; each keeps its relative gain): group_host[i] in [0, n_groups) is
 * the group of sensor i, coef_host [n_groups][n_int[0] + 3] the groups'
 * profiles (FP64, uploaded as FP32), gain_host (nullable, default 1) the
 * per-sensor gains multiplying them.  Knot grid as ants_lrf_create.  Usable
 * wherever a RADIAL set is (search, simulation, evaluation, forms, refit and
 * iteration); not saved (ANTS_E_UNIMPLEMENTED).  Errors: ANTS_E_ARG,
 * ANTS_E_OOM, ANTS_E_CUDA. */
ANTS_API int ants_lrf_create_grouped(ants_ctx *ctx, const ants_detector *det, const int *n_int, const double *lo,
                                     const double *hi, int n_groups, const int *group_host, const double *coef_host,
                                     const double *gain_host, ants_lrf **out);

/* An XY LRF set with symmetry classes (Sec. 6.2: sensors related by a
 * rotation or reflection of the array share one LRF): class_host[i] in [0,
 * n_classes) is sensor i's class, op_host[i] in [0, 24) its operation M
 * (the rotation by (op mod 12) x 30 degrees, preceded for op >= 12 by the
 * reflection y -> -y) about centre[2]; coef_host [n_classes][n_coef] the
 * classes' XY LRFs in their representatives' frames, gain_host (nullable)
 * per-sensor gains.  eta_i(p) = g_i F_class(i)(M_i^T (p - c) + c); a point is
 * inside the domain when every mapped point lies in the XY box.  Used by the
 * plain search (through the per-node kernel), the variants, the
 * minimisation, the simulator, evaluation, the refit (each class refitted to
 * its members' mapped samples, gains kept) and the iteration; not by the
 * precision and learned forms or batches, not saved (ANTS_E_UNIMPLEMENTED).
 * Errors: ANTS_E_ARG, ANTS_E_OOM, ANTS_E_CUDA. */
ANTS_API int ants_lrf_create_symmetric(ants_ctx *ctx, const ants_detector *det, const int *n_int, const double *lo,
                                       const double *hi, int n_classes, const int *class_host, const int *op_host,
                                       const double *centre, const double *coef_host, const double *gain_host,
                                       ants_lrf **out);

/* Fit an XY LRF set with symmetry classes from samples (Sec. 6.2): each
 * class's LRF by FP64 least squares (as ants_lrf_fit) to its members'
 * samples mapped into the representative's frame, M_i^T (p - c) + c, with
 * values vals_host[e][i] / gain_host[i] (gains nullable = 1); mapped points
 * outside the XY box are left out.  pts_host [n_pts][2], vals_host
 * [n_pts][n_sensors]; classes and operations as ants_sensor_symmetry gives
 * them.  Errors: as ants_lrf_fit. */
ANTS_API int ants_lrf_fit_symmetric(ants_ctx *ctx, const ants_detector *det, const int *n_int, const double *lo,
                                    const double *hi, int n_classes, const int *class_host, const int *op_host,
                                    const double *centre, long n_pts, const double *pts_host,
                                    const double *vals_host, const double *gain_host, double ridge, ants_lrf **out);

/* Classes by the rotation and reflection symmetry of the array (Sec. 6.2):
 * the centre is the mean sensor position; an operation (as above) is a
 * symmetry when it maps every sensor within tol of a sensor; sensors in index
 * order open a class unless already reached, and each symmetry (in table
 * order) maps the class's first sensor onto the unassigned sensor it reaches,
 * recording that operation.  Outputs class_host[n], op_host[n], centre_out[2],
 * *n_classes_out.  Host only.  Errors: ANTS_E_ARG. */
ANTS_API int ants_sensor_symmetry(const ants_detector *det, double tol, int *class_host, int *op_host,
                                  double *centre_out, int *n_classes_out);

/* Groups by distance from the array's centre (Sec. 6.2): the centre is the
 * mean sensor position; sensors in order of increasing distance d (ties by
 * index) start a new group when d exceeds the distance of the current
 * group's first sensor by more than tol (mm).  group_host [n_sensors]
 * receives each sensor's group (0 = innermost), *n_groups_out their count.
 * Host only.  Errors: ANTS_E_ARG. */
ANTS_API int ants_sensor_rings(const ants_detector *det, double tol, int *group_host, int *n_groups_out);

/* LRF sets of the other parameterisation schemes (Sec. 6.1.1, 6.1.2), one
 * coefficient set per sensor, coef_host [n_sensors][n_coef]:
 *   ANTS_LRF_COMPOSITE: the axial part, n_int_r + 3 coefficients of a cubic
 *     B-spline in r on [0, hi_r], followed by the XY part, (n_int[0] + 3) *
 *     (n_int[1] + 3) coefficients on the box lo[0..1] .. hi[0..1] (x
 *     fastest).  Defined where r <= hi_r and (x, y) is inside the box.
 *   ANTS_LRF_AXIAL_Z: one spline of (r, z): axis 0 = r on [0, hi[0]] (lo[0]
 *     must be 0) with n_int[0] intervals, axis 1 = z on [lo[1], hi[1]]; (n_int[0]
 *     + 3) * (n_int[1] + 3) coefficients, r fastest.
 *   ANTS_LRF_SLICED: n_planes (2..64) XY splines on the box lo[0..1] .. hi[0..1]
 *     with planes z_j = lo[2] + j (hi[2] - lo[2]) / (n_planes - 1); between
 *     two planes the value is (1 - w) f_j + w f_{j+1}; n_planes * (n_int[0] +
 *     3) * (n_int[1] + 3) coefficients, plane by plane.
 * Reconstruction with these sets evaluates every node on its own (the
 * per-node kernel of ANTS_CGS_VARIANT); the precision and learned forms, the
 * batched run, the iterative refit and save / load take the first three
 * types only.  Errors: ANTS_E_ARG, ANTS_E_OOM, ANTS_E_CUDA. */
ANTS_API int ants_lrf_create_scheme(ants_ctx *ctx, const ants_detector *det, int type, const int *n_int,
                                    const double *lo, const double *hi, int n_int_r, double hi_r, int n_planes,
                                    const double *coef_host, ants_lrf **out);

/* Fit an LRF set of one of those schemes by FP64 least squares on the device
 * (Sec. 6.1.1, 6.1.2).  pts_host [n_pts][d] (COMPOSITE: x, y; AXIAL_Z and
 * SLICED: x, y, z), vals_host [n_pts][n_sensors].  COMPOSITE: per sensor the
 * axial part is fitted first to (r_i, v_i), then the XY part to the residual
 * v_i - A_i(r_i) (a sample beyond the axial part's reach gives a zero
 * residual).  AXIAL_Z: per sensor one fit of (r_i, z).  SLICED: the XY
 * splines of plane j are fitted to the samples whose nearest plane is j.
 * Each fit retries with the ridge of ants_lrf_fit when singular.
 * Synchronous.  Errors: as ants_lrf_fit. */
ANTS_API int ants_lrf_fit_scheme(ants_ctx *ctx, const ants_detector *det, int type, const int *n_int,
                                 const double *lo, const double *hi, int n_int_r, double hi_r, int n_planes,
                                 long n_pts, const double *pts_host, const double *vals_host, double ridge,
                                 ants_lrf **out);

/* Copy the FP64 coefficients ([n_sets][n_coef]) to coef_host; `count` is
 * the capacity in doubles and must be >= n_sets*n_coef.  *n_sets_out and
 * *n_coef_out (nullable) receive the shape.  Errors: ANTS_E_ARG. */
ANTS_API int ants_lrf_coefficients(const ants_lrf *lrf, double *coef_host, size_t count,
                                   int *n_sets_out, int *n_coef_out);

/* Copy the per-sensor gain factors ([n_sensors]: a RADIAL LRF's factors,
 * 1 otherwise) to gain_host; `count` is the capacity in doubles and must be
 * >= n_sensors.  Errors: ANTS_E_ARG. */
ANTS_API int ants_lrf_gains(const ants_lrf *lrf, double *gain_host, size_t count);

/* Evaluate eta_i (the LRFs of Sec. 6, 6.1) at n_pts points for all sensors: pts_dev[n_pts][dim] FP32
 * (dim = 2 for RADIAL/XY, 3 for XYZ), out_dev[n_pts][n_sensors] FP32.
 * Points outside the LRF domain give NaN.  Asynchronous on `stream`.
 * Errors: ANTS_E_ARG, ANTS_E_CUDA. */
ANTS_API int ants_lrf_eval(const ants_lrf *lrf, const float *pts_dev, long n_pts, int dim,
                           float *out_dev, void *stream);

/* Save / load an LRF set (versioned little-endian binary file: header,
 * grid, gains, FP64 coefficients).  load binds the LRF to `det`, whose
 * sensor count must match the file.  Errors: ANTS_E_IO, ANTS_E_SHAPE,
 * ANTS_E_ARG, ANTS_E_OOM, ANTS_E_CUDA. */
ANTS_API int ants_lrf_save(const ants_lrf *lrf, const char *path);
ANTS_API int ants_lrf_load(ants_ctx *ctx, const ants_detector *det, const char *path,
                           ants_lrf **out);

ANTS_API void ants_lrf_free(ants_lrf *lrf);

/* ------------------------------------------------------------------------ */
/* Reconstruction (Sec. 5.1.2 maximum likelihood, 5.1.2.2 contracting grids)  */
/* ------------------------------------------------------------------------ */

/* Reconstruct n_events events.
 *   method: ANTS_CGS_PLAIN with params = const ants_cgs_params*,
 *     ANTS_GEMM_TOPK with params = const ants_gemm_params* (no start_xyz_dev,
 *     no trace_dev), or ANTS_MLP_SEEDED with params = const
 *     ants_mlp_seeded_params* (no start_xyz_dev; trace_dev then records the
 *     refine grids), ANTS_CGS_VARIANT with params = const
 *     ants_cgs_variant_params* (no start_xyz_dev), or ANTS_MINIMIZE with
 *     params = const ants_minimize_params* (trace_dev [n_events][1]).
 *   signals_dev: [n_events][n_sensors] row-major, element type signal_dtype
 *     (ANTS_F32, or ANTS_F16: widened to FP32 in library-owned device
 *     chunks of up to 2^20 events, so the results equal those of the FP32
 *     values); n_sensors must equal the LRF's.
 *   start_xyz_dev: nullable [n_events][3] FP32 start positions; NULL = the
 *     centroid (Sec. 5.1.1) clamped into the XY domain of an XY/XYZ LRF,
 *     with z = params->z0 (Sec. 5.1.2.1 start options).
 *   Outputs (FP32 unless stated): xyz_dev [n_events][3] (z = 0 for 2D
 *   LRFs), E_dev [n_events] = sum s / sum eta at the result (Sec. 5.1.2.2),
 *   logL_dev [n_events] = sum_i [s_i ln mu_i - mu_i - lgamma(s_i+1)] with
 *   mu_i = E eta_i (Poisson), status_dev [n_events] int32 ants_evt_status.
 *   trace_dev: nullable [n_events][iters] int16, the flat index of the node
 *   chosen on each grid (-1 for events that were not searched).
 * The likelihood is Poisson with the energy profiled out: each node scores
 * F = sum_i s_i ln eta_i - S ln sum_i eta_i (S = sum s), eta_i floored at
 * 1e-30; nodes outside the LRF domain score -inf (RADIAL: every sensor
 * within r <= hi[0]; XY/XYZ: inside the box).
 * n_events == 0 is a no-op.  Asynchronous on `stream`.
 * Errors: ANTS_E_ARG, ANTS_E_SHAPE, ANTS_E_UNIMPLEMENTED, ANTS_E_CUDA. */
ANTS_API int ants_reconstruct(ants_ctx *ctx, const ants_lrf *lrf, int method, const void *params,
                              const void *signals_dev, int signal_dtype, long n_events,
                              int n_sensors, const float *start_xyz_dev, float *xyz_dev,
                              float *E_dev, float *logL_dev, int32_t *status_dev,
                              int16_t *trace_dev, void *stream);

/* The same reconstruction with HOST buffers (signals_host [n_events]
 * [n_sensors], outputs xyz_host [n_events][3], E_host, logL_host,
 * status_host; nullable start_xyz_host, plain search and minimisation only),
 * any method.
 * The library streams the events through device buffers owned by the
 * context in chunks; for the plain search it overlaps the host-to-device
 * copy, the search and the device-to-host copy on two internal streams, for
 * the two forms (which use the context's scratch buffers) the chunks run in
 * turn.  Page-locked host memory gives full copy bandwidth.
 * Synchronous: returns when the outputs are in host memory.
 * Errors: as ants_reconstruct, plus ANTS_E_OOM. */
ANTS_API int ants_reconstruct_host(ants_ctx *ctx, const ants_lrf *lrf, int method,
                                   const void *params, const void *signals_host, int signal_dtype,
                                   long n_events, int n_sensors, const float *start_xyz_host,
                                   float *xyz_host, float *E_host, float *logL_host,
                                   int32_t *status_host);

/* Poisson deviance D = 2 sum_i [s_i ln(s_i/mu_i) - (s_i - mu_i)] (s_i = 0:
 * 2 mu_i) with mu_i = E eta_i(xyz) and E = S/H, for each event at the given
 * position xyz_dev [n_events][3] -- a goodness-of-fit statistic for the
 * event filters of Sec. 5.2.  D_dev [n_events]; NaN where xyz is outside the
 * LRF domain.  Asynchronous on `stream`. */
ANTS_API int ants_deviance(ants_ctx *ctx, const ants_lrf *lrf, const float *signals_dev, long n_events,
                           int n_sensors, const float *xyz_dev, float *D_dev, void *stream);

/* Simulate events first_event .. first_event + n_events - 1 from an LRF set:
 * source uniform in the region (z uniform in [z_lo, z_hi] for XYZ LRFs, else
 * 0), energy E uniform in e0 (1 +- e_spread), signal of sensor i Poisson with
 * mean E eta_i(source) (the mean response an LRF describes, Sec. 6) and, with
 * spe_sigma > 0, each photo-electron contributing N(1, spe_sigma^2) (the
 * normal single photo-electron response of Sec. 4.2.5), clamped at 0.
 * Random numbers: Philox4x32-10 keyed by `seed`; event e uses counters
 * (e, 0xFFFFFFFF, *) for its source and (e, i, *) for sensor i, so any range
 * of events can be generated independently and reproducibly.
 * signals_dev [n_events][n_sensors] FP32; truth_dev (nullable)
 * [n_events][4] = (x, y, z, E).  Asynchronous on `stream`. */
ANTS_API int ants_simulate_events(ants_ctx *ctx, const ants_lrf *lrf, const ants_sim_params *params,
                                  uint64_t seed, long first_event, long n_events, float *signals_dev,
                                  float *truth_dev, void *stream);

/* ------------------------------------------------------------------------ */
/* Global-grid log-response table (precision form)                           */
/* ------------------------------------------------------------------------ */

/* Tabulate T[g][i] = ln p_i(g) - m_i on the nx x ny cell centres g of an XY
 * LRF's box, p_i = eta_i / sum_j eta_j and m_i = mean_g ln p_i(g), stored as
 * BF16 [nx*ny][n_sensors].  With the energy profiled out (E = S/H,
 * Sec. 5.1.2.2) the Poisson log-likelihood of an event at g is
 * sum_i s_i ln p_i(g) plus a term of the event alone, so the scores
 * sum_i s_i T[g][i] rank the grid points exactly as the likelihood does (the
 * m_i shift every score of an event equally and keep |T| small for BF16).
 * Synchronous.  XY LRFs, n_sensors a multiple of 8, nx*ny <= 2^20. */
ANTS_API int ants_logtable_create(ants_ctx *ctx, const ants_lrf *lrf, int nx, int ny, ants_logtable **out);

/* Copy the table as FP32 (table_host [nx*ny][n_sensors], nullable) and the
 * centring constants m (mean_host [n_sensors], nullable).  Synchronous.
 * Errors: ANTS_E_ARG, ANTS_E_CUDA. */
ANTS_API int ants_logtable_values(const ants_logtable *table, float *table_host, float *mean_host);

/* Top-K grid points of each event by score sum_i s_i T[g][i] (the profiled
 * likelihood of Sec. 5.1.2, 5.1.2.2 ranked over a global grid): score_dev and
 * index_dev [n_events][top_k], descending score, ties to the lower index,
 * top_k in [1, 8].  Signals FP32 (rounded to BF16 for the product).
 * Asynchronous.  A bounded device-side wait that runs out sets the context's
 * fault word (ants_ctx_fault); the outputs are then undefined.
 * Errors: ANTS_E_ARG, ANTS_E_SHAPE (n_sensors differs from the table's),
 * ANTS_E_CUDA. */
ANTS_API int ants_logtable_topk(ants_ctx *ctx, const ants_logtable *table, const float *signals_dev,
                                long n_events, int n_sensors, int top_k, float *score_dev,
                                int32_t *index_dev, void *stream);
ANTS_API void ants_logtable_free(ants_logtable *table);

/* ------------------------------------------------------------------------ */
/* Batched reconstruction of several detectors in one persistent launch      */
/* ------------------------------------------------------------------------ */

/* One detector's share of a batch: its LRF set (with the detector bound to
 * it), search settings, device signals and outputs as in ants_reconstruct. */
typedef struct {
    const ants_lrf *lrf;
    ants_cgs_params params;
    const float *signals_dev;    /* [n_events][n_sensors of the LRF] */
    long n_events;
    const float *start_xyz_dev;  /* nullable */
    float *xyz_dev;
    float *E_dev;
    float *logL_dev;
    int32_t *status_dev;
    int16_t *trace_dev;          /* nullable [n_events][iters] */
} ants_batch_item;

/* Launch shape of a batch: events per work unit, warps per block (1..8),
 * blocks per SM (1..32). */
typedef struct {
    int unit_events;
    int warps_per_block;
    int blocks_per_sm;
} ants_batch_config;

/* Build a plan: the work units (unit_events events of one detector each)
 * sorted by cost (nodes x iterations x sensors x events) largest first, and a
 * CUDA graph that resets a work counter and launches one persistent kernel in
 * which every warp takes units from that counter and runs the per-event
 * contracting-grid search of the unit's detector (Sec. 5.1.2.2; any mix of
 * RADIAL, XY and XYZ LRFs).  Items and their buffers must outlive the plan.
 * cfg nullable (16 events per unit, 8 warps per block, 4 blocks per SM).
 * Errors: ANTS_E_ARG, ANTS_E_CUDA, ANTS_E_OOM. */
ANTS_API int ants_batch_plan_create(ants_ctx *ctx, int n_items, const ants_batch_item *items,
                                    const ants_batch_config *cfg, ants_batch_plan **out);

/* Launch the plan's graph on `stream` (asynchronous).  Calls with one plan
 * must not overlap (they share the work counter).
 * Errors: ANTS_E_ARG, ANTS_E_CUDA. */
ANTS_API int ants_batch_run(ants_batch_plan *plan, void *stream);

/* Choose the launch shape: time every candidate (units of 4/16/64 events,
 * 4/8 warps per block, 2/4/8 blocks per SM) on the first events_per_item
 * events of every detector (<= 0: 2048) and keep the fastest.  With
 * cache_path, a previous choice for the same batch signature is reused, and
 * a new choice is appended to that text file.  Synchronous.  The plan is
 * rebuilt with the choice; *chosen (nullable) receives it.  A cache file
 * that cannot be opened is skipped (no error).  get_config copies the plan's
 * current shape.  Errors: ANTS_E_ARG, ANTS_E_OOM, ANTS_E_CUDA. */
ANTS_API int ants_batch_autotune(ants_batch_plan *plan, const char *cache_path, long events_per_item,
                                 ants_batch_config *chosen);
ANTS_API int ants_batch_get_config(const ants_batch_plan *plan, ants_batch_config *cfg);
ANTS_API void ants_batch_plan_free(ants_batch_plan *plan);

/* ------------------------------------------------------------------------ */
/* Learned proposal network                                                  */
/* ------------------------------------------------------------------------ */

/* Create a network for n_in inputs (the sensor count) with He-normal hidden
 * and Xavier-normal output weights from `seed`, zero biases.  The network
 * plays the part of the neural-network reconstruction of Sec. 5.1.3; the
 * paper does not specify its architecture.  Errors: ANTS_E_ARG, ANTS_E_OOM,
 * ANTS_E_CUDA. */
ANTS_API int ants_mlp_create(ants_ctx *ctx, int n_in, const ants_mlp_config *cfg, uint64_t seed,
                             ants_mlp **out);
ANTS_API void ants_mlp_free(ants_mlp *mlp);

/* Shape: inputs, hidden width, number of parameters (nullable outputs).
 * Errors: ANTS_E_ARG. */
ANTS_API int ants_mlp_shape(const ants_mlp *mlp, int *n_in, int *n_hidden, long *n_params);

/* FP32 parameters, concatenated in the order W1 [H][n_in], b1 [H],
 * W2 [H][H], b2 [H], W3 [3][H], b3 [3] (row-major [out][in]).  set resets the
 * optimiser state.  count must equal (get: be at least) n_params.
 * Synchronous.  Errors: ANTS_E_ARG, ANTS_E_CUDA. */
ANTS_API int ants_mlp_set_params(ants_mlp *mlp, const float *params_host, long count);
ANTS_API int ants_mlp_get_params(const ants_mlp *mlp, float *params_host, long count);

/* Network outputs for device signals [n_events][n_sensors]: out_dev
 * [n_events][3] raw outputs; start_xyz_dev (nullable) [n_events][3] =
 * (o0 xy_scale, o1 xy_scale, 0); E_dev (nullable, needs start_xyz_dev)
 * = exp(o2 loge_std + loge_mean).  Uses the context's device scratch.
 * Errors: ANTS_E_ARG, ANTS_E_SHAPE (n_sensors differs from n_in),
 * ANTS_E_OOM, ANTS_E_CUDA. */
ANTS_API int ants_mlp_forward(ants_ctx *ctx, const ants_mlp *mlp, const float *signals_dev,
                              long n_events, int n_sensors, int bf16, float *out_dev,
                              float *start_xyz_dev, float *E_dev, void *stream);

/* Mean squared error of the network on device signals and truth
 * [n_events][4] = (x, y, z, E), and its gradient (same layout as the
 * parameters) -- for checking the backward pass.  Synchronous.
 * Errors: ANTS_E_ARG, ANTS_E_SHAPE, ANTS_E_OOM, ANTS_E_CUDA. */
ANTS_API int ants_mlp_loss_grad(ants_ctx *ctx, const ants_mlp *mlp, const float *signals_dev,
                                const float *truth_dev, long n_events, int n_sensors, int bf16,
                                float *loss_host, float *grads_host);

/* Train on device signals and truth [n_events][4] (x, y, z, E).  The first
 * (1 - monitor_frac) of the events are shuffled into batches every epoch;
 * the rest is the monitor set.  Synchronous; bitwise reproducible for a
 * given seed.  report nullable.  Sec. 5.1.3: the training set is split
 * off a monitoring set against over-fitting.
 * Errors: ANTS_E_ARG, ANTS_E_SHAPE, ANTS_E_OOM, ANTS_E_CUDA. */
ANTS_API int ants_mlp_train(ants_ctx *ctx, ants_mlp *mlp, const float *signals_dev,
                            const float *truth_dev, long n_events, int n_sensors,
                            const ants_train_params *params, ants_train_report *report);

/* Save / load (versioned binary: header, config, FP32 parameters).
 * Errors: ANTS_E_ARG, ANTS_E_IO, ANTS_E_OOM, ANTS_E_CUDA. */
ANTS_API int ants_mlp_save(const ants_mlp *mlp, const char *path);
ANTS_API int ants_mlp_load(ants_ctx *ctx, const char *path, ants_mlp **out);

/* ------------------------------------------------------------------------ */
/* Reconstruction without device allocation                                   */
/* ------------------------------------------------------------------------ */

/* Bytes of the static device staging area behind
 * ants_reconstruct_host_noalloc (32 MiB). */
#define ANTS_NOALLOC_STAGE_BYTES 33554432

/* The plain contracting-grid search of ants_reconstruct_host, for callers
 * that must not allocate device memory.  The paper has no counterpart: this is a service of
 * the library, not a step of the method.
 *
 * Who needs it: programs that hand all device memory to their own pool (or
 * to another framework) at start-up, acquisition loops that cannot afford a
 * failed allocation or the device-wide synchronisation that cudaMalloc and
 * cudaFree may cause while data are streaming, and plug-ins whose host
 * application forbids allocating on its GPU.  This call stages signals and
 * results through a fixed area that the library declares statically, so it
 * calls neither cudaMalloc nor cudaFree nor any allocating library routine.
 *
 * Arguments and results are those of ants_reconstruct_host (host buffers;
 * synchronous: returns when the outputs are in host memory), restricted to
 * method ANTS_CGS_PLAIN and FP32 signals: the other methods and FP16 signals
 * return ANTS_E_UNIMPLEMENTED, because the two forms need scratch that
 * grows with the batch.  Limits and behaviour:
 *   - The staging area takes ANTS_NOALLOC_STAGE_BYTES of device memory on
 *     each GPU from the moment its module is loaded there until the process
 *     exits.  Under CUDA's default lazy module loading that is the first
 *     call of this entry point on the device (eager loading reserves it when
 *     the context is created).  A call with n_events = 0 (buffers may be
 *     NULL) does this set-up and nothing else: a caller that hands the rest
 *     of device memory to its own pool makes that call first.
 *   - The whole batch must fit it: 4*n_events*n_sensors bytes of signals,
 *     24*n_events bytes of results and, with start positions, 12*n_events
 *     more, each region rounded up to 256 bytes — about
 *     33,554,432 / (4*n_sensors + 24) events (119,835 for 64 sensors;
 *     114,910 with start positions).
 *     Larger batches are rejected with ANTS_E_ARG before any copy.
 *   - The first call on a device (with any n_events) looks up the area's
 *     device address with cudaGetSymbolAddress while that device is current
 *     and keeps it for the life of the process; make that first call before
 *     any stream capture begins.  A device reset (cudaDeviceReset) after
 *     that call is not supported: the kept address would be stale.
 *   - Every call uses the same area and leaves the last call's data in it;
 *     nothing in it has to start at zero.  Calls that overlap on the GPU (for
 *     example from two host threads on the same device at once) race on the
 *     area: serialise them.
 * Errors: as ants_reconstruct_host (ANTS_E_ARG also for a batch beyond the
 * capacity; ANTS_E_UNIMPLEMENTED for another method or signal type). */
ANTS_API int ants_reconstruct_host_noalloc(ants_ctx *ctx, const ants_lrf *lrf, int method,
                                           const void *params, const void *signals_host,
                                           int signal_dtype, long n_events, int n_sensors,
                                           const float *start_xyz_host, float *xyz_host,
                                           float *E_host, float *logL_host, int32_t *status_host);

/* ------------------------------------------------------------------------ */
/* Event filters (Sec. 5.2) and iterative LRF reconstruction (Sec. 8)         */
/* ------------------------------------------------------------------------ */

/* Centroid position (Sec. 5.1.1: x = sum X_i s_i/g_i / sum s_i/g_i with the
 * detector's relative gains g_i, sensor positions X_i) and the sum of the
 * signals of each event, as the start of an iterative reconstruction when no
 * LRF is known yet.  signals_dev [n_events][n_s] FP32; xyz_dev [n_events][3]
 * receives (x, y, 0) (NaN when the weighted sum is not > 0); sum_dev
 * [n_events] (nullable).  Accumulates in FP64.  Asynchronous on `stream`.
 * Errors: ANTS_E_ARG, ANTS_E_CUDA. */
ANTS_API int ants_event_centroid(ants_ctx *ctx, const ants_lrf *lrf, const float *signals_dev, long n_events,
                                 float *xyz_dev, float *sum_dev, void *stream);

/* Chi-squared of each event's reconstruction (Sec. 5.2): Pearson's
 * statistic sum_i (s_i - mu_i)^2 / mu_i with mu_i = E eta_i(xyz), over the
 * sensors with mu_i > 0, divided by n_s - 3 (x, y, E fitted; 1 when
 * n_s <= 3); NaN when the position or E is not finite.  FP32 (the terms'
 * differences are exact near the mean; a pairwise sum over the warp).  sum_dev (nullable) receives the sum of the
 * signals.  Asynchronous on `stream`.  Errors: ANTS_E_ARG, ANTS_E_CUDA. */
ANTS_API int ants_event_chi2(ants_ctx *ctx, const ants_lrf *lrf, const float *signals_dev, long n_events,
                             const float *xyz_dev, const float *E_dev, float *chi2_dev, float *sum_dev,
                             void *stream);

/* Select the events that were reconstructed (status ANTS_EVT_OK, finite
 * position, E and chi2) and pass every active cut (the event filters of
 * Sec. 5.2).  index_dev (capacity
 * n_events) receives the kept event indices in increasing order and
 * *n_kept_host their number.  sum_dev may be NULL when the signal-sum cut is
 * off.  Waits for the count (synchronises `stream`).
 * Errors: ANTS_E_ARG, ANTS_E_OOM, ANTS_E_CUDA. */
ANTS_API int ants_event_filter(ants_ctx *ctx, long n_events, const int32_t *status_dev, const float *xyz_dev,
                               const float *E_dev, const float *chi2_dev, const float *sum_dev,
                               const ants_event_cuts *cuts, int32_t *index_dev, long *n_kept_host, void *stream);

/* Refit `lrf` from reconstructed events (Sec. 6: LRFs from (position,
 * signal) data; Sec. 8: the positions are reconstructed ones).  The events
 * are index_dev[0..n_kept) (NULL: all n_events in order); event e gives the
 * value v_ei = s_ei / E_e of sensor i at its position, after adding the
 * seeded normal offset of (seed, cycle, e) to x and y when shift_sigma > 0
 * (Philox4x32-10 block at counter (e_lo, e_hi, 0xFFFFFFFE, cycle), Box-Muller
 * of its first two words, FP64).
 *   XY / XYZ: one FP64 least-squares fit, points (x, y[, z]), one value
 *     column per sensor.
 *   RADIAL with p->shared: one fit of the profile to every (r_ei, v_ei/g_i),
 *     r_ei the distance to sensor i, g_i the input's gains; with
 *     p->refit_gains the gains are then refitted with the new profile fixed,
 *     g_i = sum f(r) v / sum f(r)^2 (Sec. 6.3), and scaled to mean 1, the
 *     profile taking the inverse factor.
 *   RADIAL without p->shared: one fit of (r_ei, v_ei) per sensor, gains 1.
 *   RADIAL with sensor groups (ants_lrf_create_grouped; p->shared ignored):
 *     one fit per group of its sensors' (r_ei, v_ei/g_i); with
 *     p->refit_gains each sensor's gain against its group's new profile,
 *     scaled to mean 1 within the group (the group's profile taking the
 *     factor).  The output keeps the groups.
 *   XY with symmetry classes (ants_lrf_create_symmetric): one fit per class
 *     of its members' positions mapped into the class frame, values
 *     v_ei / g_i; gains and classes kept.
 * The output has the input's knot grid, sensors and relative gains.
 * Synchronous.  Errors: ANTS_E_ARG, ANTS_E_LRF (a fit stayed singular, e.g.
 * no events), ANTS_E_OOM, ANTS_E_CUDA. */
ANTS_API int ants_lrf_refit(ants_ctx *ctx, const ants_lrf *lrf, const float *signals_dev, long n_events,
                            const float *xyz_dev, const float *E_dev, const int32_t *index_dev, long n_kept,
                            const ants_refit_params *p, ants_lrf **out);

/* Iterative LRF reconstruction from flood data (Sec. 8): starting from
 * lrf_init, each of p->cycles cycles reconstructs all events with the current
 * LRFs (ants_reconstruct with p->method: ANTS_CGS_PLAIN and p->cgs, or
 * ANTS_MINIMIZE and p->minimize; the paper's procedure uses whichever
 * reconstruction is configured), computes their
 * chi-squared, keeps the events that pass p->cuts and refits the LRFs from
 * them (ants_lrf_refit with the input's grouping, p->refit_gains, the shift
 * during the first p->shift_cycles cycles with cycle = the cycle number, and
 * p->ridge).  stats_host (nullable) receives p->cycles records.  *out is a
 * new LRF set; lrf_init is not modified.  Synchronous; all work runs on the
 * context's first stream.  Errors: as the calls above; ANTS_E_LRF when a
 * cycle keeps no event. */
ANTS_API int ants_lrf_iterate(ants_ctx *ctx, const ants_lrf *lrf_init, const float *signals_dev, long n_events,
                              const ants_iter_params *p, ants_iter_stats *stats_host, ants_lrf **out);

/* Number of kernels the calling thread's last successful ants_* call
 * launched (for accounting in benchmarks). */
ANTS_API long ants_last_launch_count(void);

/* ------------------------------------------------------------------------ */
/* Optical photon transport (Sec. 4.2.3 photon tracing, 4.2.4 detection,     */
/* 4.2.6 pre-rejection, Sec. 3.5 custom interface properties)                */
/* ------------------------------------------------------------------------ */

#define ANTS_OPT_MAX_LAYERS 8

/* A stack of horizontal slabs, laterally bounded by |x| <= half_x, |y| <=
 * half_y (photons crossing those walls leave the geometry).  Layer k lies
 * between z[k] < z[k+1] (mm) and has refractive index n[k], absorption
 * length abs_len[k] and Rayleigh mean free path ray_len[k] (mm; 0 = none).
 * Below z[0] and above z[n_layers] are media of index n_below and n_above
 * (photons refracted into them leave the stack).  Boundary b (0..n_layers)
 * has custom probabilities p_abs[b] (absorption), p_spec[b] (specular
 * reflection) and p_diff[b] (Lambertian reflection), applied before Fresnel
 * (sum <= 1; the rest goes to Fresnel).  Sensors: square windows of side
 * sensor_size centred at sensor_xy_host[i] on the bottom boundary z[0], of
 * index n_sensor, with quantum efficiency qe_host[i] and, when n_ang >= 2, a
 * relative angular response ang_host[j] at incidence theta_j = j (pi/2) /
 * (n_ang - 1), linear in the angle (detection probability QE times the
 * response).  max_cycles bounds the tracing cycles of a photon; pre_reject
 * = 1 discards a photon before tracing when its detection uniform is not
 * below the largest detection probability, and uses that uniform for the
 * detection test (the same distribution of counts).  Host arrays are read
 * during the call. */
typedef struct {
    int n_layers;
    double z[ANTS_OPT_MAX_LAYERS + 1];
    double n[ANTS_OPT_MAX_LAYERS];
    double abs_len[ANTS_OPT_MAX_LAYERS];
    double ray_len[ANTS_OPT_MAX_LAYERS];
    double n_below, n_above;
    double half_x, half_y;
    double p_abs[ANTS_OPT_MAX_LAYERS + 1];
    double p_spec[ANTS_OPT_MAX_LAYERS + 1];
    double p_diff[ANTS_OPT_MAX_LAYERS + 1];
    int n_sensors;                 /* 1..256 */
    const double *sensor_xy_host;  /* [n_sensors][2] */
    double sensor_size;
    double n_sensor;
    const double *qe_host;         /* [n_sensors], 0..1 */
    int n_ang;                     /* 0 or 2..64 */
    const double *ang_host;        /* [n_ang], 0..1 */
    int max_cycles;
    int pre_reject;
} ants_optics_params;

/* The outcome of a traced photon: >= 0 the index of the detecting sensor. */
typedef enum {
    ANTS_PH_ABSORBED = -1,    /* in a layer or by an interface */
    ANTS_PH_ESCAPED = -2,     /* out of the stack or through a lateral wall */
    ANTS_PH_MAX_CYCLES = -3,  /* cycle limit reached */
    ANTS_PH_UNDETECTED = -4,  /* entered a window, failed the detection test */
    ANTS_PH_REJECTED = -5     /* discarded before tracing (pre_reject) */
} ants_photon_outcome;

/* Optical photon transport (Sec. 4.2.3-4.2.6, 3.5).
 * Trace n_photons photons from each of n_src point sources
 * src_xyz_dev[n_src][3] (FP32, mm; the source's layer: z[k] <= z < z[k+1]).
 * Each photon draws its uniforms from its own Philox4x32-10 stream with key
 * seed and counter (photon, source, 0x0F7105, block) in a fixed order:
 * [pre-rejection uniform], emission cos(theta) = 2u - 1 and phi = 2 pi u,
 * then per cycle the absorption and Rayleigh uniforms (ranges -L ln u), a
 * Rayleigh scatter's cos(theta) (phase function 1 + cos^2) and azimuth, at an
 * interface one uniform for the custom properties (when any is non-zero) and
 * two for a Lambertian direction, one for Fresnel, and one for the detection
 * test.  precision ANTS_F64 takes every decision in double precision,
 * ANTS_F32 in single.  Outputs: counts_dev[n_src][n_sensors] int32 detected
 * photons (zeroed by the call); outcome_dev (nullable) [n_src][n_photons]
 * int16 outcomes; eta_dev (nullable) [n_src][n_sensors] FP32 counts /
 * n_photons (the light response at the source positions, e.g. to fit LRFs).
 * Asynchronous on `stream`.  Errors: ANTS_E_ARG, ANTS_E_CUDA. */
ANTS_API int ants_trace_photons(ants_ctx *ctx, const ants_optics_params *params, const float *src_xyz_dev,
                                long n_src, long n_photons, uint64_t seed, int precision, int32_t *counts_dev,
                                int16_t *outcome_dev, float *eta_dev, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* ANTS_H */
