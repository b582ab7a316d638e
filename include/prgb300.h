/*
 * prgb300.h -- C ABI of the GB300 real-fluid property library (libprgb300.so).
 *
 * Per-cell real-fluid thermophysical properties of a multi-species mixture
 * (the property evaluation that arxiv 2312.04830 replaces by a DNN, Sec. 4):
 * Peng-Robinson cubic equation of state (Eq. 1) with van der Waals one-fluid
 * mixing (Sec. 2, text after Eq. 1), NASA-7 ideal-gas terms, Chung's dense-fluid
 * viscosity and conductivity (Sec. 2, last paragraph), and the inversion
 * T(h, p, Y) the solver needs because it advances enthalpy (Sec. 4.1).
 *
 * Conventions shared by every entry point:
 *  - Status: every call returns 0 (PR_OK) or a negative PR_E* code; the
 *    message of the last failure on the calling thread is pr_last_error().
 *    Arguments are validated on the host before any launch; a failed call
 *    launches nothing.  Kernels never trap: per-cell problems are reported in
 *    the per-cell status array (PR_CELL_*).
 *  - Memory: all array arguments are DEVICE pointers owned by the caller
 *    (unless stated otherwise), valid for the duration of the asynchronous
 *    work.  The library allocates only inside pr_create / surrogate_create /
 *    serve_create and frees in the matching destroy.
 *  - Layout: structure of arrays.  Cell arrays have length n.  Mass fractions
 *    are species-major: Y[k * ldY + i] for species k, cell i (ldY >= n).
 *  - Precision: PR_FP64 takes and returns double arrays; PR_FP32 and
 *    PR_MIXED take and return float arrays.
 *  - Streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy
 *    default stream).  Calls are asynchronous with respect to the host.
 *  - Units: SI.  T [K], p [Pa], Y [-] (mass fractions, sum 1 within 1e-6; not
 *    renormalised), rho [kg/m^3], Z [-], h [J/kg] (absolute, formation
 *    enthalpy included), cp [J/(kg K)], mu [Pa s], lambda [W/(m K)].
 */
#ifndef PRGB300_H
#define PRGB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int pr_status;

#define PR_OK            0
#define PR_EINVAL       -1  /* bad argument (null pointer, size, alignment, range) */
#define PR_ENOMEM       -2  /* device or host allocation failed */
#define PR_ECUDA        -3  /* a CUDA runtime call failed */
#define PR_ETIMEOUT     -4  /* a bounded wait ran out */
#define PR_ENOTREADY    -5  /* result not available yet */
#define PR_EUNSUPPORTED -6  /* option not supported by this build */

/* Per-cell status codes written to cell_status arrays. */
#define PR_CELL_OK          0  /* converged / evaluated */
#define PR_CELL_MAXIT       1  /* Newton inversion hit max_iter */
#define PR_CELL_H_RANGE     2  /* h* outside [h(60 K), h(5000 K)] or inside a jump of h(T) */
#define PR_CELL_NO_ROOT     3  /* cubic has no root with Z > B */
#define PR_CELL_BAD_INPUT   4  /* non-finite / non-positive T or p, negative Y, |sum Y - 1| > 1e-6 */
#define PR_CELL_AMBIGUOUS   5  /* two physical roots with |Delta g_res| < 1e-9 (larger Z kept) */

/* PR_MIXED: FP32 arithmetic throughout, FP64 for the cubic's root selection:
 * a cell whose FP32 cubic has one physical root, with the root count settled
 * by margins FP32 rounding cannot close (|discriminant| above 1e-4 of its
 * terms' scale, every other real root below 0.999 B), keeps that root; cells
 * with several physical roots (the residual-Gibbs choice between them) or a
 * near-degenerate cubic are solved and selected in FP64. */
typedef enum { PR_FP64 = 0, PR_FP32 = 1, PR_MIXED = 2 } pr_precision;

/* Flags of pr_species_table.flags */
#define PR_FLAG_PRINTED_CONSTANTS 1  /* use Eq. 1's printed 0.45724 / 0.07780 instead of the exact
                                        critical-point values 0.457235529 / 0.077796074 */
#define PR_FLAG_TRANSPORT_XAVG    2  /* mu, lambda = mole-fraction average of pure-species Chung
                                        values instead of Chung's mixture rules */
#define PR_FLAG_NEWTON_FP64_ONLY  4  /* PR_FP64 inversion without the FP32 warm start */

#define PR_MAX_SPECIES 32

/* Species data (HOST pointers, copied by pr_create; the caller keeps ownership).
 * W [g/mol], Tc [K], pc [Pa], omega [-], Vc [cm^3/mol], dipole [debye],
 * kappa (Chung association factor) [-], nasa_lo / nasa_hi: NASA-7 a1..a7 of
 * the low (T < T_mid) and high ranges, row-major [N][7]; T_mid [K];
 * kij: binary interaction parameters [N][N] row-major, or NULL for all zero. */
typedef struct {
    int32_t n_species;   /* 1 .. PR_MAX_SPECIES */
    int32_t flags;       /* PR_FLAG_* */
    const double *W, *Tc, *pc, *omega, *Vc, *dipole, *kappa;
    const double *nasa_lo, *nasa_hi, *T_mid;
    const double *kij;
} pr_species_table;

typedef struct pr_ctx pr_ctx;

/* Create a context on the current CUDA device: validates the table, copies
 * it to the device and derives the per-species constants there (one small
 * kernel).  Synchronous.  *out receives the handle; PR_EINVAL on a bad table
 * (n_species out of range, Tc/pc/W/Vc not positive, NaN), PR_ENOMEM/PR_ECUDA on
 * device failures. */
pr_status pr_create(const pr_species_table *tbl, pr_ctx **out);

/* Release a context (synchronises the device first).  NULL is a no-op. */
void pr_destroy(pr_ctx *ctx);

/* Forward properties, one thread per cell (Eq. 1 + mixing + NASA-7 + Chung).
 *   T, p     [n] inputs; Y [N][ldY] inputs (species-major).
 *   rho, Z, h, cp, mu, lambda  [n] outputs; any may be NULL to skip it.  When
 *            both mu and lambda are NULL the transport step is not run.
 *   cell_status [n] int32 output or NULL.
 * Cells with status PR_CELL_BAD_INPUT or PR_CELL_NO_ROOT get NaN outputs.
 * n = 0 is a no-op.  All pointers must be aligned to their element size. */
pr_status pr_props(pr_ctx *ctx, pr_precision prec, int64_t n,
                   const void *T, const void *p, const void *Y, int64_t ldY,
                   void *rho, void *Z, void *h, void *cp, void *mu, void *lambda,
                   int32_t *cell_status, void *stream);

/* pr_props plus the two further outputs the paper's networks provide to its
 * solver (Sec. 4.1), from the same evaluation:
 *   psi   [n]  d rho / d p at constant enthalpy [s^2/m^2] (the solver's
 *              compressibility), from the PR equation's partial derivatives;
 *   alpha [n]  thermal diffusivity of the enthalpy equation, lambda / cp
 *              [kg/(m s)] (the form an OpenFOAM-derived solver carries; divide
 *              by rho for m^2/s).
 * Any output may be NULL; asking for alpha runs the transport step.  Same
 * precisions, layouts, status codes and errors as pr_props. */
pr_status pr_props_ext(pr_ctx *ctx, pr_precision prec, int64_t n,
                       const void *T, const void *p, const void *Y, int64_t ldY,
                       void *rho, void *Z, void *h, void *cp, void *mu, void *lambda,
                       void *psi, void *alpha, int32_t *cell_status, void *stream);

/* Per-species outputs of the paper's networks (Sec. 4.1: the nondimensional
 * standard-state enthalpies and the mixture-averaged diffusion coefficients
 * of each species; Sec. 2: binary diffusion with a high-pressure correction).
 *   hk_RT [N][ldo]  h_k^0(T) / (R T) of the NASA-7 fit of each species;
 *   Dk    [N][ldo]  mixture-averaged diffusion coefficient [m^2/s],
 *                   D_km = (1 - Y_k) / sum_{j != k} X_j / D_kj (1 - Y_k
 *                   taken as sum_{j != k} Y_j / sum_j Y_j), with the
 *                   Chapman-Enskog binary D_kj (Neufeld's collision integral;
 *                   Lennard-Jones sigma = 0.809 Vc^(1/3), eps/k = Tc / 1.2593,
 *                   arithmetic-mean sigma_kj, geometric-mean eps_kj, pair
 *                   molar mass 2 / (1/W_k + 1/W_j)); a species with no other
 *                   species in the cell gets its self-diffusion D_kk; every
 *                   D_kj is multiplied by the factor set with
 *                   pr_set_diffusion_correction (1 when none is set).
 *   T, p [n]; Y [N][ldY]; either output may be NULL; ldo >= n.
 *   cell_status [n] int32 (NULL allowed): PR_CELL_OK or PR_CELL_BAD_INPUT
 *   (NaN outputs).  No cubic is solved: PR_MIXED computes as PR_FP32.
 * Pointers aligned to their element size; n = 0 is a no-op. */
pr_status pr_species_props(pr_ctx *ctx, pr_precision prec, int64_t n,
                           const void *T, const void *p, const void *Y, int64_t ldY,
                           void *hk_RT, void *Dk, int64_t ldo, int32_t *cell_status, void *stream);

/* High-pressure correction of the binary diffusion coefficients (Sec. 2 names
 * Takahashi's): f(T_r, p_r) = (D p) / (D p)_low-pressure as a table on the
 * caller's grid, interpolated bilinearly and held at its edge values outside,
 * evaluated at the mixture's pseudo-reduced state (Kay's rule,
 * T_r = T / sum X_k Tc_k, p_r = p / sum X_k pc_k).  Takahashi's chart is data
 * the caller supplies; the library ships none.
 *   Tr [n_Tr], pr [n_pr]: strictly increasing, finite; 2..64 points each.
 *   f [n_Tr][n_pr] (row-major, T_r rows): finite, >= 0.
 * All arrays are HOST memory, copied.  corr = NULL removes the correction.
 * Synchronises the device; do not call while work of this context runs. */
typedef struct {
    int32_t n_Tr, n_pr;
    const double *Tr, *pr, *f;
} pr_diffusion_correction;
pr_status pr_set_diffusion_correction(pr_ctx *ctx, const pr_diffusion_correction *corr);

/* Bilger's mixture fraction, the composition input of the paper's networks
 * (Sec. 4.1): Z = (beta - beta_ox) / (beta_fuel - beta_ox) with Bilger's
 * coupling function beta = 2 Z_C / W_C + Z_H / (2 W_H) - Z_O / W_O of the
 * element mass fractions Z_e, i.e. beta = sum_k Y_k (2 a_Ck + a_Hk / 2 - a_Ok)
 * / W_k.  pr_set_bilger takes HOST arrays: atoms [N][3] = carbon, hydrogen and
 * oxygen atoms per molecule of each species, Y_fuel [N] and Y_ox [N] the
 * stream compositions (PR_EINVAL when their coupling functions are equal);
 * it synchronises the device.  pr_bilger_z: Y [N][ldY], Z [n] outputs (FP64
 * or FP32 by prec; no validation, NaN propagates); PR_EINVAL before
 * pr_set_bilger.  Z leaves [0, 1] for compositions that are not mixtures of
 * the two streams (pure H2: Z > 1). */
pr_status pr_set_bilger(pr_ctx *ctx, const int32_t *atoms, const double *Y_fuel, const double *Y_ox);
pr_status pr_bilger_z(pr_ctx *ctx, pr_precision prec, int64_t n, const void *Y, int64_t ldY, void *Z,
                      void *stream);

/* Measured throughput of an arithmetic pipe on the current device, the
 * roofline denominator of the kernels it bounds (a diagnostic; synchronous,
 * about 0.1 s):
 *   PR_PEAK_FP64_FMA  FP64 flops/s (an FMA counts two), the FP64 paths;
 *   PR_PEAK_FP32_FMA  FP32 flops/s;
 *   PR_PEAK_MUFU_EX2  exp2 evaluations/s of the special-function unit.
 * Every thread runs eight independent FMA (or ex2) chains; the best of three
 * timed launches is kept.  *ops_per_s is a HOST pointer. */
#define PR_PEAK_FP64_FMA 0
#define PR_PEAK_FP32_FMA 1
#define PR_PEAK_MUFU_EX2 2
/* FP64 library calls per second (CUDA's exp, log, division, square root and
 * cube root, arguments of order one): the FP64 rate over one of these gives
 * the FP64-pipe slots a call takes, the weight of that call in the FP64
 * paths' algorithmic work. */
#define PR_PEAK_FP64_EXP 3
#define PR_PEAK_FP64_LOG 4
#define PR_PEAK_FP64_DIV 5
#define PR_PEAK_FP64_SQRT 6
#define PR_PEAK_FP64_CBRT 7
pr_status pr_measure_peak(int kind, double *ops_per_s);

/* The FP64 exponential and logarithm the FP64 property paths use (a
 * diagnostic, for their accuracy tests): y[i] = f(x[i]) for fn = 0 exp,
 * 1 expm1, 2 log, 3 log1p (the library's table-driven forms: Tang, ACM TOMS
 * 15 (1989) 144 and 16 (1990) 378), 4..7 the same functions of CUDA's math
 * library.  x, y: DEVICE arrays of n doubles; asynchronous on `stream`. */
pr_status pr_eval_math(int fn, int64_t n, const double *x, double *y, void *stream);

/* Inversion T(h*, p, Y) by safeguarded Newton on f(T) = h(T) - h*, f' = cp,
 * inside the bracket [60, 5000] K, starting from T_guess (clipped to the
 * bracket).  A Newton step that leaves the current bracket, or follows a step
 * that did not halve |f|, is replaced by bisection.  Converged when
 * |dT| <= rtol T or |f| <= rtol max(|h*|, cp T).  PR_FP64 first runs plain
 * Newton on the FP32 thermodynamics (at most 8 steps, until a step is below
 * 1e-5 T) and starts the FP64 iteration from that root, or from T_guess when
 * the FP32 steps fail or do not settle; the FP64 iteration alone decides
 * convergence, so the result meets the same FP64 tolerance
 * (PR_FLAG_NEWTON_FP64_ONLY turns the warm start off).  iters counts the
 * FP64 iterations.  PR_MIXED iterates on the mixed thermodynamics (FP64 root
 * selection, above) and re-solves in FP64, from that root, the cells where it failed and
 * those in the pseudo-boiling band (cp above 3 x the ideal-gas cp), where
 * the FP32 iteration is least reliable; there its T is the FP64 solution
 * rounded to FP32.  iters then counts both iterations.
 *   hstar, p, T_guess [n]; Y [N][ldY]; T_out [n] output;
 *   cell_status [n] (required), iters [n] (NULL allowed);
 *   max_iter in 1..1000; rtol in [1e-15, 1e-2].
 * Status per cell: PR_CELL_OK, PR_CELL_MAXIT (T_out = last iterate),
 * PR_CELL_H_RANGE (T_out clamped to the bracket end, or the jump location),
 * PR_CELL_BAD_INPUT, PR_CELL_NO_ROOT. */
pr_status pr_T_from_h(pr_ctx *ctx, pr_precision prec, int64_t n,
                      const void *hstar, const void *p, const void *Y, int64_t ldY,
                      const void *T_guess, void *T_out, int32_t *cell_status, int32_t *iters,
                      int max_iter, double rtol, void *stream);

/* ======================================================================
 * Surrogate MLP (Sec. 4: the DNN that replaces the property evaluation).
 * Inputs per cell: [log T, p, Y_1..Y_9, T_pc / T, log W] (9 species, the
 * context's order; T_pc = sum_k X_k Tc_k by Kay's rule, W the mean molar mass
 * [kg/mol], both from the raw T, Y);
 * outputs: [rho, Z, h, cp, mu, lambda] learned as [log rho, Z, h - h_ig,
 * log cp, log mu, log lambda], inputs and outputs standardised with statistics
 * of the training pool; h_ig(T, Y) = sum_k Y_k h_k(T) / W_k is the NASA-7
 * ideal-gas enthalpy (Sec. 2), evaluated exactly and added to the network's
 * departure.  Checkpoints carry format 4 (these inputs and targets and the
 * Box-Cox parameters; format 3 files, without them, still load).  Hidden
 * layers use GeLU (Sec. 4.1) in its tanh form,
 * 0.5 z (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))).  Forward and
 * backward GEMMs run on the tensor cores (BF16 operands, FP32 accumulation);
 * master weights and Adam moments are FP32.
 * ====================================================================== */

typedef struct sg_model sg_model;

typedef struct {
    int32_t width;          /* hidden width: 128, 256, 512 or 1024 */
    int32_t hidden_layers;  /* number of hidden layers, 1..8 */
    int32_t max_batch;      /* largest training batch; multiple of 128 */
    int32_t infer_chunk;    /* rows per inference chunk; multiple of 128 */
} sg_config;

#define SG_NORM_FLOATS 84  /* in_mean[13] in_std[13] out_mean[0..5] out_std[0..5] hull_lo[13] hull_hi[13]
                              out_mean[6..15] out_std[6..15] */

/* Create a model bound to `ctx` (which must hold exactly 9 species; it is
 * used for the Peng-Robinson fallback).  Weights ~ U(-1/sqrt(fan_in),
 * 1/sqrt(fan_in)) from a counter-based generator seeded by `seed`.  Allocates
 * every device buffer the model will use; synchronous. */
pr_status surrogate_create(pr_ctx *ctx, const sg_config *cfg, uint64_t seed, sg_model **out);
void surrogate_destroy(sg_model *m);

/* Number of trainable parameters (W_l [out][in] and b_l [out] per layer). */
int64_t surrogate_num_params(const sg_model *m);

/* Copy the FP32 master parameters to / from HOST memory in the order
 * W_1, b_1, ..., W_L+1, b_L+1 (row-major W [out][in]); n must equal
 * surrogate_num_params.  Synchronous. */
pr_status surrogate_get_params(const sg_model *m, float *host_dst, int64_t n);
pr_status surrogate_set_params(sg_model *m, const float *host_src, int64_t n);

/* Normalisation and training hull (SG_NORM_FLOATS floats, HOST memory). */
pr_status surrogate_get_normalization(const sg_model *m, float *host_dst);
pr_status surrogate_set_normalization(sg_model *m, const float *host_src);

/* Fit the normalisation and the training hull (per-input [min, max] widened
 * by 1 % of the range) to a pool of n states.  x: DEVICE [11][ldx] raw inputs
 * (T, p, Y_1..Y_9); y: DEVICE [n_out][ldy] raw targets (rho, Z, h, cp, mu,
 * lambda for the property networks; see SG_OPT_MODE and SG_OPT_OUTPUTS).  Rows whose features or log-targets are not finite (e.g. a
 * non-positive property) are left out.  Asynchronous on `stream`. */
pr_status surrogate_fit_normalization(sg_model *m, int64_t n, const float *x, int64_t ldx, const float *y,
                                      int64_t ldy, void *stream);

/* One training step (Sec. 4.3, with the squared error on the standardised
 * log / scaled targets, i.e. a relative-MSE loss, and Adam with beta =
 * (0.9, 0.999), eps = 1e-8): batch rows (a multiple of 128, <= max_batch)
 * are drawn from the pool x [11][ldx], y [n_out][ldy] (DEVICE, n_pool rows):
 * rows 0..batch-1 in order when sample_seed == 0 and n_pool == batch, else
 * uniformly with replacement by a counter-based hash of (sample_seed, row).
 * Outputs whose target is not finite contribute neither loss nor gradient.
 * loss_out: DEVICE float receiving the batch loss, or NULL. */
pr_status surrogate_train_step(sg_model *m, int64_t batch, int64_t n_pool, const float *x, int64_t ldx,
                               const float *y, int64_t ldy, uint64_t sample_seed, float lr, float *loss_out,
                               void *stream);

/* Loss and gradients of the first `batch` pool rows without updating the
 * model.  grad_out: DEVICE [surrogate_num_params] in the get_params order. */
pr_status surrogate_loss_grad(sg_model *m, int64_t batch, const float *x, int64_t ldx, const float *y, int64_t ldy,
                              float *loss_out, float *grad_out, void *stream);

/* Inference (FP32 I/O): T, p [n], Y [9][ldY] DEVICE inputs; out [n_out][ldo]
 * DEVICE outputs (rho, Z, h, cp, mu, lambda for the forward property network;
 * n_out = 6, or 9 with SG_OPT_OUTPUTS = SG_OUT_DK or SG_OUT_HK).  Cells with any input outside
 * the training hull are evaluated by the FP64 Peng-Robinson path instead and
 * flagged in used_fallback [n] (DEVICE uint8, NULL allowed). */
pr_status surrogate_infer(sg_model *m, int64_t n, const float *T, const float *p, const float *Y, int64_t ldY,
                          float *out, int64_t ldo, uint8_t *used_fallback, void *stream);

/* Model options.  SG_OPT_FUSED_INFER: run all layers of an inference chunk
 * in one launch.  3 (the default for widths 256 and 512 when the device
 * takes cluster launches): CTA pairs (clusters of two, tcgen05 pair MMA,
 * M = 256) that take each block of 256 rows through every layer with its
 * activations resident in shared memory, only the weights streaming from
 * L2; 1 (the default otherwise): a persistent cooperative launch whose
 * activations stay in L2-sized rings (widths that are multiples of 256, up
 * to 1024, hidden_layers x width <= 4528), 128 x 256 tiles, one CTA each;
 * 2: the same with 256 x 256 tiles on CTA pairs, falling back to 1 when the
 * device refuses that launch; 4 (widths 256 and 512, cluster launches): CTA
 * pairs whose activations alternate from layer to layer between tensor
 * memory (read as the next layer's MMA A operand) and shared memory, in
 * N-tiles of 128; 0: one GEMM launch per layer.  All give identical
 * outputs.  PR_EINVAL for an unknown option or a value the model
 * cannot take. */
#define SG_OPT_FUSED_INFER 1
/* SG_OPT_MODE: SG_MODE_FORWARD (default) or SG_MODE_INVERSE, the paper's own
 * arrangement (Sec. 4.1: the networks take enthalpy, pressure and composition
 * and return the temperature and the properties the solver needs).  Set it
 * before fitting the normalisation and training; checkpoints record it.  In
 * the inverse mode:
 *   pools:  x = [h*, p, Y_1..Y_9] (h* in J/kg), y = [T, rho, psi, mu, alpha,
 *           cp] (pr_props_ext's units; alpha = lambda / cp);
 *   inputs: [h* - h_f(Y), p, Y_1..Y_9, log T_pc, log W] with h_f(Y) = sum_k
 *           Y_k h_k(298.15 K) / W_k (formation enthalpies removed);
 *   surrogate_infer: the T argument holds h*, and out [n_out][ldo] receives
 *           [T, rho, psi, mu, alpha, cp]; cells outside the training hull get
 *           the FP64 inversion started from the network's T, then
 *           pr_props_ext's values at that T (NaN where the inversion fails). */
#define SG_OPT_MODE 2
/* SG_OPT_WAIT_LIMIT_KCYCLES: limit, in thousands of SM clock cycles, of every
 * bounded wait of the fused inference kernel (0: the default, 4e9 cycles,
 * about 2 s).  When a wait runs out the kernel stops waiting, finishes without
 * its results and flags the model: surrogate_sync_status returns PR_ETIMEOUT
 * and clears the flag, and the next call runs normally.
 * SG_OPT_TEST_STALL: test hook for that path; 1 makes layer 1 of the first
 * row block of every chunk wait for an arrival that never comes. */
#define SG_OPT_WAIT_LIMIT_KCYCLES 3
#define SG_OPT_TEST_STALL 4
/* SG_OPT_LOSS: the training loss on the standardised targets.
 * SG_LOSS_REL_MSE (default): mean squared error (relative, the targets being
 * logarithms or scaled values); SG_LOSS_L1: the paper's L1 norm (Sec. 4.3),
 * mean |y - target|, output gradient sign(y - target) / (batch * 6) with
 * sign(0) = 0.  Non-finite targets are masked in both. */
/* SG_OPT_CONFIDENCE_PPM: low-confidence test of the forward model, in parts
 * per million (0: off).  The network predicts rho and Z separately while the
 * equation of state ties them (rho Z R T = p W, W the mean molar mass of Y);
 * a cell with |rho Z R T / (p W) - 1| above the tolerance takes the FP64
 * fallback like a cell outside the hull (and is flagged in used_fallback). */
#define SG_OPT_CONFIDENCE_PPM 6
/* SG_OPT_TRANSPORT_CONFIDENCE_PPM: low-confidence test of the property models'
 * transport outputs, in parts per million (0: off).  Chung's correlation
 * (Sec. 2) is evaluated in FP32 at the network's own density -- and, for the
 * inverse and Bilger models, its own temperature -- and the cell's
 * composition; a cell whose predicted mu or lambda (inverse models: alpha cp)
 * differs from those values by more than the tolerance takes the FP64
 * fallback like a cell outside the hull (flagged in used_fallback).  No effect
 * on the per-species networks. */
#define SG_OPT_TRANSPORT_CONFIDENCE_PPM 8
/* SG_OPT_TIME_MLP: 1 records CUDA events on the call's stream around the MLP
 * launch of every inference chunk (the one launch of a fused kernel, or the
 * per-layer launches together) from now on, restarting the count; 0 stops.
 * surrogate_mlp_time reads them.  Default 0. */
#define SG_OPT_TIME_MLP 9
/* SG_OPT_OUTPUTS (the paper's dedicated networks, Sec. 4.1): with
 * SG_MODE_INVERSE or SG_MODE_BILGER inputs, the network predicts
 *   SG_OUT_PROPS  (default) T, rho, psi, mu, alpha, cp;
 *   SG_OUT_DK     the 9 mixture-averaged diffusion coefficients D_k [m^2/s]
 *                 (pr_species_props; learned as logarithms);
 *   SG_OUT_HK     the 9 standard-state enthalpies h_k / (R T);
 *   SG_OUT_SINGLE + j, j = 0..5: one of T, rho, psi, mu, alpha, cp alone
 *                 (one dedicated network per property, as the paper trains
 *                 them; learned as its logarithm).
 * surrogate_infer then writes [n_out][ldo] (n_out = 9 for the per-species
 * outputs, 1 for a single property); training targets y are [n_out][ldy] of
 * the same quantities; cells outside the hull take the FP64 inversion and the
 * FP64 values at its T (per-species: with the context's correction table;
 * a single property other than T: the inversion starts from 1000 K).
 * Selecting outputs re-initialises the weights (set before fitting). */
#define SG_OPT_OUTPUTS 7
#define SG_OUT_PROPS 0
#define SG_OUT_DK 1
#define SG_OUT_HK 2
#define SG_OUT_SINGLE 3
#define SG_OPT_LOSS 5
#define SG_LOSS_REL_MSE 0
#define SG_LOSS_L1 1
#define SG_MODE_FORWARD 0
#define SG_MODE_INVERSE 1
/* SG_MODE_BILGER (the paper's network inputs, Sec. 4.1-4.2): as
 * SG_MODE_INVERSE (inputs h*, p, Y; outputs T, rho, psi, mu, alpha, cp;
 * FP64 fallback outside the hull), but the network sees only
 * [h* - h_f(Y), p, BoxCox(Z)], Z Bilger's mixture fraction of Y (the
 * context's pr_set_bilger table, required before selecting the mode) and
 * BoxCox(Z) = ((Z + shift)^lambda - 1) / lambda (log at lambda = 0) with the
 * parameters of surrogate_set_boxcox (default lambda = 1, shift = 1e-3: Z
 * itself, shifted).  Set mode and Box-Cox parameters before fitting and
 * training. */
#define SG_MODE_BILGER 2
pr_status surrogate_set_option(sg_model *m, int option, int value);

/* Current value of an option (host int *value).  For SG_OPT_FUSED_INFER it
 * is the kernel the next inference runs: 0 per-layer launches, 1 single
 * CTAs, 2 CTA pairs, 3 resident activations, 4 activations alternating
 * between tensor and shared memory.  PR_EINVAL for an unknown
 * option or a null pointer. */
pr_status surrogate_get_option(const sg_model *m, int option, int *value);

/* Box-Cox parameters of Bilger's mixture fraction in SG_MODE_BILGER (the
 * paper applies the transform to the mixture fraction, Sec. 4.2): lambda in
 * [-10, 10], shift in (0, 1].  Stored in checkpoints (format 4). */
pr_status surrogate_set_boxcox(sg_model *m, double lambda, double shift);

/* Synchronise the device and report PR_ETIMEOUT if a tensor-core kernel gave
 * up waiting on one of its barriers since the last call (the flag is then
 * cleared). */
pr_status surrogate_sync_status(sg_model *m);

/* Device time of the MLP launches recorded since SG_OPT_TIME_MLP was set to 1
 * or since the last call (host double *ms: the sum of the event intervals in
 * milliseconds; host int64_t *launches: their number), then restarts the
 * count.  Waits for the last recorded event.  PR_EINVAL for null arguments. */
pr_status surrogate_mlp_time(sg_model *m, double *ms, int64_t *launches);

/* Checkpoint (HOST file): weights, Adam moments, step count, normalisation. */
pr_status surrogate_save(const sg_model *m, const char *path);
pr_status surrogate_load(sg_model *m, const char *path);

/* ======================================================================
 * Continuous-batching property server (many simulations sharing one GPU).
 * Requests carry FP32 fields in HOST memory (pinned memory keeps the copies
 * asynchronous; pageable memory works but its copies block the worker) and a
 * precision.  A worker thread admits requests in arrival order while their
 * device buffers fit in the HBM budget, cuts them into `chunk`-cell pieces,
 * fills batches of up to `max_slots` pieces of one (kind, precision)
 * round-robin across every admitted request of that path, and runs each batch
 * by replaying a CUDA graph captured for its path and (power-of-two) slot
 * count: gather the pieces, evaluate them, scatter the results.  Results do
 * not depend on batch composition.  The worker makes its CUDA calls outside
 * the request lock, so submitting and polling never wait behind a launch.
 * The model (if any) must not be used by other calls while the server runs.
 * ====================================================================== */

typedef struct sv_server sv_server;

#define SV_PROPS     0   /* out [6][n]: rho, Z, h, cp, mu, lambda */
#define SV_T_FROM_H  1   /* out [n]: T; status [n] per-cell PR_CELL_* codes */

/* Precision of a request.  Inputs and outputs stay FP32; the FP64 paths widen
 * the inputs, compute in FP64 (pr_props / pr_T_from_h with PR_FP64, inversion
 * tolerance 1e-12) and round the results.
 *   SV_PREC_SERVER  the server's own path: SV_PROPS through the surrogate with
 *                   its FP64 PR fallback (the FP32 PR path when the server has
 *                   no model); SV_T_FROM_H in sv_config.newton_precision
 *   SV_PREC_FP64    the FP64 PR path
 *   SV_PREC_MIXED   PR_MIXED (FP32 with FP64 root selection / band re-solve)
 *   SV_PREC_FP32    the FP32 PR path
 * The FP32 and mixed inversions stop at rtol 1e-6. */
#define SV_PREC_SERVER 0
#define SV_PREC_FP64   1
#define SV_PREC_MIXED  2
#define SV_PREC_FP32   3

typedef struct {
    int32_t kind;        /* SV_PROPS or SV_T_FROM_H */
    int32_t precision;   /* SV_PREC_* */
    int64_t n;           /* cells, >= 1 */
    const float *T;      /* SV_PROPS: T [n]; SV_T_FROM_H: initial guess [n] (HOST) */
    const float *p;      /* [n] (HOST) */
    const float *Y;      /* [9][n] species-major (HOST) */
    const float *h;      /* SV_T_FROM_H: h* [n] (HOST); NULL for SV_PROPS */
    float *out;          /* HOST output (see kind); written when the request is done */
    int32_t *status;     /* SV_T_FROM_H per-cell status [n] (HOST) or NULL */
} sv_request;

typedef struct {
    int32_t chunk;             /* cells per batch slot: multiple of 128 */
    int32_t max_slots;         /* slots per batch, 1..256 */
    int32_t newton_precision;  /* PR_FP64, PR_MIXED or PR_FP32: SV_T_FROM_H requests at SV_PREC_SERVER */
    int32_t pad;
    size_t hbm_budget_bytes;   /* device memory for admitted requests' buffers */
} sv_config;

typedef struct {
    uint64_t submitted, completed, batches, slots_used, slots_launched;
    int64_t cells;             /* cells of completed requests */
    size_t bytes_in_use, peak_bytes_in_use;
    size_t queued, active;
} sv_stats;

/* Create a server (allocates the HBM budget, staging and descriptor tables,
 * captures its graphs, starts the worker).  model may be NULL. */
pr_status serve_create(pr_ctx *ctx, sg_model *model, const sv_config *cfg, sv_server **out);

/* Queue a request; *ticket identifies it.  The host arrays must stay valid
 * (and `out` untouched) until the request is done.  A request that cannot fit
 * in the budget even alone completes with result PR_ENOMEM. */
pr_status serve_submit(sv_server *s, const sv_request *req, uint64_t *ticket);

/* Non-blocking status: *done = 1 when finished; then *result (PR_OK or an
 * error) and *latency_ms (submit to completion, host clock) are set. */
pr_status serve_poll(sv_server *s, uint64_t ticket, int *done, pr_status *result, double *latency_ms);

/* Block until the request is done or timeout_ms passes (PR_ETIMEOUT). */
pr_status serve_wait(sv_server *s, uint64_t ticket, double timeout_ms, pr_status *result, double *latency_ms);

pr_status serve_stats(sv_server *s, sv_stats *out);

/* Stop the worker, wait for the device, release everything. */
void serve_destroy(sv_server *s);

/* Plain tensor-core GEMM with the kernel the MLP uses: D[M][N] (FP32,
 * row pitch ldd) = A[M][K] * B[N][K]^T with A, B BF16 K-major (row pitches lda,
 * ldb elements), FP32 accumulation.  K a positive multiple of 64; N = 16, 64 or
 * a multiple of 128; any M >= 1.  DEVICE pointers, 16-byte aligned.  err_flag:
 * DEVICE int set to 1 if a barrier wait inside the kernel ran out. */
pr_status mlp_gemm_bf16(int64_t M, int64_t N, int64_t K, const void *A, int64_t lda, const void *B, int64_t ldb,
                        float *D, int64_t ldd, int *err_flag, void *stream);

/* ----------------------------------------------------------------------
 * Allocation-free fallback evaluation.  The paper has no counterpart: this
 * entry point exists for host programs that cannot call cudaMalloc (for
 * example a solver that owns all device memory through its own pool, or one
 * held to a device-memory budget fixed in advance).
 *
 * For every cell i < n with mask[i] != 0, evaluates the FP64 Peng-Robinson
 * properties from FP32 inputs (the same step surrogate_infer applies to cells
 * outside the training hull) and writes rho, Z, h, cp, mu, lambda as FP32 to
 * out[q * ldo + i], q = 0..5; cells with mask[i] == 0 are left untouched.
 * T, p [n], Y [N][ldY], mask [n] (uint8) and out [6][ldo] are DEVICE pointers
 * owned by the caller.
 *
 * It allocates nothing: the compacted cell list lives in a fixed scratch array
 * compiled into the library (PR_NOALLOC_MAX_CELLS indices plus a counter,
 * about 4 MB), which every GPU that loads the library holds until the process
 * exits.  n > PR_NOALLOC_MAX_CELLS is rejected with PR_EINVAL.  pr_create
 * looks up the scratch array's device address on the context's device, so
 * this call needs no set-up of its own; it must be made with the context's
 * device current (PR_EINVAL otherwise).  Every call shares the one scratch
 * array and clears its counter first; calls whose work overlaps on the GPU
 * (e.g. on two streams at once, or from two contexts on one device) race on
 * it.  Asynchronous on `stream`. */
#define PR_NOALLOC_MAX_CELLS (1 << 20)
pr_status pr_fallback_props_noalloc(pr_ctx *ctx, int64_t n, const float *T, const float *p, const float *Y,
                                    int64_t ldY, const uint8_t *mask, float *out, int64_t ldo, void *stream);

/* Thread-local message of the last failed call on this thread ("" if none). */
const char *pr_last_error(void);

/* Library version string. */
const char *pr_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PRGB300_H */
