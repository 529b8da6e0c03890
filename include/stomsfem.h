/*
 * stomsfem.h -- C ABI of the GB300 (sm_103a) StoMsFEM local-upscaling library.
 *
 * The library computes, on one GPU, the data-parallel hot path of the
 * stochastic multiscale finite element method of Hou, Li and Zhang
 * ("Exploring the locally low dimensional structure in solving random
 * elliptic PDEs"): for every (random sample, coarse cell) pair it builds
 * the fine-grid Q1 stiffness of the sampled coefficient, solves the cell
 * problems that give the multiscale basis, forms the upscaled stiffness
 * and load, and then assembles and solves each sample's coarse system.
 * Beside this plain path (FP64, FP32, FP32 + FP64 refinement) it offers
 * the paper's other forms of the local upscaling -- the Petrov-Galerkin
 * form, the oscillatory boundary condition of the cell problems, random
 * interpolation in the local parameters, the reduced basis (also with an
 * affine coefficient) -- a learned surrogate, the coarse solve with mixed
 * boundary data, the pieces of the two-level Monte Carlo estimator, and
 * plans that replay a batch's whole step as one CUDA graph.
 *
 * Conventions shared by every call
 *  - Unit square, zero Dirichlet data on its boundary (except
 *    stomsfem_coarse_solve_bc, which takes its own), constant load f.
 *    Fine grid nf x nf square elements (h = 1/nf); coarse grid nc x nc
 *    cells (H = 1/nc); rho = nf/nc must be an integer.
 *  - Arrays are row-major and y-major: coefficient a[s][ey][ex] (one value
 *    per fine element, evaluated at its centroid); coarse nodal vectors
 *    u[s][J*(nc+1)+I].  Cell index cell = cy*nc + cx.
 *  - Quad corner order SW, SE, NE, NW.  K_e is packed as its upper triangle
 *    row by row: (0,0)(0,1)(0,2)(0,3)(1,1)(1,2)(1,3)(2,2)(2,3)(3,3).
 *  - Every pointer argument named as device memory must point to device
 *    memory of the current CUDA device; the caller owns all arrays.  All
 *    calls are asynchronous on `stream` (NULL = legacy default stream)
 *    unless stated otherwise; arguments are validated on the host before
 *    any launch and a failing call launches nothing.
 *  - Return value: STOMSFEM_OK (0) or a negative STOMSFEM_E* code;
 *    stomsfem_last_error() gives a one-line message for the calling thread.
 */
#ifndef STOMSFEM_H
#define STOMSFEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* stomsfem_stream_t; /* same object as cudaStream_t */

enum {
  STOMSFEM_OK = 0,
  STOMSFEM_EINVAL = -1,   /* bad argument or descriptor */
  STOMSFEM_ENOMEM = -2,   /* workspace too small / allocation failed */
  STOMSFEM_ECUDA = -3,    /* a CUDA runtime call failed (message has details) */
  STOMSFEM_ENOTSPD = -4,  /* Cholesky breakdown in at least one unit */
  STOMSFEM_ETIMEOUT = -5, /* a bounded device wait expired */
  STOMSFEM_EVERSION = -6  /* bad or incompatible serialized object */
};

enum { STOMSFEM_FP64 = 0, STOMSFEM_FP32_REFINED = 1, STOMSFEM_FP32 = 2 };
enum { STOMSFEM_FIELD_EXP = 0, STOMSFEM_FIELD_EXP_SIGMOID = 1, STOMSFEM_FIELD_AFFINE = 2 };
/* Boundary data of the cell problems (stomsfem_upscale_bc). */
enum { STOMSFEM_BC_BILINEAR = 0, STOMSFEM_BC_OSCILLATORY = 1 };

typedef struct {
  int32_t nf; /* fine elements per side */
  int32_t nc; /* coarse cells per side, nf % nc == 0 */
  double f;   /* constant load */
} stomsfem_grid;

/* Coefficient model (the nonlinear transform of Sec. 2.1.3 applied to an
 * affine expansion in localized bumps):
 *   z(x)  = sum_i xi_i exp(-|x - c_i|^2 / width^2),
 *           c_i = ((bx + 1/2)/nbx, (by + 1/2)/nby),  i = by*nbx + bx;
 *   EXP:          a = exp(scale * z)
 *   EXP_SIGMOID:  a = exp(contrast_log / (1 + exp(-gain * z)))
 *   AFFINE:       a = gain + scale * z   (Eq. RBaffine: affine in xi, gain
 *                 the mean level; positive while gain > |scale| max|z|)  */
typedef struct {
  int32_t kind;
  int32_t nbx, nby;
  double width;
  double scale;
  double contrast_log;
  double gain;
} stomsfem_field;

const char* stomsfem_version(void);
const char* stomsfem_last_error(void);

/* Failure-path self test (no paper counterpart): one CTA waits, with a limit
 * of `iters` polls of about 100 ns, on an mbarrier that nothing arrives at
 * -- the same bounded wait the tensor-core kernels use -- and reports the
 * outcome in *status_host (STOMSFEM_ETIMEOUT when the limit ran out).
 * Synchronous; the device stays usable afterwards.  1 <= iters <= 2^20. */
int stomsfem_selftest_wait_timeout(int32_t iters, int32_t* status_host);

/* Self test of the table-driven FP64 exponential that the coefficient
 * sampler uses (no paper counterpart): out[i] = exp(t[i]) for device arrays
 * of n doubles, stream-ordered.  EINVAL for n < 0 or NULL pointers. */
int stomsfem_selftest_exp(const double* t, int32_t n, double* out, stomsfem_stream_t stream);

/* Measured peak of the non-tensor FMA pipe (no paper counterpart; the
 * denominator of the upscaling kernels' ALU roofline): every SM runs 8
 * blocks of 256 threads, each thread 8 independent FMA chains (FP32: 16384
 * steps, FP64: 512 steps), timed with CUDA events after a warm-up launch,
 * best of three.  *tflops_host = 2 x FMAs / time in TFLOP/s.  precision
 * STOMSFEM_FP32 or STOMSFEM_FP64.  Allocates a small device buffer and
 * synchronises the device.  EINVAL on a bad precision or NULL. */
int stomsfem_selftest_fma_rate(int32_t precision, float* tflops_host);

/* Measured throughput of the warp-level tensor-core instructions (no paper
 * counterpart; the A/B of the cell factorisation's engines rests on it):
 * kind 0 mma.sync m16n8k8 TF32, kind 1 m16n8k16 BF16, FP32 accumulation,
 * 8 independent accumulator chains per warp, 8 blocks of 256 threads per
 * SM, best of three timed launches.  *tflops_host = 2 x MACs / time.
 * Allocates a small device buffer and synchronises the device. */
int stomsfem_selftest_mma_rate(int32_t kind, float* tflops_host);

/* Coefficient sampling (Sec. 2.1.3, the parametrized coefficient of
 * Eq. MsFEB2).  xi: device [S][nbx*nby] float64; a: device [S][nf][nf]
 * float64, a value per fine element at its centroid ((ex+1/2)h, (ey+1/2)h).
 * Errors: EINVAL for bad sizes. */
int stomsfem_sample_coef(const stomsfem_grid* grid, const stomsfem_field* field,
                         const double* xi, int32_t S, double* a, stomsfem_stream_t stream);

/* The same sampling at a chosen arithmetic precision: STOMSFEM_FP64 is
 * stomsfem_sample_coef; STOMSFEM_FP32 evaluates the bump sums and the
 * exponentials in FP32 (a is still stored as float64), for the FP32
 * upscaling form whose cell matrices are FP32 anyway: relative error of a
 * about |scale * z| x 1e-6 (EXP) and contrast_log * gain * 1e-6
 * (EXP_SIGMOID).  Errors: as stomsfem_sample_coef, and EINVAL for any other
 * precision. */
int stomsfem_sample_coef_precision(const stomsfem_grid* grid, const stomsfem_field* field,
                                   const double* xi, int32_t S, int32_t precision, double* a,
                                   stomsfem_stream_t stream);

/* Scratch needed by stomsfem_upscale for one unit in flight ("slot") and
 * the recommended total (a slot per unit the whole GPU keeps in flight, plus
 * 8 (nc^2 + 1) bytes, rounded up to 256, for the cell lists of the FP32
 * form).  Each slot holds one unit's banded Cholesky factor and solution
 * vectors. */
int stomsfem_upscale_workspace_size(const stomsfem_grid* grid, int32_t max_oversample,
                                    int32_t precision, size_t* slot_bytes,
                                    size_t* recommended_bytes);

/* Simultaneous local upscaling of S samples: for every (sample, cell) unit
 * solve the four cell problems of Eq. MsFEB on the fine mesh (bilinear
 * boundary data on the patch = the cell enlarged by oversample[cell] fine
 * elements on each side and clipped to the domain, Remark on oversampling),
 * recombine the patch solutions into the basis that is nodal at the cell
 * corners, and form the upscaled stiffness and load of Eq. stiffness_local
 * on the cell.  In the FP32 form without phi output, cells without
 * oversampling use K_e(l,m) = p_l^T A p_m - y_l . y_m with y the forward
 * solutions (the Galerkin identity of the cell problem; no back
 * substitution); with an oversample array and room at the end of the
 * workspace for the cell lists, those cells and the others run as two
 * launches.
 *   a            device [S][nf][nf] float64 coefficient
 *   oversample   device [nc*nc] int8 layer widths, or NULL for none; every
 *                entry must lie in [0, max_oversample] (units with an
 *                out-of-range entry get status EINVAL and NaN outputs)
 *   precision    STOMSFEM_FP64: everything in FP64.
 *                STOMSFEM_FP32_REFINED: FP32 factor and solves, FP64
 *                  residuals (refine_iters steps of iterative refinement)
 *                  and FP64 K_e/b_e accumulation.
 *                STOMSFEM_FP32: FP32 throughout, results stored as FP64.
 *   Ke           device [S][nc*nc][10] float64 (packed upper triangle)
 *   be           device [S][nc*nc][4] float64
 *   phi          device [S][nc*nc][4][(rho+1)^2] float64 basis on the cell
 *                nodes, or NULL
 *   unit_status  device [S][nc*nc] int32 or NULL: 0 on success; k+1 when
 *                pivot k of the unit's patch matrix was not positive; -1
 *                for an oversample entry outside [0, max_oversample];
 *                STOMSFEM_ENOTSPD when the corner matrix of the
 *                oversampling recombination is singular.  Failed units
 *                get NaN outputs.
 *   workspace    device scratch of workspace_bytes (>= the slots of one
 *                block: 8 in the FP32 forms, 4 in FP64, with the default
 *                factorisation engine; 4 with a tensor-core engine chosen
 *                through stomsfem_upscale_engine; more slots = more units
 *                in flight)
 * Errors: EINVAL (sizes, pointers, precision, bandwidth > 64), ENOMEM
 * (workspace below one block of slots), ECUDA. */
int stomsfem_upscale(const stomsfem_grid* grid, const double* a, const int8_t* oversample,
                     int32_t max_oversample, int32_t S, int32_t precision, int32_t refine_iters,
                     double* Ke, double* be, double* phi, int32_t* unit_status, void* workspace,
                     size_t workspace_bytes, stomsfem_stream_t stream);

/* Allocation-free variant of stomsfem_upscale (the paper has no counterpart;
 * this is a library convenience).  For callers that cannot allocate device
 * memory where they upscale -- code running inside another framework's
 * memory pool or a plugin that must not grow the device footprint, loops
 * that must not take cudaMalloc's implicit synchronisation, programs that
 * only receive device pointers -- the scratch is a fixed 64 MiB file-scope
 * device array instead of a caller workspace; inputs and outputs are the
 * caller's, with the same meaning and layout as in stomsfem_upscale.
 *  - The array is reserved on a device when the library module holding it
 *    is loaded there (by default, at the first call of this function on
 *    that device) and is held until the process exits.
 *  - The first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture.  The address is cached per device and
 *    context: after a device reset (cudaDeviceReset, or the primary context
 *    released and created again) the old address is invalid, and the next
 *    call, seeing a new context, looks it up again (make that call outside
 *    a stream capture too).
 *  - Every call uses the same array.  Nothing in it needs to start at zero
 *    (each unit overwrites what it reads), but calls that can overlap on
 *    the GPU (different streams, or different host threads) race on it and
 *    must be serialised by the caller.
 *  - Errors: EINVAL when the slots of one block of the upscaling launch do
 *    not fit in the array (message gives the sizes): 8 slots in the FP32
 *    forms (two units per warp), 4 in FP64 (stomsfem_upscale_workspace_size
 *    gives the slot size); plus those of stomsfem_upscale.  This entry point
 *    always runs the default factorisation engine.  Fewer slots than the workspace
 *    path may mean lower throughput. */
int stomsfem_upscale_noalloc(const stomsfem_grid* grid, const double* a, const int8_t* oversample,
                             int32_t max_oversample, int32_t S, int32_t precision,
                             int32_t refine_iters, double* Ke, double* be, double* phi,
                             int32_t* unit_status, stomsfem_stream_t stream);

/* Size in bytes of the static scratch array used by stomsfem_upscale_noalloc. */
size_t stomsfem_upscale_static_scratch_bytes(void);

/* Scratch needed by stomsfem_coarse_solve. */
int stomsfem_coarse_workspace_size(const stomsfem_grid* grid, int32_t S, size_t* bytes);

/* Coarse assembly and solve (Eq. upscaleSUF) with zero Dirichlet data on
 * the boundary nodes, plus the running Monte Carlo moments of Eq.
 * MCestimate.  Ke [S][nc*nc][10], be [S][nc*nc][4] device float64;
 * u device [S][(nc+1)^2] float64 (boundary entries 0).  mean, m2 device
 * [(nc+1)^2] float64 and count device [1] float64 are running accumulators
 * (all zero before the first batch), merged with this batch's moments:
 * mean = M[u], m2 = sum (u - mean)^2 over all samples so far, so the MC
 * variance is m2/count.  mean/m2/count may all be NULL to skip the
 * moments.  Errors: EINVAL, ENOMEM, ECUDA; a sample whose coarse matrix
 * is not positive definite gets NaN in u. */
int stomsfem_coarse_solve(const stomsfem_grid* grid, const double* Ke, const double* be,
                          int32_t S, double* u, double* mean, double* m2, double* count,
                          void* workspace, size_t workspace_bytes, stomsfem_stream_t stream);

/* ---------------------------------------------------------------------
 * Plans (no paper counterpart: the Monte Carlo driver of Sec. 4.1.1 for
 * one batch shape).  A plan owns the intermediate device buffers of a step
 * over S samples -- a [S][nf][nf], Ke [S][nc*nc][10], be [S][nc*nc][4] and
 * the upscaling and coarse workspaces -- and runs
 *   stomsfem_sample_coef_precision (FP32 arithmetic for the FP32 form)
 *   -> stomsfem_upscale -> stomsfem_coarse_solve (+ moments)
 * with launch shapes chosen by stomsfem_plan_tune and the whole step
 * captured once as a CUDA graph.
 * ------------------------------------------------------------------- */
typedef struct stomsfem_plan stomsfem_plan; /* opaque, library-owned */

/* oversample: device [nc*nc] or NULL (owned by the caller, must outlive
 * the plan); precision and refine_iters as stomsfem_upscale.  Allocates
 * device memory (synchronous).  EINVAL on bad arguments, ENOMEM/ECUDA. */
int stomsfem_plan_create(const stomsfem_grid* grid, const stomsfem_field* field, const int8_t* oversample,
                         int32_t max_oversample, int32_t S, int32_t precision, int32_t refine_iters,
                         stomsfem_plan** out);
int stomsfem_plan_destroy(stomsfem_plan* plan);

/* Factorisation engines of the FP32 forms' cell problems (launch choices,
 * no paper counterpart):
 *   STOMSFEM_ENGINE_AUTO     the default (BLOCKED);
 *   STOMSFEM_ENGINE_BLOCKED  banded Cholesky with FP32 FMA updates, two
 *                            units per warp, column blocks of 8, any half
 *                            bandwidth <= 64;
 *   STOMSFEM_ENGINE_TC3      banded Cholesky whose trailing updates run on
 *                            the tensor cores (mma TF32) with every operand
 *                            split exactly into three TF32 parts (six
 *                            products; rounding no worse than FP32), one
 *                            unit per warp, needs 4 <= nf/nc and a half
 *                            bandwidth <= 40;
 *   STOMSFEM_ENGINE_TC2      the same with two parts (three products, about
 *                            2^-21 per product: several times the FP32
 *                            rounding; offered for measurement, never
 *                            picked by the tuner);
 *   STOMSFEM_ENGINE_WIDE     the FMA factorisation with one unit per warp
 *                            and column blocks of 16, any half bandwidth
 *                            <= 64 (Galerkin form without oscillatory
 *                            data).
 * FP64 always uses its own FMA factorisation (BLOCKED). */
enum {
  STOMSFEM_ENGINE_AUTO = 0,
  STOMSFEM_ENGINE_BLOCKED = 1,
  STOMSFEM_ENGINE_TC3 = 2,
  STOMSFEM_ENGINE_TC2 = 3,
  STOMSFEM_ENGINE_WIDE = 4
};

/* Unit orders of the persistent upscaling launches (launch choices):
 *   STOMSFEM_ORDER_CELL   cells fastest (a warp's consecutive units are
 *                         neighbouring cells of one sample);
 *   STOMSFEM_ORDER_PATCH  by patch size, largest first: the cells sorted by
 *                         decreasing oversampling, the samples fastest
 *                         within a cell, so that the longest units start
 *                         first and the launch ends on the shortest ones.
 * Results do not depend on the order. */
enum { STOMSFEM_ORDER_CELL = 0, STOMSFEM_ORDER_PATCH = 1 };

/* Autotuner: runs the step on xi (device [S][nbx*nby]; u device
 * [S][(nc+1)^2] receives the solutions, no moments) under launch choices
 * and keeps the fastest.  Coordinate descent from (all CTAs per SM, split,
 * BLOCKED, ORDER_CELL): first the engine (FP32 forms: BLOCKED, WIDE, and
 * TC3 where the patches are eligible), then the unit order (with
 * oversampling: CELL or PATCH), then the split (FP32 form with
 * oversampling: the separate forward-only launch for the unoversampled
 * cells or one launch), then at most 1, 2 or all resident upscaling CTAs
 * per SM; each candidate is timed over two runs with CUDA events after one
 * untimed run.  Host outputs, any may be NULL: blocks per SM (0 meaning all
 * that fit), split flag, the best time per step in ms; the engine and the
 * order through stomsfem_plan_info.  Synchronises `stream`; drops the
 * captured graph.  The FP32 results depend on the split and engine
 * choices within the FP32 tolerance. */
int stomsfem_plan_tune(stomsfem_plan* plan, const double* xi, double* u, int32_t* blocks_per_sm,
                       int32_t* split_fp32, float* ms_best, stomsfem_stream_t stream);

/* stomsfem_upscale with an explicit factorisation engine for the FP32
 * forms (STOMSFEM_ENGINE_*; ignored in FP64) and unit order
 * (STOMSFEM_ORDER_*; the patch order needs oversampling and room for the
 * cell lists past the slots of one block, else it falls back to the cell
 * order); same arguments, layout and errors otherwise, plus EINVAL for an
 * unknown engine or order, or an engine the form or patches are not
 * eligible for.  Results of different engines agree within the form's
 * tolerance; the order does not change them. */
int stomsfem_upscale_engine(const stomsfem_grid* grid, const double* a, const int8_t* oversample,
                            int32_t max_oversample, int32_t S, int32_t precision, int32_t refine_iters,
                            int32_t engine, int32_t order, double* Ke, double* be, double* phi,
                            int32_t* unit_status, void* workspace, size_t workspace_bytes,
                            stomsfem_stream_t stream);

/* Sets the launch choice without timing: blocks per SM (0 = all that fit),
 * split flag (0 or 1), engine (STOMSFEM_ENGINE_*), unit order
 * (STOMSFEM_ORDER_*).  Drops the captured graph.  EINVAL for values out of
 * range or an engine the plan's form or patches are not eligible for. */
int stomsfem_plan_set_choice(stomsfem_plan* plan, int32_t blocks_per_sm, int32_t split_fp32, int32_t engine,
                             int32_t order);

/* One step: xi (device [S][nbx*nby]) -> u (device [S][(nc+1)^2]) and the
 * running moments (mean, m2, count as stomsfem_coarse_solve, or all NULL).
 * With use_graph != 0 on a created stream the step is captured as a CUDA
 * graph on first use and replayed afterwards; it is captured again when
 * the stream or any of the five pointers changes.  The default streams
 * run the launches directly.  Stream-ordered. */
int stomsfem_plan_step(stomsfem_plan* plan, const double* xi, double* u, double* mean, double* m2,
                       double* count, int32_t use_graph, stomsfem_stream_t stream);

/* The plan's launch choice (engine: the one AUTO resolves to for this
 * plan; unit order), whether a graph is instantiated, and the device
 * memory it owns (host outputs, any may be NULL). */
int stomsfem_plan_info(const stomsfem_plan* plan, int32_t* blocks_per_sm, int32_t* split_fp32,
                       int32_t* engine, int32_t* order, int32_t* graph_ready, size_t* device_bytes);

/* Device time of the upscaling launches (the cell-list kernel and the one
 * or two upscale_kernel launches) of the plan's most recent step, in ms:
 * two timing events of the plan are recorded around them in every step
 * (inside the captured graph as external event nodes).  Waits for the
 * second event (a host wait on that step's upscaling, not on the
 * stream).  EINVAL before the first step. */
int stomsfem_plan_upscale_ms(stomsfem_plan* plan, float* ms);

/* ---------------------------------------------------------------------
 * Local KL parametrization (Sec. 2.1.1, Def. of the local KL expansion,
 * Eqs. localCov, localKL, local_KL_truncation).  On the patch P_m of every
 * coarse cell (the cell plus an oversampling layer of `oversample` fine
 * elements, clipped to the domain) the field's covariance restricted to
 * P_m has eigenpairs (lambda_k, f_k), int_P f_k^2 = 1; a field sample
 * kappa has the local parameters
 *   xi_k = lambda_k^{-1/2} int_P (kappa - kappa_bar) f_k,  k < K_m,
 * and kappa ~ kappa_bar + sum_k sqrt(lambda_k) xi_k f_k on P_m.  The field
 * is piecewise constant on the fine elements (centroid values), integrals
 * use the midpoint rule (weight h^2 per element), so the patch operator is
 * h^2 C_m between element centroids and f_k = u_k / h (u_k orthonormal).
 * ------------------------------------------------------------------- */
typedef struct stomsfem_local_kl stomsfem_local_kl; /* opaque, library-owned */
enum { STOMSFEM_KL_BUMPS = 0, STOMSFEM_KL_GAUSSIAN = 1 };

/* Offline stage on the GPU (FP64, one CTA per cell, Jacobi eigensolver).
 * cov_kind STOMSFEM_KL_BUMPS: the covariance of the bump fields'
 * log-coefficient s z, s^2 var sum_i psi_i(x) psi_i(y) (field: nbx, nby,
 * width, scale; var the variance of each xi_i, 1/3 for U[-1,1], 1 for
 * N(0,1)); STOMSFEM_KL_GAUSSIAN: sigma^2 exp(-|x - y|^2 / beta^2) (field
 * may be NULL).  Modes kept: with energy > 0 the fewest whose eigenvalues
 * reach that share of the patch's spectrum, else kmax; at most kmax (1..32)
 * and only positive eigenvalues (> 1e-12 lambda_1).  k_out host [nc*nc]
 * (or NULL) receives K_m.  Patches of at most 112 fine elements.
 * Synchronises `stream`.  EINVAL on bad arguments, ECUDA. */
int stomsfem_local_kl_build(const stomsfem_grid* grid, int32_t oversample, int32_t cov_kind,
                            const stomsfem_field* field, double var, double beta, double sigma, int32_t kmax,
                            double energy, stomsfem_local_kl** out, int32_t* k_out, stomsfem_stream_t stream);
int stomsfem_local_kl_destroy(stomsfem_local_kl* kl);
/* Host copies (either may be NULL): lam [nc*nc][kmax] (descending, 0 past
 * K_m) and the projection weights w [nc*nc][kmax][112], w_k(e) = h u_k(e) /
 * sqrt(lambda_k) over the patch's elements in y-major order (0 past the
 * patch and past K_m).  Synchronous. */
int stomsfem_local_kl_modes(const stomsfem_local_kl* kl, double* lam_host, double* w_host);
/* Online stage: kappa device [S][nf][nf] (the field, e.g. log a),
 * kappa_bar device [nf][nf] or NULL (zero mean) -> xi device
 * [S][nc*nc][kmax] (0 past K_m), xi_k = sum_e w_k(e) (kappa_e -
 * kappa_bar_e), FP64.  Stream-ordered. */
int stomsfem_local_kl_project(const stomsfem_local_kl* kl, const double* kappa, const double* kappa_bar,
                              int32_t S, double* xi, stomsfem_stream_t stream);

/* ---------------------------------------------------------------------
 * Two-level Monte Carlo (Remark in Sec. 4.1.1, Eq. MCmean2level):
 *   M2 = mean over N_H samples of u_H
 *      + mean over N_h other samples of (u_h - u_H at the coarse nodes),
 * u_h the standard Q1 FEM on the fine grid.  The pieces below compose it:
 * stomsfem_coarse_solve (u_H and its moments), stomsfem_fine_fem (u_h),
 * stomsfem_restrict_to_coarse (the differences) and stomsfem_mc_moments.
 * ------------------------------------------------------------------- */

/* Scratch needed by stomsfem_fine_fem for S samples (nf <= 64: the banded
 * factors of the warps in flight; larger nf: the multigrid hierarchy, the
 * CG vectors and the FP64 operator of all S samples, about 139 bytes per
 * fine node and sample).  EINVAL for an nf above 64 that does not halve down to 16 or
 * less. */
int stomsfem_fine_fem_workspace_size(const stomsfem_grid* grid, int32_t S, size_t* bytes);

/* Standard Q1 FEM on the fine grid with zero Dirichlet data and load f
 * (element matrices a_e K_ref, load f h^2/4 per element corner).
 *  - nf <= 64: one warp per sample on the blocked banded Cholesky of the
 *    coarse solve (NaN for a sample whose matrix is not positive
 *    definite); stream-ordered.
 *  - nf > 64 (nf = c 2^k, c <= 16): conjugate gradients in FP64 on all S
 *    samples at once, preconditioned by one multigrid V-cycle in FP32
 *    (bilinear prolongation, or operator-dependent prolongation when the
 *    batch's coefficient contrast max a / min a exceeds 1e3; Galerkin
 *    coarse operators, damped Jacobi
 *    smoothing), until every sample's recursively updated CG residual is
 *    at most 1e-13 of its load (at most 400 iterations, else ENOTSPD;
 *    ENOTSPD too as soon as a residual is not finite);
 *    the true residual b - A u then sits at the FP64 rounding floor
 *    (about eps || |A| |u| ||, e.g. 2e-11 of the load on a 1024^2
 *    lognormal medium); synchronises `stream` (convergence is checked on
 *    the host every four iterations).
 * a device [S][nf][nf], u device [S][(nf+1)^2] (boundary entries 0). */
int stomsfem_fine_fem(const stomsfem_grid* grid, const double* a, int32_t S, double* u, void* workspace,
                      size_t workspace_bytes, stomsfem_stream_t stream);

/* d [S][(nc+1)^2] = u_fine [S][(nf+1)^2] at the coarse nodes, minus
 * u_coarse [S][(nc+1)^2] when it is not NULL (device arrays). */
int stomsfem_restrict_to_coarse(const stomsfem_grid* grid, const double* u_fine, const double* u_coarse,
                                int32_t S, double* d, stomsfem_stream_t stream);

/* Running Monte Carlo moments of S samples u [S][n] (device) merged into
 * mean [n], m2 [n] and count [1] (device, zero before the first batch), as
 * stomsfem_coarse_solve does for its solutions. */
int stomsfem_mc_moments(int32_t n, int32_t S, const double* u, double* mean, double* m2, double* count,
                        stomsfem_stream_t stream);

/* Merges a second set of running moments (mean_b [n], m2_b [n], count_b
 * [1], device; e.g. another rank's, gathered after a multi-GPU run) into
 * (mean, m2, count) in place, by the pairwise update of Chan, Golub and
 * LeVeque: the result equals the moments of both sample sets together (up
 * to rounding).  A zero count_b leaves the first set unchanged.
 * Stream-ordered.  EINVAL on n <= 0 or a NULL pointer. */
int stomsfem_mc_merge(int32_t n, double* mean, double* m2, double* count, const double* mean_b,
                      const double* m2_b, const double* count_b, stomsfem_stream_t stream);

/* Petrov-Galerkin form of stomsfem_upscale (Eq. stiffness_local_petrov;
 * the form the paper uses with oversampling): same cell problems, same
 * arguments, but the test functions are the cell's bilinear nodal
 * functions q_l', so
 *   Ke [S][nc*nc][16]  S_ll' = int_cell a grad phi_l . grad q_l', row-major
 *                      (row l = trial basis function, column l' = test),
 *   be [S][nc*nc][4]   b_l = int_cell f q_l = f H^2 / 4 (deterministic).
 * Without oversampling S_ll' equals the Galerkin matrix (phi_l' - q_l'
 * vanishes on the cell boundary and phi_l is discrete-harmonic), so those
 * cells give the symmetric 16 entries.  Workspace, precision, refinement,
 * phi output, statuses and errors as stomsfem_upscale. */
int stomsfem_upscale_pg(const stomsfem_grid* grid, const double* a, const int8_t* oversample,
                        int32_t max_oversample, int32_t S, int32_t precision, int32_t refine_iters,
                        double* Ke, double* be, double* phi, int32_t* unit_status, void* workspace,
                        size_t workspace_bytes, stomsfem_stream_t stream);

/* Local upscaling with a choice of boundary data for the cell problems:
 * bc = STOMSFEM_BC_BILINEAR is stomsfem_upscale (pg = 0) or
 * stomsfem_upscale_pg (pg = 1); bc = STOMSFEM_BC_OSCILLATORY gives every
 * patch edge the oscillatory data of the short-correlation example's MsFEM
 * (Sec. 5.3): each nodal function interpolates its two corner values
 * linearly in the edge's harmonic coordinate sum_{e<k} 1/a_e / sum_e 1/a_e
 * (a_e the patch element next to edge segment e, the reduced problem
 * (a u')' = 0 along the edge) instead of in arc length.  In a medium that
 * does not vary along an edge the two coincide there.  Arguments, layouts
 * (Ke 10 entries per unit, or 16 with pg = 1), workspace (that of
 * stomsfem_upscale_workspace_size), statuses and errors as those calls; with
 * oscillatory data every cell takes the back-substitution route in one
 * launch, also in FP32.  Errors: EINVAL also for pg not 0 or 1 and an
 * unknown bc. */
int stomsfem_upscale_bc(const stomsfem_grid* grid, int32_t pg, int32_t bc, const double* a,
                        const int8_t* oversample, int32_t max_oversample, int32_t S, int32_t precision,
                        int32_t refine_iters, double* Ke, double* be, double* phi, int32_t* unit_status,
                        void* workspace, size_t workspace_bytes, stomsfem_stream_t stream);

/* Scratch needed by stomsfem_coarse_solve_pg. */
int stomsfem_coarse_pg_workspace_size(const stomsfem_grid* grid, int32_t S, size_t* bytes);

/* Coarse solve of the Petrov-Galerkin system: U with
 * sum_I U_I S(phi_I, q_J) = b_J for every interior coarse node J (row J
 * collects S_e[I_loc][J_loc] over the cells around J; zero Dirichlet data),
 * by banded LU without pivoting (half bandwidth nc), one warp per sample.
 * Ke [S][nc*nc][16], be [S][nc*nc][4] from stomsfem_upscale_pg; u, mean,
 * m2, count as stomsfem_coarse_solve.  A sample whose elimination meets a
 * zero or non-finite pivot gets NaN in u.  Errors: EINVAL (also nc < 2 or
 * nc > 64), ENOMEM, ECUDA. */
int stomsfem_coarse_solve_pg(const stomsfem_grid* grid, const double* Ke, const double* be, int32_t S,
                             double* u, double* mean, double* m2, double* count, void* workspace,
                             size_t workspace_bytes, stomsfem_stream_t stream);

/* Scratch needed by stomsfem_coarse_solve_bc for the form pg (0 Galerkin,
 * 1 Petrov-Galerkin). */
int stomsfem_coarse_bc_workspace_size(const stomsfem_grid* grid, int32_t pg, int32_t S, size_t* bytes);

/* Coarse solve with mixed boundary data, the boundary conditions of the
 * anisotropy study of the high-contrast example (Sec. 5.2, Eqs.
 * xsquarewave and ysquarewave: prescribed values on node lines, zero flux
 * on the rest of the boundary).  Every coarse node is an unknown:
 *   dirichlet [(nc+1)^2] uint8 (device)  nonzero: u is prescribed there
 *                                        (any node, interior lines too),
 *   g         [(nc+1)^2] float64 (device) the prescribed values (read
 *                                        where dirichlet is nonzero),
 * node (i, j) at j*(nc+1)+i, shared by the S samples.  The other nodes
 * carry the natural condition (zero flux on the boundary).  pg = 0:
 * Galerkin, K = Ke [S][nc*nc][10] and b = be [S][nc*nc][4] of
 * stomsfem_upscale, symmetric elimination of the prescribed nodes and the
 * blocked banded Cholesky (half bandwidth nc + 2); pg = 1:
 * Petrov-Galerkin, K [S][nc*nc][16] and b [S][nc*nc][4] of
 * stomsfem_upscale_pg, banded LU without pivoting.  One warp per sample.
 * u [S][(nc+1)^2] takes every node (g at the prescribed ones); mean, m2,
 * count as stomsfem_coarse_solve.  The caller makes the problem well posed
 * (at least one prescribed node in every part of the domain the cells
 * connect): a sample whose factorisation meets a non-positive (pg = 0) or
 * a zero or non-finite (pg = 1) pivot gets NaN in u.  Errors: EINVAL (also
 * nc > 62, pg not 0 or 1), ENOMEM (workspace below two slots), ECUDA. */
int stomsfem_coarse_solve_bc(const stomsfem_grid* grid, int32_t pg, const double* K, const double* b,
                             const uint8_t* dirichlet, const double* g, int32_t S, double* u, double* mean,
                             double* m2, double* count, void* workspace, size_t workspace_bytes,
                             stomsfem_stream_t stream);

/* ---------------------------------------------------------------------
 * Reduced-basis (POD) upscaling, Sec. 3.2 (Eq. KLphi, Eqs. localRB and
 * localRBsystem, Algs. 3 and 4), for cells without oversampling.
 * ------------------------------------------------------------------- */
typedef struct stomsfem_pod stomsfem_pod; /* opaque, owned by the library */

/* Offline stage (Alg. 3).  Inputs are training snapshots of the multiscale
 * basis as produced by stomsfem_upscale (phi output, oversample NULL) and
 * the training coefficients:
 *   phi_snap  device [S_train][nc*nc][4][(rho+1)^2] float64
 *   a_train   device [S_train][nf][nf] float64
 * Per cell: phibar_l = training mean of phi_l; abar = training mean of a;
 * KL expansion of the centred interior snapshots (the four l stacked, one
 * basis per cell) in the energy inner product int abar grad u . grad v
 * (footnote of Eq. KLphi); modes kept while sqrt(lambda_q/lambda_1) >= tol,
 * at most max_rank; or, if ranks_in (host [nc*nc]) is not NULL, exactly
 * ranks_in[cell] modes.  ranks_out (host [nc*nc], may be NULL) receives the
 * ranks.  Limits: 2 <= rho <= 32, 1 <= max_rank <= 27.  For rho <= 8 the
 * KL eigenproblem is the interior-node covariance's ((rho-1)^2 wide); for
 * 8 < rho <= 32 it is solved in snapshot space (the 4 S_train x 4 S_train
 * matrix X^T Abar X / (4 S_train) of the centred snapshots X, whose
 * nonzero eigenvalues are the covariance's, modes X v / sqrt(4 S_train
 * lambda)): S_train <= 24 there, and the eigenvalues past 4 S_train read 0.
 * Allocates the handle's device memory and synchronises `stream` before
 * returning.  Errors: EINVAL, ENOTSPD (training-mean energy matrix, rho <=
 * 8), ECUDA. */
int stomsfem_pod_build(const stomsfem_grid* grid, const double* phi_snap, const double* a_train,
                       int32_t S_train, double tol, int32_t max_rank, const int32_t* ranks_in,
                       stomsfem_pod** out, int32_t* ranks_out, stomsfem_stream_t stream);
/* The same call under the name of the method's offline step ("build the
 * POD basis"); identical arguments, results and errors. */
int stomsfem_build_pod(const stomsfem_grid* grid, const double* phi_snap, const double* a_train,
                       int32_t S_train, double tol, int32_t max_rank, const int32_t* ranks_in,
                       stomsfem_pod** out, int32_t* ranks_out, stomsfem_stream_t stream);

/* Offline stage with one reduced basis per basis function (the patch study
 * of Sec. 5.1 expands phi^1, phi^2, phi^3 separately): per cell and
 * l = 1..3, the KL expansion of the centred interior snapshots of phi_l
 * alone in the same energy inner product, truncated by the same rule at
 * most max_rank_per_l modes (or exactly ranks_in[cell][l], host
 * [nc*nc][3]); phi_4 follows online from the partition of unity,
 * phi_4 = 1 - phi_1 - phi_2 - phi_3.  The extended basis is
 * W = [phibar_1..4, V_1, V_2, V_3] (each V_l in a block of max_rank_per_l
 * columns), the online reduced systems block diagonal (one per l, one
 * right-hand side each).  ranks_out host [nc*nc][3] or NULL.  Limits:
 * 2 <= rho <= 8, 1 <= max_rank_per_l <= 9.  The handle serves
 * stomsfem_pod_upscale, stomsfem_pod_set_affine / _upscale_affine, save and
 * load like a shared-basis one.  Errors as stomsfem_pod_build. */
int stomsfem_pod_build_per_l(const stomsfem_grid* grid, const double* phi_snap, const double* a_train,
                             int32_t S_train, double tol, int32_t max_rank_per_l, const int32_t* ranks_in,
                             stomsfem_pod** out, int32_t* ranks_out, stomsfem_stream_t stream);

/* Frees the handle (synchronous). */
int stomsfem_pod_destroy(stomsfem_pod* pod);

/* Copies all KL eigenvalues, host [nc*nc][(rho-1)^2] (per-l handles:
 * [nc*nc][3][(rho-1)^2]), descending per cell (and l) (synchronous). */
int stomsfem_pod_eigenvalues(const stomsfem_pod* pod, double* lam_host);

/* Checkpoint of the offline stage, so that the online stage (Alg. 4) can run
 * in another process without repeating Alg. 3.  Serialises the basis W,
 * load weights, eigenvalues, BF16 element tensors and ranks into the
 * caller's host buffer: with host_buf NULL only *bytes is set (the size
 * needed); ENOMEM if buf_bytes is smaller (then *bytes holds the size).
 * Format: magic "STMFPOD1" ("STMFPODL" for per-l bases), format version,
 * byte-order probe, dimensions, arrays in native byte order.  Synchronous. */
int stomsfem_pod_save(const stomsfem_pod* pod, void* host_buf, size_t buf_bytes, size_t* bytes);
/* Rebuilds a handle from a stomsfem_pod_save buffer.  EVERSION if the magic
 * tag, format version or byte order differ; EINVAL if the buffer is
 * truncated or its dimensions are inconsistent.  Synchronous. */
int stomsfem_pod_load(const void* host_buf, size_t buf_bytes, stomsfem_pod** out);

/* Scratch of stomsfem_pod_upscale for S samples (BF16 copy of a by cell,
 * [nc*nc][S rounded up to 128][rho^2 rounded up to 64], and the FP32
 * reduced matrices [nc*nc][S rounded up to 128][packed pairs rounded up to
 * 16]; about 4 MB per sample at H/h = 32 on a 64 x 64 coarse grid). */
int stomsfem_pod_workspace_size(const stomsfem_pod* pod, int32_t S, size_t* bytes);

/* Online stage (Alg. 4) for S samples a (device [S][nf][nf] float64):
 * G = W^T A(omega) W for the extended basis W = [phibar, V] as one
 * tensor-core GEMM per cell (BF16 operands, FP32 accumulation; K = the
 * cell's rho^2 elements in steps of 64; by default each operand carried as
 * a BF16 pair, value and BF16 of the remainder, and three products
 * summed, about 16 significant bits in G: see stomsfem_pod_set_gemm_split),
 * the r x r
 * Galerkin system (V^T A V) c_l = -V^T A phibar_l in FP32, then
 * refine_iters FP64 refinement steps whose residual is formed with the fine
 * 9-point stencil of A(omega) (0 = none: K_e and b_e from the FP32 reduced
 * quantities).  Outputs as in stomsfem_upscale (Ke [S][nc*nc][10], be
 * [S][nc*nc][4], unit_status [S][nc*nc] or NULL: 0, ENOTSPD, ETIMEOUT).
 * The refinement needs rho <= 8.  Errors: EINVAL, ENOMEM (workspace),
 * ECUDA. */
int stomsfem_pod_upscale(stomsfem_pod* pod, const double* a, int32_t S, int32_t refine_iters,
                         double* Ke, double* be, int32_t* unit_status, void* workspace,
                         size_t workspace_bytes, stomsfem_stream_t stream);

/* The online GEMM's operand precision (no paper counterpart): split = 1
 * (the default) both operands as BF16 (hi, lo) pairs and three tensor-core
 * products per K step (hi hi + hi lo + lo hi); split = 0 one BF16 product
 * (8 significant bits in G: enough where the reduced matrices are well
 * conditioned, e.g. the H/h = 8 workloads; at contrast 10^4 and H/h = 32
 * the reduced Cholesky then meets non-positive pivots).  EINVAL for a NULL
 * handle or another value. */
int stomsfem_pod_set_gemm_split(stomsfem_pod* pod, int32_t split);

/* Affine structure of the coefficient (Sec. 3.2.2, Eqs. RBaffine and
 * localAF) for an affine field (field->kind == STOMSFEM_FIELD_AFFINE,
 * a = gain + scale z): with the cell's local parameters xi_m (bump i local
 * when exp(-d^2/width^2) >= tau, as stomsfem_local_vars; the others are
 * dropped), every reduced quantity of the handle's basis
 * W = [phibar_1..4, V] splits as
 *   W^T A(xi) W = gain G_0 + scale sum_k xi_k G_k,
 *   G_0 = sum_e W_e^T K_ref W_e,  G_k = sum_e psi_k(x_e) W_e^T K_ref W_e,
 * computed here once per cell in FP64 (stored FP32).  grid must be the
 * handle's and rho <= 8; EINVAL for another field kind or more than 16
 * local parameters.  Allocates device memory, synchronises `stream`.  The parts
 * are not part of stomsfem_pod_save; call again after a load. */
int stomsfem_pod_set_affine(stomsfem_pod* pod, const stomsfem_grid* grid, const stomsfem_field* field,
                            double tau, stomsfem_stream_t stream);

/* Online stage with the affine parts (Alg. 4 without the fine grid): per
 * (sample, cell) unit the reduced quantities are assembled from xi
 * (device [S][nbx*nby]) in shared memory, then solved as in
 * stomsfem_pod_upscale (FP32 reduced Cholesky, K_e and b_e from the
 * reduced quantities; refine_iters > 0 runs the FP64 stencil refinement,
 * which needs a, device [S][nf][nf]; a may be NULL otherwise).  No
 * workspace.  Ke [S][nc*nc][10], be [S][nc*nc][4], unit_status as
 * stomsfem_pod_upscale.  EINVAL if stomsfem_pod_set_affine was not called. */
int stomsfem_pod_upscale_affine(stomsfem_pod* pod, const double* xi, const double* a, int32_t S,
                                int32_t refine_iters, double* Ke, double* be, int32_t* unit_status,
                                stomsfem_stream_t stream);

/* ---------------------------------------------------------------------
 * Learned surrogate of the local upscaled quantities (stands in for the
 * random-interpolation model of S^m(xi_m), b^m(xi_m), Sec. 3.1, Algs. 1-2;
 * the cell problem depends on the local parameters xi_m only, Eq. MsFEB2).
 * Cells without oversampling.  Per patch family an MLP
 *   16 -> 128 -> 128 -> 128 -> 16 (GELU), weights [out][in] per layer,
 *   flat FP32 layout per family: W1[128][16] b1[128] W2[128][128] b2[128]
 *   W3[128][128] b3[128] W4[16][128] b4[16]  (37264 floats),
 * maps the zero-padded xi_m to y; targets y_0..9 = K_e/abar - K_ref,
 * y_10..12 = b_l/(f H^2) - 1/4 (abar = mean of a over the cell).
 * ------------------------------------------------------------------- */
typedef struct stomsfem_surrogate stomsfem_surrogate; /* opaque, library-owned */

typedef struct {
  int32_t steps;      /* Adam steps (minibatches of 64 rows per family) */
  double lr, lr_min;  /* cosine decay from lr to lr_min */
  double beta1, beta2, eps;
  uint64_t seed;      /* minibatch selection (splitmix64 of seed, family, step, row) */
  int32_t fp32_products; /* 0: BF16 products, FP32 accumulation (the training
                            mode); 1: FP32 products and activations (the
                            slower check mode, for comparisons with FP64) */
} stomsfem_surrogate_cfg;

/* Local parameters of every cell (host computation, no GPU): variable i is
 * local to a cell when exp(-d^2/width^2) >= tau, d the distance from bump
 * centre i to the closed cell rectangle; per cell sorted by the centre's
 * offset from the cell's south-west corner (y then x).  Cells with equal
 * offset lists form one family.  Outputs (host, any may be NULL):
 * k_per_cell [nc*nc], var_ids [nc*nc][16] (-1 padded), family [nc*nc],
 * n_families.  EINVAL if a cell has more than 16 local variables. */
int stomsfem_local_vars(const stomsfem_grid* grid, const stomsfem_field* field, double tau,
                        int32_t* k_per_cell, int32_t* var_ids, int32_t* family,
                        int32_t* n_families);

/* Seeded Xavier-uniform initial weights for n_families networks into the
 * host buffer w_host [n_families][37264] (flat layout above): each weight
 * lim (2 u - 1), lim = sqrt(6 / (fan_in + fan_out)), u uniform in [0, 1)
 * from the top 53 bits of SplitMix64(seed ^ family << 48 ^ parameter
 * index); biases zero.  Host only; EINVAL for n_families < 1 or NULL. */
int stomsfem_surrogate_init_weights(int32_t n_families, uint64_t seed, float* w_host);

/* Creates a surrogate with the given initial weights (host [nfam][37264],
 * e.g. from stomsfem_surrogate_init_weights; query nfam with
 * stomsfem_local_vars).  Allocates device memory (synchronous). */
int stomsfem_surrogate_create(const stomsfem_grid* grid, const stomsfem_field* field, double tau,
                              const float* init_weights, stomsfem_surrogate** out,
                              int32_t* n_families);
int stomsfem_surrogate_destroy(stomsfem_surrogate* sg);
/* Copies the FP32 master weights to host [nfam][37264] (synchronous). */
int stomsfem_surrogate_weights(const stomsfem_surrogate* sg, float* w_host);

/* Checkpoint / resume of a surrogate (no paper counterpart; the paper's
 * interpolation tables play this role for Alg. 1-2): grid, field, tau, the
 * FP32 master weights, Adam moments, step count and the per-family training
 * input box, into the caller's host buffer (host_buf NULL: size only;
 * ENOMEM if too small).  Format: magic "STMFSUR1", format version,
 * byte-order probe, then fields in native byte order.  Synchronous. */
int stomsfem_surrogate_save(const stomsfem_surrogate* sg, void* host_buf, size_t buf_bytes, size_t* bytes);
/* Rebuilds a surrogate from a stomsfem_surrogate_save buffer; the families
 * are re-derived from grid, field and tau and must match the stored count.
 * Training resumes at the stored step.  EVERSION on a foreign or other-
 * version buffer; EINVAL if truncated or inconsistent.  Synchronous. */
int stomsfem_surrogate_load(const void* host_buf, size_t buf_bytes, stomsfem_surrogate** out,
                            int32_t* n_families);

/* Trains on the S samples' (xi, a, K_e, b_e) (device: xi [S][nbx*nby],
 * a [S][nf][nf], Ke [S][nc*nc][10], be [S][nc*nc][4], from the plain
 * upscaler): one fused forward/backward/Adam kernel, one CTA per family;
 * every 10th row of a family is held out.  loss_hist (host [steps] or NULL)
 * receives the family-averaged training loss per step.  Allocates the
 * training rows and synchronises `stream`.  Successive calls continue the
 * Adam state and step count. */
int stomsfem_surrogate_train(stomsfem_surrogate* sg, const stomsfem_surrogate_cfg* cfg,
                             const double* xi, const double* a, const double* Ke, const double* be,
                             int32_t S, float* loss_hist, stomsfem_stream_t stream);

/* One forward/backward pass of the training kernel on a batch of exactly 64
 * rows, no update: weights device [37264], X device [64][16], T device
 * [64][16] (targets; columns 13..15 ignored), grad device [37264] receives
 * d loss / d weights for loss = mean over rows and the 13 used outputs of
 * (y - T)^2; loss device [1] or NULL.  fp32_products as in
 * stomsfem_surrogate_cfg.  Stream-ordered, allocates nothing.  For
 * gradient checks. */
int stomsfem_surrogate_grad(const float* weights, const float* X, const float* T, int32_t fp32_products,
                            float* grad, float* loss, stomsfem_stream_t stream);

/* Scratch of stomsfem_surrogate_infer for S samples. */
int stomsfem_surrogate_workspace_size(const stomsfem_surrogate* sg, int32_t S, size_t* bytes);

/* Inference with fallback for S samples (device: xi [S][nbx*nby],
 * a [S][nf][nf]).  Every (sample, cell) unit goes through its family's
 * network on the tensor cores (BF16 operands, FP32 accumulation, one
 * 128-unit tile per CTA); the 10 outputs are projected onto symmetric
 * zero-row-sum matrices and scaled by abar.  Error indicator, per unit:
 * an input outside the family's training range (1% margin); for the x- and
 * y-linear corner vectors v, v^T K v outside [ahar (1 - delta),
 * abar (1 + delta)] (harmonic and arithmetic cell means of a: the energy
 * bounds of the cell problem with affine data); K not positive definite
 * on the complement of the constants.  With an ensemble partner
 * (stomsfem_surrogate_set_partner), also: the partner network's K_e on the
 * same inputs differs from this one's by more than tol relative.  Flagged
 * units (fell_back device [S][nc*nc] uint8: 1 by the rules above, 2 by the
 * ensemble test, 0 accepted) are recomputed by the plain FP64 upscaler in
 * the same call.  Outputs Ke [S][nc*nc][10], be [S][nc*nc][4] (device).
 * A device-side wait that ran out flags every unit (all fall back). */
int stomsfem_surrogate_infer(stomsfem_surrogate* sg, const double* xi, const double* a, int32_t S,
                             double delta, double* Ke, double* be, uint8_t* fell_back,
                             void* workspace, size_t workspace_bytes, stomsfem_stream_t stream);

/* Ensemble indicator (the a-posteriori detection of Sec. 3.2 read as the
 * disagreement of two independently trained networks; no paper formula):
 * stomsfem_surrogate_infer on sg also runs `partner` (a second surrogate of
 * the same grid, local variables and families, trained from other initial
 * weights; not owned, it must outlive its use) and sends to the fallback
 * every unit the rules accepted whose two K_e differ by more than tol
 * (||K1 - K2|| > tol ||K1||, Euclidean norm over the 10 packed entries).
 * partner NULL removes it.  Changes the workspace size
 * (stomsfem_surrogate_workspace_size: query again).  Not part of
 * stomsfem_surrogate_save.  EINVAL: sg NULL, partner == sg, tol < 0, or a
 * partner of other families. */
int stomsfem_surrogate_set_partner(stomsfem_surrogate* sg, const stomsfem_surrogate* partner, double tol);

/* ---------------------------------------------------------------------
 * Random interpolation of the local upscaled quantities (Sec. 3.1,
 * Algorithms 1 and 2; accuracy: Thm. approx_S).  Cells without
 * oversampling.  Per cell, bump i is an interpolated direction with degree
 * nu_i >= 1 when its strength g_i = max over the closed cell of
 * |d log a / d xi_i| (scale exp(-d^2/w^2) for the exponential field,
 * |contrast_log gain| / 4 exp(-d^2/w^2) for the sigmoid one) makes
 * 2 (g_i/2)^(nu+1) / (nu+1)! > eps for every smaller nu (nu capped at
 * nu_max); other bumps are frozen at xi_i = 0.  Directions are ordered by
 * degree, then by the bump's offset from the cell's south-west corner
 * (y, then x); cells with equal (offset, degree) lists form one family and
 * share one interpolant, built on the family's first cell.  The family's
 * collocation grid is the tensor product of nu_i + 1 nodes per direction
 * (last direction fastest): Chebyshev points of the first kind or
 * Legendre zeros on [-1, 1].
 * ------------------------------------------------------------------- */
enum { STOMSFEM_RI_CHEBYSHEV = 0, STOMSFEM_RI_LEGENDRE = 1 };
typedef struct stomsfem_ri stomsfem_ri; /* opaque, library-owned */

/* The plan of stomsfem_ri_build without building it (host, no GPU).
 * Outputs (host, any may be NULL): family [nc*nc]; var_ids [nc*nc][16]
 * (bump index per direction in table order, -1 padded); nu [nc*nc][16]
 * (0 padded); n_families; n_points (grid points over all families).
 * EINVAL: bad arguments, nu_max outside [1, 8], a cell with more than 16
 * directions, a family with more than 64 node slots or 2048 grid points. */
int stomsfem_ri_plan(const stomsfem_grid* grid, const stomsfem_field* field, double eps, int32_t nu_max,
                     int32_t* family, int32_t* var_ids, int32_t* nu, int32_t* n_families,
                     int64_t* n_points);

/* Offline stage (Alg. 1): for every grid point of every family one
 * coefficient sample (the family's directions at the point's nodes, every
 * other xi 0), the family's first cell upscaled by the FP64 path; the
 * K_e (10) and b_e (4) entries are the interpolation data.  Allocates
 * device memory, synchronises `stream`.  Errors as stomsfem_ri_plan, plus
 * ENOMEM / ECUDA. */
int stomsfem_ri_build(const stomsfem_grid* grid, const stomsfem_field* field, double eps, int32_t nu_max,
                      int32_t nodes, stomsfem_ri** out, int32_t* n_families, stomsfem_stream_t stream);
int stomsfem_ri_destroy(stomsfem_ri* ri);
/* The FP64 interpolation data, host [n_points][14] (K_e packed, then b_e),
 * families in order, each family's grid points last direction fastest.
 * Synchronous. */
int stomsfem_ri_values(const stomsfem_ri* ri, double* V_host, int64_t n_points);
/* Checkpoint of an interpolation handle (no paper counterpart; the
 * interpolation data are the offline stage's whole output): grid, field,
 * eps, nu_max, node family and the FP64 data, into the caller's host
 * buffer (host_buf NULL: size only; ENOMEM if too small).  Format: magic
 * "STMFRIT1", format version, byte-order probe, then fixed-width fields in
 * native byte order.  Synchronous. */
int stomsfem_ri_save(const stomsfem_ri* ri, void* host_buf, size_t buf_bytes, size_t* bytes);
/* Rebuilds a handle from a stomsfem_ri_save buffer without the offline
 * solves: the plan is re-derived from the stored grid, field, eps and
 * nu_max and must have the stored number of grid points.  EVERSION on a
 * foreign or other-version buffer; EINVAL if truncated or inconsistent.
 * Allocates device memory (synchronous). */
int stomsfem_ri_load(const void* host_buf, size_t buf_bytes, stomsfem_ri** out, int32_t* n_families);

/* Scratch of stomsfem_ri_upscale for S samples. */
int stomsfem_ri_workspace_size(const stomsfem_ri* ri, int32_t S, size_t* bytes);
/* Online stage (Alg. 2) for S samples (device: xi [S][nbx*nby], a
 * [S][nf][nf] or NULL).  Per (sample, cell) unit the tensor Lagrange
 * interpolant of the 14 entries at the cell's local parameters (second
 * barycentric form per direction, FP32 sum over the family's grid held in
 * shared memory, two units per thread), written as FP64 to Ke [S][nc*nc][10], be [S][nc*nc][4].
 * A unit with a local parameter outside [-1, 1] (or NaN) is upscaled
 * directly by the FP64 path from `a` in the same call, fell_back = 1; with
 * a == NULL it gets NaN entries and fell_back = 2.  Other units:
 * fell_back = 0.  Errors: EINVAL, ENOMEM (workspace), ECUDA. */
int stomsfem_ri_upscale(stomsfem_ri* ri, const double* xi, const double* a, int32_t S, double* Ke,
                        double* be, uint8_t* fell_back, void* workspace, size_t workspace_bytes,
                        stomsfem_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* STOMSFEM_H */
