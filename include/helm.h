/*
 * helm.h - C ABI of the GB300 (sm_103a) library for the learned multigrid-augmented
 * Helmholtz solver of Lerer, Ben-Yair and Treister (arXiv 2306.17486).
 *
 * The library solves the h^2-scaled discrete heterogeneous Helmholtz system
 *
 *     h^2 A u = h^2 g,   A = -Delta_h - omega^2 kappa^2 (1 - gamma i)        (Eq. 1-3)
 *
 * on an nx x ny grid (zero Dirichlet values outside, absorbing layer in gamma) with
 * flexible GMRES (Saad 1993), preconditioned either by a shifted-Laplacian multigrid
 * V-cycle (Section 3.2, Algorithm 1, Eq. 4, 6, 8) or by the encoder-solver U-Net with
 * its implicit coarsest layer composed with that V-cycle (Section 4).
 *
 * Conventions shared by every call
 *   - Complex vectors are interleaved (re, im) float32 ("complex64") or float64
 *     ("complex128"), row-major [batch][ny][nx], one right-hand side per batch item.
 *   - Every pointer argument named *_dev, and every vector argument of the hot calls,
 *     is DEVICE memory owned by the caller; the library never frees it.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Hot calls are
 *     asynchronous and stream-ordered; they allocate nothing: scratch comes from the
 *     caller's workspace, whose size helm_workspace_size() returns.
 *   - Return value: HELM_OK (0) or a negative HELM_E* code; helm_last_error_string()
 *     describes the last failure on the calling thread.  Per-right-hand-side
 *     non-convergence is not a call error: it is reported in helm_fgmres_stats.status.
 *   - Device kernels never spin unboundedly: a wait that times out sets a bit in the
 *     device error word, read (and cleared) with helm_device_errors().
 */
#ifndef HELM_H
#define HELM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---------------------------------------------------------------- */
#define HELM_OK 0
#define HELM_EINVAL (-1)     /* bad argument (null pointer, non-positive size, ...)        */
#define HELM_ESHAPE (-2)     /* grid not divisible as required (see each call)            */
#define HELM_ECUDA (-3)      /* a CUDA runtime / driver call failed                       */
#define HELM_ENOMEM (-4)     /* setup allocation failed                                   */
#define HELM_ETIMEOUT (-5)   /* a device-side bounded wait gave up (device error word set) */
#define HELM_EWORKSPACE (-6) /* workspace smaller than helm_workspace_size()              */
#define HELM_ESTATE (-7)     /* call made in the wrong state (e.g. backward without a
                                training forward)                                        */

/* ---- per-RHS solver status (helm_fgmres_stats.status) ---------------------------- */
#define HELM_STATUS_ACTIVE 0
#define HELM_STATUS_CONVERGED 1
#define HELM_STATUS_MAXIT 2
#define HELM_STATUS_NONFINITE 3

/* ---- device error word bits ------------------------------------------------------ */
#define HELM_DEVERR_TMA_WAIT 1u   /* a TMA completion wait ran out                       */
#define HELM_DEVERR_MMA_WAIT 2u   /* a tensor-core completion wait ran out               */

/* ---- convolution modes (helm_conv_bf16) ----------------------------------------- */
#define HELM_CONV_S1 0 /* 3x3, stride 1, zero padding 1                                  */
#define HELM_CONV_S2 1 /* 3x3, stride 2, padding 1: output H/2 x W/2                      */
#define HELM_CONV_T2 2 /* 3x3 transposed, stride 2, padding 1, output padding 1: 2H x 2W  */
#define HELM_CONV_T1 3 /* 3x3 transposed, stride 1, padding 1 (= S1 with flipped kernel)  */

typedef struct helm_problem helm_problem; /* one slowness model + frequency + multigrid  */

/* ---- boundary conditions outside the grid (helm_mg_opts.bc) ------------------------
 * Each replaces the ghost value next to a boundary node u_b by c u_b, which adds c per
 * boundary side to the node's mass term; the stencil kernels are the same for all.   */
#define HELM_BC_DIRICHLET 0  /* c = 0: zero padding, the paper's setting (Section 3.4)       */
#define HELM_BC_NEUMANN 1    /* c = 1: replication padding (Section 3.4, remark on Neumann)  */
#define HELM_BC_SOMMERFELD 2 /* c = 1 - i omega h kappa_b: first-order outgoing-wave
                                condition du/dn + i omega kappa u = 0 (Section 3.1 names
                                Sommerfeld as an alternative to the absorbing layer)     */

/* Multigrid options (Section 3.2 / 3.4); also the problem's boundary condition. */
typedef struct {
  int levels;            /* grid levels incl. the finest (>= 2); nx, ny divisible by 2^levels */
  double beta;           /* imaginary shift of Eq. (4), alpha = 1 (paper: 0.5)              */
  double omega_jacobi;   /* damped-Jacobi weight (0.8)                                       */
  int coarse_iters;      /* GMRES iterations with Jacobi right-preconditioning on the
                            coarsest grid (Section 3.4; default 10, run to the full count)  */
  int sl_includes_gamma; /* 0: SL mass (1 - beta i); 1: (1 - (beta + gamma) i)               */
  int boundary_fix;      /* 1: coarse grids keep the low-side Dirichlet boundary at the
                            fine position (ghost-point correction of the first row/col);
                            Dirichlet problems only                                         */
  int bc;                /* HELM_BC_*: the operator's boundary condition (default
                            Dirichlet); every multigrid level is rediscretised with it,
                            with kappa_l = sqrt(restricted kappa^2) and h_l = 2^l h       */
} helm_mg_opts;

/* Fill `o` with the defaults above (levels = 3). */
void helm_mg_opts_default(helm_mg_opts* o);

/*
 * Create a problem (Section 3.1): copies kappa (device, float32 [ny][nx], slowness
 * including the absorbing-layer cells), builds on the device
 *   gamma(x) = gamma0 + max((d_x/abl)^2, (d_y/abl)^2)   (absorbing layer, quadratic ramp)
 *   mass_A   = (omega h)^2 kappa^2 (1 - gamma i)        (fine Helmholtz operator, Eq. 3)
 *   mass_SL,l = (omega h 2^l)^2 kappa_l^2 (1 - beta i)  (SL operator per level, Eq. 4),
 *              kappa_l^2 the full-weighting average of kappa^2 (Eq. 8)
 * and the damped Jacobi inverse diagonals omega_J / (4 - mass_SL,l).
 * omega_h is omega times the grid spacing (10 points per wavelength: 2 pi / 10).
 * Returns HELM_ESHAPE unless nx, ny are even and divisible by 2^levels.
 * The problem owns its device arrays until helm_problem_destroy().
 */
int helm_problem_create(const float* kappa_dev, int nx, int ny, int abl, double omega_h, double gamma0,
                        const helm_mg_opts* opts, void* stream, helm_problem** out);
int helm_problem_destroy(helm_problem* p);

/* Recompute problem p's setup fields (those of helm_problem_create: Section 3.1 Eq. 1-3,
 * Section 3.2 Eq. 4 and 8) in place for a new slowness model kappa_dev (same
 * grid, absorbing layer, gamma0 and multigrid options) and frequency omega_h; the
 * problem's device arrays keep their addresses, so work captured against them (a
 * helm_solver_plan) stays valid.  A network's cached encodings of p become stale:
 * call helm_cnn_set_problem again.  Synchronises `stream`. */
int helm_problem_update(helm_problem* p, const float* kappa_dev, double omega_h, void* stream);

/* Grid size of multigrid level `level` (0 = finest). */
int helm_problem_level_shape(const helm_problem* p, int level, int* nx, int* ny);

/* Copy a setup field to caller device memory `out_dev` (complex64 [ny_l][nx_l] unless
 * noted): which = 0 mass_A (level must be 0), 1 mass_SL at `level`, 2 damped inverse
 * Jacobi diagonal at `level`, 3 gamma (float32, level 0), 4 kappa (float32, level 0). */
int helm_problem_get_field(const helm_problem* p, int which, int level, void* out_dev, void* stream);

/*
 * Workspace bytes needed by any hot call below for `batch` right-hand sides and
 * FGMRES restart length `restart` (cnn may be NULL: SL-multigrid only).
 */
typedef struct helm_cnn helm_cnn;
int helm_workspace_size(const helm_problem* p, const helm_cnn* cnn, int batch, int restart, size_t* bytes);

/*
 * y = h^2 A x  (Eq. 3 with the absorbing-layer gamma; 5-point stencil, zero outside).
 * x, y: complex64 [batch][ny][nx], distinct buffers.  No workspace.
 */
int helm_helmholtz_apply(const helm_problem* p, const void* x, void* y, int batch, void* stream);

/*
 * r = h^2 b - h^2 A x evaluated in FP64 arithmetic (the true residual of Section 5's
 * stopping rule): b complex64, x complex128, r complex64, rnorm2_dev (nullable) receives
 * ||r||^2 per RHS as float64 [batch].  Workspace as returned by helm_workspace_size.
 */
int helm_helmholtz_residual_fp64(const helm_problem* p, const void* b, const void* x, void* r,
                                 double* rnorm2_dev, int batch, void* ws, size_t ws_bytes, void* stream);

/*
 * z = V(r): one shifted-Laplacian V(1,1) cycle from a zero initial guess (Algorithm 1
 * applied recursively): damped Jacobi pre-sweep, full-weighting restriction of the
 * residual, coarse correction (coarsest level: coarse_iters GMRES iterations with a
 * Jacobi right preconditioner), bilinear prolongation, damped Jacobi post-sweep.
 * r, z: complex64 [batch][ny][nx].  Workspace as returned by helm_workspace_size.
 */
int helm_slmg_vcycle(const helm_problem* p, const void* r, void* z, int batch, void* ws, size_t ws_bytes,
                     void* stream);

/*
 * z = V(r) exactly as helm_slmg_vcycle (Section 3.2, Algorithm 1), without a workspace
 * argument: the scratch is a
 * fixed device array inside the library of HELM_VCYCLE_STATIC_BYTES (16 MiB), resident
 * on every device the library is loaded on.  The paper has no counterpart: it is for
 * callers that cannot pass or allocate scratch (e.g. a preconditioner callback of an
 * external Krylov solver).  The call allocates nothing.
 *   - Scratch need per call: the V-cycle's coarse-level buffers for `batch` RHS, about
 *     2.2 MB per RHS at 576^2 with 4 levels (7 RHS fit).  A call that needs more
 *     returns HELM_EWORKSPACE before launching anything.
 *   - Nothing in the scratch has to start at zero: every element is written before it
 *     is read within one call.
 *   - The first call on a device looks up the array's address (cudaGetSymbolAddress)
 *     and keeps it for the life of the process; make that first call before any stream
 *     capture, and do not use this entry point on a device after cudaDeviceReset.
 *   - All calls on one device share the one array: calls that may overlap in time
 *     (different streams, or threads without ordering) race on it.  Order them on one
 *     stream.
 *   - The current device must be the problem's device (else HELM_EINVAL).
 */
#define HELM_VCYCLE_STATIC_BYTES ((size_t)16 << 20)
int helm_slmg_vcycle_static(const helm_problem* p, const void* r, void* z, int batch, void* stream);

/* FGMRES options. */
typedef struct {
  int restart;      /* FGMRES(m) restart length (paper: 10)                                */
  double rtol;      /* stop when ||b - A x|| <= rtol ||b|| (true FP64 residual)             */
  int maxit;        /* cap on Arnoldi steps per RHS (paper: 2000)                           */
  int warmup_iters; /* with a CNN: first cycle of this many steps with the V-cycle only
                       (Section 4.1: typically 3); ignored without a CNN                   */
  int reorth;       /* 0: classical Gram-Schmidt; 1: CGS with selective re-orthogonalisation
                       (second pass when ||w|| drops below ||w_0||/sqrt 2); 2: always CGS2   */
  int cnn_every;    /* with a CNN: the composed preconditioner on Arnoldi steps j with
                       j mod cnn_every == 0, the V-cycle alone on the others (FGMRES admits
                       a different preconditioner per step); 1 = every step, the paper's
                       method (default); must be >= 1                                      */
  int fallback;     /* with a CNN, 1 (default): a right-hand side falls back to the plain
                       V-cycle for the rest of its solve when a restart cycle with the
                       network reduces its true residual by less than 5 %, or when a step
                       with the network gives a non-finite Arnoldi column (that step is
                       discarded, the cycle ends with the steps before it); 0: the network
                       stays in use (a stalled RHS runs on to maxit, a non-finite column
                       ends the RHS with HELM_STATUS_NONFINITE)                           */
} helm_fgmres_opts;

/* Per-RHS result. */
typedef struct {
  int iters;           /* Arnoldi steps performed (= preconditioner applications)         */
  int status;          /* HELM_STATUS_*                                                   */
  double rel_res_est;  /* last Givens residual estimate / ||b||                           */
  double rel_res_true; /* ||b - A x|| / ||b|| in FP64 at exit                             */
} helm_fgmres_stats;

void helm_fgmres_opts_default(helm_fgmres_opts* o);

/*
 * Right-preconditioned flexible GMRES on h^2 A x = b for `batch` right-hand sides.
 * b: complex64 [batch][ny][nx]; x: complex128 [batch][ny][nx], in: initial guess,
 * out: solution (accumulated in FP64; the Krylov vectors are FP32).
 * cnn: NULL for the SL V-cycle preconditioner, else the composed preconditioner
 *   z = e + V(r - A e), e = s Net(r / s), s = RMS(r)  (Section 4.1), with the warm-up cycle.
 * maxit_dev: nullable device int [batch] per-RHS caps (min with opts->maxit).
 * stats_dev: device helm_fgmres_stats [batch] written at exit.
 * The call synchronises `stream` once per restart cycle to test for completion.
 */
int helm_fgmres_solve(const helm_problem* p, const helm_cnn* cnn, const void* b, void* x, int batch,
                      const helm_fgmres_opts* opts, const int* maxit_dev, helm_fgmres_stats* stats_dev,
                      void* ws, size_t ws_bytes, void* stream);

/*
 * A captured solver for repeated solves of one batch shape (mixed-size serving: one
 * plan per grid size): the FGMRES of helm_fgmres_solve (Section 4.1; Saad 1993).  helm_solver_plan_create binds the problem, the network (NULL:
 * SL V-cycle only), the right-hand-side buffer b (complex64 [batch][ny][nx]), the
 * solution buffer x (complex128, the initial guess is zero), the options and the
 * workspace (helm_workspace_size), runs every kind of restart cycle once, then records
 * each kind (the network's warm-up cycle and a regular cycle) as a CUDA graph on
 * `stream`, which must be a non-default stream.  In the captured cycles the network
 * runs on every right-hand side of the batch and the output of those that fell back to
 * the V-cycle (helm_fgmres_opts.fallback) is zeroed on the device, so no host decision
 * is needed inside a cycle; per right-hand side the arithmetic is that of
 * helm_fgmres_solve.
 * helm_solver_plan_solve solves for the current contents of b: the restart setup, then
 * one graph launch per restart cycle with one host read of the active count between
 * launches; per-RHS statistics as in helm_fgmres_solve.  Between solves the caller may
 * overwrite b, update the problem in place (helm_problem_update) and recompute the
 * network's encodings (helm_cnn_set_problem); changing the network's parameters needs a
 * new plan (HELM_ESTATE), as do encodings computed for another problem.  The buffers
 * and workspace must stay allocated while the plan lives.
 */
typedef struct helm_solver_plan helm_solver_plan;
int helm_solver_plan_create(const helm_problem* p, const helm_cnn* cnn, const void* b, void* x, int batch,
                            const helm_fgmres_opts* opts, void* ws, size_t ws_bytes, void* stream,
                            helm_solver_plan** out);
int helm_solver_plan_solve(helm_solver_plan* plan, const int* maxit_dev, helm_fgmres_stats* stats_dev, void* stream);
int helm_solver_plan_destroy(helm_solver_plan* plan);

/*
 * One convolution of the encoder-solver network on the tcgen05 tensor cores
 * (Sections 4.4, 5.3): x BF16 NHWC [batch][hi][wi][cin], w FP32 in the layout of the
 * paper's PyTorch modules ([cout][cin][3][3] for S1/S2, [cin][cout][3][3] for T1/T2,
 * [cout][cin] when taps == 1), packed to BF16 in `ws`.  Output
 *   y    = act(scale * acc + shift) + add1 + add2   (BF16 NHWC, nullable)
 *   yraw = acc                                      (FP32 NHWC, nullable)
 * scale/shift nullable (1, 0); act 1 = softplus; add1 [batch][ho][wo][cout] BF16,
 * add2 the same or [1][ho][wo][cout] with add2_bcast = 1 (both nullable).
 * cin <= 2 or a multiple of 8 (one of the network's layer shapes); cout a multiple
 * of 16.  HELM_EINVAL for shapes without a kernel instance.
 */
int helm_conv_bf16(const void* x, int batch, int hi, int wi, int cin, const float* w, int cout, int taps, int mode,
                   const float* scale, const float* shift, int act, const void* add1, const void* add2,
                   int add2_bcast, void* y, float* yraw, void* ws, size_t ws_bytes, void* stream);

/*
 * One evaluation-mode inverted bottleneck of the solver network (Section 4.4: the
 * MobileNetV2 block, expansion 6) in one fused kernel, the layer the network executes:
 *   y = x + BN2(P softplus(BN1(dw3x3(softplus(BN0(E x))))))
 * x, y: BF16 NHWC [batch][h][w][c], distinct; c = 16, 32 or 64.  Weights FP32 in the
 * PyTorch module layouts: w_exp [6c][c] (1x1), w_dw [6c][3][3] (depthwise, zero
 * padding), w_proj [c][6c] (1x1); the 1x1 weights are rounded to BF16 and the depthwise
 * weights to FP16 inside.  bn0, bn1 (FP32 [2][6c]) and bn2 (FP32 [2][c]) are folded
 * evaluation-mode BatchNorms, scale then shift.  ws: device scratch for the packed
 * weights (>= 4 c 6c + 512 bytes; HELM_EWORKSPACE otherwise).
 */
int helm_ib_bf16(const void* x, int batch, int h, int w, int c, const float* w_exp, const float* bn0,
                 const float* w_dw, const float* bn1, const float* w_proj, const float* bn2, void* y, void* ws,
                 size_t ws_bytes, void* stream);

/*
 * The implicit layer (Section 4.2, Eq. 14) as the network executes it: channel k and
 * k + c/2 of x (BF16 NHWC [batch][m][m][c], c a multiple of 8) form complex channel k,
 * which is zero-padded to 2m x 2m, transformed, multiplied by ghat[k] (complex64
 * [c/2][2m][2m], the Green's function of Eq. 15 after crop and DFT, as returned by
 * helm_cnn_get_ghat), transformed back and cropped to the top-left m x m block; y has
 * x's layout, distinct from x.  HELM_ESHAPE for m beyond the shared-memory limit (about
 * 111; helm_implicit_3pass_bf16 takes larger maps).
 */
int helm_implicit_bf16(const void* x, int batch, int m, int c, const void* ghat, void* y, void* stream);

/*
 * The same layer on an m_y x m_x map (the coarsest map of a rectangular grid; the paper's
 * grids are square, its out-of-distribution models of Section 5.1 are rectangles): x, y
 * BF16 NHWC [batch][my][mx][c], each complex channel zero-padded to 2m_y x 2m_x, and
 * ghat complex64 [c/2][2my][2mx] (helm_cnn_get_ghat_rect).  HELM_ESHAPE when the map
 * exceeds shared memory or 2m_x or 2m_y has a prime factor above 17.
 */
int helm_implicit_rect_bf16(const void* x, int batch, int my, int mx, int c, const void* ghat, void* y,
                            void* stream);

/*
 * The same layer (Section 4.2, Eq. 14) in three passes through a global intermediate,
 * for maps whose
 * m_y x 2m_x intermediate exceeds a CTA's shared memory (m about 112 and above: the
 * coarsest maps of grids from about 1792^2 up): the row transforms into the workspace,
 * the column transforms with the product by ghat in place, then the inverse row
 * transforms into y.  Arguments as helm_implicit_rect_bf16, plus a device workspace of
 * helm_implicit_3pass_workspace_size bytes (batch * c/2 * my * 2mx complex64;
 * HELM_EWORKSPACE if smaller).  The network switches to this form by itself when the
 * one-CTA form does not fit (its workspace includes the intermediate).  HELM_ESHAPE when
 * 2m_x or 2m_y exceeds 2048 or has a prime factor above 17.
 */
int helm_implicit_3pass_bf16(const void* x, int batch, int my, int mx, int c, const void* ghat, void* y, void* ws,
                             size_t ws_bytes, void* stream);
int helm_implicit_3pass_workspace_size(int batch, int my, int mx, int c, size_t* bytes);

/* Launch-shape tuning table (process-wide, read at launch time; captured solver plans
 * keep the shapes they were captured with).  A knob's value for a layer of height
 * `height` run on `batch` images overrides the kernel family's launch heuristic.
 * Lookup order: (height, batch), (height, any batch: batch 0), (any: height 0 and
 * batch 0).  Value 0 removes an entry; values are clamped to what the kernel supports.
 * HELM_EINVAL for an unknown knob or negative arguments.  The autotuner of the Python
 * package fills it from timings.  Knobs:
 *   HELM_TUNE_CONV_ROWS  most output rows per convolution segment (a CTA's unit of
 *                        work; the heuristic takes as many as the shared-memory budget
 *                        allows, up to 32)
 *   HELM_TUNE_IB_SH      output rows per work unit of the 16/32-channel inverted
 *                        bottleneck (a multiple of 4; the heuristic balances the units
 *                        over the SMs)
 *   HELM_TUNE_IMPLICIT_3PASS  1: the network's implicit layer on maps of m_y rows runs
 *                        in three passes (helm_implicit_3pass_bf16) even where the
 *                        one-CTA form fits (the heuristic takes three passes only
 *                        where it does not)                                            */
#define HELM_TUNE_CONV_ROWS 0
#define HELM_TUNE_IB_SH 1
#define HELM_TUNE_IMPLICIT_3PASS 2
#define HELM_TUNE_KNOBS 3
int helm_tune_set(int knob, int height, int batch, int value);
int helm_tune_get(int knob, int height, int batch, int* value);
int helm_tune_clear(void);

/* Number of kernels the library has launched in this process (all devices). */
unsigned long long helm_launch_count(void);

/* Opt-in profiler: between helm_profile_begin() and helm_profile_end() every kernel
 * launch is bracketed by CUDA events on its own stream; helm_profile_end() waits for
 * them and aggregates per kernel name.  helm_profile_read(i, ...) returns the i-th
 * kernel name (library-owned string), its launch count and total device time (ms).
 * Host-side only; recording adds two events per launch. */
int helm_profile_begin(void);
int helm_profile_end(int* nkernels);
int helm_profile_read(int idx, const char** name, long* launches, double* total_ms);

/* ---- the encoder-solver network (Sections 4.1-4.4, 5.3) ---------------------------- */
typedef struct {
  int c0;             /* channels of the first level (16; kernels exist for 16)           */
  int expansion;      /* inverted-bottleneck expansion factor (6)                         */
  int skip_threshold; /* grids below this size keep the coarsest level at I/8 (512)       */
  int literal_green;  /* 0: Eq. (15) read as conj(K)/(|K|^2+eps); 1: literal K/(K^2+eps) */
  int explicit_unet;  /* 0: the implicit U-Net (Section 4.2); 1: the explicit U-Net that
                         Section 6 compares it with, the same network without the implicit
                         step at the coarsest level (no "s.imp.K" parameter, no G_hat)     */
} helm_cnn_desc;

/* Create a network (the encoder-solver U-Net of Sections 4.1-4.4 with the sizes of
 * Section 5.3; all parameters owned by the caller, see helm_cnn_set_params); the
 * handle owns BN running statistics (initialised to mean 0, var 1), packed BF16
 * weights, the Green's functions per coarsest size and the encodings of one problem. */
int helm_cnn_create(const helm_cnn_desc* desc, helm_cnn** out);
int helm_cnn_destroy(helm_cnn* c);

/* Parameter table: a flat FP32 vector; entry idx has a name (library-owned string),
 * ndim <= 4 dims in `shape`, and starts at element `offset`.  Conv weights use the
 * PyTorch module layouts ([co][ci][3][3], transposed [ci][co][3][3], 1x1 [co][ci]);
 * "s.imp.K" is [2][nk][3][3] (real, imaginary parts of the implicit kernels). */
int helm_cnn_num_params(const helm_cnn* c, size_t* n);
int helm_cnn_param_info(const helm_cnn* c, int idx, const char** name, int* ndim, int* shape, size_t* offset);
/* BatchNorm table: running statistics are a flat FP32 vector, BN idx at `roff`:
 * mean [C] then variance [C]. */
int helm_cnn_num_bn(const helm_cnn* c, int* n);
int helm_cnn_bn_info(const helm_cnn* c, int idx, const char** name, int* C, size_t* roff);

/* Use the caller's FP32 parameter vector (device, kept alive by the caller).  Marks the
 * derived state stale; it is rebuilt (packing, BN folding, G_hat, Eq. 15) on next use. */
int helm_cnn_set_params(helm_cnn* c, const float* params_dev, void* stream);
int helm_cnn_set_running(helm_cnn* c, const float* running_dev, void* stream);
int helm_cnn_get_running(helm_cnn* c, float* out_dev, void* stream);

/* Run the encoder (evaluation-mode BN) on problem p's slowness model and cache the
 * encodings (Section 4.1: once per slowness model, reused for every RHS and
 * iteration).  Needed again after helm_cnn_set_params.  The grid may be a rectangle
 * (ny x nx, both sides divisible by 16) for inference (set_problem, apply with train = 0,
 * the composed preconditioner): every layer then runs per axis, the coarsest map is
 * m_y x m_x, and the solver's last downsampling is skipped when the shorter side is below
 * the skip threshold.  Training needs a square grid (HELM_ESHAPE otherwise). */
int helm_cnn_set_problem(helm_cnn* c, const helm_problem* p, void* ws, size_t ws_bytes, void* stream);

/* e = s Net(r / s), s = RMS of r over the grid (Eq. 16's SolverNet with the residual
 * normalisation of this library), r, e complex64 [batch][ny][nx].  train = 0: evaluation-mode BN with the
 * cached encodings.  train = 1: batch-statistics BN, encoder run on p in training mode
 * inside the call, activations saved in `ws` for helm_cnn_precond_backward, running
 * statistics updated (momentum 0.1). */
int helm_cnn_apply(const helm_problem* p, helm_cnn* c, const void* r, void* e, int batch, int train, void* ws,
                   size_t ws_bytes, void* stream);

/* Bytes of the training workspace for a training forward over `nprob` slowness models
 * (helm_cnn_train_forward, or helm_cnn_apply(train = 1) with nprob = 1) followed by
 * helm_cnn_precond_backward at this batch size (activations, raw BN inputs, statistics,
 * gradients of every activation, reduction partials). */
int helm_cnn_train_workspace_size(const helm_problem* p, const helm_cnn* c, int batch, int nprob, size_t* bytes);

/* Training-mode forward over a batch whose samples come from several slowness models
 * (Section 4.3, Eq. 16: each pair carries its own kappa): sample b belongs to
 * probs[b / (batch / nprob)] (batch divisible by nprob, equal grids).  The encoder runs
 * on the nprob models, batch-statistics BN, activations saved in ws for
 * helm_cnn_precond_backward, running statistics updated. */
int helm_cnn_train_forward(const helm_problem* const* probs, int nprob, helm_cnn* c, const void* r, void* e,
                           int batch, void* ws, size_t ws_bytes, void* stream);

/* Backward of the last training-mode forward (helm_cnn_train_forward or
 * helm_cnn_apply(train = 1)) that used the same workspace, for the network part
 * e = s Net(r / s), s = RMS(r) of Section 4.1 (Eq. 16's SolverNet; the V-cycle is not
 * differentiated):
 *   grad_e      complex64 [batch][N][N], dLoss/dRe e + i dLoss/dIm e
 *   grad_params FP32 in the parameter layout, overwritten; covers the solver and the
 *               encoder (the encodings receive the batch sum of their gradients)
 *   grad_r      nullable; complex64 [batch][N][N] receives dLoss/dRe r + i dLoss/dIm r,
 *               the scale s's own dependence on r included (a zero sample gets zero)
 *   r           the forward's input (complex64, caller-owned); needed only with grad_r
 * HELM_EINVAL if grad_r is given without r or aliases it; HELM_ESTATE without a
 * preceding training forward. */
int helm_cnn_precond_backward(const helm_problem* p, helm_cnn* c, const void* r, const void* grad_e, void* grad_r,
                              float* grad_params, int batch, void* ws, size_t ws_bytes, void* stream);

/* Eq. (16): loss = (1/batch) sum |e_pred - e_true|^2 over n complex entries (all
 * batch items), written as float64 to loss_dev; grad (nullable, complex64 like e_pred)
 * receives 2 (e_pred - e_true) / batch.  ws: >= 4096 bytes of device scratch. */
int helm_mse_loss(const void* e_pred, const void* e_true, long n, int batch, double* loss_dev, void* grad, void* ws,
                  void* stream);

/* One Adam step (the optimiser of Section 5.3; bias-corrected, step >= 1) on n FP32
 * parameters, moments m, v. */
int helm_adam_step(float* params, const float* grads, float* m, float* v, long n, double lr, double beta1,
                   double beta2, double eps, int step, void* stream);

/* Save the network to the file `path`: its descriptor, the FP32 parameters (the vector
 * set by helm_cnn_set_params), the BN running statistics and the Green's function G_hat
 * of every coarsest size m the handle holds for these parameters (Section 4.2: G_hat is
 * computed from the learned kernel once and stored as part of the network), followed by
 * a hash of the contents.  Host I/O; synchronises `stream`.  HELM_ESTATE without
 * parameters, HELM_EINVAL if the file cannot be written. */
int helm_cnn_save(helm_cnn* c, const char* path, void* stream);

/* Load a file written by helm_cnn_save into a handle created with the same descriptor:
 * the parameters are copied to params_dev (caller-owned device FP32 [num_params], which
 * becomes the handle's parameter vector as if passed to helm_cnn_set_params), the
 * running statistics into the handle, and the stored G_hat become the handle's Green's
 * functions without an Eq. 15 rebuild.  HELM_EINVAL if the file is missing, truncated,
 * fails its hash, or was saved from another descriptor or parameter table (then
 * nothing is changed); synchronises `stream`.  Needs helm_cnn_set_problem afterwards. */
int helm_cnn_load(helm_cnn* c, const char* path, float* params_dev, void* stream);

/* Copy G_hat (Eq. 15, after crop and DFT) for coarsest size m to out_dev, complex64
 * [nk][2m][2m]; builds it if needed.  HELM_ESTATE for an explicit U-Net. */
int helm_cnn_get_ghat(helm_cnn* c, int m, void* out_dev, void* stream);
/* The same for an m_y x m_x coarsest map: complex64 [nk][2my][2mx], Eq. 15 on the
 * 6m_y x 6m_x periodic grid.  Rectangular G_hat are derived on demand and not stored by
 * helm_cnn_save. */
int helm_cnn_get_ghat_rect(helm_cnn* c, int my, int mx, void* out_dev, void* stream);

/* The composed preconditioner of Section 4.1: z = e + V(r - A e), e = s Net(r/s), s = RMS(r). */
int helm_cnn_precond_apply(const helm_problem* p, helm_cnn* c, const void* r, void* z, int batch, void* ws,
                           size_t ws_bytes, void* stream);

/*
 * Training pairs of Section 4.3, Eq. (17): for random x (complex64 [batch][N][N]),
 * b = A x (with the problem's gamma, 0.05 in training), x_tilde = FGMRES with the SL
 * V-cycle from x0 = 0 run for exactly iters_dev[i] steps (1 <= iters <= max_iters <= 32,
 * one cycle), e = x - x_tilde and r = b - A x_tilde (FP64 evaluation), written as
 * complex64; normalise = 1 scales both by 1/RMS(r_i) (RMS over the grid).  Workspace:
 * helm_datagen_workspace_size().
 */
int helm_datagen_pairs(const helm_problem* p, const void* x, const int* iters_dev, void* e, void* r, int batch,
                       int max_iters, int normalise, void* ws, size_t ws_bytes, void* stream);
int helm_datagen_workspace_size(const helm_problem* p, int batch, int max_iters, size_t* bytes);

/*
 * Random vectors x of the training pairs (Section 4.3: a smooth random error plus noise):
 *   x_b = f_b / RMS(f_b) + noise (n_b0 + i n_b1),  f_b = G w_b0 + i G w_b1,
 * G the periodic Gaussian filter of standard deviation `sigma` cells along both axes
 * (weights exp(-t^2 / (2 sigma^2)) for |t| <= ceil(3 sigma), normalised to sum 1), RMS
 * over the grid.  white: device float [batch][4][n][n], the planes w_b0, w_b1, n_b0, n_b1
 * of standard normal numbers drawn by the caller; x: device complex64 [batch][n][n]
 * (written).  Stream-ordered, no workspace.  HELM_EINVAL unless 0 < sigma <= 8 and
 * noise >= 0.
 */
int helm_training_field(const float* white, int batch, int n, float sigma, float noise, void* x, void* stream);

/* Read and clear the device error word (HELM_DEVERR_* bits) of the current device. */
int helm_device_errors(unsigned int* flags);

/* Human-readable description of the last error on this thread ("" if none). */
const char* helm_last_error_string(void);

/* Library version string. */
const char* helm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* HELM_H */
