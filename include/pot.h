/*
 * pot.h -- C ABI of libpot.so: generalized Laguerre cells, the partial
 * optimal transport Newton solve and the explicit fluid step on one B300.
 *
 * Paper: "More Power to the Particles: Analytic Geometry for Partial Optimal
 * Transport-based Fluid Simulation" (arXiv 2601.05765).
 *
 * Conventions (every entry point):
 *  - Array arguments are DEVICE pointers on the context's device, owned by the
 *    caller, unless stated otherwise.  Positions are AoS (n,3) row-major.
 *    Indices of sites are 0..n-1 in the caller's order.
 *  - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *    stream.  Work is enqueued on that stream; a call returns after its own
 *    small host reads (status words, scalars) have completed, so outputs are
 *    ready for later work on the same stream.
 *  - The library owns its workspace inside the opaque context (allocated by
 *    pot_create); no other call allocates device memory.
 *  - Every call returns an int status (POT_OK = 0) and never aborts or prints.
 *    On error the array outputs are undefined; stats structs are filled as
 *    far as the call got.
 *  - The domain is an axis-aligned box [lo, hi].
 *  - Weights psi: the ball of site i has radius sqrt(psi_i); psi_i <= 0 gives
 *    an empty cell.
 *  - A context is not thread-safe: one call at a time per context.
 */
#ifndef POT_H
#define POT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define POT_OK 0
#define POT_ERR_INVALID_ARG 1         /* NULL pointer, n <= 0, n > n_max, bad box, ... */
#define POT_ERR_CUDA 2                /* a CUDA runtime call failed */
#define POT_ERR_NEIGHBOUR_OVERFLOW 3  /* a cell has more than k_max cutting bisectors */
#define POT_ERR_COINCIDENT_SITES 4    /* two sites at distance 0 cut each other's ball */
#define POT_ERR_EMPTY_CELL_AT_START 5 /* Newton start has a cell of volume 0 */
#define POT_ERR_NOT_CONVERGED 6       /* Newton iteration cap reached */
#define POT_ERR_LINESEARCH_FAILED 7   /* KMT step not found within max_halvings */
#define POT_ERR_POLYGON_OVERFLOW 8    /* a facet polygon exceeded its edge capacity */
#define POT_ERR_CAPACITY 9            /* CSR capacity too small for the Hessian */
#define POT_ERR_PCG_BREAKDOWN 10      /* PCG met p.Mp <= 0 (matrix not SPD) */
#define POT_ERR_TOO_LARGE 11          /* n above the no-alloc entry point's maximum */

/* ---- types ------------------------------------------------------------ */
typedef struct pot_ctx pot_ctx;

/* Axis-aligned box domain [lo, hi] (Sec. 2.2: the cells live in the box). */
typedef struct {
  double lo[3];
  double hi[3];
} pot_domain;

/* CSR of M = -grad^2 K (the Hessian of Eq. 2 with its sign flipped so that M
 * is symmetric positive definite):
 *   M_ij = -|B_ij| / (2 |p_i - p_j|) for every restricted bisector facet B_ij
 *          with area above 4e-7 psi_i (1e-13 psi_i in FP64),
 *   M_ii = sum_j |B_ij| / (2 |p_i - p_j|) + |K_i| / (2 sqrt(psi_i)),
 * |K_i| the free-surface (spherical patch) area.  Every row holds its
 * diagonal; columns ascend within a row.  The caller allocates row_ptr (n+1),
 * cols and vals (cap each); the call writes nnz (also when it exceeds cap,
 * then it returns POT_ERR_CAPACITY and leaves cols/vals undefined). */
typedef struct {
  int32_t* row_ptr;
  int32_t* cols;
  float* vals;
  int64_t cap;
  int64_t nnz;
} pot_csr;

typedef struct {
  int32_t* row_ptr;
  int32_t* cols;
  double* vals;
  int64_t cap;
  int64_t nnz;
} pot_csr_f64;

/* Per-call statistics of lgc_compute_cells*. */
typedef struct {
  int64_t n_empty;    /* cells of volume 0 */
  int64_t n_planes;   /* total cutting planes (walls + bisectors) */
  int64_t nnz;        /* Hessian entries incl. the diagonal */
  int64_t error_site; /* site index behind an error status, else -1 */
  int32_t max_planes; /* largest cutting-plane count of one cell */
  float ms_grid;      /* device time: grid build + sort */
  float ms_cells;     /* device time: candidates + cell geometry */
  float ms_csr;       /* device time: CSR assembly */
} pot_cell_stats;

/* Newton / fluid-step parameters (pot_default_params fills the defaults). */
typedef struct {
  double tol;           /* stop when max_i |V_i - nu_i| / nu_i <= tol (1e-4) */
  int32_t max_newton;   /* Newton iteration cap (100, Sec. 7) */
  int32_t max_halvings; /* KMT step halvings per iteration (30) */
  int32_t max_pcg;      /* PCG iteration cap per Newton step (2000) */
  int32_t pcg_chunk;    /* PCG iterations per host-driven batch of launches (16;
                           see pcg_host_loop) */
  double pcg_rtol;      /* PCG relative residual; <= 0 selects the adaptive
                           forcing term (default) */
  double dt;            /* fluid step (2e-3) */
  double eps;           /* spring length of the pressure force (0.01, Sec. 5) */
  double gravity[3];    /* (0, 0, -9.81) */
  double wall_margin;   /* sites are clamped to [lo+m, hi-m] (1e-6) */
  int32_t warm_start;   /* 0: previous psi; 1: learned MLP start; 2: psi
                           extrapolated from the previous two steps */
  int32_t substeps;     /* pot_fluid_step takes this many explicit steps of
                           dt / substeps (0 or 1: one step of dt) */
  double mu;            /* viscosity (Eq. 4; 0: none) */
  double gamma;         /* surface tension (Sec. 5; 0: none) */
  double mu_wall;       /* fluid-wall affinity of the viscosity (walls at rest; 0: none) */
  double gamma_wall;    /* the walls' part of the surface tension: surface tension times
                           the fluid's affinity to the walls (Sec. 5; 0: none) */
  int32_t pcg_host_loop; /* 0: each PCG solve runs on the device alone (one
                           persistent cooperative kernel for up to 2^17 rows,
                           else a CUDA graph whose while node repeats the two
                           iteration kernels); 1: the host launches the two
                           kernels pcg_chunk iterations at a time and checks
                           for convergence between batches (slower; every
                           launch visible to a profiler) */
  int32_t reserved_params; /* 0 */
} pot_params;

/* Statistics of one Newton solve (and of the solve inside a fluid step). */
typedef struct {
  int32_t status;
  int32_t newton_iters;
  int32_t pcg_iters;   /* total over the solve */
  int32_t halvings;    /* total KMT halvings */
  int32_t cell_evals;  /* evaluations of all cells (incl. line search) */
  int32_t grid_builds;
  double err_max;      /* final max_i |V_i - nu_i| / nu_i */
  double err_l2;       /* final ||nu - V||_2 */
  double err_start;    /* max relative error at the start */
  double ms_total;     /* host wall time of the call */
  double ms_cells;     /* device time in cell evaluations */
  double ms_pcg;       /* device time in PCG */
  int64_t nnz;         /* Hessian entries of the last assembly */
  int32_t mlp_used;    /* warm start: 1 if the MLP start was kept */
  int32_t mlp_fallback;/* warm start: 1 if the MLP start was rejected */
  int32_t repairs;     /* empty cells at the start whose weight was raised */
  int32_t passes;      /* security-ball passes over all cell evaluations */
  int64_t error_site;  /* caller index of a site behind the last cell error, else -1 */
  int32_t visc_iters;  /* PCG iterations of the viscosity solves (fluid step) */
  int32_t reserved;
  double ms_visc;      /* host wall time of the viscosity / surface-tension update */
} pot_solve_stats;

/* ---- context ---------------------------------------------------------- */

/* Create a context on `device` for up to n_max sites and k_max (<= 1024)
 * candidate bisectors per cell, and allocate all its workspace.  A cell is
 * built from the bisectors whose plane cuts its ball and meets the cell's
 * security ball (a ball around the cell's previous centroid that the cell
 * is verified not to leave, Sec. 4); in packed fluid that is about 15-40
 * planes, in strongly compressed fluid (sites much closer than nu^(1/3))
 * cells reach past several neighbours and need more.  A cell that needs
 * more than k_max gives POT_ERR_NEIGHBOUR_OVERFLOW.  Workspace: about
 * 16 k_max + 1000 bytes per site for each precision in precision_mask
 * (about 9.9 GB for the FP32 entry points at 2M sites and k_max 246).
 * Newton solves and fluid steps on the same sites reuse the previous
 * solve's cell centres.
 * precision_mask: bit 0 = FP32 geometry (mixed-precision entry points),
 * bit 1 = FP64 entry points (*_f64).
 * Returns POT_ERR_INVALID_ARG / POT_ERR_CUDA on failure (*ctx = NULL). */
int pot_create(pot_ctx** ctx, int device, int64_t n_max, int32_t k_max, int32_t precision_mask);

/* Free the context and its workspace.  NULL is accepted. */
int pot_destroy(pot_ctx* ctx);

/* Static string for a status code. */
const char* pot_status_string(int status);

/* Default parameters (see pot_params). */
void pot_default_params(pot_params* p);

/* Number of CUDA kernel launches this library has issued in this process
 * (all contexts and devices), for launch accounting by callers. */
int64_t pot_kernel_launches(void);

/* FP32 FMA throughput of the current device in TFLOP/s (not in the paper:
 * the denominator of the cell kernel's roofline, whose work is FP32
 * arithmetic).  Runs one warm-up and five timed launches of a kernel of
 * independent FMA chains on `stream` at full occupancy (CUDA events, best
 * launch; 2 FLOP per FMA); ms_out (optional) gets that launch's time.
 * sink: a caller-owned device buffer of at least (SM count x 8) floats that
 * the kernel never writes in practice (it only writes an impossible value).
 * Errors: POT_ERR_INVALID_ARG (NULL sink or tflops), POT_ERR_CUDA. */
int pot_measure_fp32_peak(void* stream, float* sink, double* tflops, double* ms_out);

/* Device time of the cell kernel (clipping, restriction and analytic
 * quantities, Sec. 3.2-3.4) accumulated over this context's evaluations since
 * the last reset, measured with CUDA events on the caller's stream around each
 * launch: the number of launches (one per security-ball pass), the cells
 * they processed and the milliseconds.  Any output pointer may be NULL;
 * reset != 0 clears the counters after reading them.
 * Errors: POT_ERR_INVALID_ARG for a NULL context. */
int pot_cell_kernel_time(pot_ctx* ctx, int reset, int64_t* launches, int64_t* cells, double* ms);

/* State of the last FP32 cell evaluation in this context, per site in the
 * caller order of that evaluation (n sites, device arrays, any may be
 * NULL): the security ball (centre offset from the site, 3 values per site,
 * and radius; Sec. 4's contributing-neighbour problem), the cell's extent
 * from that centre, and the number of planes (walls + candidate bisectors)
 * the cell was built from (0 for an empty cell or one that overflowed).
 * Errors: POT_ERR_INVALID_ARG when n does not match that evaluation. */
int pot_cell_diagnostics(pot_ctx* ctx, void* stream, int64_t n, float* center_offset,
                         float* radius, float* extent, int32_t* planes);

/* ---- generalized Laguerre cells (Eq. 1, Sec. 3.2-3.4, Algorithm 2) ------ */

/* Build every generalized Laguerre cell
 *   C_i = box ∩ B(p_i, sqrt(psi_i)) ∩ {x : |x-p_i|^2 - psi_i <= |x-p_j|^2 - psi_j, all j}
 * and evaluate analytically:
 *   volumes[i] = |C_i| (pyramid decomposition, Sec. 3.2, Algorithm 2),
 *   grad[i]    = targets[i] - |C_i|  (dK/dpsi_i, Sec. 3.1; -|C_i| if targets is NULL),
 *   hess       = M = -grad^2 K in CSR (Eq. 2, see pot_csr), optional (NULL),
 *   centroids  = (n,3) cell centroids c_i (pressure force, Sec. 5), optional,
 *   karea      = |K_i| free-surface area (Sec. 3.3), optional.
 * Inputs: pos (n,3) float, psi (n) float, targets (n) double or NULL.
 * FP32 geometry; grad in FP64.  Cells whose FP32 rounding could exceed
 * 1e-5 of their volume or of their Hessian diagonal (small against their
 * ball, a small diagonal, or two facet lines crossing inside a disk at a
 * sine below 1.5e-2) are recomputed from the same inputs in FP64.
 * Errors: POT_ERR_NEIGHBOUR_OVERFLOW, POT_ERR_COINCIDENT_SITES,
 *         POT_ERR_POLYGON_OVERFLOW (stats->error_site names a site),
 *         POT_ERR_CAPACITY (hess->nnz > hess->cap). */
int lgc_compute_cells(pot_ctx* ctx, void* stream, int64_t n, const float* pos, const float* psi,
                      const double* targets, const pot_domain* dom, float* volumes, double* grad,
                      pot_csr* hess, float* centroids, float* karea, pot_cell_stats* stats);

/* Same in FP64 throughout (pos, psi, volumes, centroids, karea, hess values). */
int lgc_compute_cells_f64(pot_ctx* ctx, void* stream, int64_t n, const double* pos,
                          const double* psi, const double* targets, const pot_domain* dom,
                          double* volumes, double* grad, pot_csr_f64* hess, double* centroids,
                          double* karea, pot_cell_stats* stats);

/* ---- cell evaluation without allocation ----------------------------------- */

/* The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory: plugins whose host application owns
 * every device allocation (a fixed arena with no room for, or no permission
 * to make, cudaMalloc calls of its own), and real-time loops where a
 * cudaMalloc/cudaFree pair would stall the device at the wrong moment.
 *
 * Computes what lgc_compute_cells computes, except the Hessian (volumes,
 * grad, centroids, karea; same meaning, layout and FP32/FP64 split), with
 * no context and no allocation: all scratch memory is one file-scope device
 * array inside libpot.so sized for n <= 8192 sites and 64 cutting bisectors
 * per cell (5,333,504 bytes, held by every GPU that loads the library until
 * the process exits).  The caller passes device inputs and outputs as usual;
 * centroids, karea and grad may be NULL.
 *  - n > 8192 returns POT_ERR_TOO_LARGE before any device work.
 *  - The first call on each device looks up the array's device address with
 *    that device current (the calling thread's current device is used);
 *    make that first call before any stream capture.  `stream` must belong
 *    to the current device (POT_ERR_INVALID_ARG otherwise).
 *  - Every call shares the array and overwrites the previous call's
 *    contents; calls whose work overlaps on the GPU race on it (a host mutex
 *    serialises calls from several threads, and each call waits for its own
 *    stream before returning, also when it returns an error).
 * Errors: as lgc_compute_cells (no POT_ERR_CAPACITY), plus POT_ERR_TOO_LARGE.
 * Timing fields of stats stay 0. */
int lgc_compute_cells_noalloc(void* stream, int64_t n, const float* pos, const float* psi,
                              const double* targets, const pot_domain* dom, float* volumes,
                              double* grad, float* centroids, float* karea, pot_cell_stats* stats);

/* ---- Newton solve (Algorithm 1 with KMT steps) --------------------------- */

/* Find the weights psi with |C_i(psi)| = targets[i] for all i (partial OT,
 * Sec. 2.2) by damped Newton (Algorithm 1).  A start with empty cells is
 * repaired first: each empty cell's weight is raised to
 * max_j (psi_j - d_ij^2) + 0.25 d*^2, which puts its site inside its own cell
 * (stats->repairs counts them).  Then M u = nu - V(psi) is solved by
 * Jacobi-preconditioned CG (Sec. 7), then the KMT step: alpha = 1, 1/2, ...
 * until min V(psi + alpha u) >= eps0 and
 * ||nu - V(psi + alpha u)||_2 <= (1 - alpha/2) ||nu - V(psi)||_2,
 * eps0 = 1/2 min(min nu, min V(psi_start)).  Stops when
 * max_i |V_i - nu_i| / nu_i <= params->tol.
 * psi_inout: start (must give non-empty cells) in, solution out.
 * Mixed precision: FP32 geometry and matrix; the residual sums and PCG dot
 * products accumulate the FP32 terms in double-float (about 44 bits) and
 * give FP64 scalars, and the KMT test and step lengths run in FP64.  This
 * entry point stops at 0.9 params->tol on its FP32-evaluated error, a
 * margin for the FP32 rounding of the volumes (about 1e-6 of the target),
 * so the weights meet params->tol in exact arithmetic; its KMT test also
 * accepts the same decrease of the max relative error (the l2 norm of an
 * FP32 evaluation stalls at its rounding floor).  Errors:
 * POT_ERR_EMPTY_CELL_AT_START (if the repair fails),
 * POT_ERR_NOT_CONVERGED, POT_ERR_LINESEARCH_FAILED, geometry errors.
 * psi_inout holds the last accepted iterate on NOT_CONVERGED. */
int pot_newton_solve(pot_ctx* ctx, void* stream, int64_t n, const float* pos, const double* targets,
                     float* psi_inout, const pot_domain* dom, const pot_params* params,
                     pot_solve_stats* stats);

/* Same with FP64 geometry, matrix and PCG vectors; stops at params->tol and
 * takes the l2 KMT test alone. */
int pot_newton_solve_f64(pot_ctx* ctx, void* stream, int64_t n, const double* pos,
                         const double* targets, double* psi_inout, const pot_domain* dom,
                         const pot_params* params, pot_solve_stats* stats);

/* ---- fluid step (Sec. 5, Gallouet-Merigot scheme) ------------------------ */

/* One explicit step, all on the device:
 *   x <- x + dt v, clamped to [lo+m, hi-m] (velocity component through the
 *        wall set to 0);
 *   psi <- Newton solve at the new x, warm-started from psi;
 *   v <- v + dt (g + (c_i - x_i) / eps^2)   (pressure spring F_p, Sec. 5).
 * With params->mu > 0 or params->gamma > 0 the velocity update is the
 * semi-implicit one of Eq. 4 (unit mass) over the P1 Laplacian of Eq. 3,
 * whose weights |B_ij| / (2 d_ij) come from the converged cells:
 *   (I/dt + mu (D - W)) v <- v/dt + (c - x)/eps^2 + g + gamma L x,
 * one Jacobi-PCG solve per component (relative residual 1e-6 in FP32,
 * 1e-11 in FP64); params->mu_wall > 0 adds walls at rest, mu_wall times the
 * cell's wall facets' weight |B_iw| / (2 h_iw) on the diagonal (Sec. 5's
 * fluid-boundary term); params->gamma_wall != 0 adds the walls' part of the
 * surface tension, each wall facet acting as the facet to a neighbour placed
 * cbrt(|V_i|) beyond the wall (Sec. 5): gamma_wall times
 * sum_w |B_iw| / (2 h_iw) (h_iw + cbrt(|V_i|)) n_w on the right-hand side
 * (n_w the wall's outward normal); the free surface adds no Laplacian term.
 * With params->warm_start = 2, Newton starts from psi + (psi - psi_prev),
 * psi_prev the weights at the start of the previous pot_fluid_step on this
 * context with the same n (none after pot_create, pot_clear_history or a
 * pot_newton_solve: then from psi); a start with an empty cell or a geometry
 * error, or from which Newton does not converge, falls back to psi (stats:
 * mlp_used / mlp_fallback).
 * With params->substeps = k > 1 this is done k times with dt / k, stopping
 * at the first substep whose solve fails; stats then sums the substeps'
 * counts and times and keeps their largest start and final errors.
 * pos, vel (n,3) and psi (n) are updated in place. */
int pot_fluid_step(pot_ctx* ctx, void* stream, int64_t n, float* pos, float* vel, float* psi,
                   const double* targets, const pot_domain* dom, const pot_params* params,
                   pot_solve_stats* stats);

int pot_fluid_step_f64(pot_ctx* ctx, void* stream, int64_t n, double* pos, double* vel,
                       double* psi, const double* targets, const pot_domain* dom,
                       const pot_params* params, pot_solve_stats* stats);

/* Forget the weight history of warm_start = 2 (a new run on the same
 * context).  Errors: POT_ERR_INVALID_ARG for a NULL context. */
int pot_clear_history(pot_ctx* ctx);

/* Several fluids (Sec. 5's per-pair viscosity coefficients): per-site
 * factors f (device, n floats, caller order, owned by the caller and read by
 * every later viscous pot_fluid_step with this n) make the pair coefficient
 * mu_ij = params->mu (f_i + f_j) / 2.  NULL clears them (mu_ij = mu).
 * Errors: POT_ERR_INVALID_ARG (NULL context; n out of range with factors). */
int pot_set_viscosity_factors(pot_ctx* ctx, int64_t n, const float* factors);

/* ---- learned warm start (not in the paper) ------------------------------- */

/* A small MLP predicts each site's new weight from its neighbourhood:
 * inputs (80 BF16 values per site, row-major): offsets to the up to 24
 * nearest other sites closer than 2 h, by increasing distance,
 * divided by h = nu^(1/3) (zero-padded); psi_prev / h^2; v dt / h; the
 * previous weight change (psi_prev - psi_old) / h^2 (0 without history);
 * 3 zeros.
 * Network: 80 -> 128 -> 128 -> 128 (ReLU) -> 1, BF16 weights and activations,
 * FP32 accumulation on the tcgen05 tensor cores.  Prediction:
 * psi_start = psi_prev + h^2 * clamp(output, -1, 1).  Parameters are one FP32 vector of
 * pot_mlp_num_params() values: W1 (80 x 128, row = input), b1 (128),
 * W2 (128 x 128), b2, W3 (128 x 128), b3, w4 (128), b4 (1). */
typedef struct pot_mlp pot_mlp;

/* Model with workspace for inference on up to max_rows rows (training batches
 * up to 16384 rows, multiples of 8).  Parameters start at zero. */
int pot_mlp_create(pot_mlp** mlp, int device, int64_t max_rows);
int pot_mlp_destroy(pot_mlp* mlp);
int pot_mlp_num_params(void);

/* Copy parameters in/out (device FP32 vectors); set also resets Adam. */
int pot_mlp_set_params(pot_mlp* mlp, void* stream, const float* params);
int pot_mlp_get_params(pot_mlp* mlp, void* stream, float* params);

/* out[r] = MLP(x[r]) for rows x (rows x 80 BF16, device). */
int pot_mlp_forward(pot_mlp* mlp, void* stream, int64_t rows, const uint16_t* x, float* out);

/* Rows idx[0..batch) of the dataset (x_all: n_all x 80 BF16, y_all: n_all
 * FP32 targets) form one batch; loss = mean (out - y)^2.
 * pot_mlp_gradients writes d loss / d params (FP32, pot_mlp_num_params
 * values) and the loss (device scalar), without updating;
 * pot_mlp_train_step takes one Adam step (beta 0.9 / 0.999, eps 1e-8) with
 * learning rate lr and writes the batch loss before the step.
 * batch <= 16384 and a multiple of 8. */
int pot_mlp_gradients(pot_mlp* mlp, void* stream, int64_t n_all, const uint16_t* x_all,
                      const float* y_all, const int32_t* idx, int64_t batch, float* grads,
                      float* loss);
int pot_mlp_train_step(pot_mlp* mlp, void* stream, int64_t n_all, const uint16_t* x_all,
                       const float* y_all, const int32_t* idx, int64_t batch, float lr,
                       float* loss);

/* Status of the model's kernels since the last check (a bounded tensor-core
 * wait that ran out reports POT_ERR_CUDA); clears it. */
int pot_mlp_check(pot_mlp* mlp, void* stream);

/* Features (n x 80 BF16, caller order) at the positions and velocities the
 * next pot_fluid_step will solve at (x + dt v clamped into the box, same rule),
 * with psi as the previous weights and psi_old as the weights one step before
 * them (NULL: no history, the change feature is 0).  Uses ctx's grid
 * workspace. */
int pot_mlp_features(pot_ctx* ctx, pot_mlp* mlp, void* stream, int64_t n, const float* pos,
                     const float* vel, const float* psi, const float* psi_old,
                     const double* targets, const pot_domain* dom, const pot_params* params,
                     uint16_t* feat);

/* Inputs of the model: 77 (default: the 24 neighbour offsets, the previous
 * weight, the velocity and the previous weight change; the prediction
 * corrects the extrapolation psi + (psi - psi_old)) or 76 (the inputs the
 * warm-start configuration names, without the weight change: input 77 is
 * 0 and the prediction corrects the previous weights, psi + h^2 y).  The
 * features (pot_mlp_features) and the fluid step's warm start follow the
 * choice.  Errors: POT_ERR_INVALID_ARG (mlp NULL, n_inputs not 76 or 77). */
int pot_mlp_set_inputs(pot_mlp* mlp, int32_t n_inputs);

/* Weight history of the warm start.  Each warm-started pot_fluid_step keeps
 * its starting weights (caller order) as the next step's psi_old, valid while
 * the site count stays n.  This call seeds the history with psi_old (device,
 * n values, caller order), or clears it (psi_old NULL).  Errors:
 * POT_ERR_INVALID_ARG when n exceeds the model's max_rows. */
int pot_mlp_set_history(pot_mlp* mlp, void* stream, int64_t n, const float* psi_old);

/* Attach a model to a context (NULL detaches; the context does not own it).
 * pot_fluid_step then starts Newton from psi + (psi - psi_old) + h^2 y, y
 * the MLP's output clamped to [-1, 1] (psi_old from the history; without it
 * that term is 0), when params->warm_start is 1, and falls back to
 * plain Newton from the previous weights when the prediction fails the KMT
 * precondition (an empty cell, or a geometry error) or when Newton from it
 * does not converge (stats: mlp_used / mlp_fallback).  FP32 path only. */
int pot_set_warm_start(pot_ctx* ctx, pot_mlp* mlp);

/* ---- first hit of camera rays (Sec. 6, finding the first cell) -------- */

/* Pinhole camera: rays from origin through the pixel centres; right =
 * forward x up, the image's up = right x forward; fov_y the vertical field
 * of view in radians, the horizontal one from width / height; row 0 at the
 * top. */
typedef struct {
  double origin[3];
  double forward[3];
  double up[3];
  double fov_y;
  int32_t width, height;
} pot_camera;

/* Depth and normal of the first point of each camera ray inside the fluid:
 * the union of the generalized Laguerre cells of Eq. 1, which is the union
 * of the balls B(p_i, sqrt(psi_i)) inside the box dom.  pos (n,3), psi (n),
 * karea (n, optional: the cells' free-surface areas |K_i|, e.g. from
 * lgc_compute_cells; balls of cells with |K_i| = 0 are skipped, which leaves
 * the first hit unchanged) are device arrays in caller order.  depth
 * (height x width, row-major): the ray parameter t of the hit (the distance
 * from the origin), -1 when the ray misses; normal (3 per pixel, optional):
 * unit outward normal of the sphere hit, 0 when none.  Device buffers
 * written on `stream`; no graphics API.  Uses ctx's FP32 grid workspace.
 * Errors: POT_ERR_INVALID_ARG (NULL pointers, n out of range, an FP64-only
 * context, width or height <= 0, fov_y outside (0, 3.14), degenerate
 * forward/up), POT_ERR_CUDA. */
int pot_render_depth(pot_ctx* ctx, void* stream, int64_t n, const float* pos, const float* psi,
                     const float* karea, const pot_domain* dom, const pot_camera* cam,
                     float* depth, float* normal);

/* ---- traversal of the fluid volume (Sec. 6, volume traversal) --------- */

/* Walk each camera ray through the fluid cell by cell: the generalized
 * Laguerre cells of Eq. 1 at (pos, psi) are evaluated first (as
 * lgc_compute_cells does), then one thread per pixel goes from cell to cell
 * across the restricted bisector facets, leaves the fluid through a free
 * surface (a spherical patch) or the box, and finds the next entry through
 * the air as the next ball along the ray (the fluid is the union of the
 * balls inside the box).  Per pixel (height x width, row-major, device
 * buffers written on `stream`): first: the ray parameter t of the first
 * point in the fluid (-1: none); thickness: the length of the ray inside
 * the fluid; last: t of the last exit (-1: none); visits (optional, int32):
 * the cells visited.  pos (n,3), psi (n) device arrays in caller order.
 * Camera as in pot_render_depth; no graphics API.  Uses ctx's FP32
 * workspace (its cell data are overwritten).
 * Errors: POT_ERR_INVALID_ARG (NULL pointers, n out of range, an FP64-only
 * context, a bad camera or box), the geometry errors of lgc_compute_cells,
 * POT_ERR_CUDA. */
int pot_render_volume(pot_ctx* ctx, void* stream, int64_t n, const float* pos, const float* psi,
                      const pot_domain* dom, const pot_camera* cam, float* first,
                      float* thickness, float* last, int32_t* visits);

/* ---- smoothed free surface (Sec. 6, surface smoothing) ----------------- */

/* Sphere-trace each camera ray to the smoothed free surface: the cells at
 * (pos, psi) are evaluated first (as lgc_compute_cells does); at a ray
 * point x the closest site i (least |x - p_i| - r_i) and its Laguerre
 * neighbourhood (the sites sharing a restricted facet with it) give the
 * signed distance f = smin_k(d_(1), d_(2)), the cubic polynomial smooth
 * union of the two nearest spheres of that set with smoothing radius
 * k_smooth (smin_k(a, b) = min(a, b) - k h^3 / 6, h = max(k - |a - b|, 0)
 * / k).  A ray point farther than k/6 from every ball jumps to the next
 * entry into the balls grown by k/6; otherwise the march steps by f (at
 * least 1e-4 k) and stops at f <= 1e-3 k, after at most 1024 evaluations.
 * Per pixel (height x width, row-major, device buffers written on
 * `stream`): depth: t of the hit (-1: none); normal (3 per pixel,
 * optional): the unit gradient of f there (0: none); steps (optional,
 * int32): evaluations of f taken.  pos (n,3), psi (n) device arrays in
 * caller order.  Camera as in pot_render_depth; no graphics API.  Uses
 * ctx's FP32 workspace (its cell data are overwritten).
 * Errors: POT_ERR_INVALID_ARG (NULL pointers, n out of range, an FP64-only
 * context, k_smooth not positive and finite, a bad camera or box), the
 * geometry errors of lgc_compute_cells, POT_ERR_CUDA. */
int pot_render_smooth(pot_ctx* ctx, void* stream, int64_t n, const float* pos, const float* psi,
                      const pot_domain* dom, const pot_camera* cam, float k_smooth, float* depth,
                      float* normal, int32_t* steps);

#ifdef __cplusplus
}
#endif

#endif /* POT_H */
