// Damped Newton with KMT steps (Algorithm 1) and the explicit fluid step
// (Sec. 5), driven from the host; every per-site step runs in the kernels of
// cells.cu / pcg.cu.  The only device-to-host traffic per Newton iteration is
// the FP64 residual summary (max relative error, squared l2 norm, min volume)
// read after each cell evaluation, and the PCG done flag once per chunk.
//
// Readings of Algorithm 1 (its printed form is garbled):
//   - the Newton system is M u = nu - V(psi), M = -grad^2 K (Eq. 2);
//   - the KMT step halves alpha from 1 until min V(psi + alpha u) >= eps0 and
//     ||nu - V(psi + alpha u)||_2 <= (1 - alpha/2) ||nu - V(psi)||_2, with
//     eps0 = 1/2 min(min nu, min V(psi_start)); the FP32-geometry path also
//     accepts that decrease of the max relative error (see the line search);
//   - the start is the given psi (psi = 0 would give empty cells);
//   - convergence: max_i |V_i - nu_i| / nu_i <= tol (relative, Sec. 7).
#include <chrono>
#include <math.h>

#include "pot_internal.cuh"

namespace pot {
namespace {

// stopping test of the FP32-geometry path: err <= kMixedStop * tol
constexpr double kMixedStop = 0.9;

template <typename T>
__global__ void k_accept(int64_t n, const V4<T>* __restrict__ sxp, T* base) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n) base[s] = sxp[s].w;
}

__global__ void k_nu_min(int64_t n, const double* __restrict__ snu, double* part) {
  double m = 1e300;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    m = fmin(m, snu[i]);
  for (int off = 16; off > 0; off >>= 1) m = fmin(m, __shfl_down_sync(kFull, m, off));
  __shared__ double sh[8];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); w++) m = fmin(m, sh[w]);
    part[blockIdx.x] = m;
  }
}

__global__ void k_min_final(const double* __restrict__ part, int nb, double* out) {
  double m = 1e300;  // one warp: strided, then a shuffle tree
  for (int b = threadIdx.x; b < nb; b += 32) m = fmin(m, part[b]);
  for (int off = 16; off > 0; off >>= 1) m = fmin(m, __shfl_down_sync(kFull, m, off));
  if (threadIdx.x == 0) *out = m;
}

// x <- x + dt v, clamped into [lo+m, hi-m]; velocity through a wall -> 0
template <typename T>
__global__ void k_advect(int64_t n, T* pos, T* vel, T dt, Box<T> box, T margin) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
#pragma unroll
  for (int k = 0; k < 3; k++) {
    T x = pos[3 * i + k] + dt * vel[3 * i + k];
    T v = vel[3 * i + k];
    T lo = box.lo[k] + margin, hi = box.hi[k] - margin;
    if (x < lo) {
      x = lo;
      if (v < T(0)) v = T(0);
    } else if (x > hi) {
      x = hi;
      if (v > T(0)) v = T(0);
    }
    pos[3 * i + k] = x;
    vel[3 * i + k] = v;
  }
}

// v <- v + dt (g + (c_i - x_i) / eps^2)  (pressure spring, Sec. 5); psi out
template <typename T>
__global__ void k_velocity(int64_t n, const int32_t* __restrict__ perm,
                           const V4<T>* __restrict__ sxp, const T* __restrict__ cen,
                           const T* __restrict__ psi_base, T* vel, T* psi, T dt, T inv_eps2,
                           T gx, T gy, T gz) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  int64_t o = perm[s];
  const V4<T> p = sxp[s];
  vel[3 * o + 0] += dt * (gx + (cen[3 * s + 0] - p.x) * inv_eps2);
  vel[3 * o + 1] += dt * (gy + (cen[3 * s + 1] - p.y) * inv_eps2);
  vel[3 * o + 2] += dt * (gz + (cen[3 * s + 2] - p.z) * inv_eps2);
  psi[o] = psi_base[s];
}

// Extrapolated start (Sec. 5 steps are smooth in time): psi_start =
// psi^k + (psi^k - psi^{k-1}), from the weights at the start of this step
// (psi, caller order) and of the previous one (hist); a non-positive value
// keeps psi^k.  The plain start psi^k is kept in fb (sorted) for the
// fallback; the largest new weight raises psi_max.
template <typename T>
__global__ void k_extrapolate(int64_t n, const int32_t* __restrict__ perm, const T* __restrict__ psi,
                              const T* __restrict__ hist, V4<T>* sxp, T* psi_base, T* fb,
                              T* psi_max) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  T v = T(0);
  if (s < n) {
    const int64_t o = perm[s];
    const T p = psi[o];
    v = p + (p - hist[o]);
    if (!(v > T(0))) v = p;
    fb[s] = p;
    sxp[s].w = v;
    psi_base[s] = v;
  }
  block_max_to(v > T(0) ? v : T(0), psi_max);
}

// Semi-implicit velocity update with viscosity and surface tension (Sec. 5,
// Eq. 4, unit mass) over the P1 Laplacian of Eq. 3, whose weights
// w_ij = |B_ij| / (2 d_ij) are the converged cells' off-diagonal Hessian
// entries with the sign flipped (vals = -w):
//   (I/dt + mu (D - W) + mu_wall Dw) v^{k+1} = v^k/dt + (c - x)/eps^2 + g + gamma L x + T_w,
//   D = diag(sum_j w_ij), (L x)_i = sum_j w_ij (x_j - x_i), Dw = diag of the
//   wall facets' weights |B_iw| / (2 h_iw) (walls at rest: no-slip), T_w the
//   walls' part of the surface tension, gamma_wall sum_w |B_iw| / (2 h_iw)
//   (h_iw + cbrt |V_i|) n_w (a neighbour cbrt |V_i| beyond each wall).
// This kernel forms the right-hand side per sorted site (into b, 3 per
// site) and the system's diagonal (into diag).
// With per-site factors f (several fluids), mu_ij = mu (f_i + f_j) / 2 (the
// per-pair coefficients of Sec. 5); the row's entries become the system's
// off-diagonal -mu_ij w_ij in place (each thread owns its row).
template <typename T>
__global__ void k_visc_rhs(int64_t n, const int32_t* __restrict__ perm,
                           const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ cols,
                           T* vals, const V4<T>* __restrict__ sxp, const T* cen,
                           const T* __restrict__ vel, const float* __restrict__ factors,
                           const T* __restrict__ wallw, T mu_wall, const T* __restrict__ wallv,
                           const T* __restrict__ vol, T gamma_wall, T dt, T inv_eps2, T gx, T gy,
                           T gz, T mu, T gamma, T* b, T* diag) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const V4<T> p = sxp[i];
  const T fi = factors ? (T)factors[perm[i]] : T(1);
  T msum = T(0), lx = T(0), ly = T(0), lz = T(0);
  for (int k = row_ptr[i]; k < row_ptr[i + 1]; k++) {
    const T wij = -vals[k];
    const int j = cols[k];
    const V4<T> q = sxp[j];
    const T mij = factors ? mu * T(0.5) * (fi + (T)factors[perm[j]]) : mu;
    msum += mij * wij;
    vals[k] = -mij * wij;
    lx += wij * (q.x - p.x);
    ly += wij * (q.y - p.y);
    lz += wij * (q.z - p.z);
  }
  const int64_t o = perm[i];
  T tx = T(0), ty = T(0), tz = T(0);
  if (gamma_wall != T(0)) {
    // the walls' part of the surface tension: each wall facet is the facet
    // to a neighbour cbrt(|V_i|) beyond the wall, weight |B| / (2 h):
    // sum_w |B|/(2h) (h + cbrt V) n = sum |B| n / 2 + cbrt V sum |B| n / (2h)
    const T* wv = wallv + 6 * i;
    const T cv = cbrt(fmax(vol[i], T(0)));
    tx = gamma_wall * (wv[0] + cv * wv[3]);
    ty = gamma_wall * (wv[1] + cv * wv[4]);
    tz = gamma_wall * (wv[2] + cv * wv[5]);
  }
  const T bx = vel[3 * o + 0] / dt + (cen[3 * i + 0] - p.x) * inv_eps2 + gx + gamma * lx + tx;
  const T by = vel[3 * o + 1] / dt + (cen[3 * i + 1] - p.y) * inv_eps2 + gy + gamma * ly + ty;
  const T bz = vel[3 * o + 2] / dt + (cen[3 * i + 2] - p.z) * inv_eps2 + gz + gamma * lz + tz;
  b[3 * i + 0] = bx;
  b[3 * i + 1] = by;
  b[3 * i + 2] = bz;
  // no-slip walls: the wall facets' Laplacian weight towards zero velocity
  diag[i] = T(1) / dt + msum + mu_wall * wallw[i];
}

// component c of b (sorted) as the PCG right-hand side
template <typename T>
__global__ void k_visc_b(int64_t n, const T* __restrict__ b, int c, double* rhs) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) rhs[i] = (double)b[3 * i + c];
}

// component c of the new velocity (caller order): the solution u, or dt b
// when there is no viscosity (the system is then I/dt)
template <typename T>
__global__ void k_visc_store(int64_t n, const int32_t* __restrict__ perm, const T* __restrict__ u,
                             const T* __restrict__ b, int c, T dt, T* vel) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  vel[3 * (int64_t)perm[i] + c] = u ? u[i] : dt * b[3 * i + c];
}

// psi <- src (sorted), the current weights for evaluation and the base;
// psi_max follows (reset by the caller)
template <typename T>
__global__ void k_set_psi(int64_t n, const T* __restrict__ src, V4<T>* sxp, T* base, T* psi_max) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  T v = T(0);
  if (s < n) {
    v = src[s];
    sxp[s].w = v;
    base[s] = v;
  }
  block_max_to(v > T(0) ? v : T(0), psi_max);
}

template <typename T>
__global__ void k_unsort_psi(int64_t n, const int32_t* __restrict__ perm, const T* __restrict__ base,
                             T* psi) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n) psi[perm[s]] = base[s];
}

double now_ms() {
  return std::chrono::duration<double, std::milli>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct EvTimer {
  cudaEvent_t a, b;
  cudaStream_t st;
  EvTimer(pot_ctx* ctx, int k, cudaStream_t s) : a(ctx->ev[2 * k]), b(ctx->ev[2 * k + 1]), st(s) {
    cudaEventRecord(a, st);
  }
  double stop() {
    cudaEventRecord(b, st);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    return ms;
  }
};

// one full evaluation + status + residual summary
template <typename T>
int eval_and_reduce(pot_ctx* ctx, cudaStream_t st, int64_t n, const pot_domain* dom,
                    double res[6], pot_solve_stats* S) {
  EvTimer tm(ctx, 0, st);
  // the residual summary and the status word come back with the last
  // pass's wait
  const int ce = cells_eval<T>(ctx, st, n, dom, true, true);
  int64_t site;
  int code;
  if (ctx->tail_ready) {
    code = status_on_host(ctx, &site);  // also clears the device status
  } else {
    if (ce == POT_OK) POT_CHECK(residuals<T>(ctx, st, n, nullptr));
    code = read_status(ctx, st, &site);
  }
  if (ce == POT_OK)
    for (int k = 0; k < 6; k++) res[k] = ctx->h_pinned[k];
  S->ms_cells += tm.stop();
  S->cell_evals++;
  S->passes += ctx->last_passes;
  if (code != POT_OK) S->error_site = site;
  return code != POT_OK ? code : ce;
}

}  // namespace

// Newton solve in sorted space.  Requires grid_build (sxp.w = psi_base = start).
// psi_fallback (sorted, optional): weights to restart from when the given
// start fails the KMT precondition -- an empty cell (the bound eps0 needs
// min V > 0) or a geometry error.
template <typename T>
int newton_sorted_impl(pot_ctx* ctx, cudaStream_t st, int64_t n, const pot_domain* dom,
                       const pot_params* P, pot_solve_stats* S, const T* psi_fallback);

// The evaluations of one solve share the grid order: the candidate pass
// keeps its neighbour lists across them.
template <typename T>
int newton_sorted(pot_ctx* ctx, cudaStream_t st, int64_t n, const pot_domain* dom,
                  const pot_params* P, pot_solve_stats* S, const T* psi_fallback = nullptr) {
  Work<T>& w = ctx->work<T>();
  w.verlet = true;
  const int status = newton_sorted_impl<T>(ctx, st, n, dom, P, S, psi_fallback);
  w.verlet = false;
  return status;
}

template <typename T>
int newton_sorted_impl(pot_ctx* ctx, cudaStream_t st, int64_t n, const pot_domain* dom,
                       const pot_params* P, pot_solve_stats* S, const T* psi_fallback) {
  Work<T>& w = ctx->work<T>();
  double res[6];
  if (psi_fallback) {
    int code = eval_and_reduce<T>(ctx, st, n, dom, res, S);
    const bool bad = code != POT_OK || !(res[2] > 0.0);
    if (bad) {
      S->mlp_fallback = 1;
      POT_CUDA(cudaMemsetAsync(w.psi_max, 0, sizeof(T), st));
      note_launch();
      k_set_psi<T><<<blocks_for(n, 256), 256, 0, st>>>(n, psi_fallback, w.sxp, w.psi_base, w.psi_max);
      POT_CHECK(eval_and_reduce<T>(ctx, st, n, dom, res, S));
    } else {
      S->mlp_used = 1;
    }
  } else {
    POT_CHECK(eval_and_reduce<T>(ctx, st, n, dom, res, S));
  }
  S->err_start = res[0];
  // empty cells at the start (sites pushed deep into a heavier neighbour's
  // cell by a fast step): raise their weights until every site is inside its
  // own cell, then start Algorithm 1 from the repaired weights
  for (int rep = 0; rep < 32 && !(res[2] > 0.0); rep++) {
    int repaired = 0;
    POT_CHECK(repair_empty<T>(ctx, st, n, &repaired));
    if (repaired == 0) break;
    S->repairs += repaired;
    POT_CHECK(eval_and_reduce<T>(ctx, st, n, dom, res, S));
  }
  S->err_max = res[0];
  S->err_l2 = sqrt(res[1]);
  if (!(res[2] > 0.0)) return POT_ERR_EMPTY_CELL_AT_START;
  // cell extents of the accepted iterate seed the security radii of the trials
  POT_CUDA(cudaMemcpyAsync(w.rcell_acc, w.rcell, n * sizeof(T), cudaMemcpyDeviceToDevice, st));
  w.have_acc = true;
  note_launch();
  k_nu_min<<<kRedBlocks, 256, 0, st>>>(n, ctx->snu, ctx->red);
  note_launch();
  k_min_final<<<1, 32, 0, st>>>(ctx->red, kRedBlocks, ctx->red_out);
  POT_CUDA(cudaMemcpyAsync(ctx->h_pinned, ctx->red_out, sizeof(double), cudaMemcpyDeviceToHost, st));
  POT_CUDA(cudaStreamSynchronize(st));
  const double eps0 = 0.5 * fmin(ctx->h_pinned[0], res[2]);
  // The FP32-geometry path stops at kMixedStop * tol on its FP32-evaluated
  // error: the margin of 0.1 tol (1e-5 at tol = 1e-4) covers the rounding
  // of the FP32 volumes (measured against the FP64 oracle at about 1e-6 of
  // the target, ten times below it), so that the volumes meet tol exactly
  const double tol_stop = sizeof(T) == 4 ? kMixedStop * P->tol : P->tol;
  double err = res[0], gnorm = sqrt(res[1]);
  for (int it = 0;; it++) {
    S->newton_iters = it;
    S->err_max = err;
    S->err_l2 = gnorm;
    if (err <= tol_stop) return POT_OK;
    if (it >= P->max_newton) return POT_ERR_NOT_CONVERGED;
    int64_t nnz_off = 0;
    POT_CHECK(csr_compact<T>(ctx, st, n, nullptr));  // its size is read after the PCG's wait
    // inexact Newton: the linear residual only needs to be small against
    // the distance still to go to the tolerance, and far from it no smaller
    // than the error the next Newton step leaves anyway (about err^2)
    double rtol = P->pcg_rtol;
    if (!(rtol > 0.0)) rtol = fmin(0.1, fmax(1e-7, fmax(0.1 * P->tol / err, 0.02 * err)));
    int iters = 0;
    {
      EvTimer tm(ctx, 1, st);
      int ps = pcg_solve<T>(ctx, st, n, nnz_off, rtol, P->max_pcg, P->pcg_chunk,
                            P->pcg_host_loop != 0, &iters, nullptr);
      S->ms_pcg += tm.stop();
      S->pcg_iters += iters;
      S->nnz = csr_nnz(ctx) + n;
      if (ps != POT_OK) return ps;
    }
    double alpha = 1.0;
    bool accepted = false;
    for (int hv = 0; hv <= P->max_halvings; hv++) {
      POT_CHECK(psi_update<T>(ctx, st, n, alpha));
      // a trial whose balls grew past the cell kernel's capacities is a
      // rejected step (halve), not a failure of the solve
      const int code = eval_and_reduce<T>(ctx, st, n, dom, res, S);
      if (code != POT_OK && code != POT_ERR_NEIGHBOUR_OVERFLOW && code != POT_ERR_POLYGON_OVERFLOW)
        return code;
      // KMT: a sufficient decrease of the l2 norm (FP64 path: the test of
      // Algorithm 1 as read, nothing else).  The FP32-geometry path also
      // accepts the same decrease of the max relative error that the
      // stopping test measures: its l2 norm over many cells reaches the FP32
      // rounding floor (about 1e-6 nu per cell) while a few worst cells are
      // still above the tolerance, where the l2 test alone stalls
      const double fac = 1.0 - 0.5 * alpha;
      const bool l2_ok = sqrt(res[1]) <= fac * gnorm;
      const bool max_ok = sizeof(T) == 4 && res[0] <= fac * err;
      if (code == POT_OK && res[2] >= eps0 && (l2_ok || max_ok)) {
        accepted = true;
        break;
      }
      alpha *= 0.5;
      S->halvings++;
    }
    if (!accepted) {
      // back to the last accepted weights, with their cells
      POT_CHECK(psi_update<T>(ctx, st, n, 0.0));
      POT_CHECK(eval_and_reduce<T>(ctx, st, n, dom, res, S));
      return POT_ERR_LINESEARCH_FAILED;
    }
    note_launch();
    k_accept<T><<<blocks_for(n, 256), 256, 0, st>>>(n, w.sxp, w.psi_base);
    POT_CUDA(cudaMemcpyAsync(w.rcell_acc, w.rcell, n * sizeof(T), cudaMemcpyDeviceToDevice, st));
    err = res[0];
    gnorm = sqrt(res[1]);
  }
}

template <typename T>
int newton_solve(pot_ctx* ctx, cudaStream_t st, int64_t n, const T* pos, const double* targets,
                 T* psi_inout, const pot_domain* dom, const pot_params* P, pot_solve_stats* S) {
  double t0 = now_ms();
  POT_CHECK(grid_build<T>(ctx, st, n, pos, psi_inout, targets, dom));
  S->grid_builds++;
  Work<T>& w = ctx->work<T>();
  w.use_hint = true;  // security balls start from the last solve's cells
  w.hist_n = -1;      // weights from outside a run of fluid steps: no history
  int status = newton_sorted<T>(ctx, st, n, dom, P, S);
  if (status == POT_OK || status == POT_ERR_NOT_CONVERGED || status == POT_ERR_LINESEARCH_FAILED) {
    note_launch();
    k_unsort_psi<T><<<blocks_for(n, 256), 256, 0, st>>>(n, ctx->perm, w.psi_base, psi_inout);
    POT_CHECK(store_hint<T>(ctx, st, n));
  }
  POT_CUDA(cudaStreamSynchronize(st));
  S->status = status;
  S->ms_total = now_ms() - t0;
  return status;
}

namespace {

// One explicit step of length dt (Sec. 5): advect and clamp, Newton at the
// new positions warm-started from psi, velocities from the centroids.
template <typename T>
int fluid_substep(pot_ctx* ctx, cudaStream_t st, int64_t n, T* pos, T* vel, T* psi,
                  const double* targets, const pot_domain* dom, const pot_params* P, double dt,
                  pot_solve_stats* S) {
  double t0 = now_ms();
  Box<T> box;
  for (int k = 0; k < 3; k++) {
    box.lo[k] = (T)dom->lo[k];
    box.hi[k] = (T)dom->hi[k];
  }
  note_launch();
  k_advect<T><<<blocks_for(n, 256), 256, 0, st>>>(n, pos, vel, (T)dt, box, (T)P->wall_margin);
  POT_CHECK(grid_build<T>(ctx, st, n, pos, psi, targets, dom));
  S->grid_builds++;
  ctx->work<T>().use_hint = true;  // security balls start from the last step's cells
  const T* fallback = nullptr;
  if (sizeof(T) == 4 && P->warm_start == 1 && ctx->mlp) {
    float* prev = nullptr;
    POT_CHECK(mlp_warm_start(ctx, ctx->mlp, st, n, (const float*)vel, (const float*)psi,
                             (float)dt, &prev));
    fallback = (const T*)prev;
  } else if (P->warm_start == 2) {
    Work<T>& w = ctx->work<T>();
    if (w.hist_n == n) {
      note_launch();
      k_extrapolate<T><<<blocks_for(n, 256), 256, 0, st>>>(n, ctx->perm, psi, w.psi_hist, w.sxp,
                                                           w.psi_base, w.psi_fb, w.psi_max);
      POT_CUDA(cudaGetLastError());
      fallback = w.psi_fb;
    }
    // this step's starting weights are the next step's history
    POT_CUDA(cudaMemcpyAsync(w.psi_hist, psi, n * sizeof(T), cudaMemcpyDeviceToDevice, st));
    w.hist_n = n;
  }
  int status = newton_sorted<T>(ctx, st, n, dom, P, S, fallback);
  if (fallback && S->mlp_used &&
      (status == POT_ERR_NOT_CONVERGED || status == POT_ERR_LINESEARCH_FAILED)) {
    // Newton from the learned start failed: plain Newton from the previous
    // weights judges the step
    S->mlp_used = 0;
    S->mlp_fallback = 1;
    Work<T>& w = ctx->work<T>();
    POT_CUDA(cudaMemsetAsync(w.psi_max, 0, sizeof(T), st));
    note_launch();
    k_set_psi<T><<<blocks_for(n, 256), 256, 0, st>>>(n, fallback, w.sxp, w.psi_base, w.psi_max);
    status = newton_sorted<T>(ctx, st, n, dom, P, S, nullptr);
  }
  if (status == POT_OK || status == POT_ERR_NOT_CONVERGED || status == POT_ERR_LINESEARCH_FAILED) {
    Work<T>& w = ctx->work<T>();
    const bool viscous =
        P->mu > 0.0 || P->gamma > 0.0 || P->mu_wall > 0.0 || P->gamma_wall != 0.0;
    const bool solve = P->mu > 0.0 || P->mu_wall > 0.0;
    if (viscous) {
      // Eq. 4 over the converged cells: right-hand side from the old
      // velocities, the weights written out (k_velocity with dt = 0 leaves
      // the velocities alone), then one solve per component
      const double tv = now_ms();
      int64_t nnz_off = 0;
      POT_CHECK(csr_compact<T>(ctx, st, n, &nnz_off));
      note_launch();
      k_visc_rhs<T><<<blocks_for(n, 256), 256, 0, st>>>(
          n, ctx->perm, ctx->row_ptr, ctx->csr_cols, w.csr_vals, w.sxp, w.cen, vel,
          ctx->visc_factors_n == n ? ctx->visc_factors : nullptr, w.wallw, (T)P->mu_wall,
          w.wallv, w.vol, (T)P->gamma_wall, (T)dt,
          (T)(1.0 / (P->eps * P->eps)), (T)P->gravity[0], (T)P->gravity[1], (T)P->gravity[2],
          (T)P->mu, (T)P->gamma, w.vel_s, w.diag);
      POT_CUDA(cudaGetLastError());
      note_launch();
      k_velocity<T><<<blocks_for(n, 256), 256, 0, st>>>(
          n, ctx->perm, w.sxp, w.cen, w.psi_base, vel, psi, T(0), T(0), T(0), T(0), T(0));
      for (int c = 0; c < 3; c++) {
        if (solve) {
          note_launch();
          k_visc_b<T><<<blocks_for(n, 256), 256, 0, st>>>(n, w.vel_s, c, ctx->grad);
          int iters = 0;
          const double rtol = sizeof(T) == 4 ? 1e-6 : 1e-11;
          POT_CHECK(pcg_solve<T>(ctx, st, n, nnz_off, rtol, P->max_pcg, P->pcg_chunk,
                                 P->pcg_host_loop != 0, &iters, nullptr));
          S->visc_iters += iters;
        }
        note_launch();
        k_visc_store<T><<<blocks_for(n, 256), 256, 0, st>>>(n, ctx->perm, solve ? w.u : nullptr,
                                                            w.vel_s, c, (T)dt, vel);
      }
      POT_CUDA(cudaGetLastError());
      POT_CUDA(cudaStreamSynchronize(st));
      S->ms_visc += now_ms() - tv;
    } else {
      note_launch();
      k_velocity<T><<<blocks_for(n, 256), 256, 0, st>>>(
          n, ctx->perm, w.sxp, w.cen, w.psi_base, vel, psi, (T)dt, (T)(1.0 / (P->eps * P->eps)),
          (T)P->gravity[0], (T)P->gravity[1], (T)P->gravity[2]);
    }
    POT_CHECK(store_hint<T>(ctx, st, n));
  }
  POT_CUDA(cudaStreamSynchronize(st));
  S->status = status;
  S->ms_total = now_ms() - t0;
  return status;
}

}  // namespace

// P->substeps explicit steps of dt / substeps (at least one), stopping at
// the first that fails; S sums the counts and times of the substeps and
// keeps the largest start and final errors.
template <typename T>
int fluid_step(pot_ctx* ctx, cudaStream_t st, int64_t n, T* pos, T* vel, T* psi,
               const double* targets, const pot_domain* dom, const pot_params* P,
               pot_solve_stats* S) {
  const int k = P->substeps > 1 ? P->substeps : 1;
  if (k == 1) return fluid_substep<T>(ctx, st, n, pos, vel, psi, targets, dom, P, P->dt, S);
  const double dt = P->dt / k;
  pot_solve_stats acc = *S;
  int status = POT_OK;
  for (int i = 0; i < k && status == POT_OK; i++) {
    pot_solve_stats s1;
    memset(&s1, 0, sizeof(s1));
    s1.error_site = -1;
    status = fluid_substep<T>(ctx, st, n, pos, vel, psi, targets, dom, P, dt, &s1);
    acc.newton_iters += s1.newton_iters;
    acc.pcg_iters += s1.pcg_iters;
    acc.halvings += s1.halvings;
    acc.cell_evals += s1.cell_evals;
    acc.grid_builds += s1.grid_builds;
    acc.repairs += s1.repairs;
    acc.passes += s1.passes;
    acc.ms_total += s1.ms_total;
    acc.ms_cells += s1.ms_cells;
    acc.ms_pcg += s1.ms_pcg;
    acc.visc_iters += s1.visc_iters;
    acc.ms_visc += s1.ms_visc;
    acc.err_start = i == 0 ? s1.err_start : fmax(acc.err_start, s1.err_start);
    acc.err_max = i == 0 ? s1.err_max : fmax(acc.err_max, s1.err_max);
    acc.err_l2 = i == 0 ? s1.err_l2 : fmax(acc.err_l2, s1.err_l2);
    acc.nnz = s1.nnz;
    acc.mlp_used |= s1.mlp_used;
    acc.mlp_fallback |= s1.mlp_fallback;
    if (s1.error_site >= 0) acc.error_site = s1.error_site;
    acc.status = status;
  }
  *S = acc;
  return status;
}

#define POT_NINST(T)                                                                             \
  template int newton_solve<T>(pot_ctx*, cudaStream_t, int64_t, const T*, const double*, T*,    \
                               const pot_domain*, const pot_params*, pot_solve_stats*);         \
  template int fluid_step<T>(pot_ctx*, cudaStream_t, int64_t, T*, T*, T*, const double*,        \
                             const pot_domain*, const pot_params*, pot_solve_stats*);
POT_NINST(float)
POT_NINST(double)

}  // namespace pot
