// C ABI of libpot.so (declared in include/pot.h): argument checks, context
// and workspace, and the entry points that chain the kernels of grid.cu,
// cells.cu, pcg.cu and newton.cu.
#include <math.h>
#include <string.h>

#include <new>

#include "pot_internal.cuh"

namespace pot {
template <typename T>
int newton_solve(pot_ctx*, cudaStream_t, int64_t, const T*, const double*, T*, const pot_domain*,
                 const pot_params*, pot_solve_stats*);
template <typename T>
int fluid_step(pot_ctx*, cudaStream_t, int64_t, T*, T*, T*, const double*, const pot_domain*,
               const pot_params*, pot_solve_stats*);
}  // namespace pot

namespace pot {
std::atomic<long long> g_launches{0};
}  // namespace pot

using namespace pot;

namespace {

template <typename P>
int alloc(P** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  return cudaMalloc((void**)p, count * sizeof(P)) == cudaSuccess ? POT_OK : POT_ERR_CUDA;
}

template <typename T>
int alloc_work(Work<T>& w, int64_t n, int64_t k, int64_t gcap, int sms) {
  POT_CHECK(alloc(&w.sxp, n));
  POT_CHECK(alloc(&w.psi_base, n));
  POT_CHECK(alloc(&w.vol, n));
  POT_CHECK(alloc(&w.karea, n));
  POT_CHECK(alloc(&w.diag, n));
  POT_CHECK(alloc(&w.cen, 3 * n));
  POT_CHECK(alloc(&w.stage_vals, n * k));
  POT_CHECK(alloc(&w.csr_vals, n * k));
  POT_CHECK(alloc(&w.u, n));
  POT_CHECK(alloc(&w.x, n));
  POT_CHECK(alloc(&w.r, n));
  POT_CHECK(alloc(&w.z, n));
  POT_CHECK(alloc(&w.p0, n));
  POT_CHECK(alloc(&w.p1, n));
  POT_CHECK(alloc(&w.zp, 2 * n));
  POT_CHECK(alloc(&w.q, n));
  POT_CHECK(alloc(&w.vel_s, 3 * n));
  POT_CHECK(alloc(&w.psi_max, 1));
  POT_CHECK(alloc(&w.nu_max, 1));
  POT_CHECK(alloc(&w.srad, n));
  POT_CHECK(alloc(&w.srad_lo, n));
  POT_CHECK(alloc(&w.soff, 3 * n));
  POT_CHECK(alloc(&w.hint, 4 * n));
  POT_CHECK(alloc(&w.wallw, n));
  POT_CHECK(alloc(&w.wallv, 6 * n));
  POT_CHECK(alloc(&w.psi_hist, n));
  POT_CHECK(alloc(&w.psi_fb, n));
  POT_CHECK(alloc(&w.rcell_acc, n));
  POT_CHECK(alloc(&w.rcell, n));
  POT_CHECK(alloc(&w.vlist, n * (int64_t)kVerletCap));
  POT_CHECK(alloc(&w.vcount, n));
  POT_CHECK(alloc(&w.vreach, n));
  POT_CHECK(alloc(&w.gmax, gcap + 1));
  w.ccap = gcap / 8 + 4096;
  POT_CHECK(alloc(&w.cmax, w.ccap));
  POT_CHECK(alloc(&w.cnb, w.ccap));
  // cells with more planes than the cell kernel takes (kSmallPlanes) exist
  // only when the lists may hold that many
  if (k + 6 > kSmallPlanes) {
    w.big_warps = sms * kBigWarpsPerSm;
    POT_CHECK(alloc(&w.big_pl, (int64_t)w.big_warps * kBigPlanes));
    POT_CHECK(alloc(&w.big_d, (int64_t)w.big_warps * kBigPlanes));
    POT_CHECK(alloc(&w.big_j, (int64_t)w.big_warps * kBigPlanes));
  }
  return POT_OK;
}

template <typename T>
void free_work(Work<T>& w) {
  void* ptrs[] = {w.sxp, w.psi_base, w.vol,  w.karea, w.diag, w.cen, w.stage_vals, w.csr_vals,
                  w.u,   w.x,        w.r,    w.z,     w.p0,   w.p1,  w.q,          w.vel_s,
                  w.psi_max, w.nu_max, w.srad, w.srad_lo, w.soff, w.hint, w.rcell_acc, w.rcell, w.gmax,
                  w.big_pl, w.big_d, w.big_j, w.psi_hist, w.psi_fb, w.wallw, w.vlist, w.vcount,
                  w.vreach, w.wallv, w.zp, w.cmax, w.cnb};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  w = Work<T>();
}

bool finite_box(const pot_domain* d) {
  if (!d) return false;
  for (int k = 0; k < 3; k++)
    if (!(isfinite(d->lo[k]) && isfinite(d->hi[k]) && d->hi[k] > d->lo[k])) return false;
  return true;
}

int check_ctx(pot_ctx* ctx, int64_t n, int need) {
  if (!ctx || n <= 0 || n > ctx->n_max) return POT_ERR_INVALID_ARG;
  if (!(ctx->mask & need)) return POT_ERR_INVALID_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return POT_ERR_CUDA;
  return POT_OK;
}

bool check_params(const pot_params* p) {
  return p && p->tol > 0.0 && p->max_newton >= 0 && p->max_halvings >= 0 && p->max_pcg > 0 &&
         p->pcg_chunk > 0 && isfinite(p->dt) && p->eps > 0.0 && p->substeps >= 0 &&
         p->mu >= 0.0 && p->gamma >= 0.0 && p->mu_wall >= 0.0 && isfinite(p->mu) &&
         isfinite(p->gamma) && isfinite(p->mu_wall) && isfinite(p->gamma_wall) &&
         (p->pcg_host_loop == 0 || p->pcg_host_loop == 1);
}

template <typename T, typename CSR>
int compute_cells(pot_ctx* ctx, void* stream, int64_t n, const T* pos, const T* psi,
                  const double* targets, const pot_domain* dom, T* volumes, double* grad, CSR* hess,
                  T* centroids, T* karea, pot_cell_stats* stats) {
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->error_site = -1;
  }
  POT_CHECK(check_ctx(ctx, n, sizeof(T) == 4 ? 1 : 2));
  if (!pos || !psi || !finite_box(dom)) return POT_ERR_INVALID_ARG;
  if (hess && (!hess->row_ptr || (hess->cap > 0 && (!hess->cols || !hess->vals)))) return POT_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t* ev = ctx->ev;
  cudaEventRecord(ev[0], st);
  POT_CHECK(grid_build<T>(ctx, st, n, pos, psi, targets, dom));
  cudaEventRecord(ev[1], st);
  const int ce = cells_eval<T>(ctx, st, n, dom, grad != nullptr);
  cudaEventRecord(ev[2], st);
  int64_t site = -1;
  int code = read_status(ctx, st, &site);  // also clears the device status
  if (code == POT_OK) code = ce;
  if (code) {
    if (stats) stats->error_site = site;
    return code;
  }
  double res[6];
  POT_CHECK(residuals<T>(ctx, st, n, res));
  POT_CHECK(unsort_outputs<T>(ctx, st, n, volumes, grad, centroids, karea, nullptr));
  int64_t nnz = 0;
  cudaEventRecord(ev[3], st);
  if (hess) {
    int s = csr_user<T>(ctx, st, n, hess->row_ptr, hess->cols, hess->vals, hess->cap, &nnz);
    hess->nnz = nnz;
    if (s != POT_OK) return s;
  }
  cudaEventRecord(ev[4], st);
  POT_CUDA(cudaEventSynchronize(ev[4]));
  if (stats) {
    stats->n_empty = (int64_t)res[3];
    stats->n_planes = (int64_t)res[4];
    stats->max_planes = (int32_t)res[5];
    stats->nnz = nnz;
    cudaEventElapsedTime(&stats->ms_grid, ev[0], ev[1]);
    cudaEventElapsedTime(&stats->ms_cells, ev[1], ev[2]);
    cudaEventElapsedTime(&stats->ms_csr, ev[3], ev[4]);
  }
  return POT_OK;
}

}  // namespace

extern "C" {

int64_t pot_kernel_launches(void) { return g_launches.load(); }

int pot_cell_diagnostics(pot_ctx* ctx, void* stream, int64_t n, float* center_offset, float* radius,
                         float* extent, int32_t* planes) {
  if (!ctx) return POT_ERR_INVALID_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return POT_ERR_CUDA;
  return cell_diagnostics(ctx, (cudaStream_t)stream, n, center_offset, radius, extent, planes);
}

int pot_cell_kernel_time(pot_ctx* ctx, int reset, int64_t* launches, int64_t* cells, double* ms) {
  if (!ctx) return POT_ERR_INVALID_ARG;
  if (launches) *launches = ctx->kc_launches;
  if (cells) *cells = ctx->kc_cells;
  if (ms) *ms = ctx->kc_ms;
  if (reset) {
    ctx->kc_launches = 0;
    ctx->kc_cells = 0;
    ctx->kc_ms = 0.0;
  }
  return POT_OK;
}

void pot_default_params(pot_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->tol = 1e-4;
  p->max_newton = 100;
  p->max_halvings = 30;
  p->max_pcg = 2000;
  p->pcg_chunk = 16;
  p->pcg_rtol = 0.0;
  p->dt = 2e-3;
  p->eps = 0.01;
  p->gravity[0] = 0.0;
  p->gravity[1] = 0.0;
  p->gravity[2] = -9.81;
  p->wall_margin = 1e-6;
  p->warm_start = 0;
}

int pot_set_viscosity_factors(pot_ctx* ctx, int64_t n, const float* factors) {
  if (!ctx || (factors && (n <= 0 || n > ctx->n_max))) return POT_ERR_INVALID_ARG;
  ctx->visc_factors = factors;
  ctx->visc_factors_n = factors ? n : -1;
  return POT_OK;
}

int pot_clear_history(pot_ctx* ctx) {
  if (!ctx) return POT_ERR_INVALID_ARG;
  ctx->wf.hist_n = -1;
  ctx->wd.hist_n = -1;
  return POT_OK;
}

const char* pot_status_string(int status) {
  switch (status) {
    case POT_OK: return "ok";
    case POT_ERR_INVALID_ARG: return "invalid argument";
    case POT_ERR_CUDA: return "CUDA runtime error";
    case POT_ERR_NEIGHBOUR_OVERFLOW: return "more than k_max cutting bisectors in a cell";
    case POT_ERR_COINCIDENT_SITES: return "coincident sites";
    case POT_ERR_EMPTY_CELL_AT_START: return "empty cell at the Newton start";
    case POT_ERR_NOT_CONVERGED: return "Newton did not converge within max_newton";
    case POT_ERR_LINESEARCH_FAILED: return "KMT line search failed";
    case POT_ERR_POLYGON_OVERFLOW: return "facet polygon exceeded its edge capacity";
    case POT_ERR_CAPACITY: return "CSR capacity too small";
    case POT_ERR_PCG_BREAKDOWN: return "PCG breakdown (matrix not positive definite)";
    case POT_ERR_TOO_LARGE: return "more sites than the no-alloc entry point holds (8192)";
    default: return "unknown status";
  }
}

int pot_destroy(pot_ctx* ctx) {
  if (!ctx) return POT_OK;
  cudaSetDevice(ctx->device);
  void* ptrs[] = {ctx->keys,     ctx->perm,    ctx->iperm,    ctx->cell_count, ctx->cell_start,
                  ctx->cand,     ctx->meta,    ctx->row_cnt,  ctx->row_ptr,    ctx->ucnt,
                  ctx->csr_cols, ctx->scan_tmp, ctx->snu,     ctx->grad,       ctx->red,
                  ctx->red_out,  ctx->pcg_red, ctx->pcg_ctl,  ctx->err, ctx->need, ctx->need_count, ctx->big_list,
                  ctx->fix_list};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (int k = 0; k < 2; k++) {
    if (ctx->pcg_exec[k]) cudaGraphExecDestroy(ctx->pcg_exec[k]);
    if (ctx->pcg_graph[k]) cudaGraphDestroy(ctx->pcg_graph[k]);
  }
  free_work(ctx->wf);
  free_work(ctx->wd);
  if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
  for (auto& e : ctx->ev)
    if (e) cudaEventDestroy(e);
  delete ctx;
  return POT_OK;
}

int pot_create(pot_ctx** out, int device, int64_t n_max, int32_t k_max, int32_t precision_mask) {
  if (!out) return POT_ERR_INVALID_ARG;
  *out = nullptr;
  if (n_max <= 0 || n_max > (int64_t)1 << 30 || k_max <= 0 || k_max > kMaxK ||
      (precision_mask & 3) == 0)
    return POT_ERR_INVALID_ARG;
  if (n_max * (int64_t)k_max >= ((int64_t)1 << 31)) return POT_ERR_INVALID_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return POT_ERR_CUDA;
  pot_ctx* ctx = new (std::nothrow) pot_ctx();
  if (!ctx) return POT_ERR_CUDA;
  ctx->device = device;
  ctx->n_max = n_max;
  ctx->k_max = k_max;
  ctx->mask = precision_mask & 3;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  ctx->sm_count = sms > 0 ? sms : 148;
  ctx->grid_cap = n_max * 8 > (1 << 16) ? n_max * 8 : (1 << 16);
  const int64_t n = n_max, k = k_max;
  int s = POT_OK;
#define A(ptr, cnt) \
  if (s == POT_OK) s = alloc(&(ptr), (size_t)(cnt));
  A(ctx->keys, n);
  A(ctx->perm, n);
  A(ctx->iperm, n);
  A(ctx->cell_count, ctx->grid_cap + 1);
  A(ctx->cell_start, ctx->grid_cap + 1);
  A(ctx->cand, n * k);
  A(ctx->meta, n);
  A(ctx->row_cnt, n + 1);
  A(ctx->row_ptr, n + 1);
  A(ctx->ucnt, n + 1);
  A(ctx->csr_cols, n * k);
  ctx->scan_tmp_len = (ctx->grid_cap + 2047) / 2048 + 2;
  A(ctx->scan_tmp, ctx->scan_tmp_len);
  A(ctx->snu, n);
  A(ctx->grad, n);
  A(ctx->red, 6 * kRedBlocks);
  A(ctx->red_out, 8);
  A(ctx->pcg_red, pcg_red_len(ctx->sm_count));
  A(ctx->pcg_ctl, kPcgCtlWords);
  A(ctx->err, 2);
  A(ctx->need, n);
  A(ctx->need_count, 4);
  A(ctx->big_list, n);
  if (precision_mask & 1) A(ctx->fix_list, n);
#undef A
  if (s == POT_OK && (ctx->mask & 1)) s = alloc_work(ctx->wf, n, k, ctx->grid_cap, ctx->sm_count);
  if (s == POT_OK && (ctx->mask & 2)) s = alloc_work(ctx->wd, n, k, ctx->grid_cap, ctx->sm_count);
  if (s == POT_OK && cudaMallocHost((void**)&ctx->h_pinned, 64 * sizeof(double)) != cudaSuccess)
    s = POT_ERR_CUDA;
  for (auto& e : ctx->ev)
    if (s == POT_OK && cudaEventCreate(&e) != cudaSuccess) s = POT_ERR_CUDA;
  if (s == POT_OK) {
    int32_t reset[2] = {0, 0x7fffffff};
    if (cudaMemcpy(ctx->err, reset, sizeof(reset), cudaMemcpyHostToDevice) != cudaSuccess)
      s = POT_ERR_CUDA;
  }
  if (s != POT_OK) {
    pot_destroy(ctx);
    return s;
  }
  *out = ctx;
  return POT_OK;
}

int lgc_compute_cells(pot_ctx* ctx, void* stream, int64_t n, const float* pos, const float* psi,
                      const double* targets, const pot_domain* dom, float* volumes, double* grad,
                      pot_csr* hess, float* centroids, float* karea, pot_cell_stats* stats) {
  return compute_cells<float, pot_csr>(ctx, stream, n, pos, psi, targets, dom, volumes, grad, hess,
                                       centroids, karea, stats);
}

int lgc_compute_cells_f64(pot_ctx* ctx, void* stream, int64_t n, const double* pos,
                          const double* psi, const double* targets, const pot_domain* dom,
                          double* volumes, double* grad, pot_csr_f64* hess, double* centroids,
                          double* karea, pot_cell_stats* stats) {
  return compute_cells<double, pot_csr_f64>(ctx, stream, n, pos, psi, targets, dom, volumes, grad,
                                            hess, centroids, karea, stats);
}

int pot_newton_solve(pot_ctx* ctx, void* stream, int64_t n, const float* pos, const double* targets,
                     float* psi_inout, const pot_domain* dom, const pot_params* params,
                     pot_solve_stats* stats) {
  pot_solve_stats local;
  pot_solve_stats* S = stats ? stats : &local;
  memset(S, 0, sizeof(*S));
  S->error_site = -1;
  POT_CHECK(check_ctx(ctx, n, 1));
  if (!pos || !targets || !psi_inout || !finite_box(dom) || !check_params(params))
    return POT_ERR_INVALID_ARG;
  return newton_solve<float>(ctx, (cudaStream_t)stream, n, pos, targets, psi_inout, dom, params, S);
}

int pot_newton_solve_f64(pot_ctx* ctx, void* stream, int64_t n, const double* pos,
                         const double* targets, double* psi_inout, const pot_domain* dom,
                         const pot_params* params, pot_solve_stats* stats) {
  pot_solve_stats local;
  pot_solve_stats* S = stats ? stats : &local;
  memset(S, 0, sizeof(*S));
  S->error_site = -1;
  POT_CHECK(check_ctx(ctx, n, 2));
  if (!pos || !targets || !psi_inout || !finite_box(dom) || !check_params(params))
    return POT_ERR_INVALID_ARG;
  return newton_solve<double>(ctx, (cudaStream_t)stream, n, pos, targets, psi_inout, dom, params, S);
}

int pot_fluid_step(pot_ctx* ctx, void* stream, int64_t n, float* pos, float* vel, float* psi,
                   const double* targets, const pot_domain* dom, const pot_params* params,
                   pot_solve_stats* stats) {
  pot_solve_stats local;
  pot_solve_stats* S = stats ? stats : &local;
  memset(S, 0, sizeof(*S));
  S->error_site = -1;
  POT_CHECK(check_ctx(ctx, n, 1));
  if (!pos || !vel || !targets || !psi || !finite_box(dom) || !check_params(params))
    return POT_ERR_INVALID_ARG;
  return fluid_step<float>(ctx, (cudaStream_t)stream, n, pos, vel, psi, targets, dom, params, S);
}

int pot_fluid_step_f64(pot_ctx* ctx, void* stream, int64_t n, double* pos, double* vel,
                       double* psi, const double* targets, const pot_domain* dom,
                       const pot_params* params, pot_solve_stats* stats) {
  pot_solve_stats local;
  pot_solve_stats* S = stats ? stats : &local;
  memset(S, 0, sizeof(*S));
  S->error_site = -1;
  POT_CHECK(check_ctx(ctx, n, 2));
  if (!pos || !vel || !targets || !psi || !finite_box(dom) || !check_params(params))
    return POT_ERR_INVALID_ARG;
  return fluid_step<double>(ctx, (cudaStream_t)stream, n, pos, vel, psi, targets, dom, params, S);
}

}  // extern "C"
