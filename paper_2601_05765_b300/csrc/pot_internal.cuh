// Internal declarations of libpot.so (not part of the C ABI).
//
// Data layout in HBM.  Inside the library every per-site array is in
// grid-sorted order ("sorted space"); the C ABI maps to and from the
// caller's order.
//   sxp[s]      V4<T> (x, y, z, psi) of the s-th site in grid order
//   perm[s]     caller index of sorted site s; iperm is its inverse
//   cell_start  first sorted site of each grid cell (exclusive scan of counts)
//   cand        per cell up to k_max sorted indices of the bisectors that cut
//               its ball (row s at s*k_max, ascending); the cell kernel
//               rewrites each row in place into its Hessian column list
//   meta[s]     cutting-plane count | wall mask << 8 | flags
//   stage_vals  per cell the off-diagonal Hessian values of its row (row s at s*k_max)
//   vol, karea, diag, cen  per-cell outputs of the cell kernel
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "../../include/pot.h"

namespace pot {

constexpr int kWarp = 32;
constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxK = 1024;        // candidate bisectors per cell (k_max <= 1024)
constexpr int kPlaneCap = 252;     // planes of a cell kept without bisecting its security radius
constexpr int kSmallPlanes = 32;   // planes of a cell in the cell kernel (32-bit crossing sets)
constexpr int kVerletCap = 160;    // sites of a neighbour list of the candidate pass
constexpr float kVerletReach = 1.05f;  // a list's reach over the reach it was built for
constexpr int kBigPlanes = kMaxK + 6;  // planes of a cell in the big-cell kernel
constexpr int kBigWarpsPerSm = 8;  // warps of the big-cell kernel per SM
constexpr int kMaxLines = 24;      // edges of one facet polygon
constexpr int kCellWarps = 4;      // warps per block of the cell kernel
constexpr int kCellsPerWarp = 32;  // cells per warp task
// facet arc counts carry, from bit 16 up, the count of ill-conditioned
// vertices (two lines crossing inside a disk with sine below kIllSine)
constexpr int kIllFlag = 1 << 16;
constexpr int kArcMask = kIllFlag - 1;
constexpr float kIllSine = 1.5e-2f;

// meta word written by the candidate kernel
constexpr int kMetaPlanes = 0x7ff;  // planes (walls + candidates) <= kMaxK + 6
constexpr int kMetaWallShift = 11;  // 6 wall bits
constexpr int kMetaEmpty = 1 << 17;
constexpr int kMetaRetry = 1 << 18;  // candidate list overflowed: redo at a smaller radius
constexpr int kMaxPasses = 48;       // security-radius passes of one cell evaluation
// need[] bits of a cell during an evaluation
constexpr uint8_t kNeedPending = 1;  // to be (re)built in the next pass
constexpr uint8_t kNeedBig = 2;      // needs more planes than the cell kernel's window

// device status words: [0] error code (max over sites), [1] smallest site with that error
enum { kErrCode = 0, kErrSite = 1 };

template <typename T>
struct alignas(4 * sizeof(T)) V4 {
  T x, y, z, w;
};

template <typename T>
struct Real;
template <>
struct Real<float> {
  // relative area (of psi_i) below which a bisector facet is not emitted
  static constexpr float kEmitArea = 4e-7f;
  // a plane exactly through the site moves outward by this fraction of r
  static constexpr float kZeroShift = 9.313225746154785e-10f;  // 2^-30
};
template <>
struct Real<double> {
  static constexpr double kEmitArea = 1e-13;
  static constexpr double kZeroShift = 9.094947017729282e-13;  // 2^-40
};

// Explicitly rounded arithmetic: the candidate kernel and the cell kernel
// must take the same decisions on the same inputs, so the steps that decide
// (squared distance, plane offset) are pinned against FMA contraction.
__device__ __forceinline__ float r_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double r_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float r_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double r_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float r_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double r_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float r_div(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ double r_div(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ float r_sqrt(float a) { return __fsqrt_rn(a); }
__device__ __forceinline__ double r_sqrt(double a) { return __dsqrt_rn(a); }

// Sums of FP32 products carried as an unevaluated pair hi + lo of floats
// (double-float): each product a b is split exactly into p + e (one FMA)
// and each addition is Knuth's error-free two-sum, so a thread's partial
// over a few terms keeps about 44 bits while running on FP32 units alone
// (the FP64 units of this GPU issue at a small fraction of the FP32 rate).
// The partial becomes a double once, for the FP64 block and grid sums.
struct DF {
  float hi = 0.f, lo = 0.f;
};
__device__ __forceinline__ void df_add_prod(DF& s, float a, float b) {
  const float p = a * b;
  const float e = fmaf(a, b, -p);  // p + e = a b exactly
  const float t = s.hi + p;
  const float bp = t - s.hi;
  const float err = (s.hi - (t - bp)) + (p - bp);  // s.hi + p = t + err exactly
  s.hi = t;
  s.lo += err + e;
}
__device__ __forceinline__ void df_add(DF& s, const DF& o) {
  const float t = s.hi + o.hi;
  const float bp = t - s.hi;
  const float err = (s.hi - (t - bp)) + (o.hi - bp);  // s.hi + o.hi = t + err exactly
  s.hi = t;
  s.lo += err + o.lo;
}
__device__ __forceinline__ double df_value(const DF& s) { return (double)s.hi + (double)s.lo; }

// Max of the non-negative values m of a block's threads into *out, one
// atomic per block (non-negative IEEE values order like their bit patterns
// read as signed integers).  Every thread of the block must call it.
template <typename T>
__device__ __forceinline__ void block_max_to(T m, T* out) {
  __shared__ T sh[32];
  for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_down_sync(kFull, m, off));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)((blockDim.x + 31) >> 5); w++) m = fmax(m, sh[w]);
    if (m > T(0)) {
      if (sizeof(T) == 4)
        atomicMax((int*)out, __float_as_int((float)m));
      else
        atomicMax((unsigned long long*)out, (unsigned long long)__double_as_longlong((double)m));
    }
  }
}

// Bisector (radical) plane of sites i and j seen from i (Eq. 1):
// points y - p_i with y.n <= h, n = (p_j - p_i)/d,
// h = (d^2 + psi_i - psi_j) / (2 d).  Returns d2 (0 for coincident sites).
template <typename T>
__device__ __forceinline__ T bisector(const V4<T>& pi, const V4<T>& pj, T& dx, T& dy, T& dz, T& d,
                                      T& h) {
  dx = r_sub(pj.x, pi.x);
  dy = r_sub(pj.y, pi.y);
  dz = r_sub(pj.z, pi.z);
  T d2 = r_add(r_add(r_mul(dx, dx), r_mul(dy, dy)), r_mul(dz, dz));
  d = r_sqrt(d2);
  h = r_div(r_add(d2, r_sub(pi.w, pj.w)), r_add(d, d));
  return d2;
}

// A plane exactly through the site is moved outward by r * kZeroShift: the
// limit of the site moving into its own cell (stays right when several
// planes meet at the site, e.g. a site on a box corner).
template <typename T>
__device__ __forceinline__ T fix_zero(T h, T r) {
  return h == T(0) ? r * Real<T>::kZeroShift : h;
}

// Signed distance from the site to wall w (0..5 = -x,+x,-y,+y,-z,+z), positive inside.
template <typename T>
__device__ __forceinline__ T wall_offset(const V4<T>& p, int w, const T* lo, const T* hi) {
  int ax = w >> 1;
  T pk = ax == 0 ? p.x : (ax == 1 ? p.y : p.z);
  return (w & 1) ? r_sub(hi[ax], pk) : r_sub(pk, lo[ax]);
}

template <typename T>
struct Box {
  T lo[3];
  T hi[3];
};

// Grid over the domain box: cell (cx,cy,cz) has key (cz*dim1 + cy)*dim0 + cx.
template <typename T>
struct GridParams {
  T lo[3];
  T cs;
  T inv_cs;
  int dim[3];
};

// Per-precision workspace.
template <typename T>
struct Work {
  V4<T>* sxp = nullptr;     // sorted (x,y,z,psi)
  T* psi_base = nullptr;    // accepted psi (sorted)
  T* vol = nullptr;
  T* karea = nullptr;
  T* diag = nullptr;
  T* cen = nullptr;         // 3 per site
  T* stage_vals = nullptr;  // n_max * k_max
  T* csr_vals = nullptr;    // n_max * k_max (off-diagonal, compacted)
  T* u = nullptr;           // Newton direction
  T* x = nullptr;           // PCG vectors
  T* r = nullptr;
  T* z = nullptr;
  T* p0 = nullptr;
  T* p1 = nullptr;
  T* zp = nullptr;          // PCG: (z, p) interleaved, 2 per site
  T* q = nullptr;
  T* vel_s = nullptr;       // sorted velocities, 3 per site
  T* psi_max = nullptr;     // device scalar: max psi of the current evaluation
  T* nu_max = nullptr;      // device scalar: max target volume (grid build)
  T* srad = nullptr;        // per cell: security radius of the current pass
  T* srad_lo = nullptr;     // per cell: largest radius found too small in this evaluation
  T* soff = nullptr;        // per cell: security ball centre - site (3 per cell)
  T* rcell_acc = nullptr;   // per cell: rcell at the last accepted Newton iterate
  T* rcell = nullptr;       // per cell: farthest point of the cell from its security centre
  T* hint = nullptr;        // caller order: centroid - site and extent from it (4 per site)
  V4<T>* big_pl = nullptr;  // big-cell kernel: planes of each warp's cell (kBigPlanes per warp)
  T* big_d = nullptr;
  int* big_j = nullptr;
  int big_warps = 0;        // warps of the big-cell kernel (0: no big cells possible)
  T* gmax = nullptr;        // per grid cell: largest psi of its sites
  T* cmax = nullptr;        // per coarse cell (f x f x f grid cells): largest psi of its sites
  T* cnb = nullptr;         // per coarse cell: largest psi over its 3 x 3 x 3 coarse neighbourhood
  int64_t ccap = 0;         // coarse cells cmax and cnb hold
  double grid_pmax = 0.0;   // largest psi at the grid build
  GridParams<T> grid{};
  bool grid_valid = false;
  bool have_rcell = false;  // rcell belongs to the current grid order
  bool have_acc = false;    // rcell_acc belongs to the current grid order
  int64_t hint_n = -1;      // sites the hint was written for (-1: none)
  T* wallw = nullptr;       // walls' P1 Laplacian weight per cell (sorted)
  T* wallv = nullptr;       // per cell (sorted): sum over wall facets of |B| n / 2 and of |B| n / (2h)
  T* psi_hist = nullptr;    // weights at the start of the last fluid step (caller order)
  T* psi_fb = nullptr;      // plain start kept while an extrapolated one is tried (sorted)
  int64_t hist_n = -1;      // sites psi_hist was written for (-1: none)
  bool use_hint = false;    // this grid order's first evaluation starts from the hint
  int32_t* vlist = nullptr; // candidate pass: per-site neighbour lists (kVerletCap per site)
  int32_t* vcount = nullptr;
  T* vreach = nullptr;      // reach each list was built with (0: none; cleared by the grid build)
  bool verlet = false;      // evaluations of the current solve keep and reuse the lists
};

}  // namespace pot

struct pot_mlp;

struct pot_ctx {
  pot_mlp* mlp = nullptr;  // learned warm-start model (pot_set_warm_start), not owned
  const float* visc_factors = nullptr;  // per-site viscosity factors (caller's, caller order)
  int64_t visc_factors_n = -1;          // sites they were given for
  int device = 0;
  int64_t n_max = 0;
  int32_t k_max = 0;
  int32_t mask = 0;
  int64_t grid_cap = 0;
  int sm_count = 148;
  uint32_t* keys = nullptr;
  int32_t* perm = nullptr;
  int32_t* iperm = nullptr;
  int32_t* cell_count = nullptr;  // grid_cap + 1
  int32_t* cell_start = nullptr;  // grid_cap + 1
  int32_t* cand = nullptr;        // n_max * k_max
  int32_t* meta = nullptr;
  int32_t* row_cnt = nullptr;     // n_max + 1
  int32_t* row_ptr = nullptr;     // n_max + 1
  int32_t* ucnt = nullptr;        // n_max + 1 (caller-order row counts)
  int32_t* csr_cols = nullptr;    // n_max * k_max
  int32_t* scan_tmp = nullptr;
  int64_t scan_tmp_len = 0;
  double* snu = nullptr;          // sorted targets
  double* grad = nullptr;         // sorted gradient nu - V
  double* red = nullptr;          // reduction partials
  double* red_out = nullptr;      // reduction results (device)
  double* pcg_red = nullptr;      // PCG reduction partials
  int32_t* pcg_ctl = nullptr;     // PCG control words
  // PCG iteration loop as a CUDA graph with a device-side while node, one
  // per precision ([0] float, [1] double), built for pcg_graph_n rows
  cudaGraph_t pcg_graph[2] = {nullptr, nullptr};
  cudaGraphExec_t pcg_exec[2] = {nullptr, nullptr};
  int64_t pcg_graph_n[2] = {-1, -1};
  int32_t* err = nullptr;         // device status words
  uint8_t* need = nullptr;        // per cell: still to be (re)built in this evaluation
  int32_t* need_count = nullptr;  // device counters: cells to rebuild, big cells, FP64 cells listed, next chunk of the cell kernel
  int32_t* big_list = nullptr;    // cells with more planes than the shared window holds
  int32_t* fix_list = nullptr;    // FP32 cells re-evaluated in FP64 (ill-conditioned)
  int last_passes = 0;            // security-radius passes of the last cell evaluation
  bool tail_ready = false;        // residuals and status of the last evaluation are on the host
  int64_t kc_launches = 0;        // cell-kernel timer: launches, cells processed, device ms
  int64_t kc_cells = 0;
  double kc_ms = 0.0;
  double* h_pinned = nullptr;     // pinned host scalars
  cudaEvent_t ev[8] = {};
  pot::Work<float> wf;
  pot::Work<double> wd;
  template <typename T>
  pot::Work<T>& work();
};

template <>
inline pot::Work<float>& pot_ctx::work<float>() { return wf; }
template <>
inline pot::Work<double>& pot_ctx::work<double>() { return wd; }

namespace pot {

#define POT_CUDA(call)                          \
  do {                                          \
    cudaError_t e_ = (call);                    \
    if (e_ != cudaSuccess) return POT_ERR_CUDA; \
  } while (0)

#define POT_CHECK(call)          \
  do {                           \
    int s_ = (call);             \
    if (s_ != POT_OK) return s_; \
  } while (0)

// kernel launches issued by this library in this process (pot_kernel_launches)
extern std::atomic<long long> g_launches;
inline void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
inline void note_launches(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

inline int blocks_for(int64_t n, int threads) { return (int)((n + threads - 1) / threads); }

constexpr int kRedBlocks = 296;  // partial count of the deterministic reductions

// exclusive scan of n int32 values: out[k] = sum_{i<k} in[i]; out[n] = total.
// in may alias out.  Enqueued on the stream; no host sync.
int scan_exclusive(pot_ctx* ctx, cudaStream_t st, const int32_t* in, int32_t* out, int64_t n);

// Grid build, sort and gather into sorted space (grid.cu).  One host sync.
template <typename T>
int grid_build(pot_ctx* ctx, cudaStream_t st, int64_t n, const T* pos, const T* psi,
               const double* targets, const pot_domain* dom);

// Cell evaluation in sorted space (cells.cu): candidates + geometry.  With
// tail_resid, every pass also enqueues the residual summary and a copy of
// the status word before its wait, so that after the last pass both are on
// the host (ctx->tail_ready) without a further wait.
template <typename T>
int cells_eval(pot_ctx* ctx, cudaStream_t st, int64_t n, const pot_domain* dom, bool want_grad,
               bool tail_resid = false);
// keep the last evaluation's cell centres and extents (caller order) as the
// security-ball hint of the next Newton solve on the same sites
template <typename T>
int store_hint(pot_ctx* ctx, cudaStream_t st, int64_t n);
int cell_diagnostics(pot_ctx* ctx, cudaStream_t st, int64_t n, float* off, float* rad, float* ext,
                     int32_t* planes);

// FP64 reductions over sorted cells:
// out = {max |V-nu|/nu, sum (nu-V)^2, min V, #empty, #planes, max planes}.  Host
// sync; with out NULL only enqueued (the values are at ctx->h_pinned[0..5]
// after the caller's next wait on the stream).
template <typename T>
int residuals(pot_ctx* ctx, cudaStream_t st, int64_t n, double out[6]);

// raise the weights of empty cells so that each site lies inside its own
// cell (cells.cu); *repaired = number of cells changed.  Needs a preceding
// cells_eval (volumes, grid maxima).
template <typename T>
int repair_empty(pot_ctx* ctx, cudaStream_t st, int64_t n, int* repaired);

// read and clear the device status word; returns a POT status
int read_status(pot_ctx* ctx, cudaStream_t st, int64_t* site);
// the same from the copy already on the host (ctx->h_pinned + 8, written
// by a wait that followed the copy); clears the device word if set
int status_on_host(pot_ctx* ctx, int64_t* site);

// internal CSR (off-diagonal, sorted space) from the staged rows; nnz on host
// (nnz_off NULL: not waited for; csr_nnz reads it after the next wait)
template <typename T>
int csr_compact(pot_ctx* ctx, cudaStream_t st, int64_t n, int64_t* nnz_off);
int64_t csr_nnz(const pot_ctx* ctx);

// caller-order CSR with the diagonal
template <typename T>
int csr_user(pot_ctx* ctx, cudaStream_t st, int64_t n, int32_t* row_ptr, int32_t* cols, T* vals,
             int64_t cap, int64_t* nnz);

// scatter sorted per-site outputs back to caller order (NULL outputs skipped)
template <typename T>
int unsort_outputs(pot_ctx* ctx, cudaStream_t st, int64_t n, T* vol, double* grad, T* cen,
                   T* karea, T* psi);

// psi_trial = psi_base + alpha * u written into sxp.w; updates psi_max
template <typename T>
int psi_update(pot_ctx* ctx, cudaStream_t st, int64_t n, double alpha);

// learned warm start (mlp.cu): features of the sorted sites, the MLP, and
// psi_pred = psi_prev + h^2 out into sxp.w / psi_base; *psi_prev points to the
// kept previous weights (sorted)
int mlp_warm_start(pot_ctx* ctx, pot_mlp* mm, cudaStream_t st, int64_t n, const float* vel,
                   const float* psi, float dt, float** psi_prev);

// PCG (pcg.cu): solve M u = grad (sorted space) into work.u
constexpr int kPcgMaxBlocksPerSm = 8;
constexpr int kPcgCtlWords = 16;    // ctx->pcg_ctl
int pcg_blocks(int sm_count);       // largest grid of the PCG kernels
size_t pcg_red_len(int sm_count);   // doubles of ctx->pcg_red
template <typename T>
int pcg_solve(pot_ctx* ctx, cudaStream_t st, int64_t n, int64_t nnz_off, double rtol, int max_iter,
              int chunk, bool host_loop, int* iters, double* rel_res);

}  // namespace pot
