// Jacobi-preconditioned conjugate gradients for M u = nu - V (Sec. 7: CG with
// a Jacobi preconditioner), M = -grad^2 K stored as its diagonal plus the
// off-diagonal CSR in sorted space.
//
// Two kernels per iteration, no host round trip:
//   k_spmv:   beta from the device partials; p_new = z + beta p_old fused into
//             the gather of the SpMV (p double-buffered); q = M p_new;
//             partial sums of p_new . q
//   k_update: alpha = rz / pq; x += alpha p; r -= alpha q; z = r / diag;
//             partial sums of r . z and r . r
// Dot products accumulate in FP64 (per-thread, then fixed-order block and
// grid reductions, so the result is deterministic).  Every block re-reduces
// the previous kernel's partials and takes the same decision (converged,
// breakdown), so no grid-wide barrier is needed.  The host checks the done
// flag once per chunk of iterations.
#include "pot_internal.cuh"

namespace pot {
namespace {

constexpr int kPcgThreads = 256;
constexpr int kTpr = 8;  // threads per CSR row

enum { kRZ0 = 0, kRZ1 = 1, kPQ = 2, kRR = 3, kRR0 = 4, kSlots = 5 };
enum { kDone = 0, kItA = 1, kItB = 2, kBreak = 3, kIters = 4 };

// Sum of nb partials, same order in every block; result broadcast.
__device__ __forceinline__ double sum_partials(const double* __restrict__ part, int nb) {
  __shared__ double sh;
  if (threadIdx.x < 32) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += 32) s += part[b];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(kFull, s, off);
    if (threadIdx.x == 0) sh = s;
  }
  __syncthreads();
  double v = sh;
  __syncthreads();
  return v;
}

__device__ __forceinline__ void block_partial(double v, double* out) {
  __shared__ double sh[kPcgThreads / 32];
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(kFull, v, off);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kPcgThreads / 32; w++) s += sh[w];
    out[blockIdx.x] = s;
  }
  __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(kPcgThreads)
    k_pcg_init(int64_t n, const double* __restrict__ b, const T* __restrict__ diag, T* x, T* r,
               T* z, T* p0, double* part, int nb, int32_t* ctl) {
  double rz = 0.0, rr = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    T ri = (T)b[i];
    T zi = diag[i] > T(0) ? ri / diag[i] : T(0);
    x[i] = T(0);
    r[i] = ri;
    z[i] = zi;
    p0[i] = T(0);
    rz += (double)ri * (double)zi;
    rr += (double)ri * (double)ri;
  }
  block_partial(rz, part + kRZ0 * nb);
  block_partial(rr, part + kRR * nb);
  block_partial(rr, part + kRR0 * nb);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctl[kDone] = 0;
    ctl[kItA] = 0;
    ctl[kItB] = 0;
    ctl[kBreak] = 0;
    ctl[kIters] = 0;
  }
}

template <typename T>
__global__ void __launch_bounds__(kPcgThreads)
    k_spmv(int64_t n, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ cols,
           const T* __restrict__ vals, const T* __restrict__ diag, const T* __restrict__ z,
           T* pa, T* pb, T* q, double* part, int nb, int32_t* ctl, double rtol2, int max_iter) {
  if (ctl[kDone]) return;
  const int it = ctl[kItA];
  const double rr = sum_partials(part + kRR * nb, nb);
  const double rr0 = sum_partials(part + kRR0 * nb, nb);
  if (rr <= rtol2 * rr0 || it >= max_iter) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      ctl[kDone] = 1;
      ctl[kIters] = it;
    }
    return;
  }
  const double rz = sum_partials(part + ((it & 1) ? kRZ1 : kRZ0) * nb, nb);
  const double rzp = sum_partials(part + ((it & 1) ? kRZ0 : kRZ1) * nb, nb);
  const T beta = it == 0 ? T(0) : (T)(rz / rzp);
  const T* __restrict__ pold = (it & 1) ? pb : pa;
  T* pnew = (it & 1) ? pa : pb;
  const int sub = threadIdx.x & (kTpr - 1);
  double pq = 0.0;
  const int64_t groups = (int64_t)gridDim.x * (blockDim.x / kTpr);
  // rows rounded up to a multiple of the group count: every lane of a warp
  // runs the same number of iterations (the shuffles use the full mask)
  const int64_t n_round = ((n + groups - 1) / groups) * groups;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kTpr; i < n_round;
       i += groups) {
    T acc = T(0);
    T pi = T(0);
    if (i < n) {
      const int a = row_ptr[i], e = row_ptr[i + 1];
      for (int k = a + sub; k < e; k += kTpr) {
        const int j = cols[k];
        acc += vals[k] * (z[j] + beta * pold[j]);
      }
      pi = z[i] + beta * pold[i];
    }
#pragma unroll
    for (int off = kTpr / 2; off > 0; off >>= 1) acc += __shfl_xor_sync(kFull, acc, off);
    if (i < n && sub == 0) {
      const T qi = diag[i] * pi + acc;
      pnew[i] = pi;
      q[i] = qi;
      pq += (double)pi * (double)qi;
    }
  }
  block_partial(pq, part + kPQ * nb);
  if (blockIdx.x == 0 && threadIdx.x == 0) ctl[kItB] = it;
}

template <typename T>
__global__ void __launch_bounds__(kPcgThreads)
    k_update(int64_t n, const T* __restrict__ diag, T* x, T* r, T* z, const T* __restrict__ pa,
             const T* __restrict__ pb, const T* __restrict__ q, double* part, int nb,
             int32_t* ctl) {
  if (ctl[kDone]) return;
  const int it = ctl[kItB];
  const double rz = sum_partials(part + ((it & 1) ? kRZ1 : kRZ0) * nb, nb);
  const double pq = sum_partials(part + kPQ * nb, nb);
  if (!(pq > 0.0)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      ctl[kBreak] = 1;
      ctl[kDone] = 1;
      ctl[kIters] = it;
    }
    return;
  }
  const T alpha = (T)(rz / pq);
  const T* __restrict__ p = (it & 1) ? pa : pb;
  double rzn = 0.0, rr = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    x[i] += alpha * p[i];
    const T ri = r[i] - alpha * q[i];
    const T zi = diag[i] > T(0) ? ri / diag[i] : T(0);
    r[i] = ri;
    z[i] = zi;
    rzn += (double)ri * (double)zi;
    rr += (double)ri * (double)ri;
  }
  block_partial(rzn, part + ((it & 1) ? kRZ0 : kRZ1) * nb);
  block_partial(rr, part + kRR * nb);
  if (blockIdx.x == 0 && threadIdx.x == 0) ctl[kItA] = it + 1;
}

}  // namespace

template <typename T>
int pcg_solve(pot_ctx* ctx, cudaStream_t st, int64_t n, int64_t nnz_off, double rtol, int max_iter,
              int chunk, int* iters, double* rel_res) {
  (void)nnz_off;
  Work<T>& w = ctx->work<T>();
  const int nb = ctx->sm_count * 2;
  double* part = ctx->pcg_red;
  if (chunk < 1) chunk = 1;
  note_launch();
  k_pcg_init<T><<<nb, kPcgThreads, 0, st>>>(n, ctx->grad, w.diag, w.u, w.r, w.z, w.p0, part, nb,
                                            ctx->pcg_ctl);
  const double rtol2 = rtol * rtol;
  int launched = 0;
  int32_t* hctl = (int32_t*)(ctx->h_pinned + 16);
  for (;;) {
    for (int k = 0; k < chunk; k++) {
      note_launch();
      k_spmv<T><<<nb, kPcgThreads, 0, st>>>(n, ctx->row_ptr, ctx->csr_cols, w.csr_vals, w.diag,
                                            w.z, w.p0, w.p1, w.q, part, nb, ctx->pcg_ctl, rtol2,
                                            max_iter);
      note_launch();
      k_update<T><<<nb, kPcgThreads, 0, st>>>(n, w.diag, w.u, w.r, w.z, w.p0, w.p1, w.q, part, nb,
                                              ctx->pcg_ctl);
    }
    launched += chunk;
    POT_CUDA(cudaGetLastError());
    POT_CUDA(cudaMemcpyAsync(hctl, ctx->pcg_ctl, 5 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    POT_CUDA(cudaStreamSynchronize(st));
    if (hctl[kDone] || launched > max_iter + chunk) break;
  }
  *iters = hctl[kIters];
  if (rel_res) *rel_res = -1.0;
  if (hctl[kBreak]) return POT_ERR_PCG_BREAKDOWN;
  return POT_OK;
}

template int pcg_solve<float>(pot_ctx*, cudaStream_t, int64_t, int64_t, double, int, int, int*,
                              double*);
template int pcg_solve<double>(pot_ctx*, cudaStream_t, int64_t, int64_t, double, int, int, int*,
                               double*);

}  // namespace pot
