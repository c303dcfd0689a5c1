// Jacobi-preconditioned conjugate gradients for M u = nu - V (Sec. 7: CG with
// a Jacobi preconditioner), M = -grad^2 K stored as its diagonal plus the
// off-diagonal CSR in sorted space.
//
// Systems of up to kPcgCoopMaxRows rows run as one persistent cooperative
// kernel (k_pcg_coop, below) when the device supports cooperative launches.
// Larger ones take two kernels per iteration, no host round trip:
//   k_spmv:   beta = rz / rz_prev; p_new = z + beta p_old fused into the
//             gather of the SpMV; q = M p_new; p_new . q
//   k_update: alpha = rz / pq; x += alpha p_new; r -= alpha q;
//             z = r D^-1 (D^-1 formed once per solve); r . z and r . r;
//             convergence test
// z and p are stored interleaved, (z_j, p_j) per row: the SpMV gathers both
// with one 8-byte (16-byte in FP64) load per entry, and k_update writes the
// pair (z_new, p_new) of its row.
// Dot products accumulate per thread, then per block (fixed tree), then
// over blocks by the last block to finish (an arrival counter after a
// memory fence), which adds the block partials in index order and publishes
// the scalars, the next step length and the decisions (converged,
// breakdown) for the next kernel: exactly in FP64 for FP64 vectors, in
// double-float on the FP32 units for FP32 vectors (this GPU's FP64 units
// issue at a small fraction of the FP32 rate).  The result is deterministic
// and no block re-reads all partials.
//
// The iterations run as a CUDA graph: a while node whose body is the two
// kernels, built once per context, precision and row count (the tolerance
// and iteration cap live in device memory, set by k_pcg_init).  Thread 0 of
// k_update's block 0 alone ends the loop (cudaGraphSetConditional): when an
// earlier kernel has set the done flag, or when its own trip counter passes
// the cap + 1, so the loop ends even if the done flag were never set.  The
// host waits once per solve.  Without the graph (its construction failed,
// or the caller asked for host-driven launches, pot_params.pcg_host_loop)
// the same kernels run in chunks from the host, which checks the done flag
// once per chunk.
#include "pot_internal.cuh"

namespace pot {
namespace {

constexpr int kPcgThreads = 256;
constexpr int kTpr = 2;  // threads per CSR row (about 10 entries per row)

// Partial sums of dot products: exact FP64 sums of the products of FP64
// vectors; double-float sums (FP32 units only) of FP32 vectors, kept in
// double-float through the block and grid sums and converted to FP64 once,
// for the scalars.  A partial travels between blocks in one 8-byte word (a
// double, or the two floats of a double-float).
template <typename T>
struct Dot {
  double s = 0.0;
  __device__ __forceinline__ void add(T a, T b) { s += a * b; }
  __device__ __forceinline__ void merge(const Dot& o) { s += o.s; }
  __device__ __forceinline__ Dot down(int off) const {
    Dot d;
    d.s = __shfl_down_sync(kFull, s, off);
    return d;
  }
  __device__ __forceinline__ double pack() const { return s; }
  __device__ __forceinline__ static Dot unpack(double w) {
    Dot d;
    d.s = w;
    return d;
  }
  __device__ __forceinline__ double value() const { return s; }
};
template <>
struct Dot<float> {
  DF s;
  __device__ __forceinline__ void add(float a, float b) { df_add_prod(s, a, b); }
  __device__ __forceinline__ void merge(const Dot& o) { df_add(s, o.s); }
  __device__ __forceinline__ Dot down(int off) const {
    Dot d;
    d.s.hi = __shfl_down_sync(kFull, s.hi, off);
    d.s.lo = __shfl_down_sync(kFull, s.lo, off);
    return d;
  }
  __device__ __forceinline__ double pack() const {
    return __hiloint2double(__float_as_int(s.hi), __float_as_int(s.lo));
  }
  __device__ __forceinline__ static Dot unpack(double w) {
    Dot d;
    d.s.hi = __int_as_float(__double2hiint(w));
    d.s.lo = __int_as_float(__double2loint(w));
    return d;
  }
  __device__ __forceinline__ double value() const { return df_value(s); }
};

// z and p of one row, stored together
template <typename T>
struct alignas(2 * sizeof(T)) ZP {
  T z, p;
};

// partial-sum arrays (nb packed partials each) and scalars at the end of
// pcg_red; the step lengths alpha and beta, formed once per iteration by
// the last block of the kernel before, sit in the scalars' last two
// doubles as T values
enum { kPartA = 0, kPartB = 1, kPartC = 2, kParts = 3 };
enum { kRZ = 0, kRZP = 1, kPQ = 2, kRR = 3, kRR0 = 4, kRtol2 = 5, kSteps = 6, kScalars = 8 };
template <typename T>
__device__ __forceinline__ T* steps(double* scal) {  // [0] alpha, [1] beta
  return reinterpret_cast<T*>(scal + kSteps);
}
// control words (ctx->pcg_ctl holds 8)
enum { kDone = 0, kIt = 1, kBreak = 2, kIters = 3, kArrive = 4, kTrips = 5, kMaxIt = 6,
       kBar = 8, kTimeout = 9 };
static_assert(kTimeout < kPcgCtlWords, "control words");
// tries of a block's wait at the grid barrier of the persistent solve (about
// 100 ns each) before it gives up and reports a timeout
constexpr int kBarrierSpins = 1 << 24;
// largest system solved by the persistent kernel
constexpr int64_t kPcgCoopMaxRows = 1 << 17;

// Block sum of v (fixed tree) into thread 0's return value.
template <typename T>
__device__ __forceinline__ Dot<T> block_sum(Dot<T> v) {
  __shared__ double sh[kPcgThreads / 32];
  for (int off = 16; off > 0; off >>= 1) v.merge(v.down(off));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v.pack();
  __syncthreads();
  Dot<T> s;
  if (threadIdx.x == 0)
    for (int w = 0; w < kPcgThreads / 32; w++) s.merge(Dot<T>::unpack(sh[w]));
  __syncthreads();
  return s;
}

// Publish up to three block partials; returns true in every thread of the
// block that arrived last (which then sees every block's partials).
template <typename T>
__device__ __forceinline__ bool arrive(double* part, int nb, int count, const Dot<T>& a,
                                       const Dot<T>& b, const Dot<T>& c, int32_t* ctl) {
  __shared__ bool last;
  const Dot<T> sa = block_sum(a);
  const Dot<T> sb = count > 1 ? block_sum(b) : Dot<T>();
  const Dot<T> sc = count > 2 ? block_sum(c) : Dot<T>();
  if (threadIdx.x == 0) {
    part[kPartA * nb + blockIdx.x] = sa.pack();
    if (count > 1) part[kPartB * nb + blockIdx.x] = sb.pack();
    if (count > 2) part[kPartC * nb + blockIdx.x] = sc.pack();
    __threadfence();
    last = atomicAdd(&ctl[kArrive], 1) == nb - 1;
  }
  __syncthreads();
  if (last) __threadfence();
  return last;
}

// Sum of nb partials in index order (strided per thread, fixed tree), in
// thread 0; called by the last block only.
template <typename T>
__device__ __forceinline__ Dot<T> sum_parts(const double* part, int nb) {
  Dot<T> s;
  for (int b = threadIdx.x; b < nb; b += kPcgThreads) s.merge(Dot<T>::unpack(__ldcg(part + b)));
  return block_sum(s);
}

// Grid-wide barrier of the persistent solve (a cooperative launch, every
// block resident): thread 0 of each block publishes the block's writes and
// adds one arrival to a counter that only grows; the block goes on once the
// counter reaches `target` (gen x blocks).  The wait is bounded: after
// kBarrierSpins tries, or when another block has given up, the block sets
// the timeout word and returns false, and the solve stops with an error.
__device__ __forceinline__ bool grid_barrier(int32_t* counter, int32_t* timeout, int target) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(counter, 1);
    int spins = 0;
    bool good = true;
    while (*(volatile int32_t*)counter < target) {
      if (*(volatile int32_t*)timeout != 0 || ++spins > kBarrierSpins) {
        atomicExch(timeout, 1);
        good = false;
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
    ok = good ? 1 : 0;
  }
  __syncthreads();
  return ok != 0;
}

template <typename T>
__global__ void __launch_bounds__(kPcgThreads)
    k_pcg_init(int64_t n, const double* __restrict__ b, const T* __restrict__ diag,
               T* __restrict__ x, T* __restrict__ r, T* __restrict__ dinv, ZP<T>* __restrict__ zp,
               double* part, double* scal, int nb, int32_t* ctl, double rtol2, int max_iter) {
  Dot<T> rz, rr;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const T d = diag[i];
    const T di = d > T(0) ? T(1) / d : T(0);
    const T ri = (T)b[i];
    const T zi = ri * di;
    x[i] = T(0);
    r[i] = ri;
    dinv[i] = di;
    zp[i] = ZP<T>{zi, T(0)};
    rz.add(ri, zi);
    rr.add(ri, ri);
  }
  if (arrive(part, nb, 2, rz, rr, Dot<T>(), ctl)) {
    const Dot<T> rzs = sum_parts<T>(part + kPartA * nb, nb);
    const Dot<T> rrs = sum_parts<T>(part + kPartB * nb, nb);
    if (threadIdx.x == 0) {
      const double trz = rzs.value(), trr = rrs.value();
      steps<T>(scal)[1] = T(0);  // beta of the first iteration
      scal[kRZ] = trz;
      scal[kRZP] = 1.0;
      scal[kRR] = trr;
      scal[kRR0] = trr;
      scal[kRtol2] = rtol2;
      ctl[kIt] = 0;
      ctl[kBreak] = 0;
      ctl[kIters] = 0;
      ctl[kTrips] = 0;
      ctl[kMaxIt] = max_iter;
      ctl[kDone] = (trr <= 0.0 || max_iter <= 0) ? 1 : 0;
      ctl[kArrive] = 0;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kPcgThreads)
    k_spmv(int64_t n, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ cols,
           const T* __restrict__ vals, const T* __restrict__ diag, const ZP<T>* __restrict__ zp,
           T* __restrict__ pnew, T* __restrict__ q, double* part, double* scal, int nb,
           int32_t* ctl) {
  if (ctl[kDone]) return;
  const int it = ctl[kIt];
  const T beta = steps<T>(scal)[1];
  const int sub = threadIdx.x & (kTpr - 1);
  Dot<T> pq;
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
      // unrolled so that the loads of several entries are in flight at once
#pragma unroll 2
      for (int k = a + sub; k < e; k += kTpr) {
        const ZP<T> v = zp[cols[k]];
        acc += vals[k] * (v.z + beta * v.p);
      }
      const ZP<T> v = zp[i];
      pi = v.z + beta * v.p;
    }
#pragma unroll
    for (int off = kTpr / 2; off > 0; off >>= 1) acc += __shfl_xor_sync(kFull, acc, off);
    if (i < n && sub == 0) {
      const T qi = diag[i] * pi + acc;
      pnew[i] = pi;
      q[i] = qi;
      pq.add(pi, qi);
    }
  }
  if (arrive(part, nb, 1, pq, Dot<T>(), Dot<T>(), ctl)) {
    const Dot<T> pqs = sum_parts<T>(part + kPartA * nb, nb);
    if (threadIdx.x == 0) {
      const double tpq = pqs.value();
      scal[kPQ] = tpq;
      steps<T>(scal)[0] = (T)(scal[kRZ] / tpq);  // alpha
      if (!(tpq > 0.0)) {  // M not positive definite along p: breakdown
        ctl[kBreak] = 1;
        ctl[kIters] = it;
        ctl[kDone] = 1;
      }
      ctl[kArrive] = 0;
    }
  }
}

// rows of k_update in flight per thread (their loads issued together; two
// in FP64 for registers), and its blocks per SM (one wave)
template <typename T>
constexpr int kUpdRows = sizeof(T) == 4 ? 4 : 2;
constexpr int kUpdBlocksPerSm = 4;

template <typename T, bool kGraph>
__global__ void __launch_bounds__(kPcgThreads, kUpdBlocksPerSm)
    k_update(int64_t n, const T* __restrict__ dinv, T* __restrict__ x, T* __restrict__ r,
             ZP<T>* __restrict__ zp, const T* __restrict__ pnew, const T* __restrict__ q,
             double* part, double* scal, int nb, int32_t* ctl, cudaGraphConditionalHandle loop) {
  if (kGraph && blockIdx.x == 0 && threadIdx.x == 0) {
    // the only writer of the loop condition and of the trip counter
    const int trips = ctl[kTrips] + 1;
    ctl[kTrips] = trips;
    if (ctl[kDone] || trips > ctl[kMaxIt] + 1) cudaGraphSetConditional(loop, 0u);
  }
  if (ctl[kDone]) return;
  const int max_iter = ctl[kMaxIt];
  const int it = ctl[kIt];
  const T alpha = steps<T>(scal)[0];
  Dot<T> rzn, rr;
  const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n;
       i0 += kUpdRows<T> * nthr) {
    T pv[kUpdRows<T>], xv[kUpdRows<T>], rv[kUpdRows<T>], qv[kUpdRows<T>], dv[kUpdRows<T>];
#pragma unroll
    for (int u = 0; u < kUpdRows<T>; u++) {
      const int64_t i = i0 + u * nthr;
      if (i < n) {
        pv[u] = pnew[i];
        xv[u] = x[i];
        rv[u] = r[i];
        qv[u] = q[i];
        dv[u] = dinv[i];
      }
    }
#pragma unroll
    for (int u = 0; u < kUpdRows<T>; u++) {
      const int64_t i = i0 + u * nthr;
      if (i < n) {
        const T ri = rv[u] - alpha * qv[u];
        const T zi = ri * dv[u];
        x[i] = xv[u] + alpha * pv[u];
        r[i] = ri;
        zp[i] = ZP<T>{zi, pv[u]};
        rzn.add(ri, zi);
        rr.add(ri, ri);
      }
    }
  }
  if (arrive(part, nb, 2, rzn, rr, Dot<T>(), ctl)) {
    const Dot<T> rzs = sum_parts<T>(part + kPartA * nb, nb);
    const Dot<T> rrs = sum_parts<T>(part + kPartB * nb, nb);
    if (threadIdx.x == 0) {
      const double trz = rzs.value(), trr = rrs.value();
      steps<T>(scal)[1] = (T)(trz / scal[kRZ]);  // beta of the next iteration
      scal[kRZP] = scal[kRZ];
      scal[kRZ] = trz;
      scal[kRR] = trr;
      ctl[kIt] = it + 1;
      if (trr <= scal[kRtol2] * scal[kRR0] || it + 1 >= max_iter) {
        ctl[kIters] = it + 1;
        ctl[kDone] = 1;
      }
      ctl[kArrive] = 0;
    }
  }
}

// The whole solve in one cooperative launch: every block stays resident and
// the phases of an iteration are separated by grid barriers instead of
// kernel boundaries.  Per iteration: (1) p_new = z + beta p_old fused into
// the SpMV's gather, q = M p_new, partial p.q; barrier; alpha = r.z / p.q
// from the partials summed in index order by every block; (2) x += alpha p,
// r -= alpha q, z = r D^-1 (D^-1 formed once), partials of r.z and r.r;
// barrier; beta and the convergence test, again from the ordered sums, so
// every block takes the same decisions.  Data other blocks wrote within the
// launch is read through L2 (ld.cg): an SM's L1 is not kept coherent.
// Thread 0 of each block forms the scalars; the block gets the step length
// and the decision through shared memory.
template <typename T>
__global__ void __launch_bounds__(kPcgThreads, 4)
    k_pcg_coop(int64_t n, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ cols,
               const T* __restrict__ vals, const T* __restrict__ diag,
               const double* __restrict__ b, T* x, T* r, T* z, T* pa, T* pb, T* q, T* dinv,
               double* part, int nb, int32_t* ctl, double rtol2, int max_iter) {
  const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double* Ppq = part + kPartA * nb;
  double* Prz = part + kPartB * nb;
  double* Prr = part + kPartC * nb;
  int32_t* counter = ctl + kBar;
  int32_t* timeout = ctl + kTimeout;
  int gen = 0;
  // thread 0 of every block forms the scalars from the ordered partial sums
  // (the same bits in every block) and hands the block the step length and
  // the decision
  __shared__ T s_step;
  __shared__ int s_state;  // 0: go on, 1: converged or at the cap, 2: breakdown
  double trz = 0.0, trr0 = 0.0;
  Dot<T> rz0, rr0;
  for (int64_t i = tid; i < n; i += nthr) {
    const T d = diag[i];
    const T di = d > T(0) ? T(1) / d : T(0);
    const T ri = (T)b[i];
    const T zi = ri * di;
    dinv[i] = di;
    x[i] = T(0);
    r[i] = ri;
    z[i] = zi;
    pa[i] = T(0);
    rz0.add(ri, zi);
    rr0.add(ri, ri);
  }
  {
    const Dot<T> rzb = block_sum(rz0), rrb = block_sum(rr0);
    if (threadIdx.x == 0) {
      Prz[blockIdx.x] = rzb.pack();
      Prr[blockIdx.x] = rrb.pack();
    }
  }
  if (!grid_barrier(counter, timeout, ++gen * nb)) return;
  {
    const Dot<T> rzs = sum_parts<T>(Prz, nb), rrs = sum_parts<T>(Prr, nb);
    if (threadIdx.x == 0) {
      trz = rzs.value();
      trr0 = rrs.value();
      s_step = T(0);  // beta of the first iteration
      s_state = !(trr0 > 0.0) || max_iter <= 0 ? 1 : 0;
    }
    __syncthreads();
  }
  int it = 0;
  bool brk = false;
  bool done = s_state != 0;
  const int sub = threadIdx.x & (kTpr - 1);
  const int64_t groups = nthr / kTpr;
  // rows rounded up to a multiple of the group count: every lane of a warp
  // runs the same number of row iterations (full-mask shuffles)
  const int64_t n_round = ((n + groups - 1) / groups) * groups;
  while (!done) {
    const T beta = s_step;
    const T* pold = (it & 1) ? pb : pa;
    T* pnew = (it & 1) ? pa : pb;
    Dot<T> pqt;
    for (int64_t i = tid / kTpr; i < n_round; i += groups) {
      T acc = T(0), pi = T(0);
      if (i < n) {
        const int a = row_ptr[i], e = row_ptr[i + 1];
#pragma unroll 4
        for (int k = a + sub; k < e; k += kTpr) {
          const int j = cols[k];
          acc += vals[k] * (__ldcg(z + j) + beta * __ldcg(pold + j));
        }
        pi = __ldcg(z + i) + beta * __ldcg(pold + i);
      }
#pragma unroll
      for (int off = kTpr / 2; off > 0; off >>= 1) acc += __shfl_xor_sync(kFull, acc, off);
      if (i < n && sub == 0) {
        const T qi = diag[i] * pi + acc;
        pnew[i] = pi;
        q[i] = qi;
        pqt.add(pi, qi);
      }
    }
    {
      const Dot<T> pqb = block_sum(pqt);
      if (threadIdx.x == 0) Ppq[blockIdx.x] = pqb.pack();
    }
    if (!grid_barrier(counter, timeout, ++gen * nb)) return;
    {
      const Dot<T> pqs = sum_parts<T>(Ppq, nb);
      if (threadIdx.x == 0) {
        const double tpq = pqs.value();
        if (tpq > 0.0)
          s_step = (T)(trz / tpq);  // alpha
        else
          s_state = 2;  // M not positive definite along p: breakdown
      }
      __syncthreads();
    }
    if (s_state == 2) {
      brk = true;
      break;
    }
    const T alpha = s_step;
    Dot<T> rzt, rrt;
    for (int64_t i = tid; i < n; i += nthr) {
      x[i] += alpha * __ldcg(pnew + i);
      const T ri = r[i] - alpha * __ldcg(q + i);
      const T zi = ri * dinv[i];
      r[i] = ri;
      z[i] = zi;
      rzt.add(ri, zi);
      rrt.add(ri, ri);
    }
    {
      const Dot<T> rzb = block_sum(rzt), rrb = block_sum(rrt);
      if (threadIdx.x == 0) {
        Prz[blockIdx.x] = rzb.pack();
        Prr[blockIdx.x] = rrb.pack();
      }
    }
    if (!grid_barrier(counter, timeout, ++gen * nb)) return;
    it++;
    {
      const Dot<T> rzs = sum_parts<T>(Prz, nb), rrs = sum_parts<T>(Prr, nb);
      if (threadIdx.x == 0) {
        const double trz_new = rzs.value(), trr = rrs.value();
        s_step = (T)(trz_new / trz);  // beta of the next iteration
        trz = trz_new;
        s_state = trr <= rtol2 * trr0 || it >= max_iter ? 1 : 0;
      }
      __syncthreads();
    }
    done = s_state != 0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctl[kIters] = it;
    ctl[kIt] = it;
    ctl[kBreak] = brk ? 1 : 0;
    ctl[kDone] = 1;
  }
}

}  // namespace

int pcg_blocks(int sm_count) { return sm_count * kPcgMaxBlocksPerSm; }
size_t pcg_red_len(int sm_count) { return (size_t)kParts * pcg_blocks(sm_count) + kScalars; }

namespace {

// k_update's grid: one wave at kUpdBlocksPerSm blocks per SM, at most nb
// (its partials use the same arrays)
int upd_blocks(const pot_ctx* ctx, int nb) {
  const int b = ctx->sm_count * kUpdBlocksPerSm;
  return b < nb ? b : nb;
}

// The while-node graph of the PCG iterations for n rows (see the top).
template <typename T>
int build_graph(pot_ctx* ctx, int64_t n, int nb, double* part, double* scal) {
  const int k = sizeof(T) == 4 ? 0 : 1;
  if (ctx->pcg_exec[k]) cudaGraphExecDestroy(ctx->pcg_exec[k]);
  if (ctx->pcg_graph[k]) cudaGraphDestroy(ctx->pcg_graph[k]);
  ctx->pcg_exec[k] = nullptr;
  ctx->pcg_graph[k] = nullptr;
  ctx->pcg_graph_n[k] = -1;
  Work<T>& w = ctx->work<T>();
  cudaGraph_t g = nullptr;
  POT_CUDA(cudaGraphCreate(&g, 0));
  ctx->pcg_graph[k] = g;
  cudaGraphConditionalHandle loop;
  POT_CUDA(cudaGraphConditionalHandleCreate(&loop, g, 1u, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = loop;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cnode;
  POT_CUDA(cudaGraphAddNode(&cnode, g, nullptr, nullptr, 0, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  // kernel arguments (copied into the graph when the nodes are added)
  int64_t an = n;
  const int32_t* row_ptr = ctx->row_ptr;
  const int32_t* cols = ctx->csr_cols;
  const T* vals = w.csr_vals;
  const T* diag = w.diag;
  const T* dinv = w.x;
  ZP<T>* zp = (ZP<T>*)w.zp;
  const ZP<T>* zpc = zp;
  T *x = w.u, *r = w.r, *pnew = w.p1, *q = w.q;
  const T *pnewc = w.p1, *qc = w.q;
  int anb = nb;
  int anbu = upd_blocks(ctx, nb);
  int32_t* ctl = ctx->pcg_ctl;
  void* a1[] = {&an, &row_ptr, &cols, &vals, &diag, &zpc, &pnew, &q, &part, &scal, &anb, &ctl};
  cudaKernelNodeParams k1 = {};
  k1.func = (void*)k_spmv<T>;
  k1.gridDim = dim3(nb);
  k1.blockDim = dim3(kPcgThreads);
  k1.kernelParams = a1;
  cudaGraphNode_t n1, n2;
  POT_CUDA(cudaGraphAddKernelNode(&n1, body, nullptr, 0, &k1));
  void* a2[] = {&an, &dinv, &x, &r, &zp, &pnewc, &qc, &part, &scal, &anbu, &ctl, &loop};
  cudaKernelNodeParams k2 = {};
  k2.func = (void*)k_update<T, true>;
  k2.gridDim = dim3(anbu);
  k2.blockDim = dim3(kPcgThreads);
  k2.kernelParams = a2;
  POT_CUDA(cudaGraphAddKernelNode(&n2, body, &n1, 1, &k2));
  POT_CUDA(cudaGraphInstantiate(&ctx->pcg_exec[k], g, 0));
  ctx->pcg_graph_n[k] = n;
  return POT_OK;
}

}  // namespace

template <typename T>
int pcg_solve(pot_ctx* ctx, cudaStream_t st, int64_t n, int64_t nnz_off, double rtol, int max_iter,
              int chunk, bool host_loop, int* iters, double* rel_res) {
  (void)nnz_off;
  Work<T>& w = ctx->work<T>();
  // one full wave of the SpMV kernel: as many blocks as fit on the SMs
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spmv<T>, kPcgThreads, 0) !=
          cudaSuccess ||
      per_sm < 1)
    per_sm = 2;
  if (per_sm > kPcgMaxBlocksPerSm) per_sm = kPcgMaxBlocksPerSm;
  const int nb = ctx->sm_count * per_sm;
  double* part = ctx->pcg_red;
  double* scal = ctx->pcg_red + (size_t)kParts * pcg_blocks(ctx->sm_count);
  if (chunk < 1) chunk = 1;
  const double rtol2 = rtol * rtol;
  int32_t* hctl = (int32_t*)(ctx->h_pinned + 16);
  // the persistent solve (one cooperative launch) for systems small enough
  // that launches and kernel tails dominate an iteration, when the device
  // can hold every block at once; otherwise the graph below, whose gathers
  // keep the L1 cache (measured on the 2M splash: 2.86 ms of PCG per step
  // with the graph, 3.25 ms with the persistent kernel; the 1000-site block:
  // 12.6 -> 9.3 ms per FP64 solve with the persistent kernel)
  int coop = 0, per_coop = 0;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, ctx->device);
  if (coop && !host_loop && n <= kPcgCoopMaxRows &&
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_coop, k_pcg_coop<T>, kPcgThreads,
                                                            0) == cudaSuccess &&
      per_coop >= 1) {
    if (per_coop > kPcgMaxBlocksPerSm) per_coop = kPcgMaxBlocksPerSm;
    int nbc = ctx->sm_count * per_coop;
    POT_CUDA(cudaMemsetAsync(ctx->pcg_ctl, 0, kPcgCtlWords * sizeof(int32_t), st));
    int64_t an = n;
    const int32_t* row_ptr = ctx->row_ptr;
    const int32_t* cols = ctx->csr_cols;
    const T* vals = w.csr_vals;
    const T* diag = w.diag;
    const double* bvec = ctx->grad;
    T *x = w.u, *r = w.r, *z = w.z, *pa = w.p0, *pb = w.p1, *q = w.q, *dinv = w.x;
    int32_t* ctl = ctx->pcg_ctl;
    double art = rtol2;
    int amax = max_iter;
    void* args[] = {&an, &row_ptr, &cols, &vals, &diag, &bvec, &x, &r, &z, &pa, &pb, &q, &dinv,
                    &part, &nbc, &ctl, &art, &amax};
    if (cudaLaunchCooperativeKernel((void*)k_pcg_coop<T>, nbc, kPcgThreads, args, 0, st) ==
        cudaSuccess) {
      note_launch();
      POT_CUDA(cudaMemcpyAsync(hctl, ctx->pcg_ctl, kPcgCtlWords * sizeof(int32_t),
                               cudaMemcpyDeviceToHost, st));
      POT_CUDA(cudaStreamSynchronize(st));
      if (hctl[kTimeout]) return POT_ERR_CUDA;  // a barrier wait ran out
      *iters = hctl[kIters];
      if (rel_res) *rel_res = -1.0;
      return hctl[kBreak] ? POT_ERR_PCG_BREAKDOWN : POT_OK;
    }
    cudaGetLastError();  // not launched: the graph path below
  }
  // the arrival counter must start at zero
  POT_CUDA(cudaMemsetAsync(ctx->pcg_ctl + kArrive, 0, sizeof(int32_t), st));
  note_launch();
  k_pcg_init<T><<<nb, kPcgThreads, 0, st>>>(n, ctx->grad, w.diag, w.u, w.r, w.x, (ZP<T>*)w.zp,
                                            part, scal, nb, ctx->pcg_ctl, rtol2, max_iter);
  POT_CUDA(cudaGetLastError());
  const int gk = sizeof(T) == 4 ? 0 : 1;
  bool graph = !host_loop && ctx->pcg_exec[gk] && ctx->pcg_graph_n[gk] == n;
  if (!graph && !host_loop) {
    graph = build_graph<T>(ctx, n, nb, part, scal) == POT_OK;
    if (!graph) cudaGetLastError();  // clear it: the chunked loop below runs instead
  }
  if (graph) {
    POT_CUDA(cudaGraphLaunch(ctx->pcg_exec[gk], st));
    POT_CUDA(cudaMemcpyAsync(hctl, ctx->pcg_ctl, 8 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    POT_CUDA(cudaStreamSynchronize(st));
    // launches: the kernels of every trip of the loop
    note_launches(2 * (int64_t)hctl[kTrips]);
  } else {
    int launched = 0;
    for (;;) {
      for (int k = 0; k < chunk; k++) {
        note_launch();
        k_spmv<T><<<nb, kPcgThreads, 0, st>>>(n, ctx->row_ptr, ctx->csr_cols, w.csr_vals, w.diag,
                                              (const ZP<T>*)w.zp, w.p1, w.q, part, scal, nb,
                                              ctx->pcg_ctl);
        note_launch();
        k_update<T, false><<<upd_blocks(ctx, nb), kPcgThreads, 0, st>>>(
            n, w.x, w.u, w.r, (ZP<T>*)w.zp, w.p1, w.q, part, scal, upd_blocks(ctx, nb),
            ctx->pcg_ctl, cudaGraphConditionalHandle{});
      }
      launched += chunk;
      POT_CUDA(cudaGetLastError());
      POT_CUDA(cudaMemcpyAsync(hctl, ctx->pcg_ctl, 8 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
      POT_CUDA(cudaStreamSynchronize(st));
      if (hctl[kDone] || launched > max_iter + chunk) break;
    }
  }
  *iters = hctl[kDone] ? hctl[kIters] : hctl[kIt];
  if (rel_res) *rel_res = -1.0;
  if (hctl[kBreak]) return POT_ERR_PCG_BREAKDOWN;
  return POT_OK;
}

template int pcg_solve<float>(pot_ctx*, cudaStream_t, int64_t, int64_t, double, int, int, bool,
                              int*, double*);
template int pcg_solve<double>(pot_ctx*, cudaStream_t, int64_t, int64_t, double, int, int, bool,
                               int*, double*);

}  // namespace pot
