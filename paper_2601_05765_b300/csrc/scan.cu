// Exclusive prefix sum of int32 arrays (grid cell counts, Hessian row counts).
// Three passes: per-tile totals, a one-block scan of the totals, and the
// per-tile scan with its offset.  Deterministic and safe in place.
#include "pot_internal.cuh"

namespace pot {
namespace {

constexpr int kScanThreads = 512;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int warp_incl_scan(int v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    int t = __shfl_up_sync(kFull, v, off);
    if (lane >= off) v += t;
  }
  return v;
}

// exclusive scan of one value per thread over a block of kScanThreads;
// *total receives the block sum
__device__ __forceinline__ int block_excl_scan(int v, int* total) {
  __shared__ int warp_off[kScanThreads / 32];
  __shared__ int block_tot;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  constexpr int nw = kScanThreads / 32;
  int inc = warp_incl_scan(v);
  if (lane == 31) warp_off[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    int t = lane < nw ? warp_off[lane] : 0;
    int ti = warp_incl_scan(t);
    if (lane < nw) warp_off[lane] = ti - t;
    if (lane == nw - 1) block_tot = ti;
  }
  __syncthreads();
  int res = inc - v + warp_off[wid];
  *total = block_tot;
  __syncthreads();
  return res;
}

__global__ void k_tile_sums(const int32_t* __restrict__ in, int64_t n, int32_t* __restrict__ sums) {
  int64_t base = (int64_t)blockIdx.x * kScanTile;
  int s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; k++) {
    int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
    if (i < n) s += in[i];
  }
  int tot;
  block_excl_scan(s, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// one block scans the nb tile totals in chunks and writes the grand total
__global__ void k_scan_sums(int32_t* sums, int64_t nb, int32_t* out_total) {
  int carry = 0;
  for (int64_t base = 0; base < nb; base += kScanThreads) {
    int64_t i = base + threadIdx.x;
    int v = i < nb ? sums[i] : 0;
    int tot;
    int ex = block_excl_scan(v, &tot);
    if (i < nb) sums[i] = ex + carry;
    carry += tot;
  }
  if (threadIdx.x == 0) *out_total = carry;
}

__global__ void k_tile_scan(const int32_t* in, int32_t* out, int64_t n,
                            const int32_t* __restrict__ sums) {
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int v[kScanItems];
  int s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; k++) {
    int64_t i = base + k;
    v[k] = i < n ? in[i] : 0;
    s += v[k];
  }
  int tot;
  int ex = block_excl_scan(s, &tot) + sums[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanItems; k++) {
    int64_t i = base + k;
    if (i < n) out[i] = ex;
    ex += v[k];
  }
}

}  // namespace

int scan_exclusive(pot_ctx* ctx, cudaStream_t st, const int32_t* in, int32_t* out, int64_t n) {
  if (n <= 0) {
    POT_CUDA(cudaMemsetAsync(out, 0, sizeof(int32_t), st));
    return POT_OK;
  }
  int64_t nb = (n + kScanTile - 1) / kScanTile;
  if (nb + 1 > ctx->scan_tmp_len) return POT_ERR_INVALID_ARG;
  note_launch();
  k_tile_sums<<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, ctx->scan_tmp);
  note_launch();
  k_scan_sums<<<1, kScanThreads, 0, st>>>(ctx->scan_tmp, nb, out + n);
  note_launch();
  k_tile_scan<<<(unsigned)nb, kScanThreads, 0, st>>>(in, out, n, ctx->scan_tmp);
  POT_CUDA(cudaGetLastError());
  return POT_OK;
}

}  // namespace pot
