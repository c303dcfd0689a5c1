// Learned warm start for the Newton solve (not in the paper): features from
// each site's 24 nearest neighbours, previous weight, velocity and previous
// weight change, and a BF16 MLP 80 -> 128 -> 128 -> 128 -> 1 (ReLU) whose
// output is the change of the weight in units of h^2 (h = nu^(1/3)).  Plain
// Newton from the previous weights stays the fallback.
//
// Every GEMM (forward layers, back-propagation, weight gradients) runs on the
// 5th-generation tensor cores: one CTA computes a 128 x 128 FP32 tile in
// tensor memory with tcgen05.mma (kind::f16, BF16 operands, FP32
// accumulation) issued by one thread, operands staged in shared memory in
// the canonical K-major no-swizzle layout (8-row x 16-byte core matrices;
// descriptor LBO = stride between core matrices along K, SBO = along M/N),
// completion signalled through an mbarrier by tcgen05.commit, results read
// back with tcgen05.ld for fused epilogues (bias + ReLU + BF16 pack, the
// 128 -> 1 head, the ReLU mask of back-propagation, FP32 split-K partials).
// Every wait is bounded; a timeout sets the error word and the kernel still
// frees its tensor memory.
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <new>

#include "pot_internal.cuh"

typedef __nv_bfloat16 bf16;

namespace pot {
namespace {

constexpr int kIn = 80, kFeat = 77, kHid = 128, kKnn = 24;
constexpr int kTM = 128;  // rows of a tile (and N of every GEMM)
constexpr int kKC = 64;   // K staged per chunk
constexpr int kGemmThreads = 128;
constexpr int kGemmSmem = 56 * 1024;  // keeps <= 4 CTAs per SM: 4 x 128 TMEM columns
constexpr int kTrainMax = 16384;      // largest training batch
constexpr int kSplitK = 512;          // rows of the batch per split of a weight-gradient GEMM
constexpr uint32_t kWaitLimit = 1u << 22;  // try_wait may suspend: a few seconds at most

constexpr int oW1 = 0, ob1 = oW1 + kIn * kHid, oW2 = ob1 + kHid, ob2 = oW2 + kHid * kHid,
              oW3 = ob2 + kHid, ob3 = oW3 + kHid * kHid, ow4 = ob3 + kHid, ob4 = ow4 + kHid,
              kParams = ob4 + 1;

enum { kModeF32 = 0, kModeHidden = 1, kModeHead = 2, kModeDx = 3 };

struct GemmArgs {
  const bf16* A;  // M x K, row stride lda (K contiguous)
  int64_t lda, M;
  const bf16* B;  // Nrows x K, row stride ldb (K contiguous); C = A B^T
  int64_t ldb;
  int Nrows;
  int64_t K, ksplit;
  int mode, ncols;
  float* C;  // kModeF32: partial tile of split s at C + s*M*ldc
  int64_t ldc;
  const float* bias;
  bf16* H;  // row-major output (ldh)
  int64_t ldh;
  bf16* HT;  // transposed output (ldht), optional
  int64_t ldht;
  const float* w4;
  const float* b4;
  float* out;
  const bf16* mask;  // kModeDx: ReLU mask source, row-major (ldm)
  int64_t ldm;
  int32_t* err;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// tcgen05 shared-memory matrix descriptor, no swizzle, version 1
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo & 0x3FFFF) >> 4) << 16;
  d |= (uint64_t)((sbo & 0x3FFFF) >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor: D f32, A and B bf16, both K-major, M = N = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTM >> 3) << 17) |
                            ((uint32_t)(kTM >> 4) << 24);

__device__ __forceinline__ void umma(uint32_t tmem, uint64_t da, uint64_t db, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(da), "l"(db), "r"(kIdesc), "r"(acc));
}

__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t phase) {
  uint32_t done = 0;
  for (uint32_t it = 0; it < kWaitLimit && !done; it++) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(smem_u32(mbar)), "r"(phase)
        : "memory");
  }
  return done != 0;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k = 0; k < 16; k++) v[k] = __uint_as_float(r[k]);
}

// stage rows [row0, row0+128) x k [k0, k0+64) of a K-contiguous matrix into
// the core-matrix layout (zero outside rows < nrows, k < kend)
__device__ __forceinline__ void stage(uint8_t* s, const bf16* src, int64_t ld, int64_t row0,
                                      int64_t nrows, int64_t k0, int64_t kend) {
  for (int q = threadIdx.x; q < kTM * (kKC / 8); q += kGemmThreads) {
    const int r = q >> 3, kc = q & 7;
    const int64_t gr = row0 + r, kk = k0 + kc * 8;
    uint4 v = make_uint4(0, 0, 0, 0);
    if (gr < nrows && kk < kend) v = *(const uint4*)(src + gr * ld + kk);
    *(uint4*)(s + ((r >> 3) * (kKC / 8) + kc) * 128 + (r & 7) * 16) = v;
  }
}

__global__ void __launch_bounds__(kGemmThreads) k_gemm(GemmArgs g) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = base;
  uint8_t* sB = base + kTM * kKC * 2;
  uint64_t* mbar = (uint64_t*)(sB + kTM * kKC * 2);
  uint32_t* tslot = (uint32_t*)(mbar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t row0 = (int64_t)blockIdx.x * kTM;
  const int split = blockIdx.y;
  const int64_t kbeg = (int64_t)split * g.ksplit;
  const int64_t kend = kbeg + g.ksplit < g.K ? kbeg + g.ksplit : g.K;

  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"(kTM));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;

  uint32_t phase = 0;
  bool ok = true;
  bool first = true;
  for (int64_t k0 = kbeg; k0 < kend; k0 += kKC) {
    stage(sA, g.A, g.lda, row0, g.M, k0, kend);
    stage(sB, g.B, g.ldb, 0, g.Nrows, k0, kend);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int j = 0; j < kKC / 16; j++) {
        // two core matrices (32 bytes of K) per MMA of K = 16
        uint64_t da = umma_desc(smem_u32(sA) + j * 256, 128, (kKC / 8) * 128);
        uint64_t db = umma_desc(smem_u32(sB) + j * 256, 128, (kKC / 8) * 128);
        umma(tmem, da, db, (first && j == 0) ? 0u : 1u);
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_u32(mbar))
          : "memory");
    }
    first = false;
    const bool done = mbar_wait(mbar, phase);
    phase ^= 1u;
    ok = __syncthreads_and(done) != 0;
    if (!ok) break;
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  if (!ok || first) {
    if (!ok) {
      // report, then give the MMAs in flight one more bounded wait before
      // the tensor memory is freed
      if (tid == 0) atomicExch(&g.err[kErrCode], POT_ERR_CUDA);
      mbar_wait(mbar, phase ^ 1u);
    }
  } else {
    const int trow = warp * 32 + lane;
    const int64_t grow = row0 + trow;
    const bool valid = grow < g.M;
    float acc = 0.f;
    for (int c0 = 0; c0 < kTM; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (!valid) continue;
      if (g.mode == kModeF32) {
        float* dst = g.C + ((int64_t)split * g.M + grow) * g.ldc;
#pragma unroll
        for (int k = 0; k < 16; k++)
          if (c0 + k < g.ncols) dst[c0 + k] = v[k];
        continue;
      }
      __align__(16) bf16 hb[16];
#pragma unroll
      for (int k = 0; k < 16; k++) {
        const int col = c0 + k;
        float x = v[k];
        if (g.mode == kModeDx) {
          x = (col < g.ncols && __bfloat162float(g.mask[grow * g.ldm + col]) > 0.f) ? x : 0.f;
        } else {
          x = fmaxf(x + g.bias[col], 0.f);
        }
        hb[k] = __float2bfloat16_rn(x);
        if (g.mode == kModeHead) acc += __bfloat162float(hb[k]) * g.w4[col];
      }
      if (g.H) {
        uint4* dst = (uint4*)(g.H + grow * g.ldh + c0);
        dst[0] = *(const uint4*)&hb[0];
        dst[1] = *(const uint4*)&hb[8];
      }
      if (g.HT) {
#pragma unroll
        for (int k = 0; k < 16; k++)
          if (c0 + k < g.ncols) g.HT[(int64_t)(c0 + k) * g.ldht + grow] = hb[k];
      }
    }
    if (g.mode == kModeHead && valid) g.out[grow] = acc + g.b4[0];
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTM));
}

// ---------------------------------------------------------------------------
// fused inference: the three layers and the head of one 128-row tile in one
// CTA.  The tile's activations never leave the SM: each layer's epilogue
// (bias + ReLU + BF16, the same roundings as the layer-by-layer path) writes
// them into shared memory in the core-matrix layout as the next layer's A
// operand, while the next weight matrix is staged into the B buffer.  One
// 128x128 FP32 accumulator in TMEM serves all three layers.

constexpr int kFusedSmem = 2 * kTM * kHid * 2 + 1024 + 64;

// rows [row0, row0+128) x k [0, K) of a K-contiguous matrix (K a multiple
// of 8) into the core-matrix layout with K/8 core matrices per 8-row group
// (zero rows past nrows).  Each thread issues all of its 16-byte loads
// before its shared-memory stores, so they are in flight together.
template <int K>
__device__ __forceinline__ void stage_k(uint8_t* s, const bf16* src, int64_t ld, int64_t row0,
                                        int64_t nrows) {
  constexpr int kc8 = K / 8;
  constexpr int kPer = kTM * kc8 / kGemmThreads;
  static_assert(kTM * kc8 % kGemmThreads == 0, "whole 16-byte chunks per thread");
  uint4 v[kPer];
#pragma unroll
  for (int i = 0; i < kPer; i++) {
    const int q = threadIdx.x + i * kGemmThreads;
    const int r = q / kc8, kc = q - r * kc8;
    const int64_t gr = row0 + r;
    v[i] = gr < nrows ? *(const uint4*)(src + gr * ld + kc * 8) : make_uint4(0, 0, 0, 0);
  }
#pragma unroll
  for (int i = 0; i < kPer; i++) {
    const int q = threadIdx.x + i * kGemmThreads;
    const int r = q / kc8, kc = q - r * kc8;
    *(uint4*)(s + ((r >> 3) * kc8 + kc) * 128 + (r & 7) * 16) = v[i];
  }
}

// issue K/16 MMAs (A, B in the layout of stage_k) into tmem, then commit to
// mbar; thread 0 only
__device__ __forceinline__ void issue_layer(uint32_t tmem, uint8_t* sA, uint8_t* sB, int K,
                                            uint64_t* mbar) {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t sbo = (uint32_t)(K / 8) * 128;
  for (int j = 0; j < K / 16; j++) {
    const uint64_t da = umma_desc(smem_u32(sA) + j * 256, 128, sbo);
    const uint64_t db = umma_desc(smem_u32(sB) + j * 256, 128, sbo);
    umma(tmem, da, db, j == 0 ? 0u : 1u);
  }
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(mbar))
      : "memory");
}

__global__ void __launch_bounds__(kGemmThreads) k_mlp_infer(const bf16* __restrict__ x, int64_t M,
                                                            const bf16* __restrict__ wt1,
                                                            const bf16* __restrict__ wt2,
                                                            const bf16* __restrict__ wt3,
                                                            const float* __restrict__ p,
                                                            float* __restrict__ out, int32_t* err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = base;
  uint8_t* sB = base + kTM * kHid * 2;
  uint64_t* mbar = (uint64_t*)(sB + kTM * kHid * 2);
  uint32_t* tslot = (uint32_t*)(mbar + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int64_t row0 = (int64_t)blockIdx.x * kTM;

  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"(kTM));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::);
  }
  // layer 1 operands: the input tile (K = 80) and W1 (128 x 80)
  stage_k<kIn>(sA, x, kIn, row0, M);
  stage_k<kIn>(sB, wt1, kIn, 0, kHid);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const uint32_t trow = (uint32_t)(warp * 32) << 16;  // this warp's 32 TMEM lanes
  const int r = tid;                                   // the tile row of this thread
  const int64_t grow = row0 + r;

  uint32_t phase = 0;
  bool ok = true;
  float acc = 0.f;
  for (int layer = 0; layer < 3 && ok; layer++) {
    if (tid == 0) issue_layer(tmem, sA, sB, layer == 0 ? kIn : kHid, mbar);
    ok = __syncthreads_and(mbar_wait(mbar, phase)) != 0;
    phase ^= 1u;
    if (!ok) break;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const float* bias = p + (layer == 0 ? ob1 : (layer == 1 ? ob2 : ob3));
    // the MMAs are done with sA and sB: the next weights go into sB while
    // the activations go into sA (K = 128 layout)
    if (layer < 2) stage_k<kHid>(sB, layer == 0 ? wt2 : wt3, kHid, 0, kHid);
    for (int c0 = 0; c0 < kHid; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + trow + (uint32_t)c0, v);
      __align__(16) bf16 hb[16];
#pragma unroll
      for (int k = 0; k < 16; k++) {
        hb[k] = __float2bfloat16_rn(fmaxf(v[k] + bias[c0 + k], 0.f));
        if (layer == 2) acc += __bfloat162float(hb[k]) * p[ow4 + c0 + k];
      }
      if (layer < 2) {
        const int kc = c0 / 8;
        uint8_t* d0 = sA + ((r >> 3) * (kHid / 8) + kc) * 128 + (r & 7) * 16;
        *(uint4*)d0 = *(const uint4*)&hb[0];
        *(uint4*)(d0 + 128) = *(const uint4*)&hb[8];
      }
    }
    // every thread's TMEM reads and shared-memory writes complete before
    // the next layer's MMAs read sA / sB and overwrite the accumulator
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  if (ok) {
    if (grow < M) out[grow] = acc + p[ob4];
  } else {
    // report, then give the MMAs in flight one more bounded wait before the
    // tensor memory is freed
    if (tid == 0) atomicExch(&err[kErrCode], POT_ERR_CUDA);
    mbar_wait(mbar, phase ^ 1u);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTM));
}

// ---------------------------------------------------------------------------
// kNN features

__device__ __forceinline__ int fcell(float x, float lo, float inv, int dim) {
  float f = (x - lo) * inv;
  return f < 0.f ? 0 : (f >= (float)dim ? dim - 1 : (int)f);
}

constexpr int kFeatWarps = 8;   // sites per block of k_features (one warp each)
constexpr int kCandCap = 128;   // candidate buffer of a warp

// Rank of candidate c among the first m of (d, t): the number that come
// before it in increasing distance, ties by lower sorted index (unique).
__device__ __forceinline__ int cand_rank(const float* d, const int* t, int m, float dc, int tc) {
  int rank = 0;
  for (int o = 0; o < m; o++) rank += (d[o] < dc) || (d[o] == dc && t[o] < tc);
  return rank;
}

// One warp per site (sorted order): the (up to) 24 nearest other sites with
// |d| < 2 h (h = nu^(1/3)), offsets / h by increasing distance (ties by
// lower sorted index); psi / h^2; v dt / h; the previous weight change / h^2
// (0 without history); zero padding to 80.  feat row = out_perm ? out_perm[s]
// : s.  The lanes share the scan of the grid cells that meet the ball of
// radius 2 h (per (y, z) row, the run of cells within the ball's chord);
// sites inside the ball go to a shared buffer, which is cut back to its 24
// nearest whenever it would overflow; the final 24 are placed by their rank.
// The row is assembled in shared memory and written as ten 16-byte stores
// (2-byte stores when feat is not 16-byte aligned).
__global__ void __launch_bounds__(kFeatWarps * 32)
    k_features(int64_t n, const V4<float>* __restrict__ sxp, const int32_t* __restrict__ cell_start,
               GridParams<float> g, const float* __restrict__ vel_s,
               const float* __restrict__ dpsi_s, const double* __restrict__ snu, float dt,
               const int32_t* __restrict__ out_perm, bf16* feat) {
  __shared__ float s_d[kFeatWarps][kCandCap];
  __shared__ int s_t[kFeatWarps][kCandCap];
  __shared__ float s_kd[kFeatWarps][kKnn];
  __shared__ int s_kt[kFeatWarps][kKnn];
  __shared__ __align__(16) bf16 s_row[kFeatWarps][kIn];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t s = (int64_t)blockIdx.x * kFeatWarps + wid;
  if (s >= n) return;  // the whole warp
  float* cd = s_d[wid];
  int* ct = s_t[wid];
  const V4<float> p = sxp[s];
  const float h = (float)cbrt(snu[s]);
  const float ih = 1.f / h;
  const float R = 2.f * h;
  const float R2 = R * R;
  const float pc[3] = {p.x, p.y, p.z};
  int c0[3], c1[3];
#pragma unroll
  for (int k = 0; k < 3; k++) {
    c0[k] = fcell(pc[k] - R, g.lo[k], g.inv_cs, g.dim[k]);
    c1[k] = fcell(pc[k] + R, g.lo[k], g.inv_cs, g.dim[k]);
  }
  // squared distance from p to the slab of cell c along axis k (0 inside;
  // the outermost cells reach to infinity)
  auto slab = [&](int k, int c) {
    const float lo = g.lo[k] + c * g.cs;
    float e = fmaxf(0.f, fmaxf(lo - pc[k], pc[k] - (lo + g.cs)));
    if (c == 0 && pc[k] < lo) e = 0.f;
    if (c == g.dim[k] - 1 && pc[k] > lo) e = 0.f;
    return e * e;
  };
  // keep the kKnn nearest of the m buffered candidates at the front
  auto cut = [&](int m) {
    for (int c = lane; c < m; c += 32) {
      const float dc = cd[c];
      const int tc = ct[c];
      const int rank = cand_rank(cd, ct, m, dc, tc);
      if (rank < kKnn) {
        s_kd[wid][rank] = dc;
        s_kt[wid][rank] = tc;
      }
    }
    __syncwarp();
    if (lane < kKnn) {
      cd[lane] = s_kd[wid][lane];
      ct[lane] = s_kt[wid][lane];
    }
    __syncwarp();
  };
  const unsigned below = (1u << lane) - 1u;
  int m = 0;  // buffered candidates (the same in every lane)
  for (int z = c0[2]; z <= c1[2]; z++) {
    const float ez = slab(2, z);
    if (ez >= R2) continue;
    for (int y = c0[1]; y <= c1[1]; y++) {
      const float eyz = ez + slab(1, y);
      if (eyz >= R2) continue;
      const float rx = sqrtf(R2 - eyz);
      const int x0 = fcell(p.x - rx, g.lo[0], g.inv_cs, g.dim[0]);
      const int x1 = fcell(p.x + rx, g.lo[0], g.inv_cs, g.dim[0]);
      const int key0 = (z * g.dim[1] + y) * g.dim[0];
      const int a = cell_start[key0 + x0], b = cell_start[key0 + x1 + 1];
      for (int t0 = a; t0 < b; t0 += 32) {
        const int t = t0 + lane;
        float d2 = 0.f;
        bool in = false;
        if (t < b && t != s) {
          const V4<float> q = sxp[t];
          const float dx = q.x - p.x, dy = q.y - p.y, dz = q.z - p.z;
          d2 = dx * dx + dy * dy + dz * dz;
          in = d2 < R2;
        }
        const unsigned bal = __ballot_sync(kFull, in);
        const int nb = __popc(bal);
        if (nb == 0) continue;
        if (m + nb > kCandCap) {
          cut(m);
          m = kKnn;
        }
        if (in) {
          const int at = m + __popc(bal & below);
          cd[at] = d2;
          ct[at] = t;
        }
        m += nb;
        __syncwarp();
      }
    }
  }
  // the kKnn nearest in increasing order
  const int cnt = m < kKnn ? m : kKnn;
  for (int c = lane; c < m; c += 32) {
    const int rank = cand_rank(cd, ct, m, cd[c], ct[c]);
    if (rank < kKnn) s_kt[wid][rank] = ct[c];
  }
  __syncwarp();
  bf16* row = s_row[wid];
  if (lane < kKnn) {
    float ox = 0.f, oy = 0.f, oz = 0.f;
    if (lane < cnt) {
      const V4<float> q = sxp[s_kt[wid][lane]];
      ox = (q.x - p.x) * ih;
      oy = (q.y - p.y) * ih;
      oz = (q.z - p.z) * ih;
    }
    row[3 * lane + 0] = __float2bfloat16_rn(ox);
    row[3 * lane + 1] = __float2bfloat16_rn(oy);
    row[3 * lane + 2] = __float2bfloat16_rn(oz);
  } else if (lane == kKnn) {
    row[72] = __float2bfloat16_rn(p.w * ih * ih);
    row[73] = __float2bfloat16_rn(vel_s[3 * s + 0] * dt * ih);
    row[74] = __float2bfloat16_rn(vel_s[3 * s + 1] * dt * ih);
    row[75] = __float2bfloat16_rn(vel_s[3 * s + 2] * dt * ih);
    row[76] = __float2bfloat16_rn(dpsi_s ? dpsi_s[s] * ih * ih : 0.f);
    for (int k = kFeat; k < kIn; k++) row[k] = __float2bfloat16_rn(0.f);
  }
  __syncwarp();
  const int64_t orow = out_perm ? (int64_t)out_perm[s] : s;
  bf16* f = feat + orow * kIn;
  if ((reinterpret_cast<uintptr_t>(feat) & 15) == 0) {
    if (lane < kIn / 8) reinterpret_cast<uint4*>(f)[lane] = reinterpret_cast<const uint4*>(row)[lane];
  } else {
    for (int k = lane; k < kIn; k += 32) f[k] = row[k];
  }
}

// x <- clamp(x + dt v), v through a wall -> 0  (same rule as the fluid step)
__global__ void k_advect_copy(int64_t n, const float* __restrict__ pos, const float* __restrict__ vel,
                              float* pos1, float* vel1, float dt, Box<float> box, float margin) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int k = 0; k < 3; k++) {
    float x = pos[3 * i + k] + dt * vel[3 * i + k];
    float v = vel[3 * i + k];
    const float lo = box.lo[k] + margin, hi = box.hi[k] - margin;
    if (x < lo) {
      x = lo;
      if (v < 0.f) v = 0.f;
    } else if (x > hi) {
      x = hi;
      if (v > 0.f) v = 0.f;
    }
    pos1[3 * i + k] = x;
    vel1[3 * i + k] = v;
  }
}

// sorted velocities, and the sorted previous weight change psi - psi_old
// (caller order inputs; psi_old may be NULL)
__global__ void k_gather_vel(int64_t n, const int32_t* __restrict__ perm, const float* __restrict__ vel,
                             const float* __restrict__ psi, const float* __restrict__ psi_old,
                             float* vel_s, float* dpsi_s) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int64_t i = perm[s];
  vel_s[3 * s + 0] = vel[3 * i + 0];
  vel_s[3 * s + 1] = vel[3 * i + 1];
  vel_s[3 * s + 2] = vel[3 * i + 2];
  if (psi_old) dpsi_s[s] = psi[i] - psi_old[i];
}

// psi_pred = psi_prev + dpsi + h^2 out, written as the Newton start: the
// network corrects the linear extrapolation by the last weight change dpsi
// (0 without history); psi_prev kept
__global__ void k_apply_warm(int64_t n, const float* __restrict__ out, const double* __restrict__ snu,
                             const float* __restrict__ dpsi, V4<float>* sxp, float* psi_base,
                             float* psi_prev, float* psi_max) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float v = 0.f;
  if (s < n) {
    const float prev = sxp[s].w;
    const float h = (float)cbrt(snu[s]);
    // a loose guard on the correction: at most h^2 per step
    v = prev + (dpsi ? dpsi[s] : 0.f) + h * h * fminf(fmaxf(out[s], -1.f), 1.f);
    if (!(v > 0.f)) v = prev;  // a NaN or non-positive start keeps the previous weight
    psi_prev[s] = prev;
    sxp[s].w = v;
    psi_base[s] = v;
  }
  // the candidate search radius follows the largest new weight
  block_max_to(fmaxf(v, 0.f), psi_max);
}

// ---------------------------------------------------------------------------
// training kernels

__global__ void k_gather_batch(const bf16* __restrict__ x_all, const float* __restrict__ y_all,
                               const int32_t* __restrict__ idx, int64_t batch, int64_t n_all,
                               bf16* xb, bf16* xbT, float* yb, int32_t* err) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= batch) return;
  int64_t i = idx[r];
  if (i < 0 || i >= n_all) {  // out-of-range index: report and use row 0
    atomicExch(&err[kErrCode], POT_ERR_INVALID_ARG);
    i = 0;
  }
  const uint4* src = (const uint4*)(x_all + i * kIn);
  uint4* dst = (uint4*)(xb + r * kIn);
  for (int k = 0; k < kIn / 8; k++) dst[k] = src[k];
  for (int k = 0; k < kIn; k++) xbT[(int64_t)k * batch + r] = x_all[i * kIn + k];
  yb[r] = y_all[i];
}

// dL/dout = 2 (out - y) / B; dZ3 = dout w4 (h3 > 0) in BF16 (row-major and
// transposed); squared error per row for the loss
__global__ void k_head_bwd(int64_t batch, const float* __restrict__ out, const float* __restrict__ yb,
                           const bf16* __restrict__ h3, const float* __restrict__ w4, float* dout,
                           bf16* dz3, bf16* dz3T, float* sqerr) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= batch) return;
  const float e = out[r] - yb[r];
  const float d = 2.f * e / (float)batch;
  dout[r] = d;
  sqerr[r] = e * e;
  for (int c = 0; c < kHid; c++) {
    const float v = __bfloat162float(h3[r * kHid + c]) > 0.f ? d * w4[c] : 0.f;
    const bf16 b = __float2bfloat16_rn(v);
    dz3[r * kHid + c] = b;
    dz3T[(int64_t)c * batch + r] = b;
  }
}

// out[row] = sum_k src[row * ld + k] (* w[k]) over k < len, one block per row
template <typename S>
__global__ void k_rowsum(const S* __restrict__ src, int64_t ld, int64_t len, const float* __restrict__ w,
                         float* out, float scale) {
  const int64_t row = blockIdx.x;
  float s = 0.f;
  for (int64_t k = threadIdx.x; k < len; k += blockDim.x) {
    float v = (float)src[row * ld + k];
    if (w) v *= w[k];
    s += v;
  }
  __shared__ float sh[32];
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(kFull, s, off);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int k = 0; k < (int)(blockDim.x >> 5); k++) t += sh[k];
    out[row] = t * scale;
  }
}

__global__ void k_splitk_reduce(const float* __restrict__ part, int splits, int64_t count, float* out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  float s = 0.f;
  for (int k = 0; k < splits; k++) s += part[(int64_t)k * count + i];
  out[i] = s;
}

__global__ void k_adam(float* p, const float* __restrict__ gr, float* m, float* v, int64_t n, float lr,
                       float bc1, float bc2) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float g = gr[i];
  const float mi = 0.9f * m[i] + 0.1f * g;
  const float vi = 0.999f * v[i] + 0.001f * g * g;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + 1e-8f);
}

// BF16 copies of the matrix weights: WT (out x in) for the forward GEMMs and
// Wn (in x out) for back-propagation
__global__ void k_pack(const float* __restrict__ p, bf16* wt1, bf16* wt2, bf16* wt3, bf16* wn2,
                       bf16* wn3) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < kIn * kHid) {
    const int i = (int)(t / kHid), o = (int)(t % kHid);
    wt1[o * kIn + i] = __float2bfloat16_rn(p[oW1 + t]);
  }
  if (t < kHid * kHid) {
    const int i = (int)(t / kHid), o = (int)(t % kHid);
    const bf16 b2 = __float2bfloat16_rn(p[oW2 + t]);
    const bf16 b3 = __float2bfloat16_rn(p[oW3 + t]);
    wt2[o * kHid + i] = b2;
    wt3[o * kHid + i] = b3;
    wn2[t] = b2;
    wn3[t] = b3;
  }
}

template <typename T>
__global__ void k_fill(T* p, int64_t n, T v) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

}  // namespace
}  // namespace pot

// ---------------------------------------------------------------------------
// the model object

struct pot_mlp {
  int device = 0;
  int64_t max_rows = 0;
  int sm_count = 148;
  int64_t step = 0;
  float* params = nullptr;
  float* grads = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  bf16 *wt1 = nullptr, *wt2 = nullptr, *wt3 = nullptr, *wn2 = nullptr, *wn3 = nullptr;
  // forward workspace (max_rows)
  bf16 *x = nullptr, *h1 = nullptr, *h2 = nullptr;
  float* out = nullptr;
  // training workspace (kTrainMax)
  bf16 *xb = nullptr, *xbT = nullptr, *t1 = nullptr, *t2 = nullptr, *h1T = nullptr, *h2T = nullptr,
       *h3 = nullptr, *h3T = nullptr, *dz3 = nullptr, *dz3T = nullptr, *dz2 = nullptr,
       *dz2T = nullptr, *dz1T = nullptr;
  float *yb = nullptr, *tout = nullptr, *dout = nullptr, *sqerr = nullptr, *part = nullptr,
        *loss = nullptr;
  int32_t* err = nullptr;
  float* vel_tmp = nullptr;  // features: sorted velocities (3 x max_rows)
  float* pos_tmp = nullptr;  // features: advected positions (3 x max_rows)
  float* vel_adv = nullptr;  // features: advected velocities (3 x max_rows)
  float* psi_prev = nullptr;  // warm start: previous weights (sorted)
  float* dpsi_s = nullptr;    // features: previous weight change (sorted)
  float* psi_hist = nullptr;  // warm start: weights of the previous step (caller order)
  int64_t hist_n = -1;        // sites of psi_hist (-1: no history)
  bool use_hist = true;       // 77 inputs (the previous weight change) or 76
};

namespace pot {
namespace {

using mlp_t = pot_mlp;

int gemm(mlp_t* mm, cudaStream_t st, GemmArgs a, int splits) {
  a.err = mm->err;
  dim3 grid((unsigned)((a.M + kTM - 1) / kTM), (unsigned)splits);
  note_launch();
  k_gemm<<<grid, kGemmThreads, kGemmSmem, st>>>(a);
  POT_CUDA(cudaGetLastError());
  return POT_OK;
}

GemmArgs base_args() {
  GemmArgs a;
  memset(&a, 0, sizeof(a));
  return a;
}

// forward of `rows` rows of x (rows x 80 BF16) into out; training mode also
// keeps H^T and H3 for the backward pass (rows <= kTrainMax)
int forward(mlp_t* mm, cudaStream_t st, int64_t rows, const bf16* x, float* out, bool train) {
  const float* p = mm->params;
  if (!train) {
    // inference: all layers of a tile in one CTA (k_mlp_infer)
    note_launch();
    k_mlp_infer<<<(unsigned)((rows + kTM - 1) / kTM), kGemmThreads, kFusedSmem, st>>>(
        x, rows, mm->wt1, mm->wt2, mm->wt3, p, out, mm->err);
    POT_CUDA(cudaGetLastError());
    return POT_OK;
  }
  GemmArgs a = base_args();
  a.A = x; a.lda = kIn; a.M = rows; a.B = mm->wt1; a.ldb = kIn; a.Nrows = kHid;
  a.K = kIn; a.ksplit = kIn; a.mode = kModeHidden; a.ncols = kHid; a.bias = p + ob1;
  a.H = train ? mm->t1 : mm->h1; a.ldh = kHid;
  a.HT = train ? mm->h1T : nullptr; a.ldht = rows;
  POT_CHECK(gemm(mm, st, a, 1));
  a = base_args();
  a.A = train ? mm->t1 : mm->h1; a.lda = kHid; a.M = rows; a.B = mm->wt2; a.ldb = kHid;
  a.Nrows = kHid; a.K = kHid; a.ksplit = kHid; a.mode = kModeHidden; a.ncols = kHid;
  a.bias = p + ob2; a.H = train ? mm->t2 : mm->h2; a.ldh = kHid;
  a.HT = train ? mm->h2T : nullptr; a.ldht = rows;
  POT_CHECK(gemm(mm, st, a, 1));
  a = base_args();
  a.A = train ? mm->t2 : mm->h2; a.lda = kHid; a.M = rows; a.B = mm->wt3; a.ldb = kHid;
  a.Nrows = kHid; a.K = kHid; a.ksplit = kHid; a.mode = kModeHead; a.ncols = kHid;
  a.bias = p + ob3; a.w4 = p + ow4; a.b4 = p + ob4; a.out = out;
  a.H = train ? mm->h3 : nullptr; a.ldh = kHid;
  a.HT = train ? mm->h3T : nullptr; a.ldht = rows;
  return gemm(mm, st, a, 1);
}

// weight gradient dW (Min x 128) = A^T-layout (Min x batch) . dZ^T (128 x batch)^T
int weight_grad(mlp_t* mm, cudaStream_t st, const bf16* aT, int64_t Min, const bf16* dzT,
                int64_t batch, float* dst) {
  const int splits = (int)((batch + kSplitK - 1) / kSplitK);
  GemmArgs a = base_args();
  a.A = aT; a.lda = batch; a.M = Min; a.B = dzT; a.ldb = batch; a.Nrows = kHid;
  a.K = batch; a.ksplit = kSplitK; a.mode = kModeF32; a.ncols = kHid; a.C = mm->part; a.ldc = kHid;
  POT_CHECK(gemm(mm, st, a, splits));
  const int64_t cnt = Min * kHid;
  note_launch();
  k_splitk_reduce<<<blocks_for(cnt, 256), 256, 0, st>>>(mm->part, splits, cnt, dst);
  return POT_OK;
}

// forward + backward of one batch (rows of xb / xbT / yb already in place)
int fwd_bwd(mlp_t* mm, cudaStream_t st, int64_t batch) {
  float* g = mm->grads;
  const float* p = mm->params;
  POT_CHECK(forward(mm, st, batch, mm->xb, mm->tout, true));
  note_launch();
  k_head_bwd<<<blocks_for(batch, 128), 128, 0, st>>>(batch, mm->tout, mm->yb, mm->h3, p + ow4,
                                                      mm->dout, mm->dz3, mm->dz3T, mm->sqerr);
  note_launch();
  k_rowsum<bf16><<<kHid, 256, 0, st>>>(mm->h3T, batch, batch, mm->dout, g + ow4, 1.f);
  note_launch();
  k_rowsum<float><<<1, 256, 0, st>>>(mm->dout, batch, batch, nullptr, g + ob4, 1.f);
  note_launch();
  k_rowsum<float><<<1, 256, 0, st>>>(mm->sqerr, batch, batch, nullptr, mm->loss, 1.f / batch);
  note_launch();
  k_rowsum<bf16><<<kHid, 256, 0, st>>>(mm->dz3T, batch, batch, nullptr, g + ob3, 1.f);
  POT_CHECK(weight_grad(mm, st, mm->h2T, kHid, mm->dz3T, batch, g + oW3));
  // dZ2 = (dZ3 W3^T) (h2 > 0)
  GemmArgs a = base_args();
  a.A = mm->dz3; a.lda = kHid; a.M = batch; a.B = mm->wn3; a.ldb = kHid; a.Nrows = kHid;
  a.K = kHid; a.ksplit = kHid; a.mode = kModeDx; a.ncols = kHid; a.mask = mm->t2; a.ldm = kHid;
  a.H = mm->dz2; a.ldh = kHid; a.HT = mm->dz2T; a.ldht = batch;
  POT_CHECK(gemm(mm, st, a, 1));
  note_launch();
  k_rowsum<bf16><<<kHid, 256, 0, st>>>(mm->dz2T, batch, batch, nullptr, g + ob2, 1.f);
  POT_CHECK(weight_grad(mm, st, mm->h1T, kHid, mm->dz2T, batch, g + oW2));
  // dZ1 = (dZ2 W2^T) (h1 > 0)
  a = base_args();
  a.A = mm->dz2; a.lda = kHid; a.M = batch; a.B = mm->wn2; a.ldb = kHid; a.Nrows = kHid;
  a.K = kHid; a.ksplit = kHid; a.mode = kModeDx; a.ncols = kHid; a.mask = mm->t1; a.ldm = kHid;
  a.H = nullptr; a.HT = mm->dz1T; a.ldht = batch;
  POT_CHECK(gemm(mm, st, a, 1));
  note_launch();
  k_rowsum<bf16><<<kHid, 256, 0, st>>>(mm->dz1T, batch, batch, nullptr, g + ob1, 1.f);
  POT_CHECK(weight_grad(mm, st, mm->xbT, kIn, mm->dz1T, batch, g + oW1));
  POT_CUDA(cudaGetLastError());
  return POT_OK;
}

int pack(mlp_t* mm, cudaStream_t st) {
  note_launch();
  k_pack<<<blocks_for(kHid * kHid, 256), 256, 0, st>>>(mm->params, mm->wt1, mm->wt2, mm->wt3,
                                                        mm->wn2, mm->wn3);
  POT_CUDA(cudaGetLastError());
  return POT_OK;
}

int check_err(mlp_t* mm, cudaStream_t st) {
  int32_t h = 0;
  POT_CUDA(cudaMemcpyAsync(&h, mm->err, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  POT_CUDA(cudaStreamSynchronize(st));
  if (h) {
    POT_CUDA(cudaMemsetAsync(mm->err, 0, 2 * sizeof(int32_t), st));
    return h;
  }
  return POT_OK;
}

template <typename P>
int alloc(P** p, size_t count) {
  *p = nullptr;
  return cudaMalloc((void**)p, (count ? count : 1) * sizeof(P)) == cudaSuccess ? POT_OK
                                                                              : POT_ERR_CUDA;
}

}  // namespace

// features of sorted sites into feat (rows in sorted order, or caller order
// through out_perm); requires grid_build<float> (sxp.w = previous psi)
int mlp_features_sorted(pot_ctx* ctx, pot_mlp* mm, cudaStream_t st, int64_t n, const float* vel,
                        const float* psi, const float* psi_old, float dt, const int32_t* out_perm,
                        void* feat) {
  Work<float>& w = ctx->wf;
  note_launch();
  k_gather_vel<<<blocks_for(n, 256), 256, 0, st>>>(n, ctx->perm, vel, psi, psi_old, mm->vel_tmp,
                                                    mm->dpsi_s);
  note_launch();
  k_features<<<(unsigned)((n + kFeatWarps - 1) / kFeatWarps), kFeatWarps * 32, 0, st>>>(
      n, w.sxp, ctx->cell_start, w.grid, mm->vel_tmp, psi_old ? mm->dpsi_s : nullptr, ctx->snu,
      dt, out_perm, (bf16*)feat);
  POT_CUDA(cudaGetLastError());
  return POT_OK;
}

// warm start inside the fluid step: features, MLP, psi_pred into sxp.w /
// psi_base; the previous psi is kept in mm->psi_prev (returned)
int mlp_warm_start(pot_ctx* ctx, pot_mlp* mm, cudaStream_t st, int64_t n, const float* vel,
                   const float* psi, float dt, float** psi_prev) {
  if (!mm || n > mm->max_rows) return POT_ERR_INVALID_ARG;
  const bool hist = mm->use_hist && mm->hist_n == n;
  POT_CHECK(mlp_features_sorted(ctx, mm, st, n, vel, psi, hist ? mm->psi_hist : nullptr, dt, nullptr,
                                mm->x));
  // this step's weights are the next step's history
  POT_CUDA(cudaMemcpyAsync(mm->psi_hist, psi, n * sizeof(float), cudaMemcpyDeviceToDevice, st));
  mm->hist_n = n;
  POT_CHECK(forward(mm, st, n, mm->x, mm->out, false));
  Work<float>& w = ctx->wf;
  note_launch();
  k_apply_warm<<<blocks_for(n, 256), 256, 0, st>>>(n, mm->out, ctx->snu, hist ? mm->dpsi_s : nullptr,
                                                     w.sxp, w.psi_base, mm->psi_prev, w.psi_max);
  POT_CUDA(cudaGetLastError());
  POT_CHECK(check_err(mm, st));
  *psi_prev = mm->psi_prev;
  return POT_OK;
}

}  // namespace pot

using namespace pot;

extern "C" {

int pot_mlp_num_params(void) { return kParams; }

int pot_mlp_destroy(pot_mlp* mm) {
  if (!mm) return POT_OK;
  cudaSetDevice(mm->device);
  void* ptrs[] = {mm->params, mm->grads, mm->m,   mm->v,    mm->wt1,   mm->wt2,  mm->wt3,
                  mm->wn2,    mm->wn3,   mm->x,   mm->h1,   mm->h2,    mm->out,  mm->xb,
                  mm->xbT,    mm->t1,    mm->t2,  mm->h1T,  mm->h2T,   mm->h3,   mm->h3T,
                  mm->dz3,    mm->dz3T,  mm->dz2, mm->dz2T, mm->dz1T,  mm->yb,   mm->tout,
                  mm->dout,   mm->sqerr, mm->part, mm->loss, mm->err,  mm->vel_tmp,
                  mm->pos_tmp, mm->vel_adv, mm->psi_prev, mm->dpsi_s, mm->psi_hist};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete mm;
  return POT_OK;
}

int pot_mlp_create(pot_mlp** out, int device, int64_t max_rows) {
  if (!out) return POT_ERR_INVALID_ARG;
  *out = nullptr;
  if (max_rows <= 0 || max_rows > ((int64_t)1 << 28)) return POT_ERR_INVALID_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return POT_ERR_CUDA;
  if (cudaFuncSetAttribute(k_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmem) !=
          cudaSuccess ||
      cudaFuncSetAttribute(k_mlp_infer, cudaFuncAttributeMaxDynamicSharedMemorySize, kFusedSmem) !=
          cudaSuccess)
    return POT_ERR_CUDA;
  pot_mlp* mm = new (std::nothrow) pot_mlp();
  if (!mm) return POT_ERR_CUDA;
  mm->device = device;
  mm->max_rows = max_rows;
  const int64_t R = max_rows, T = kTrainMax;
  int s = POT_OK;
#define A(ptr, cnt) \
  if (s == POT_OK) s = alloc(&(mm->ptr), (size_t)(cnt));
  A(params, kParams); A(grads, kParams); A(m, kParams); A(v, kParams);
  A(wt1, kIn * kHid); A(wt2, kHid * kHid); A(wt3, kHid * kHid); A(wn2, kHid * kHid); A(wn3, kHid * kHid);
  A(x, R * kIn); A(h1, R * kHid); A(h2, R * kHid); A(out, R);
  A(xb, T * kIn); A(xbT, T * kIn); A(t1, T * kHid); A(t2, T * kHid); A(h1T, T * kHid);
  A(h2T, T * kHid); A(h3, T * kHid); A(h3T, T * kHid); A(dz3, T * kHid); A(dz3T, T * kHid);
  A(dz2, T * kHid); A(dz2T, T * kHid); A(dz1T, T * kHid);
  A(yb, T); A(tout, T); A(dout, T); A(sqerr, T);
  A(part, (T / kSplitK) * kHid * kHid); A(loss, 1); A(err, 2);
  A(vel_tmp, 3 * R); A(pos_tmp, 3 * R); A(vel_adv, 3 * R); A(psi_prev, R); A(dpsi_s, R);
  A(psi_hist, R);
#undef A
  if (s == POT_OK && cudaMemset(mm->err, 0, 2 * sizeof(int32_t)) != cudaSuccess) s = POT_ERR_CUDA;
  if (s == POT_OK && cudaMemset(mm->params, 0, kParams * sizeof(float)) != cudaSuccess)
    s = POT_ERR_CUDA;
  if (s != POT_OK) {
    pot_mlp_destroy(mm);
    return s;
  }
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  mm->sm_count = sms > 0 ? sms : 148;
  *out = mm;
  return POT_OK;
}

int pot_mlp_set_params(pot_mlp* mm, void* stream, const float* params) {
  if (!mm || !params) return POT_ERR_INVALID_ARG;
  if (cudaSetDevice(mm->device) != cudaSuccess) return POT_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  POT_CUDA(cudaMemcpyAsync(mm->params, params, kParams * sizeof(float), cudaMemcpyDeviceToDevice, st));
  POT_CUDA(cudaMemsetAsync(mm->m, 0, kParams * sizeof(float), st));
  POT_CUDA(cudaMemsetAsync(mm->v, 0, kParams * sizeof(float), st));
  mm->step = 0;
  POT_CHECK(pack(mm, st));
  POT_CUDA(cudaStreamSynchronize(st));
  return POT_OK;
}

int pot_mlp_get_params(pot_mlp* mm, void* stream, float* params) {
  if (!mm || !params) return POT_ERR_INVALID_ARG;
  if (cudaSetDevice(mm->device) != cudaSuccess) return POT_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  POT_CUDA(cudaMemcpyAsync(params, mm->params, kParams * sizeof(float), cudaMemcpyDeviceToDevice, st));
  POT_CUDA(cudaStreamSynchronize(st));
  return POT_OK;
}

int pot_mlp_forward(pot_mlp* mm, void* stream, int64_t rows, const uint16_t* x, float* out) {
  if (!mm || !x || !out || rows <= 0 || rows > mm->max_rows) return POT_ERR_INVALID_ARG;
  if (cudaSetDevice(mm->device) != cudaSuccess) return POT_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  POT_CHECK(forward(mm, st, rows, (const bf16*)x, out, false));
  return check_err(mm, st);
}

static int gather_batch(pot_mlp* mm, cudaStream_t st, int64_t n_all, const uint16_t* x_all,
                        const float* y_all, const int32_t* idx, int64_t batch) {
  if (!mm || !x_all || !y_all || !idx || batch <= 0 || batch > kTrainMax || batch % 8 ||
      n_all <= 0)
    return POT_ERR_INVALID_ARG;
  if (cudaSetDevice(mm->device) != cudaSuccess) return POT_ERR_CUDA;
  note_launch();
  k_gather_batch<<<blocks_for(batch, 128), 128, 0, st>>>((const bf16*)x_all, y_all, idx, batch,
                                                          n_all, mm->xb, mm->xbT, mm->yb, mm->err);
  POT_CUDA(cudaGetLastError());
  return POT_OK;
}

int pot_mlp_gradients(pot_mlp* mm, void* stream, int64_t n_all, const uint16_t* x_all,
                      const float* y_all, const int32_t* idx, int64_t batch, float* grads,
                      float* loss) {
  cudaStream_t st = (cudaStream_t)stream;
  POT_CHECK(gather_batch(mm, st, n_all, x_all, y_all, idx, batch));
  POT_CHECK(fwd_bwd(mm, st, batch));
  if (grads)
    POT_CUDA(cudaMemcpyAsync(grads, mm->grads, kParams * sizeof(float), cudaMemcpyDeviceToDevice, st));
  if (loss) POT_CUDA(cudaMemcpyAsync(loss, mm->loss, sizeof(float), cudaMemcpyDeviceToDevice, st));
  return check_err(mm, st);
}

int pot_mlp_train_step(pot_mlp* mm, void* stream, int64_t n_all, const uint16_t* x_all,
                       const float* y_all, const int32_t* idx, int64_t batch, float lr,
                       float* loss) {
  cudaStream_t st = (cudaStream_t)stream;
  POT_CHECK(gather_batch(mm, st, n_all, x_all, y_all, idx, batch));
  POT_CHECK(fwd_bwd(mm, st, batch));
  mm->step++;
  const float bc1 = 1.f - powf(0.9f, (float)mm->step);
  const float bc2 = 1.f - powf(0.999f, (float)mm->step);
  note_launch();
  k_adam<<<blocks_for(kParams, 256), 256, 0, st>>>(mm->params, mm->grads, mm->m, mm->v, kParams,
                                                     lr, bc1, bc2);
  POT_CHECK(pack(mm, st));
  if (loss) POT_CUDA(cudaMemcpyAsync(loss, mm->loss, sizeof(float), cudaMemcpyDeviceToDevice, st));
  POT_CUDA(cudaGetLastError());
  return POT_OK;
}

int pot_mlp_check(pot_mlp* mm, void* stream) {
  if (!mm) return POT_ERR_INVALID_ARG;
  return check_err(mm, (cudaStream_t)stream);
}

int pot_mlp_features(pot_ctx* ctx, pot_mlp* mm, void* stream, int64_t n, const float* pos,
                     const float* vel, const float* psi, const float* psi_old,
                     const double* targets, const pot_domain* dom, const pot_params* prm,
                     uint16_t* feat) {
  if (!ctx || !mm || !pos || !vel || !psi || !targets || !dom || !prm || !feat || n <= 0 ||
      n > ctx->n_max || n > mm->max_rows || !(ctx->mask & 1) || mm->device != ctx->device)
    return POT_ERR_INVALID_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return POT_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  Box<float> box;
  for (int k = 0; k < 3; k++) {
    box.lo[k] = (float)dom->lo[k];
    box.hi[k] = (float)dom->hi[k];
  }
  // the positions and velocities the (first sub)step solves at (same
  // advection rule, same step length)
  const float dt = (float)(prm->substeps > 1 ? prm->dt / prm->substeps : prm->dt);
  note_launch();
  k_advect_copy<<<blocks_for(n, 256), 256, 0, st>>>(n, pos, vel, mm->pos_tmp, mm->vel_adv, dt, box,
                                                     (float)prm->wall_margin);
  POT_CUDA(cudaGetLastError());
  POT_CHECK(grid_build<float>(ctx, st, n, mm->pos_tmp, psi, targets, dom));
  POT_CHECK(mlp_features_sorted(ctx, mm, st, n, mm->vel_adv, psi, mm->use_hist ? psi_old : nullptr,
                                dt, ctx->perm, feat));
  POT_CUDA(cudaStreamSynchronize(st));
  return POT_OK;
}

int pot_mlp_set_history(pot_mlp* mm, void* stream, int64_t n, const float* psi_old) {
  if (!mm || n > mm->max_rows) return POT_ERR_INVALID_ARG;
  if (cudaSetDevice(mm->device) != cudaSuccess) return POT_ERR_CUDA;
  if (!psi_old || n <= 0) {
    mm->hist_n = -1;
    return POT_OK;
  }
  cudaStream_t st = (cudaStream_t)stream;
  POT_CUDA(cudaMemcpyAsync(mm->psi_hist, psi_old, n * sizeof(float), cudaMemcpyDeviceToDevice, st));
  POT_CUDA(cudaStreamSynchronize(st));
  mm->hist_n = n;
  return POT_OK;
}

int pot_mlp_set_inputs(pot_mlp* mm, int32_t n_inputs) {
  if (!mm || (n_inputs != 76 && n_inputs != 77)) return POT_ERR_INVALID_ARG;
  mm->use_hist = n_inputs == 77;
  return POT_OK;
}

int pot_set_warm_start(pot_ctx* ctx, pot_mlp* mm) {
  if (!ctx) return POT_ERR_INVALID_ARG;
  ctx->mlp = mm;
  return POT_OK;
}

}  // extern "C"
