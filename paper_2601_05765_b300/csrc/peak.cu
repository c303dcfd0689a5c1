// FP32 FMA throughput of the device: the denominator of the cell kernel's
// roofline (its work is FP32 arithmetic; the measured peaks the bench reads
// cover only HBM copies and BF16 GEMMs).  Not part of the paper's method.
//
// Every thread runs kChains independent FMA chains (enough independent work
// to hide the FMA latency at full occupancy) for `iters` rounds; one FMA is
// 2 FLOP.  The chains' values stay finite (a = 0.9999999, b = 1e-7 keeps each
// one near b / (1 - a)); the result is written only if it takes an
// impossible value, which the compiler cannot prove, so no chain is removed.
#include "pot_internal.cuh"

namespace pot {
namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;

__global__ void __launch_bounds__(kPeakThreads)
    k_fma_peak(int iters, float a, float b, float* sink) {
  float c[kChains];
#pragma unroll
  for (int k = 0; k < kChains; k++) c[k] = (float)(threadIdx.x + k);
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int u = 0; u < 16; u++) {
#pragma unroll
      for (int k = 0; k < kChains; k++) c[k] = fmaf(c[k], a, b);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; k++) s += c[k];
  if (s == -1.0f) sink[blockIdx.x] = s;
}

}  // namespace
}  // namespace pot

using namespace pot;

extern "C" int pot_measure_fp32_peak(void* stream, float* sink, double* tflops, double* ms_out) {
  if (!sink || !tflops) return POT_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0, per_sm = 0;
  POT_CUDA(cudaGetDevice(&dev));
  POT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  POT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_peak, kPeakThreads, 0));
  if (per_sm < 1) per_sm = 1;
  const int blocks = sms * per_sm;
  const int iters = 4096;
  cudaEvent_t e0, e1;
  POT_CUDA(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return POT_ERR_CUDA;
  }
  int status = POT_OK;
  float best = 0.f;
  // one warm-up launch, then the best of five
  for (int rep = 0; rep < 6 && status == POT_OK; rep++) {
    note_launch();
    cudaEventRecord(e0, st);
    k_fma_peak<<<blocks, kPeakThreads, 0, st>>>(iters, 0.9999999f, 1e-7f, sink);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
      status = POT_ERR_CUDA;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && (best == 0.f || ms < best)) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (status != POT_OK) return status;
  const double flop = 2.0 * kChains * 16.0 * iters * (double)blocks * kPeakThreads;
  *tflops = flop / (best * 1e-3) / 1e12;
  if (ms_out) *ms_out = best;
  return POT_OK;
}
