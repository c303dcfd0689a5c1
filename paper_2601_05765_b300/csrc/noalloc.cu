// lgc_compute_cells_noalloc: cell evaluation for callers that cannot
// allocate device memory.
//
// Every scratch buffer of the evaluation (sorted sites, grid, candidate
// lists, per-cell results, security radii, reduction partials, status
// words) lives in one
// file-scope device array of fixed size, so a call allocates nothing: no
// cudaMalloc, cudaFree, pinned host memory or event.  The array is sized for
// kNoAllocMaxSites sites and k_max = 64 and is held by every GPU that loads
// the library until the process exits.
//
// Host code cannot use the array's name as a device address, so the first
// call on each device asks the runtime for the address (cudaGetSymbolAddress)
// with that device current and caches it; make that first call before any
// stream capture.  The stream must belong to the current device.  Every call
// shares the array and the next call overwrites it: the status words are
// cleared at the start of each call and the grid counts are cleared by the
// grid build.  Calls that overlap on the GPU race on the array; a host mutex
// serialises calls made from several threads, and each call waits for its
// stream before it returns, on every return path.
#include <mutex>

#include "pot_internal.cuh"

namespace pot {
namespace {

constexpr int64_t kNoAllocMaxSites = 8192;
constexpr int kNoAllocK = 64;
constexpr int64_t kNoAllocGridCap = 2 * kNoAllocMaxSites;
constexpr int64_t kNoAllocScanTmp = (kNoAllocGridCap + 2047) / 2048 + 2;
constexpr int kMaxDevices = 64;

constexpr size_t al(size_t x) { return (x + 255) & ~size_t(255); }

// byte offsets of the buffers inside the scratch array
constexpr int64_t N = kNoAllocMaxSites;
constexpr size_t oKeys = 0;
constexpr size_t oPerm = oKeys + al(4 * N);
constexpr size_t oIperm = oPerm + al(4 * N);
constexpr size_t oCount = oIperm + al(4 * N);
constexpr size_t oStart = oCount + al(4 * (kNoAllocGridCap + 1));
constexpr size_t oCand = oStart + al(4 * (kNoAllocGridCap + 1));
constexpr size_t oMeta = oCand + al(4 * N * kNoAllocK);
constexpr size_t oRowCnt = oMeta + al(4 * N);
constexpr size_t oScan = oRowCnt + al(4 * (N + 1));
constexpr size_t oSnu = oScan + al(4 * kNoAllocScanTmp);
constexpr size_t oGrad = oSnu + al(8 * N);
constexpr size_t oRed = oGrad + al(8 * N);
constexpr size_t oRedOut = oRed + al(8 * 6 * kRedBlocks);
constexpr size_t oErr = oRedOut + al(8 * 8);
constexpr size_t oSxp = oErr + al(4 * 2);
constexpr size_t oPsiBase = oSxp + al(16 * N);
constexpr size_t oVol = oPsiBase + al(4 * N);
constexpr size_t oKarea = oVol + al(4 * N);
constexpr size_t oDiag = oKarea + al(4 * N);
constexpr size_t oCen = oDiag + al(4 * N);
constexpr size_t oStage = oCen + al(12 * N);
constexpr size_t oPsiMax = oStage + al(4 * N * kNoAllocK);
constexpr size_t oNuMax = oPsiMax + al(8);
constexpr size_t oSrad = oNuMax + al(8);
constexpr size_t oSradLo = oSrad + al(4 * N);
constexpr size_t oSoff = oSradLo + al(4 * N);
constexpr size_t oRcell = oSoff + al(12 * N);
constexpr size_t oGmax = oRcell + al(4 * N);
constexpr size_t oNeed = oGmax + al(4 * (kNoAllocGridCap + 1));
constexpr size_t oNeedCount = oNeed + al(N);
constexpr size_t oBigList = oNeedCount + al(16);
constexpr size_t oFixList = oBigList + al(4 * N);
constexpr size_t kScratchBytes = oFixList + al(4 * N);
// the size the header states (5,333,504 bytes, about 5.3 MB)
static_assert(kScratchBytes == 5333504, "update the scratch size stated in pot.h");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_base[kMaxDevices] = {};
double g_noalloc_host[64];  // host scalars read back by the evaluation
const int32_t kErrInit[2] = {0, 0x7fffffff};

// device address of the scratch array on `dev` (set up once per device)
int scratch_base(int dev, unsigned char** out) {
  if (dev < 0 || dev >= kMaxDevices) return POT_ERR_INVALID_ARG;
  if (!g_noalloc_base[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return POT_ERR_CUDA;
    g_noalloc_base[dev] = p;
  }
  *out = (unsigned char*)g_noalloc_base[dev];
  return POT_OK;
}

// Waits for the call's stream on every return path once device work has
// been enqueued, so that the next call (after the mutex is released) never
// overlaps this one on the shared array, whatever status this one returns.
struct StreamDrain {
  cudaStream_t st;
  bool armed = false;
  ~StreamDrain() {
    if (armed) cudaStreamSynchronize(st);
  }
};

}  // namespace
}  // namespace pot

using namespace pot;

extern "C" int lgc_compute_cells_noalloc(void* stream, int64_t n, const float* pos,
                                         const float* psi, const double* targets,
                                         const pot_domain* dom, float* volumes, double* grad,
                                         float* centroids, float* karea, pot_cell_stats* stats) {
  if (stats) {
    *stats = pot_cell_stats();
    stats->error_site = -1;
  }
  if (n > kNoAllocMaxSites) return POT_ERR_TOO_LARGE;
  if (n <= 0 || !pos || !psi || !dom) return POT_ERR_INVALID_ARG;
  for (int k = 0; k < 3; k++)
    if (!(dom->hi[k] > dom->lo[k])) return POT_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return POT_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  // the array's address belongs to the current device: the stream must too
  // (the legacy default stream follows the current device)
  if (st != nullptr) {
    int sdev = -1;
    if (cudaStreamGetDevice(st, &sdev) != cudaSuccess) return POT_ERR_INVALID_ARG;
    if (sdev != dev) return POT_ERR_INVALID_ARG;
  }
  unsigned char* b = nullptr;
  POT_CHECK(scratch_base(dev, &b));
  // declared after the lock, so it drains the stream before the unlock
  StreamDrain drain{st};

  // a context shell whose buffers all point into the scratch array
  pot_ctx c;
  c.device = dev;
  c.n_max = kNoAllocMaxSites;
  c.k_max = kNoAllocK;
  c.mask = 1;
  c.grid_cap = kNoAllocGridCap;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  c.sm_count = sms > 0 ? sms : 148;
  c.keys = (uint32_t*)(b + oKeys);
  c.perm = (int32_t*)(b + oPerm);
  c.iperm = (int32_t*)(b + oIperm);
  c.cell_count = (int32_t*)(b + oCount);
  c.cell_start = (int32_t*)(b + oStart);
  c.cand = (int32_t*)(b + oCand);
  c.meta = (int32_t*)(b + oMeta);
  c.row_cnt = (int32_t*)(b + oRowCnt);
  c.scan_tmp = (int32_t*)(b + oScan);
  c.scan_tmp_len = kNoAllocScanTmp;
  c.snu = (double*)(b + oSnu);
  c.grad = (double*)(b + oGrad);
  c.red = (double*)(b + oRed);
  c.red_out = (double*)(b + oRedOut);
  c.err = (int32_t*)(b + oErr);
  c.h_pinned = g_noalloc_host;
  Work<float>& w = c.wf;
  w.sxp = (V4<float>*)(b + oSxp);
  w.psi_base = (float*)(b + oPsiBase);
  w.vol = (float*)(b + oVol);
  w.karea = (float*)(b + oKarea);
  w.diag = (float*)(b + oDiag);
  w.cen = (float*)(b + oCen);
  w.stage_vals = (float*)(b + oStage);
  w.psi_max = (float*)(b + oPsiMax);
  w.nu_max = (float*)(b + oNuMax);
  w.srad = (float*)(b + oSrad);
  w.srad_lo = (float*)(b + oSradLo);
  w.soff = (float*)(b + oSoff);
  w.rcell = (float*)(b + oRcell);
  w.gmax = (float*)(b + oGmax);
  c.need = (uint8_t*)(b + oNeed);
  c.need_count = (int32_t*)(b + oNeedCount);
  c.big_list = (int32_t*)(b + oBigList);  // unused: 64-plane lists fit the cell kernel's window
  c.fix_list = (int32_t*)(b + oFixList);

  // the previous call's status words are stale: clear them
  drain.armed = true;
  POT_CUDA(cudaMemcpyAsync(c.err, kErrInit, sizeof(kErrInit), cudaMemcpyHostToDevice, st));
  POT_CHECK(grid_build<float>(&c, st, n, pos, psi, targets, dom));
  const int ce = cells_eval<float>(&c, st, n, dom, grad != nullptr);
  int64_t site = -1;
  int code = read_status(&c, st, &site);
  if (code == POT_OK) code = ce;
  if (code) {
    if (stats) stats->error_site = site;
    return code;
  }
  double res[6];
  POT_CHECK(residuals<float>(&c, st, n, res));
  POT_CHECK(unsort_outputs<float>(&c, st, n, volumes, grad, centroids, karea, nullptr));
  POT_CUDA(cudaStreamSynchronize(st));
  if (stats) {
    stats->n_empty = (int64_t)res[3];
    stats->n_planes = (int64_t)res[4];
    stats->max_planes = (int32_t)res[5];
  }
  return POT_OK;
}
