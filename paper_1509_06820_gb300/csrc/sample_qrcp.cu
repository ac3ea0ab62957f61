// Partial QRCP on the sample matrix: Alg. 1 halted after b pivots, applied to
// the l x n_J sample B (the qrcp(B, b) step of Alg. 4 and Alg. 6).
//
// One cooperative launch per block of pivots.  CTA g owns a contiguous range
// of sample columns and keeps them in shared memory for the whole launch;
// columns never move between CTAs.  Each pivot step costs one grid barrier:
//   1. every CTA publishes its best trailing column: a record (norm, logical
//      position, the column's row i and the sum of squares of its rows
//      below i) and those rows;
//   2. after the barrier every CTA picks the same winner (largest norm, lowest
//      logical position on a tie), forms the reflector's scalars from the
//      winner's record while the winner's rows load, records the swap in its
//      own bookkeeping, applies the reflector to its trailing columns (4
//      lanes per column in FP64, 8 in FP32, shuffle reductions), downdates
//      their norms and computes its next candidate.
// Swaps are tracked as logical positions; at the end every column is written
// back to B at its final logical position, so B holds S = [S11 S12; 0 S22]
// in the permuted order and `swaps` the partner position of each step.
//
// Norm update (reading of Alg. 1's trailing-norm step once row j is final):
// the oracle's nrm *= sqrt(f), f = max(0, 1 - (|s_ij|/nrm)^2), with an exact
// recomputation from rows j+1.. when f * (nrm/nrm_ref)^2 <= sqrt(eps), kept
// here on squared norms: nrm^2 -= s_ij^2, recomputed when
// nrm^2 <= sqrt(eps) nrm_ref^2 -- the same quantities and the same test with
// no division or square root (FP64 costs ~16 issue cycles per warp
// instruction on this GPU); the two differ only in rounding.
#include <mutex>

#include "sample_qrcp.cuh"

namespace rq {
namespace {

using namespace sq;

template <typename T>
__global__ void __launch_bounds__(NT, 1) sample_qrcp_kernel(SampleQrcpArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  sample_qrcp_body<T>(a, blockIdx.x, gridDim.x, smem_raw);
}

size_t smem_bytes(int ell, int64_t chunk) { return sample_qrcp_smem_bytes(ell, chunk); }

constexpr size_t kSmemLimit = 216 * 1024;

int sample_grid(int64_t nc, int num_sms) {
  int64_t G = (nc + 63) / 64;
  if (G > num_sms) G = num_sms;
  if (G < 1) G = 1;
  return (int)G;
}

}  // namespace

bool sample_qrcp_fits(int ell, int64_t nc, int num_sms) {
  const int G = sample_grid(nc, num_sms);
  const int64_t chunk = (nc + G - 1) / G;
  return ell <= MAX_ELL && smem_bytes(ell, chunk) <= kSmemLimit;
}

cudaError_t launch_sample_qrcp(const SampleQrcpArgs& a, int num_sms, cudaStream_t st) {
  const int G = sample_grid(a.nc, num_sms);
  const int64_t chunk = (a.nc + G - 1) / G;
  const size_t smem = sample_qrcp_smem_bytes(a.ell, chunk, a.f32 ? 4 : 8);
  if (a.ell > MAX_ELL || smem > kSmemLimit) return cudaErrorInvalidValue;
  static std::atomic<uint64_t> attr_done_d{0}, attr_done_f{0};
  const void* kern = a.f32 ? (const void*)sample_qrcp_kernel<float>
                           : (const void*)sample_qrcp_kernel<double>;
  cudaError_t e = a.f32 ? ensure_smem_attr(sample_qrcp_kernel<float>, (int)kSmemLimit, attr_done_f)
                        : ensure_smem_attr(sample_qrcp_kernel<double>, (int)kSmemLimit, attr_done_d);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(a.bar, 0, sizeof(GridBarrier), st);
  if (e != cudaSuccess) return e;
  SampleQrcpArgs args = a;
  void* params[] = {&args};
  return cudaLaunchCooperativeKernel(kern, dim3((unsigned)G),
                                     dim3(NT), params, smem, st);
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the sample QRCP launch.
//
// Some callers cannot allocate device memory: code running while a stream is
// being captured into a CUDA graph (cudaMalloc is not a stream operation, so
// it cannot be recorded and breaks the capture), latency-critical loops that
// must not enter the driver's allocator, and processes whose device memory
// belongs to a caching pool or a fixed arena, where a direct cudaMalloc would
// fragment it or exceed its reservation.  rqrcp_sample_qrcp_noalloc serves
// them: it launches the same kernel as rqrcp_sample_qrcp, but its scratch
// (the candidate norms and columns, the grid barrier and a fallback status
// word) lives in the file-scope device array below instead of handle memory.
//
// * Size: kNoAllocScratchDoubles doubles (2*152*4 + 2*152*192 + 8, about
//   477 KB).  Every GPU that loads this library holds the array until the
//   process exits.  It covers ell <= 192 sample rows with at most 152 CTAs;
//   larger ell is rejected.
// * The array's host-side name is only a stand-in for the symbol; the first
//   call on each device looks up its device address with
//   cudaGetSymbolAddress (with that device current) and caches it.  Make that
//   first call before any stream capture.
// * Every call shares the array and it keeps the previous call's contents.
//   Each call clears the words that must start at zero (the barrier) on its
//   stream before the launch.  Calls whose kernels overlap on the GPU race on
//   the array: run them on one stream, or order them.
// * The caller's device status word is required: a timed-out wait or a
//   non-finite sample leaves dB and the swaps unusable, and the status word
//   is the only place that says so.
namespace {

constexpr int kNoAllocMaxGrid = 152;  // CTAs (one per SM, capped)
constexpr int64_t kNoAllocCand = 2LL * kNoAllocMaxGrid * 4;
constexpr int64_t kNoAllocCandCol = 2LL * kNoAllocMaxGrid * MAX_ELL;
// candidates, candidate columns, then 8 doubles for the barrier
constexpr int64_t kNoAllocScratchDoubles = kNoAllocCand + kNoAllocCandCol + 8;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once
// per device; the host-side name of the array is not a device address).
cudaError_t noalloc_scratch(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (g_noalloc_ptr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace rq

extern "C" int rqrcp_sample_qrcp_noalloc(int ell, int64_t nc, int steps, double* dB, int64_t ldb,
                                         int64_t* d_swaps, int* d_info, void* cuda_stream) {
  using namespace rq;
  if (ell < 1 || ell > MAX_ELL) return -1;
  if (nc < 1) return -2;
  if (steps < 1 || steps > ell || steps > nc) return -3;
  if (!dB) return -4;
  if (ldb < ell) return -5;
  if (!d_swaps) return -6;
  if (!d_info) return -7;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return RQRCP_ERR_CUDA;
  if (sms > kNoAllocMaxGrid) sms = kNoAllocMaxGrid;
  if (!sample_qrcp_fits(ell, nc, sms)) return RQRCP_ERR_UNSUPPORTED;
  double* scratch = nullptr;
  if (noalloc_scratch(&scratch) != cudaSuccess) return RQRCP_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  GridBarrier* bar = reinterpret_cast<GridBarrier*>(scratch + kNoAllocCand + kNoAllocCandCol);
  SampleQrcpArgs a{dB, ldb, ell, nc, steps, d_swaps, scratch, scratch + kNoAllocCand, bar, d_info};
  // launch_sample_qrcp clears the barrier words before the cooperative launch
  return launch_sample_qrcp(a, sms, st) == cudaSuccess ? RQRCP_OK : RQRCP_ERR_CUDA;
}
