// The reconstruction-error pass for callers that cannot allocate device memory.
//
// Some callers must not call cudaMalloc.  Examples: a host framework whose own
// caching allocator already holds the device's memory; code that runs under a
// fixed, pre-planned memory budget; or a pipeline that cannot afford the
// implicit device-wide synchronisation of cudaMalloc and cudaFree.
// id_reconstruct_error_noalloc serves them.  It runs the same error-pass
// kernels as id_reconstruct_error, but every scratch buffer (per-CTA partial
// sums, the three result scalars, and staging copies of J and P) lives in one
// file-scope device array of fixed size.  The library never allocates for it.
//
// The array costs about 1.1 MB on every GPU that loads the library, and each
// such GPU keeps it until the process exits.  Host code cannot use the
// array's name as a device address: on the host that name is only a
// stand-in, and a kernel handed it would fault, or, where the GPU can reach
// host memory, silently use the wrong memory.  So the first call on each
// device, with that device current, looks the address up once with
// cudaGetSymbolAddress and keeps it.  That first call should come before any
// stream capture.  All calls on a device share the array, and it keeps the
// last call's contents.  Nothing in it needs clearing: every slot a call
// reads was written earlier in the same call, and the one word that must start
// at zero (the timeout flag) is cleared at the start of every call.  Calls
// that overlap on the GPU (e.g. on two streams) race on the array.
#include <math.h>

#include <algorithm>
#include <mutex>

#include "idsk_internal.h"

namespace {

constexpr int kMaxBlocks = 2048;                      // partial-sum slots
constexpr size_t kPartOff = 0;                        // 3 doubles per CTA
constexpr size_t kOutOff = 3 * (size_t)kMaxBlocks;    // 3 result scalars, then the status word
constexpr size_t kJOff = kOutOff + 4;                 // kRecKMax int32 = 32 doubles
constexpr size_t kPOff = kJOff + idsk::kRecKMax / 2;  // P, up to ID_NOALLOC_MAX_KN
constexpr size_t kTotal = kPOff + (size_t)ID_NOALLOC_MAX_KN;

static __device__ __align__(256) double g_noalloc_scratch[kTotal];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array for the current device (looked up once).
cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = static_cast<double*>(p);
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" id_status id_reconstruct_error_noalloc(const void* d_A, int64_t lda, int64_t m,
                                                  int64_t n, int32_t dtype, const int32_t* J,
                                                  const double* P, int32_t k, double* rel_fro,
                                                  double* rel_max, void* cuda_stream) {
  if (!d_A || !J || !P || m < 1 || lda < m || n < 1 || k < 1 || k > idsk::kRecKMax)
    return ID_ERR_INVALID_ARG;
  if (dtype != ID_F32 && dtype != ID_F64) return ID_ERR_INVALID_ARG;
  if ((int64_t)k * n > (int64_t)ID_NOALLOC_MAX_KN) return ID_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  double* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return ID_ERR_CUDA;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return ID_ERR_CUDA;
  int32_t jh[idsk::kRecKMax];
  if (cudaMemcpyAsync(jh, J, sizeof(int32_t) * k, cudaMemcpyDefault, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return ID_ERR_CUDA;
  for (int u = 0; u < k; ++u)
    if (jh[u] < 0 || jh[u] >= n) return ID_ERR_INVALID_ARG;
  int* dJ = reinterpret_cast<int*>(base + kJOff);
  double* dP = base + kPOff;
  if (cudaMemcpyAsync(dJ, jh, sizeof(int32_t) * k, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(dP, P, sizeof(double) * k * n, cudaMemcpyDefault, st) != cudaSuccess)
    return ID_ERR_CUDA;
  const int nblk = std::min(8 * nsm, kMaxBlocks);
  int* dstatus = reinterpret_cast<int*>(base + kOutOff + 3);   // cleared for this call
  if (cudaMemsetAsync(dstatus, 0, sizeof(int), st) != cudaSuccess) return ID_ERR_CUDA;
  if (idsk::launch_recon_error(d_A, lda, m, n, dtype, dJ, dP, k, base + kPartOff, nblk,
                               base + kOutOff, dstatus, st) != cudaSuccess)
    return ID_ERR_CUDA;
  double o[3];
  int flag = 0;
  if (cudaMemcpyAsync(o, base + kOutOff, sizeof(o), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(&flag, dstatus, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return ID_ERR_CUDA;
  if (flag) return ID_ERR_TIMEOUT;
  if (rel_fro) *rel_fro = o[1] > 0.0 ? sqrt(o[0] / o[1]) : 0.0;
  if (rel_max) *rel_max = o[2];
  return ID_OK;
}
