// Householder QR for callers that cannot allocate device memory.
//
// Some callers of this library have no way to obtain device memory of their
// own: a plug-in that is handed only input and output pointers by a host
// application owning the device memory pool, a process that has already
// reserved the whole device for another runtime, or latency-critical code
// that must not enter the CUDA allocator.  qrctm_householder_qr_noalloc
// runs the same blocked Householder QR as qrctm_householder_qr, but takes its
// scratch (working copy, reflectors, panel partial sums, grid barrier, error
// word) from one file-scope device array instead of a caller workspace.
//
// The array is part of the loaded module: every device that loads the
// library holds kNoAllocScratchBytes of it until the process exits.  Host
// code never passes the array's name to a kernel (on the host that name is
// only a stand-in); it looks up the device address once per device with
// cudaGetSymbolAddress and passes that pointer.
#include <mutex>

#include "qrctm.h"
#include "qrctm_internal.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = 48ull << 20;   // 48 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_qr_scratch[kNoAllocScratchBytes];

std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_qr_scratch on the current device (looked up once).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (g_scratch_addr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_qr_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" qrctm_status qrctm_householder_qr_noalloc(int m, int n, const double* M, double* Q,
                                                     double* R, void* stream) {
  if (m < n || n < 1 || !M || !Q || !R) return QRCTM_ERR_INVALID_ARG;
  // the fixed scratch bounds the problem size (5184 x 144, the reduced corner
  // at chi = 144 and D = 6, fits with room to spare)
  if (n > 1024 || (long long)m * n > (1ll << 20) ||
      qrctm::qr_work_bytes(m, n) > kNoAllocScratchBytes)
    return QRCTM_ERR_WORKSPACE;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  void* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return QRCTM_ERR_CUDA;
  qrctm::QrWork w = qrctm::qr_carve(base, m, n);
  // the array keeps the previous call's contents: clear the barrier and the
  // error word, which must start at zero
  cudaError_t e = cudaMemsetAsync(w.bar, 0, sizeof(qrctm::GridBar), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(w.err, 0, sizeof(int), s);
  if (e != cudaSuccess) return QRCTM_ERR_CUDA;
  e = qrctm::householder_qr_f64(m, n, M, Q, R, w, s);
  if (e != cudaSuccess) return QRCTM_ERR_CUDA;
  int flag = 0;
  if (cudaMemcpyAsync(&flag, w.err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return QRCTM_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return QRCTM_ERR_CUDA;
  if (flag) return (flag & qrctm::ERRF_TIMEOUT) ? QRCTM_ERR_TIMEOUT : QRCTM_ERR_NUMERIC;
  return QRCTM_OK;
}
