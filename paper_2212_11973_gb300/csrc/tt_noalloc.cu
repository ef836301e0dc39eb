// QR gauge kernel without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need a
// factorisation: code running inside a memory pool that must not grow, a
// process whose allocator is owned by another framework and is not reachable
// from here, or a real-time path where a cudaMalloc (which may synchronise the
// device) is not acceptable.  tt_qr_device_noalloc serves them: its workspace is
// a fixed array in device global memory that every GPU which loads this
// library reserves for the life of the process.
//
// Scratch layout (doubles): the working copy of A (m*n), then Q (m*n) and R
// (n*n).  The job record (offsets and sizes) is a kernel argument, so the call
// queues no host-to-device copy: a copy from pageable host memory would make
// the stream wait before staging it.  The QR kernel writes every element of Q
// and R and the working copy is filled from A before the kernel runs, so
// nothing has to start at zero.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/tantrg.h"
#include "tt_kernels.h"

namespace {

constexpr size_t kScratchDoubles = size_t(1) << 21;  // 16 MiB per GPU

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

// Device address of the scratch array, looked up once per device with that
// device current.  The array's name is only a host-side handle; kernels get
// this address.
double* scratch_address(int device) {
  static std::mutex mu;
  static double* addr[256] = {nullptr};
  if (device < 0 || device >= 256) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[device]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    addr[device] = static_cast<double*>(p);
  }
  return addr[device];
}

}  // namespace

extern "C" tt_status tt_qr_device_noalloc(const double* A, int m, int n, double* Q, double* R, void* cuda_stream) {
  if (!A || !Q || !R || m < 1 || n < 1 || n > 2048 || m < n) return TT_ERR_INVALID_ARG;
  const size_t mn = (size_t)m * (size_t)n;
  if (2 * mn + (size_t)n * n > kScratchDoubles) return TT_ERR_INVALID_ARG;  // beyond the fixed scratch
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return TT_ERR_CUDA;
  }
  double* s = scratch_address(dev);
  if (!s) return TT_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  double* ws = s;
  const tt::QrJob job{0, (int64_t)mn, (int64_t)(2 * mn), m, n};
  if (cudaMemcpyAsync(ws, A, mn * sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
      tt::launch_qr_job(job, ws, st) != cudaSuccess ||
      cudaMemcpyAsync(Q, ws + mn, mn * sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(R, ws + 2 * mn, (size_t)n * n * sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
    cudaGetLastError();
    return TT_ERR_CUDA;
  }
  return TT_OK;
}
