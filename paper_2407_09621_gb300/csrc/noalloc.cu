// Host-buffer apply that allocates no device memory (no counterpart in the paper).
//
// tp_apply_host stages the host vectors through device buffers it allocates
// with cudaMalloc on first use. Some callers cannot allow that: a process
// whose device memory is handed out by its own fixed pool or budget (every
// byte reserved up front), or a caller that must not hit the allocator's
// latency or its out-of-memory failure in the middle of its work. This
// variant stages through a statically sized array in device memory, so the
// call itself only copies and launches. CUDA loads this file's module lazily
// (by default), so the array is placed on a device at the first call there,
// when cudaGetSymbolAddress needs it; that call then fails cleanly if the
// device has no room left for it.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "tp_internal.h"

namespace tp {

tp_status cuda_status(int err, const char* what);
cudaError_t launch_apply(const tp_op_s* op, void* y, const void* x, cudaStream_t s);
size_t elem_bytes(tp_precision p);

// Two halves: x staging, then y staging. Held by every GPU that loads the
// library until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_stage[2 * TP_NOALLOC_MAX_BYTES];

// Device address of g_noalloc_stage per device ordinal, looked up once per
// device (the name is a host-side stand-in, not a device address). Kept for
// the life of the process: it does not survive cudaDeviceReset.
static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[256] = {};

static tp_status noalloc_stage_address(void** out) {
  int dev = 0;
  tp_status st = cuda_status(cudaGetDevice(&dev), "tp_apply_host_noalloc: cudaGetDevice");
  if (st != TP_OK) return st;
  if (dev < 0 || dev >= 256) {
    set_error("tp_apply_host_noalloc: device ordinal %d out of range", dev);
    return TP_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_stage);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error("tp_apply_host_noalloc: the static staging array (%d bytes) is unavailable on device %d: "
                "loading it failed (%s); make the first call on a device before its memory is reserved",
                2 * TP_NOALLOC_MAX_BYTES, dev, cudaGetErrorString(e));
      return TP_ERR_CUDA;
    }
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return TP_OK;
}

}  // namespace tp

extern "C" tp_status tp_apply_host_noalloc(tp_op op, void* y_host, const void* x_host, void* stream) {
  using namespace tp;
  if (!op || !x_host || !y_host) {
    set_error("tp_apply_host_noalloc: NULL argument");
    return TP_ERR_INVALID_ARG;
  }
  const size_t bytes = (size_t)op->ndofs * elem_bytes(op->prec);
  if (bytes > (size_t)TP_NOALLOC_MAX_BYTES) {
    set_error("tp_apply_host_noalloc: vector of %zu bytes exceeds the %d-byte limit of the static staging array",
              bytes, TP_NOALLOC_MAX_BYTES);
    return TP_ERR_INVALID_ARG;
  }
  const uintptr_t xa = (uintptr_t)x_host, ya = (uintptr_t)y_host;
  if (xa < ya + bytes && ya < xa + bytes) {
    set_error("tp_apply_host_noalloc: x and y overlap");
    return TP_ERR_INVALID_ARG;
  }
  int dev = -1;
  tp_status st = cuda_status(cudaGetDevice(&dev), "tp_apply_host_noalloc: cudaGetDevice");
  if (st != TP_OK) return st;
  if (dev != op->device) {
    set_error("tp_apply_host_noalloc: device %d is current, the operator lives on device %d", dev, op->device);
    return TP_ERR_INVALID_ARG;
  }
  void* base = nullptr;
  st = noalloc_stage_address(&base);
  if (st != TP_OK) return st;
  // Both halves are fully overwritten by every call (copy in, kernel out): nothing needs clearing.
  unsigned char* dx = static_cast<unsigned char*>(base);
  unsigned char* dy = dx + TP_NOALLOC_MAX_BYTES;
  cudaStream_t s = (cudaStream_t)stream;
  st = cuda_status(cudaMemcpyAsync(dx, x_host, bytes, cudaMemcpyHostToDevice, s), "tp_apply_host_noalloc H2D");
  if (st == TP_OK) st = cuda_status(launch_apply(op, dy, dx, s), "tp_apply_host_noalloc launch");
  if (st == TP_OK)
    st = cuda_status(cudaMemcpyAsync(y_host, dy, bytes, cudaMemcpyDeviceToHost, s), "tp_apply_host_noalloc D2H");
  if (st == TP_OK) st = cuda_status(cudaStreamSynchronize(s), "tp_apply_host_noalloc sync");
  return st;
}
