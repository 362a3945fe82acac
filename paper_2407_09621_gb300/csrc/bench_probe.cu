// FMA-pipe peak probe (measurement support for the roofline, include/tp_bench.h).
#include <cuda_runtime.h>

#include "../../include/tp_bench.h"
#include "tp_internal.h"

namespace tp {

template <typename T, int ILP>
__global__ void fma_probe_kernel(T* out, int iters, T a, T b) {
  T acc[ILP];
#pragma unroll
  for (int i = 0; i < ILP; ++i) acc[i] = (T)(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < ILP; ++i) acc[i] = fma(acc[i], a, b);
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < ILP; ++i) s += acc[i];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
static tp_status run_probe(double* tflops, cudaStream_t s, int iters) {
  int dev = 0, sms = 0;
  tp_status st = cuda_status(cudaGetDevice(&dev), "cudaGetDevice");
  if (st != TP_OK) return st;
  st = cuda_status(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "cudaDeviceGetAttribute");
  if (st != TP_OK) return st;
  const int blocks = sms * 4, threads = 256;
  T* buf = nullptr;
  st = cuda_status(cudaMalloc(&buf, sizeof(T) * blocks * threads), "cudaMalloc(probe)");
  if (st != TP_OK) return st;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int r = 0; r < 7; ++r) {
    cudaEventRecord(e0, s);
    fma_probe_kernel<T, 8><<<blocks, threads, 0, s>>>(buf, iters, (T)1.0000001, (T)1e-7);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (r >= 2 && ms < best) best = ms;
  }
  st = cuda_status(cudaGetLastError(), "fma probe");
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  if (st != TP_OK) return st;
  *tflops = 2.0 * 8.0 * iters * (double)blocks * threads / (best * 1e-3) / 1e12;
  return TP_OK;
}

}  // namespace tp

extern "C" tp_status tp_bench_fma_peak(int precision, double* tflops, void* stream) {
  using namespace tp;
  if (!tflops) { set_error("tp_bench_fma_peak: NULL output"); return TP_ERR_INVALID_ARG; }
  if (precision == TP_FP64) return run_probe<double>(tflops, (cudaStream_t)stream, 4096);
  if (precision == TP_FP32) return run_probe<float>(tflops, (cudaStream_t)stream, 65536);
  set_error("tp_bench_fma_peak: precision must be TP_FP64 or TP_FP32");
  return TP_ERR_INVALID_ARG;
}
