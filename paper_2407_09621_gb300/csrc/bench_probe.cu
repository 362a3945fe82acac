// FMA-pipe peak probe: measurement support for the roofline (include/tp_bench.h).
// Built as its own library, libtp_bench.so, beside libtp.so; the method's library does not
// contain it.
#include <cuda_runtime.h>

#include <cstdio>

#include "../../include/tp_bench.h"

namespace {

thread_local char g_bench_err[256] = "";

tp_status probe_status(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return TP_OK;
  snprintf(g_bench_err, sizeof(g_bench_err), "%s: %s", what, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? TP_ERR_OOM : TP_ERR_CUDA;
}

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
tp_status run_probe(double* tflops, cudaStream_t s, int iters) {
  int dev = 0, sms = 0;
  tp_status st = probe_status(cudaGetDevice(&dev), "cudaGetDevice");
  if (st != TP_OK) return st;
  st = probe_status(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "cudaDeviceGetAttribute");
  if (st != TP_OK) return st;
  const int blocks = sms * 4, threads = 256;
  T* buf = nullptr;
  st = probe_status(cudaMalloc(&buf, sizeof(T) * blocks * threads), "cudaMalloc(probe)");
  if (st != TP_OK) return st;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  st = probe_status(cudaEventCreate(&e0), "cudaEventCreate");
  if (st == TP_OK) st = probe_status(cudaEventCreate(&e1), "cudaEventCreate");
  float best = 1e30f;
  for (int r = 0; r < 7 && st == TP_OK; ++r) {
    cudaEventRecord(e0, s);
    fma_probe_kernel<T, 8><<<blocks, threads, 0, s>>>(buf, iters, (T)1.0000001, (T)1e-7);
    cudaEventRecord(e1, s);
    st = probe_status(cudaEventSynchronize(e1), "fma probe");
    float ms = 0;
    if (st == TP_OK) st = probe_status(cudaEventElapsedTime(&ms, e0, e1), "fma probe timing");
    if (st == TP_OK && r >= 2 && ms < best) best = ms;
  }
  if (st == TP_OK) st = probe_status(cudaGetLastError(), "fma probe");
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(buf);
  if (st != TP_OK) return st;
  *tflops = 2.0 * 8.0 * iters * (double)blocks * threads / (best * 1e-3) / 1e12;
  return TP_OK;
}

}  // namespace

extern "C" tp_status tp_bench_fma_peak(int precision, double* tflops, void* stream) {
  if (!tflops) {
    snprintf(g_bench_err, sizeof(g_bench_err), "tp_bench_fma_peak: NULL output");
    return TP_ERR_INVALID_ARG;
  }
  if (precision == TP_FP64) return run_probe<double>(tflops, (cudaStream_t)stream, 4096);
  if (precision == TP_FP32) return run_probe<float>(tflops, (cudaStream_t)stream, 65536);
  snprintf(g_bench_err, sizeof(g_bench_err), "tp_bench_fma_peak: precision must be TP_FP64 or TP_FP32");
  return TP_ERR_INVALID_ARG;
}

extern "C" const char* tp_bench_last_error(void) { return g_bench_err; }
