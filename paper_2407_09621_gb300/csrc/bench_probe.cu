// Measurement support (include/tp_bench.h): the FMA-pipe peak probe for the roofline, and the
// tcgen05.mma issue-rate probe behind the tensor-core apply's design.
// Built as its own library, libtp_bench.so, beside libtp.so; the method's library does not
// contain it.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <vector>

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


// ------------------------------------------------------------------ tcgen05.mma issue rate
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
// K-major, 128-byte swizzle, 8-row groups 1024 bytes apart
__device__ __forceinline__ uint64_t sw128(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) |
         ((uint64_t)2 << 61);
}
__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// One CTA per SM; ISS warps each issue `reps` x 4 products (M = 128, N = n, K = 16, FP16 operands of
// zeros, FP32 accumulators) into their own TMEM columns, A from shared memory (ts = 0) or from TMEM
// (ts = 1, columns 448..479), B from shared memory. out[2 blk] = cycles of warp 0 from its first
// issue until its products are done. Every wait is bounded (1 s): on a timeout *err = 1.
template <int ISS>
__global__ void __launch_bounds__(128, 1) umma_issue_kernel(int n, int ts, int reps, long long* out, int* err) {
  extern __shared__ unsigned char sm_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)sm_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sA = base;           // 128 rows x 128 bytes
  unsigned char* sB = base + 16384;   // up to 256 rows x 128 bytes
  uint64_t* bar = reinterpret_cast<uint64_t*>(base + 49152);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(base + 49152 + 64);
  for (int i = threadIdx.x; i < 49152 / 16; i += 128) reinterpret_cast<uint4*>(base)[i] = make_uint4(0, 0, 0, 0);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(ISS));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)), "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const int who = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0 && who < ISS) {
    const uint32_t idesc = (1u << 4) | (((uint32_t)n >> 3) << 17) | ((128u >> 4) << 24);
    uint64_t bd[4], ad[4];
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
      bd[ks] = sw128(smem_u32(sB) + ks * 32);
      ad[ks] = sw128(smem_u32(sA) + ks * 32);
    }
    const uint32_t dcol = tmem + (uint32_t)(who * n);
    const long long t0 = clock64();
    for (int r = 0; r < reps; ++r) {
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {
        if (ts)
          asm volatile("tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, 1;\n"
                       ::"r"(dcol), "r"(tmem + 448u + 8u * ks), "l"(bd[ks]), "r"(idesc));
        else
          asm volatile("tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, 1;\n"
                       ::"r"(dcol), "l"(ad[ks]), "l"(bd[ks]), "r"(idesc));
      }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
    const uint64_t w0 = globaltimer();
    uint32_t ok = 0;
    for (int it = 0; it < (1 << 24) && !ok; ++it) {
      asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                   : "=r"(ok)
                   : "r"(smem_u32(bar)), "r"(0)
                   : "memory");
      if (!ok && (it & 31) == 31 && globaltimer() - w0 > 1000000000ull) break;
    }
    if (!ok) atomicExch(err, 1);
    if (who == 0) out[blockIdx.x] = clock64() - t0;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
}

template <int ISS>
tp_status run_umma_issue(int n, int ts, double* clk, double* tflops, cudaStream_t s) {
  int dev = 0, sms = 0;
  tp_status st = probe_status(cudaGetDevice(&dev), "cudaGetDevice");
  if (st == TP_OK) st = probe_status(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "cudaDeviceGetAttribute");
  if (st != TP_OK) return st;
  const int smem = 120 * 1024, reps = 2048 / ISS;
  st = probe_status(cudaFuncSetAttribute(umma_issue_kernel<ISS>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
                    "cudaFuncSetAttribute");
  if (st != TP_OK) return st;
  long long* d_out = nullptr;
  int* d_err = nullptr;
  st = probe_status(cudaMalloc(&d_out, sizeof(long long) * sms), "cudaMalloc(probe)");
  if (st == TP_OK) st = probe_status(cudaMalloc(&d_err, sizeof(int)), "cudaMalloc(probe)");
  if (st == TP_OK) st = probe_status(cudaMemsetAsync(d_err, 0, sizeof(int), s), "cudaMemsetAsync");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (st == TP_OK) st = probe_status(cudaEventCreate(&e0), "cudaEventCreate");
  if (st == TP_OK) st = probe_status(cudaEventCreate(&e1), "cudaEventCreate");
  float best = 1e30f;
  for (int r = 0; r < 5 && st == TP_OK; ++r) {
    cudaEventRecord(e0, s);
    umma_issue_kernel<ISS><<<sms, 128, smem, s>>>(n, ts, reps, d_out, d_err);
    cudaEventRecord(e1, s);
    st = probe_status(cudaEventSynchronize(e1), "tcgen05 issue probe");
    float ms = 0;
    if (st == TP_OK) st = probe_status(cudaEventElapsedTime(&ms, e0, e1), "tcgen05 issue probe timing");
    if (st == TP_OK && r >= 2 && ms < best) best = ms;
  }
  if (st == TP_OK) st = probe_status(cudaGetLastError(), "tcgen05 issue probe");
  int herr = 0;
  std::vector<long long> h(sms);
  if (st == TP_OK) st = probe_status(cudaMemcpy(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost), "cudaMemcpy");
  if (st == TP_OK) st = probe_status(cudaMemcpy(h.data(), d_out, sizeof(long long) * sms, cudaMemcpyDeviceToHost), "cudaMemcpy");
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(d_out);
  cudaFree(d_err);
  if (st != TP_OK) return st;
  if (herr) {
    snprintf(g_bench_err, sizeof(g_bench_err), "tcgen05 issue probe: a bounded wait gave up");
    return TP_ERR_TIMEOUT;
  }
  double cyc = 0.0;
  for (long long v : h) cyc += (double)v;
  cyc /= sms;
  const double nmma = 4.0 * reps * ISS;  // products per CTA
  *clk = cyc / nmma;
  *tflops = 2.0 * 128.0 * n * 16.0 * nmma * sms / (best * 1e-3) / 1e12;
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

extern "C" tp_status tp_bench_umma_issue(int n, int issuers, int a_in_tmem, double* clk_per_mma, double* tflops,
                                         void* stream) {
  if (!clk_per_mma || !tflops) {
    snprintf(g_bench_err, sizeof(g_bench_err), "tp_bench_umma_issue: NULL output");
    return TP_ERR_INVALID_ARG;
  }
  if ((n != 64 && n != 128 && n != 192 && n != 256) || (issuers != 1 && issuers != 2 && issuers != 4) ||
      n * issuers > (a_in_tmem ? 448 : 512)) {
    snprintf(g_bench_err, sizeof(g_bench_err),
             "tp_bench_umma_issue: n must be 64/128/192/256, issuers 1/2/4, n x issuers <= 512 (448 with A in TMEM)");
    return TP_ERR_INVALID_ARG;
  }
  const int ts = a_in_tmem ? 1 : 0;
  cudaStream_t s = (cudaStream_t)stream;
  if (issuers == 1) return run_umma_issue<1>(n, ts, clk_per_mma, tflops, s);
  if (issuers == 2) return run_umma_issue<2>(n, ts, clk_per_mma, tflops, s);
  return run_umma_issue<4>(n, ts, clk_per_mma, tflops, s);
}
