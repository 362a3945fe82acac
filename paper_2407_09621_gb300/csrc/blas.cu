// Vector kernels of the Krylov and multigrid drivers: (multi-)dot products,
// (multi-)axpy, scaling and precision conversion. Dot products accumulate in
// FP64 and reduce deterministically: one partial per block written to a
// scratch array (fixed grid), then one block sums the partials in a fixed
// order, so repeated runs give bit-identical results.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "tp_internal.h"
#include "tp_vec.h"

namespace tp {

constexpr int kRedThreads = 256;

template <typename T>
__device__ __forceinline__ double to_d(T v) { return (double)v; }
template <>
__device__ __forceinline__ double to_d<__half>(__half v) { return (double)__half2float(v); }
template <>
__device__ __forceinline__ double to_d<__nv_bfloat16>(__nv_bfloat16 v) { return (double)__bfloat162float(v); }
template <typename T>
__device__ __forceinline__ T from_d(double v) { return (T)v; }
template <>
__device__ __forceinline__ __half from_d<__half>(double v) { return __float2half_rn((float)v); }
template <>
__device__ __forceinline__ __nv_bfloat16 from_d<__nv_bfloat16>(double v) { return __float2bfloat16_rn((float)v); }

// partial[q * gridDim.x + blockIdx.x] = sum over this block's grid-stride slice of w * v_q
template <typename T, int Q>
__global__ void __launch_bounds__(kRedThreads) multi_dot_partial(long long n, const T* __restrict__ w,
                                                                  MultiPtr<T> v, int nq, double* __restrict__ partial) {
  __shared__ double red[Q][kRedThreads / 32];
  double acc[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) acc[q] = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double wi = to_d(w[i]);
#pragma unroll
    for (int q = 0; q < Q; ++q)
      if (q < nq) acc[q] = fma(wi, to_d(v.p[q][i]), acc[q]);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    double s = acc[q];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) red[q][wid] = s;
  }
  __syncthreads();
  if (threadIdx.x < Q && (int)threadIdx.x < nq) {
    double s = 0.0;
    for (int k = 0; k < kRedThreads / 32; ++k) s += red[threadIdx.x][k];
    partial[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = s;
  }
}

__global__ void reduce_partials(const double* __restrict__ partial, int nblocks, int nq, double* __restrict__ out) {
  __shared__ double red[kRedThreads / 32];
  for (int q = 0; q < nq; ++q) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += partial[(size_t)q * nblocks + b];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int k = 0; k < (int)(blockDim.x / 32); ++k) t += red[k];
      out[q] = t;
    }
    __syncthreads();
  }
}

int dot_blocks(long long n) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 152;
  }
  long long want = (n + kRedThreads - 1) / kRedThreads;
  long long cap = (long long)sms * 8;
  return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

template <typename T>
cudaError_t multi_dot(long long n, const T* w, const T* const* v, int nq, double* partial, double* out,
                      cudaStream_t s) {
  const int blocks = dot_blocks(n);
  for (int q0 = 0; q0 < nq; q0 += kMaxMulti) {
    const int m = nq - q0 < kMaxMulti ? nq - q0 : kMaxMulti;
    MultiPtr<T> mp;
    for (int q = 0; q < m; ++q) mp.p[q] = v[q0 + q];
    if (m <= 1)
      multi_dot_partial<T, 1><<<blocks, kRedThreads, 0, s>>>(n, w, mp, m, partial);
    else if (m <= 4)
      multi_dot_partial<T, 4><<<blocks, kRedThreads, 0, s>>>(n, w, mp, m, partial);
    else if (m <= 8)
      multi_dot_partial<T, 8><<<blocks, kRedThreads, 0, s>>>(n, w, mp, m, partial);
    else
      multi_dot_partial<T, kMaxMulti><<<blocks, kRedThreads, 0, s>>>(n, w, mp, m, partial);
    reduce_partials<<<1, kRedThreads, 0, s>>>(partial, blocks, m, out + q0);
  }
  return cudaGetLastError();
}

// Accumulation type of the axpy: FP64 for FP64 vectors, FP32 for FP32/FP16/BF16 vectors (the
// result is rounded to the storage type; FP64 arithmetic there would only load the slow FP64 pipe).
template <typename T> struct AxpyAcc { using A = float; };
template <> struct AxpyAcc<double> { using A = double; };

template <typename A, typename T>
__device__ __forceinline__ A to_a(T v) { return (A)to_d(v); }
template <>
__device__ __forceinline__ float to_a<float, float>(float v) { return v; }
template <>
__device__ __forceinline__ float to_a<float, __half>(__half v) { return __half2float(v); }
template <>
__device__ __forceinline__ float to_a<float, __nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename T, typename A>
__device__ __forceinline__ T from_a(A v) { return from_d<T>((double)v); }
template <>
__device__ __forceinline__ float from_a<float, float>(float v) { return v; }
template <>
__device__ __forceinline__ __half from_a<__half, float>(float v) { return __float2half_rn(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 from_a<__nv_bfloat16, float>(float v) { return __float2bfloat16_rn(v); }

// w = beta * w + sum_q c[q] * v_q   (c on the host, passed by value). w may be one of the v_q:
// every entry is read and written by the same thread.
template <typename T, int Q>
__global__ void multi_axpy_kernel(long long n, T* w, double beta, MultiPtr<T> v, MultiCoef c, int nq) {
  using A = typename AxpyAcc<T>::A;
  A cq[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) cq[q] = (A)c.c[q];
  const A b = (A)beta;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    A acc = beta == 0.0 ? A(0) : b * to_a<A>(w[i]);
#pragma unroll
    for (int q = 0; q < Q; ++q)
      if (q < nq) acc = fma(cq[q], to_a<A>(v.p[q][i]), acc);
    w[i] = from_a<T>(acc);
  }
}

int stream_blocks(long long n) {
  const long long b = (n + 255) / 256;
  const long long cap = 152LL * 16;
  return (int)(b < cap ? (b > 0 ? b : 1) : cap);
}

template <typename T>
cudaError_t multi_axpy(long long n, T* w, double beta, const T* const* v, const double* c, int nq, cudaStream_t s) {
  const int blocks = stream_blocks(n);
  if (nq == 0) {
    MultiPtr<T> mp{};
    MultiCoef mc{};
    multi_axpy_kernel<T, 1><<<blocks, 256, 0, s>>>(n, w, beta, mp, mc, 0);
    return cudaGetLastError();
  }
  for (int q0 = 0; q0 < nq; q0 += kMaxMulti) {
    const int m = nq - q0 < kMaxMulti ? nq - q0 : kMaxMulti;
    MultiPtr<T> mp;
    MultiCoef mc;
    for (int q = 0; q < m; ++q) { mp.p[q] = v[q0 + q]; mc.c[q] = c[q0 + q]; }
    const double b = q0 == 0 ? beta : 1.0;
    if (m <= 1)
      multi_axpy_kernel<T, 1><<<blocks, 256, 0, s>>>(n, w, b, mp, mc, m);
    else if (m <= 4)
      multi_axpy_kernel<T, 4><<<blocks, 256, 0, s>>>(n, w, b, mp, mc, m);
    else if (m <= 8)
      multi_axpy_kernel<T, 8><<<blocks, 256, 0, s>>>(n, w, b, mp, mc, m);
    else
      multi_axpy_kernel<T, kMaxMulti><<<blocks, 256, 0, s>>>(n, w, b, mp, mc, m);
  }
  return cudaGetLastError();
}

template <typename TO, typename TI>
__global__ void convert_kernel(long long n, TO* __restrict__ out, const TI* __restrict__ in, double scale) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = from_d<TO>(scale * to_d(in[i]));
}

template <typename TO, typename TI>
cudaError_t convert(long long n, TO* out, const TI* in, double scale, cudaStream_t s) {
  convert_kernel<TO, TI><<<stream_blocks(n), 256, 0, s>>>(n, out, in, scale);
  return cudaGetLastError();
}

template cudaError_t multi_dot<double>(long long, const double*, const double* const*, int, double*, double*, cudaStream_t);
template cudaError_t multi_dot<float>(long long, const float*, const float* const*, int, double*, double*, cudaStream_t);
template cudaError_t multi_axpy<double>(long long, double*, double, const double* const*, const double*, int, cudaStream_t);
template cudaError_t multi_axpy<float>(long long, float*, double, const float* const*, const double*, int, cudaStream_t);
template cudaError_t convert<float, double>(long long, float*, const double*, double, cudaStream_t);
template cudaError_t multi_dot<__half>(long long, const __half*, const __half* const*, int, double*, double*, cudaStream_t);
template cudaError_t multi_dot<__nv_bfloat16>(long long, const __nv_bfloat16*, const __nv_bfloat16* const*, int, double*,
                                              double*, cudaStream_t);
template cudaError_t multi_axpy<__half>(long long, __half*, double, const __half* const*, const double*, int, cudaStream_t);
template cudaError_t multi_axpy<__nv_bfloat16>(long long, __nv_bfloat16*, double, const __nv_bfloat16* const*,
                                               const double*, int, cudaStream_t);
template cudaError_t convert<__half, double>(long long, __half*, const double*, double, cudaStream_t);
template cudaError_t convert<double, __half>(long long, double*, const __half*, double, cudaStream_t);
template cudaError_t convert<__nv_bfloat16, double>(long long, __nv_bfloat16*, const double*, double, cudaStream_t);
template cudaError_t convert<double, __nv_bfloat16>(long long, double*, const __nv_bfloat16*, double, cudaStream_t);
template cudaError_t convert<double, float>(long long, double*, const float*, double, cudaStream_t);
template cudaError_t convert<double, double>(long long, double*, const double*, double, cudaStream_t);
template cudaError_t convert<float, float>(long long, float*, const float*, double, cudaStream_t);

}  // namespace tp

namespace tp {

// w = w - sum_q coef[q] v_q (coef on the DEVICE), then, in the same pass, partial dot products of the
// updated w with every v_q (if with_dots) and with itself: partial[q * gridDim.x + block], q = 0..nq
// (q = nq is |w|^2).
template <typename T, int Q>
__global__ void __launch_bounds__(kRedThreads) multi_axpy_dot_partial(long long n, T* w, MultiPtr<T> v,
                                                                       const double* __restrict__ coef, int nq,
                                                                       int with_dots, double* __restrict__ partial) {
  __shared__ double red[Q + 1][kRedThreads / 32];
  double c[Q], acc[Q + 1];
#pragma unroll
  for (int q = 0; q < Q; ++q) c[q] = q < nq ? coef[q] : 0.0;
#pragma unroll
  for (int q = 0; q <= Q; ++q) acc[q] = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double wi = to_d(w[i]);
    double vi[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      vi[q] = q < nq ? to_d(v.p[q][i]) : 0.0;
      wi = fma(-c[q], vi[q], wi);
    }
    w[i] = (T)wi;
    if (with_dots) {
#pragma unroll
      for (int q = 0; q < Q; ++q) acc[q] = fma(wi, vi[q], acc[q]);
    }
    acc[Q] = fma(wi, wi, acc[Q]);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q <= Q; ++q) {
    double s = acc[q];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) red[q][wid] = s;
  }
  __syncthreads();
  if ((int)threadIdx.x <= nq) {
    const int q = (int)threadIdx.x == nq ? Q : (int)threadIdx.x;
    double s = 0.0;
    for (int k = 0; k < kRedThreads / 32; ++k) s += red[q][k];
    partial[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = s;
  }
}

// out = in / sqrt(*nrm2) (nrm2 on the device)
template <typename T>
__global__ void scale_inv_sqrt_kernel(long long n, T* __restrict__ out, const T* __restrict__ in,
                                      const double* __restrict__ nrm2) {
  const double s = 1.0 / sqrt(*nrm2);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = (T)(s * to_d(in[i]));
}

template <typename T>
cudaError_t multi_axpy_dot(long long n, T* w, const T* const* v, const double* coef_dev, int nq, int with_dots,
                           double* partial, double* out, cudaStream_t s) {
  if (nq > kMaxMulti) {
    // longer bases: axpy chunk by chunk, then one dot/norm pass
    for (int q0 = 0; q0 < nq; q0 += kMaxMulti) {
      const int m = nq - q0 < kMaxMulti ? nq - q0 : kMaxMulti;
      MultiPtr<T> mp;
      for (int q = 0; q < m; ++q) mp.p[q] = v[q0 + q];
      multi_axpy_dot_partial<T, kMaxMulti><<<dot_blocks(n), kRedThreads, 0, s>>>(n, w, mp, coef_dev + q0, m, 0,
                                                                                 partial);
    }
    cudaError_t e = with_dots ? multi_dot<T>(n, w, v, nq, partial, out, s) : cudaSuccess;
    if (e != cudaSuccess) return e;
    const T* self[1] = {w};
    return multi_dot<T>(n, w, self, 1, partial, out + nq, s);
  }
  const int blocks = dot_blocks(n);
  MultiPtr<T> mp;
  for (int q = 0; q < nq; ++q) mp.p[q] = v[q];
  if (nq <= 4)
    multi_axpy_dot_partial<T, 4><<<blocks, kRedThreads, 0, s>>>(n, w, mp, coef_dev, nq, with_dots, partial);
  else if (nq <= 8)
    multi_axpy_dot_partial<T, 8><<<blocks, kRedThreads, 0, s>>>(n, w, mp, coef_dev, nq, with_dots, partial);
  else
    multi_axpy_dot_partial<T, kMaxMulti><<<blocks, kRedThreads, 0, s>>>(n, w, mp, coef_dev, nq, with_dots, partial);
  reduce_partials<<<1, kRedThreads, 0, s>>>(partial, blocks, nq + 1, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t scale_inv_sqrt(long long n, T* out, const T* in, const double* nrm2_dev, cudaStream_t s) {
  scale_inv_sqrt_kernel<T><<<stream_blocks(n), 256, 0, s>>>(n, out, in, nrm2_dev);
  return cudaGetLastError();
}

template cudaError_t multi_axpy_dot<double>(long long, double*, const double* const*, const double*, int, int,
                                            double*, double*, cudaStream_t);
template cudaError_t scale_inv_sqrt<double>(long long, double*, const double*, const double*, cudaStream_t);

}  // namespace tp
