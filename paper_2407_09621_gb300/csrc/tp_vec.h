// Internal vector-kernel interface (blas.cu) used by the multigrid and FGMRES drivers.
#pragma once

#include <cuda_runtime.h>

namespace tp {

constexpr int kMaxMulti = 16;  // vectors per fused multi-dot / multi-axpy launch

template <typename T>
struct MultiPtr {
  const T* p[kMaxMulti];
};
struct MultiCoef {
  double c[kMaxMulti];
};

// Blocks used by multi_dot for n entries; `partial` must hold nq_chunk * dot_blocks(n) doubles
// with nq_chunk = min(nq, kMaxMulti).
int dot_blocks(long long n);
int stream_blocks(long long n);

// out[q] = sum_i w[i] * v[q][i] for q < nq, FP64 accumulation, deterministic.
// out is a DEVICE array of nq doubles; partial is device scratch.
template <typename T>
cudaError_t multi_dot(long long n, const T* w, const T* const* v, int nq, double* partial, double* out,
                      cudaStream_t s);

// w = beta*w + sum_q c[q] v[q]; c is a host array (copied into the launch).
template <typename T>
cudaError_t multi_axpy(long long n, T* w, double beta, const T* const* v, const double* c, int nq, cudaStream_t s);

// w -= sum_q coef_dev[q] v[q] (coefficients read on the device), and in the same pass
// out[q] = v[q].w_new (if with_dots, else 0) for q < nq and out[nq] = |w_new|^2.
// `partial` must hold (min(nq, kMaxMulti) + 1) * dot_blocks(n) doubles; out has nq + 1 entries.
template <typename T>
cudaError_t multi_axpy_dot(long long n, T* w, const T* const* v, const double* coef_dev, int nq, int with_dots,
                           double* partial, double* out, cudaStream_t s);

// out = in / sqrt(*nrm2_dev)
template <typename T>
cudaError_t scale_inv_sqrt(long long n, T* out, const T* in, const double* nrm2_dev, cudaStream_t s);

// out = scale * in (with conversion).
template <typename TO, typename TI>
cudaError_t convert(long long n, TO* out, const TI* in, double scale, cudaStream_t s);

}  // namespace tp
