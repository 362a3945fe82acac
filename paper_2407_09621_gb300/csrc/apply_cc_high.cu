// The CUDA-core apply (apply_cc.cuh) for degrees 8 <= k <= 15 (9 <= n <= 16), FP64 and FP32
// vectors: one cell of n^2 threads per block. Its own translation unit so that the build
// compiles it in parallel with the n <= 8 instantiations.
#include "apply_cc.cuh"

namespace tp {

template <typename T>
static cudaError_t prepare_high_t(int n) {
  switch (n) {
    case 9: return prepare_cc_n<T, T, 9>();
    case 10: return prepare_cc_n<T, T, 10>();
    case 11: return prepare_cc_n<T, T, 11>();
    case 12: return prepare_cc_n<T, T, 12>();
    case 13: return prepare_cc_n<T, T, 13>();
    case 14: return prepare_cc_n<T, T, 14>();
    case 15: return prepare_cc_n<T, T, 15>();
    case 16: return prepare_cc_n<T, T, 16>();
  }
  return cudaErrorInvalidValue;
}

template <typename T>
static cudaError_t launch_high_t(const tp_op_s* op, void* y, const void* x, long long c0, long long c1,
                                 cudaStream_t s, const void* b) {
  switch (op->n) {
    case 9: return launch_cc_n<T, T, 9>(op, y, x, c0, c1, s, b);
    case 10: return launch_cc_n<T, T, 10>(op, y, x, c0, c1, s, b);
    case 11: return launch_cc_n<T, T, 11>(op, y, x, c0, c1, s, b);
    case 12: return launch_cc_n<T, T, 12>(op, y, x, c0, c1, s, b);
    case 13: return launch_cc_n<T, T, 13>(op, y, x, c0, c1, s, b);
    case 14: return launch_cc_n<T, T, 14>(op, y, x, c0, c1, s, b);
    case 15: return launch_cc_n<T, T, 15>(op, y, x, c0, c1, s, b);
    case 16: return launch_cc_n<T, T, 16>(op, y, x, c0, c1, s, b);
  }
  return cudaErrorInvalidValue;
}

cudaError_t prepare_apply_cc_high(const tp_op_s* op) {
  switch (op->prec) {
    case TP_FP64: return prepare_high_t<double>(op->n);
    case TP_FP32: return prepare_high_t<float>(op->n);
    default: break;
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_apply_cc_high(const tp_op_s* op, void* y, const void* x, long long c0, long long c1,
                                 cudaStream_t s, const void* b) {
  switch (op->prec) {
    case TP_FP64: return launch_high_t<double>(op, y, x, c0, c1, s, b);
    case TP_FP32: return launch_high_t<float>(op, y, x, c0, c1, s, b);
    default: break;
  }
  return cudaErrorInvalidValue;
}

}  // namespace tp
