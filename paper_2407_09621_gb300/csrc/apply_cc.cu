// Sum-factorized SIPG Laplace apply on the FMA pipes ("CUDA-core" kernel): the instantiations
// for n = k + 1 <= 8 in all four vector precisions and the dispatch over n (the kernel itself
// and its derivation are in apply_cc.cuh; 8 < n <= 16 is instantiated in apply_cc_high.cu).
#include "apply_cc.cuh"

namespace tp {

// n = 2 with FP32 arithmetic: one thread per cell (apply_cpt.cu)
cudaError_t launch_apply_cpt_range(const tp_op_s* op, void* y, const void* x, long long c0, long long c1,
                                   cudaStream_t s, const void* b);

// The CUDA-core apply of this operator runs the cell-per-thread kernel (one tile shape, 128 cells
// per block) instead of the line-per-thread one.
bool cc_cell_per_thread(const tp_op_s* op) { return op->n == 2 && op->prec != TP_FP64; }

// FP64 vectors in double-word FP32 arithmetic (apply_dd.cu)
cudaError_t launch_apply_dd_range(const tp_op_s* op, void* y, const void* x, long long c0, long long c1,
                                  cudaStream_t s, const void* b);

// n > 8, FP64 and FP32 vectors (apply_cc_high.cu)
cudaError_t prepare_apply_cc_high(const tp_op_s* op);
cudaError_t launch_apply_cc_high(const tp_op_s* op, void* y, const void* x, long long c0, long long c1,
                                 cudaStream_t s, const void* b);

template <typename TS, typename TC>
static cudaError_t prepare_cc_t(int n) {
  switch (n) {
    case 2: return prepare_cc_n<TS, TC, 2>();
    case 3: return prepare_cc_n<TS, TC, 3>();
    case 4: return prepare_cc_n<TS, TC, 4>();
    case 5: return prepare_cc_n<TS, TC, 5>();
    case 6: return prepare_cc_n<TS, TC, 6>();
    case 7: return prepare_cc_n<TS, TC, 7>();
    case 8: return prepare_cc_n<TS, TC, 8>();
  }
  return cudaErrorInvalidValue;
}

// Sets the dynamic shared-memory limit of the kernel instantiation on the current device.
cudaError_t prepare_apply_cc(const tp_op_s* op) {
  if (op->n > kMaxN) return prepare_apply_cc_high(op);
  switch (op->prec) {
    case TP_FP64: return prepare_cc_t<double, double>(op->n);
    case TP_FP32: return prepare_cc_t<float, float>(op->n);
    case TP_FP16: return prepare_cc_t<__half, float>(op->n);
    case TP_BF16: return prepare_cc_t<__nv_bfloat16, float>(op->n);
  }
  return cudaErrorInvalidValue;
}

template <typename TS, typename TC>
static cudaError_t launch_cc_t(const tp_op_s* op, void* y, const void* x, long long c0, long long c1, cudaStream_t s,
                               const void* b) {
  switch (op->n) {
    case 2: return launch_cc_n<TS, TC, 2>(op, y, x, c0, c1, s, b);
    case 3: return launch_cc_n<TS, TC, 3>(op, y, x, c0, c1, s, b);
    case 4: return launch_cc_n<TS, TC, 4>(op, y, x, c0, c1, s, b);
    case 5: return launch_cc_n<TS, TC, 5>(op, y, x, c0, c1, s, b);
    case 6: return launch_cc_n<TS, TC, 6>(op, y, x, c0, c1, s, b);
    case 7: return launch_cc_n<TS, TC, 7>(op, y, x, c0, c1, s, b);
    case 8: return launch_cc_n<TS, TC, 8>(op, y, x, c0, c1, s, b);
  }
  return cudaErrorInvalidValue;
}

// cells per block of the CUDA-core launch for n nodes and tile variant v (n > 8: one cell,
// whatever v)
int cc_tile_cells(int n, int v) {
  if (n > kMaxN) return 1;
  const int base = (128 / (n * n)) > 0 ? 128 / (n * n) : 1;
  return v == 0 ? (base / 2 > 0 ? base / 2 : 1) : (v == 1 ? base : 2 * base);
}

// Output rows of cells [c0, c1) only (the input is read wherever those cells' faces reach);
// y = A x, or y = b - A x when b is not null (b and y must not overlap x).
cudaError_t launch_apply_cc_range(const tp_op_s* op, void* y, const void* x, long long c0, long long c1,
                                  cudaStream_t s, const void* b) {
  if (op->n > kMaxN) return launch_apply_cc_high(op, y, x, c0, c1, s, b);
  if (cc_cell_per_thread(op)) return launch_apply_cpt_range(op, y, x, c0, c1, s, b);
  switch (op->prec) {
    case TP_FP64:
      return op->opts.dword ? launch_apply_dd_range(op, y, x, c0, c1, s, b)
                            : launch_cc_t<double, double>(op, y, x, c0, c1, s, b);
    case TP_FP32: return launch_cc_t<float, float>(op, y, x, c0, c1, s, b);
    case TP_FP16: return launch_cc_t<__half, float>(op, y, x, c0, c1, s, b);
    case TP_BF16: return launch_cc_t<__nv_bfloat16, float>(op, y, x, c0, c1, s, b);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_apply_cc(const tp_op_s* op, void* y, const void* x, cudaStream_t s) {
  return launch_apply_cc_range(op, y, x, 0, op->ncells, s, nullptr);
}

}  // namespace tp
