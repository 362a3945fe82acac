// The CUDA-core apply for FP64 vectors in double-word FP32 arithmetic (dword.cuh): the kernel of
// apply_cc.cuh instantiated with a dd arithmetic type. A dd value is 8 bytes like a double, so the
// kernel keeps the FP64 layout of its shared cell tensors (unpadded rows, the y-lines merged into
// the x-line buffer); the vectors stay FP64 in memory and are split on load and joined on store.
// The 1D constants are the operator's FP64 ones split into dd pairs.
#include "apply_cc.cuh"
#include "dword.cuh"

namespace tp {

template <>
__device__ __forceinline__ dd load_as<double, dd>(const double* p) {
  return dd_from_double(__ldg(p));
}
template <>
__device__ __forceinline__ void store_as<double, dd>(double* p, dd v) {
  *p = dd_to_double(v);
}

namespace {

void split_const(OpConst<dd, kMaxN>& o, const OpConst<double, kMaxN>& c) {
  auto cv = [](dd* dst, const double* src, int cnt) {
    for (int e = 0; e < cnt; ++e) dst[e] = dd_from_double_host(src[e]);
  };
  for (int d = 0; d < 3; ++d) {
    cv(o.M[d], c.M[d], kMaxN * kMaxN);
    cv(o.G[d], c.G[d], kMaxN * kMaxN);
    for (int f = 0; f < 8; ++f) cv(o.E[d][f], c.E[d][f], kMaxN);
    for (int i = 0; i < kMaxN / 2; ++i) {
      cv(o.ME[d][i], c.ME[d][i], kMaxN / 2);
      cv(o.MO[d][i], c.MO[d][i], kMaxN / 2);
      cv(o.GE[d][i], c.GE[d][i], kMaxN / 2);
      cv(o.GO[d][i], c.GO[d][i], kMaxN / 2);
    }
  }
  cv(o.d0, c.d0, kMaxN);
  cv(o.d1, c.d1, kMaxN);
  o.centro = c.centro;
}

template <int N>
cudaError_t launch_dd_n(const tp_op_s* op, void* y, const void* x, long long c0, long long c1, cudaStream_t s,
                        const void* b) {
  constexpr int CPB = cc_cells_per_block<N, 1>();
  constexpr size_t smem = cc_smem_bytes<dd, N, 1>();
  static_assert(smem <= 48 * 1024, "dd tile exceeds the default shared-memory limit");
  const long long blocks = (c1 - c0 + CPB - 1) / CPB;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  if (blocks <= 0) return cudaSuccess;
  OpConst<dd, kMaxN> P;
  split_const(P, op->c64);
  if (b)
    apply_cc_kernel<double, dd, N, 1, true><<<(unsigned)blocks, N * N * CPB, smem, s>>>(
        static_cast<const double*>(x), static_cast<double*>(y), static_cast<const double*>(b), P, op->mesh.nx,
        op->mesh.ny, op->mesh.nz, c0, c1);
  else
    apply_cc_kernel<double, dd, N, 1, false><<<(unsigned)blocks, N * N * CPB, smem, s>>>(
        static_cast<const double*>(x), static_cast<double*>(y), nullptr, P, op->mesh.nx, op->mesh.ny, op->mesh.nz, c0,
        c1);
  return cudaGetLastError();
}

}  // namespace

// Output rows of cells [c0, c1) of an FP64-vector operator (n <= 8) in double-word FP32 arithmetic;
// y = A x, or y = b - A x when b is not null.
cudaError_t launch_apply_dd_range(const tp_op_s* op, void* y, const void* x, long long c0, long long c1,
                                  cudaStream_t s, const void* b) {
  switch (op->n) {
    case 2: return launch_dd_n<2>(op, y, x, c0, c1, s, b);
    case 3: return launch_dd_n<3>(op, y, x, c0, c1, s, b);
    case 4: return launch_dd_n<4>(op, y, x, c0, c1, s, b);
    case 5: return launch_dd_n<5>(op, y, x, c0, c1, s, b);
    case 6: return launch_dd_n<6>(op, y, x, c0, c1, s, b);
    case 7: return launch_dd_n<7>(op, y, x, c0, c1, s, b);
    case 8: return launch_dd_n<8>(op, y, x, c0, c1, s, b);
  }
  return cudaErrorInvalidValue;
}

}  // namespace tp
