// Device helpers shared by the apply kernels: typed loads/stores of the vector storage types
// and the rank-2 face terms of the inverse-mass form (see apply_cc.cu for their derivation).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "tp_internal.h"

namespace tp {

template <typename TS, typename TC>
__device__ __forceinline__ TC load_as(const TS* p) { return static_cast<TC>(__ldg(p)); }
template <>
__device__ __forceinline__ float load_as<__half, float>(const __half* p) { return __half2float(__ldg(p)); }
template <>
__device__ __forceinline__ float load_as<__nv_bfloat16, float>(const __nv_bfloat16* p) {
  return __bfloat162float(__ldg(p));
}

template <typename TS, typename TC>
__device__ __forceinline__ void store_as(TS* p, TC v) { *p = static_cast<TS>(v); }
template <>
__device__ __forceinline__ void store_as<__half, float>(__half* p, float v) { *p = __float2half_rn(v); }
template <>
__device__ __forceinline__ void store_as<__nv_bfloat16, float>(__nv_bfloat16* p, float v) {
  *p = __float2bfloat16_rn(v);
}

// Adds the two faces of direction d to the line accumulator acc[] of a line whose own
// values are u[] (nodes 0..N-1 along d). src_lo / src_hi: the neighbour's line or nullptr
// at the boundary; `step` is the stride of the line inside a cell. PC is an OpConst<TC, .>.
template <typename TS, typename TC, int N, typename PC>
__device__ __forceinline__ void add_faces(TC (&acc)[N], const TC (&u)[N], const TS* src_lo, const TS* src_hi,
                                          int step, const PC& P, int d) {
  // high face
  if (src_hi) {
    TC w[N];
#pragma unroll
    for (int m = 0; m < N; ++m) w[m] = load_as<TS, TC>(src_hi + m * step);
    TC sd = P.d0[0] * w[0];
#pragma unroll
    for (int m = 1; m < N; ++m) sd = fma(P.d0[m], w[m], sd);
#pragma unroll
    for (int i = 0; i < N; ++i) acc[i] = fma(P.E[d][0][i], w[0], fma(P.E[d][1][i], sd, acc[i]));
  } else {
    TC sd = P.d1[0] * u[0];
#pragma unroll
    for (int m = 1; m < N; ++m) sd = fma(P.d1[m], u[m], sd);
#pragma unroll
    for (int i = 0; i < N; ++i) acc[i] = fma(P.E[d][4][i], u[N - 1], fma(P.E[d][5][i], sd, acc[i]));
  }
  // low face
  if (src_lo) {
    TC w[N];
#pragma unroll
    for (int m = 0; m < N; ++m) w[m] = load_as<TS, TC>(src_lo + m * step);
    TC sd = P.d1[0] * w[0];
#pragma unroll
    for (int m = 1; m < N; ++m) sd = fma(P.d1[m], w[m], sd);
#pragma unroll
    for (int i = 0; i < N; ++i) acc[i] = fma(P.E[d][2][i], w[N - 1], fma(P.E[d][3][i], sd, acc[i]));
  } else {
    TC sd = P.d0[0] * u[0];
#pragma unroll
    for (int m = 1; m < N; ++m) sd = fma(P.d0[m], u[m], sd);
#pragma unroll
    for (int i = 0; i < N; ++i) acc[i] = fma(P.E[d][6][i], u[0], fma(P.E[d][7][i], sd, acc[i]));
  }
}

// The rank-2 face terms of direction d for a line whose neighbour lines are already in registers:
// wl / wh the low / high neighbour's line (used only when has_lo / has_hi; a missing neighbour is
// a boundary face and takes the own-line form, as in add_faces).
template <typename TC, int N, typename PC>
__device__ __forceinline__ void add_faces_lines(TC (&acc)[N], const TC (&u)[N], const TC (&wl)[N], bool has_lo,
                                                const TC (&wh)[N], bool has_hi, const PC& P, int d) {
  if (has_hi) {
    TC sd = P.d0[0] * wh[0];
#pragma unroll
    for (int m = 1; m < N; ++m) sd = fma(P.d0[m], wh[m], sd);
#pragma unroll
    for (int i = 0; i < N; ++i) acc[i] = fma(P.E[d][0][i], wh[0], fma(P.E[d][1][i], sd, acc[i]));
  } else {
    TC sd = P.d1[0] * u[0];
#pragma unroll
    for (int m = 1; m < N; ++m) sd = fma(P.d1[m], u[m], sd);
#pragma unroll
    for (int i = 0; i < N; ++i) acc[i] = fma(P.E[d][4][i], u[N - 1], fma(P.E[d][5][i], sd, acc[i]));
  }
  if (has_lo) {
    TC sd = P.d1[0] * wl[0];
#pragma unroll
    for (int m = 1; m < N; ++m) sd = fma(P.d1[m], wl[m], sd);
#pragma unroll
    for (int i = 0; i < N; ++i) acc[i] = fma(P.E[d][2][i], wl[N - 1], fma(P.E[d][3][i], sd, acc[i]));
  } else {
    TC sd = P.d0[0] * u[0];
#pragma unroll
    for (int m = 1; m < N; ++m) sd = fma(P.d0[m], u[m], sd);
#pragma unroll
    for (int i = 0; i < N; ++i) acc[i] = fma(P.E[d][6][i], u[0], fma(P.E[d][7][i], sd, acc[i]));
  }
}

}  // namespace tp
