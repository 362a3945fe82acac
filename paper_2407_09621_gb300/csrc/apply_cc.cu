// Sum-factorized SIPG Laplace apply on the FMA pipes ("CUDA-core" kernel).
//
// Sec. 2.1: v = A u = sum_K P_K^T A_K P_K u, evaluated cell by cell with the
// Kronecker form of Eq. (9). With the global 1D factors, A u is
//   M_z (M_y (L_x u) + L_y (M_x u)) + L_z (M_y (M_x u)),
// where L_d is block tridiagonal. The diagonal block of L_d is the interior
// one for every cell; the off-diagonal blocks and the boundary-face
// corrections are rank 2 in the normal direction:
//   L^{c,c+1} w = v1 (-g w_0 - (d0.w)/(2h)) + d1 (w_0/(2h))
//   L^{c,c-1} w = v0 (-g w_{n-1} + (d1.w)/(2h)) + d0 (-w_{n-1}/(2h))
//   boundary at the low end  (own line u): v0 ((d0.u)/(2h)) + d0 (u_0/(2h))
//   boundary at the high end (own line u): v1 (-(d1.u)/(2h)) + d1 (-u_{n-1}/(2h))
// (v0, v1 are unit vectors because Gauss-Lobatto nodes include the end
// points). Each face of a cell therefore contributes two n x n arrays
// (alpha, beta) that are expanded along the normal after the tangential
// masses of the directions already contracted have been applied to them.
//
// Thread layout (App. A's two-dimensional block): one thread per (i, j)
// column of a cell, CPB cells per block; the z-contraction runs in registers.
// TS = storage type of the vectors, TC = arithmetic type.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "tp_internal.h"

namespace tp {

template <typename TS, typename TC>
__device__ __forceinline__ TC load_as(const TS* p) { return static_cast<TC>(*p); }
template <>
__device__ __forceinline__ float load_as<__half, float>(const __half* p) { return __half2float(*p); }
template <>
__device__ __forceinline__ float load_as<__nv_bfloat16, float>(const __nv_bfloat16* p) { return __bfloat162float(*p); }

template <typename TS, typename TC>
__device__ __forceinline__ void store_as(TS* p, TC v) { *p = static_cast<TS>(v); }
template <>
__device__ __forceinline__ void store_as<__half, float>(__half* p, float v) { *p = __float2half_rn(v); }
template <>
__device__ __forceinline__ void store_as<__nv_bfloat16, float>(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }

template <int N>
__host__ __device__ constexpr int cc_cells_per_block() { return (128 / (N * N)) > 0 ? 128 / (N * N) : 1; }

// face index f: 0 = x-, 1 = x+, 2 = y-, 3 = y+, 4 = z-, 5 = z+ ; array 2f = alpha, 2f+1 = beta
template <typename TS, typename TC, int N>
__global__ void __launch_bounds__(N * N * cc_cells_per_block<N>())
apply_cc_kernel(const TS* __restrict__ x, TS* __restrict__ y, const OpConst<TC>* __restrict__ cst,
                int nx, int ny, int nz, long long ncells) {
  constexpr int CPB = cc_cells_per_block<N>();
  constexpr int N2 = N * N, N3 = N * N * N;
  __shared__ TC sM[3][N2], sL[3][N2], sd0[N], sd1[N], sg[3], shh[3];
  __shared__ TC sU[CPB][N3], sB[CPB][N3];
  __shared__ TC sF[CPB][12][N2], sT[CPB][12][N2];

  const int tid = threadIdx.x;
  for (int e = tid; e < 3 * N2; e += blockDim.x) {
    const int d = e / N2, r = e % N2, ii = r / N, jj = r % N;
    sM[d][r] = cst->M[d][ii * kMaxN + jj];
    sL[d][r] = cst->L[d][ii * kMaxN + jj];
  }
  if (tid < N) { sd0[tid] = cst->d0[tid]; sd1[tid] = cst->d1[tid]; }
  if (tid < 3) { sg[tid] = cst->gamma[tid]; shh[tid] = cst->half_inv_h[tid]; }

  const int cs = tid / N2, t = tid % N2, i = t % N, j = t / N;
  const long long cell = (long long)blockIdx.x * CPB + cs;
  const bool valid = cell < ncells;
  const int cx = valid ? (int)(cell % nx) : 0;
  const int cy = valid ? (int)((cell / nx) % ny) : 0;
  const int cz = valid ? (int)(cell / ((long long)nx * ny)) : 0;
  const TS* xc = x + cell * N3;
  __syncthreads();

  // ---- gather: own column into shared memory
  TC u[N];
#pragma unroll
  for (int l = 0; l < N; ++l) {
    u[l] = valid ? load_as<TS, TC>(xc + l * N2 + t) : TC(0);
    sU[cs][l * N2 + t] = u[l];
  }

  // ---- face traces: alpha/beta of the six faces (raw, before tangential masses)
  if (valid) {
    const long long sx = 1, sy = nx, sz = (long long)nx * ny;
    const int co[3] = {cx, cy, cz};
    const int nc[3] = {nx, ny, nz};
    const long long st[3] = {sx, sy, sz};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      // line along direction d handled by this thread, and its slot in the face array
      long long base;  // offset of node 0 of the line inside a cell
      int step;        // stride of the line inside a cell
      int slot;
      if (d == 0) { base = (long long)i * N2 + j * N; step = 1; slot = i * N + j; }       // line (l=i, j), array [l][j]
      else if (d == 1) { base = (long long)j * N2 + i; step = N; slot = j * N + i; }      // line (l=j, i), array [l][i]
      else { base = (long long)j * N + i; step = N2; slot = j * N + i; }                  // line (j, i), array [j][i]
      const TC g = sg[d], hh = shh[d];
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        const bool nb = side ? (co[d] < nc[d] - 1) : (co[d] > 0);
        const TS* src = nb ? (xc + (side ? st[d] : -st[d]) * N3) : xc;
        TC w[N];
#pragma unroll
        for (int m = 0; m < N; ++m) w[m] = load_as<TS, TC>(src + base + m * step);
        TC alpha, beta;
        if (side == 1) {
          if (nb) {
            TC sd = 0;
#pragma unroll
            for (int m = 0; m < N; ++m) sd += sd0[m] * w[m];
            alpha = -g * w[0] - hh * sd;
            beta = hh * w[0];
          } else {
            TC sd = 0;
#pragma unroll
            for (int m = 0; m < N; ++m) sd += sd1[m] * w[m];
            alpha = -hh * sd;
            beta = -hh * w[N - 1];
          }
        } else {
          if (nb) {
            TC sd = 0;
#pragma unroll
            for (int m = 0; m < N; ++m) sd += sd1[m] * w[m];
            alpha = -g * w[N - 1] + hh * sd;
            beta = -hh * w[N - 1];
          } else {
            TC sd = 0;
#pragma unroll
            for (int m = 0; m < N; ++m) sd += sd0[m] * w[m];
            alpha = hh * sd;
            beta = hh * w[0];
          }
        }
        const int f = 2 * d + side;
        sF[cs][2 * f][slot] = alpha;
        sF[cs][2 * f + 1][slot] = beta;
      }
    }
  } else {
#pragma unroll
    for (int a = 0; a < 12; ++a) sF[cs][a][t] = TC(0);
  }
  __syncthreads();

  // ---- x contraction: a = M_x u, b = L_x u + x-face terms
  TC a[N], b[N];
#pragma unroll
  for (int l = 0; l < N; ++l) {
    TC sa = 0, sb = 0;
#pragma unroll
    for (int m = 0; m < N; ++m) {
      const TC um = sU[cs][l * N2 + j * N + m];
      sa += sM[0][i * N + m] * um;
      sb += sL[0][i * N + m] * um;
    }
    const int fs = l * N + j;
    sb += sd1[i] * sF[cs][3][fs] + sd0[i] * sF[cs][1][fs];
    if (i == N - 1) sb += sF[cs][2][fs];
    if (i == 0) sb += sF[cs][0][fs];
    a[l] = sa;
    b[l] = sb;
  }
  // tangential mass M_x on the y-face arrays (index [l][i], l = j here) and on the z-face arrays ([j][i])
#pragma unroll
  for (int q = 4; q < 12; ++q) {
    TC s = 0;
#pragma unroll
    for (int m = 0; m < N; ++m) s += sM[0][i * N + m] * sF[cs][q][j * N + m];
    sT[cs][q][j * N + i] = s;
  }
  __syncthreads();
#pragma unroll
  for (int l = 0; l < N; ++l) {
    sU[cs][l * N2 + t] = a[l];
    sB[cs][l * N2 + t] = b[l];
  }
  // z-face arrays: second tangential mass M_y (along j)
#pragma unroll
  for (int q = 8; q < 12; ++q) {
    TC s = 0;
#pragma unroll
    for (int p = 0; p < N; ++p) s += sM[1][j * N + p] * sT[cs][q][p * N + i];
    sF[cs][q][t] = s;
  }
  __syncthreads();

  // ---- y contraction: c1 = M_y b + L_y a + y-face terms, c2 = M_y a
  TC c1[N], c2[N];
#pragma unroll
  for (int l = 0; l < N; ++l) {
    TC s1 = 0, s2 = 0;
#pragma unroll
    for (int p = 0; p < N; ++p) {
      const TC ap = sU[cs][l * N2 + p * N + i];
      const TC bp = sB[cs][l * N2 + p * N + i];
      s1 += sM[1][j * N + p] * bp + sL[1][j * N + p] * ap;
      s2 += sM[1][j * N + p] * ap;
    }
    const int fs = l * N + i;
    s1 += sd1[j] * sT[cs][7][fs] + sd0[j] * sT[cs][5][fs];
    if (j == N - 1) s1 += sT[cs][6][fs];
    if (j == 0) s1 += sT[cs][4][fs];
    c1[l] = s1;
    c2[l] = s2;
  }

  // ---- z contraction in registers: v = M_z c1 + L_z c2 + z-face terms; scatter
  if (valid) {
    TS* yc = y + cell * N3;
    const TC azp = sF[cs][10][t], bzp = sF[cs][11][t], azm = sF[cs][8][t], bzm = sF[cs][9][t];
#pragma unroll
    for (int l = 0; l < N; ++l) {
      TC s = 0;
#pragma unroll
      for (int p = 0; p < N; ++p) s += sM[2][l * N + p] * c1[p] + sL[2][l * N + p] * c2[p];
      s += sd1[l] * bzp + sd0[l] * bzm;
      if (l == N - 1) s += azp;
      if (l == 0) s += azm;
      store_as<TS, TC>(yc + l * N2 + t, s);
    }
  }
}

template <typename TS, typename TC, int N>
static cudaError_t launch_cc_n(const tp_op_s* op, void* y, const void* x, cudaStream_t s) {
  constexpr int CPB = cc_cells_per_block<N>();
  const long long blocks = (op->ncells + CPB - 1) / CPB;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  apply_cc_kernel<TS, TC, N><<<(unsigned)blocks, N * N * CPB, 0, s>>>(
      static_cast<const TS*>(x), static_cast<TS*>(y), static_cast<const OpConst<TC>*>(op->dconst),
      op->mesh.nx, op->mesh.ny, op->mesh.nz, op->ncells);
  return cudaGetLastError();
}

template <typename TS, typename TC>
static cudaError_t launch_cc_t(const tp_op_s* op, void* y, const void* x, cudaStream_t s) {
  switch (op->n) {
    case 2: return launch_cc_n<TS, TC, 2>(op, y, x, s);
    case 3: return launch_cc_n<TS, TC, 3>(op, y, x, s);
    case 4: return launch_cc_n<TS, TC, 4>(op, y, x, s);
    case 5: return launch_cc_n<TS, TC, 5>(op, y, x, s);
    case 6: return launch_cc_n<TS, TC, 6>(op, y, x, s);
    case 7: return launch_cc_n<TS, TC, 7>(op, y, x, s);
    case 8: return launch_cc_n<TS, TC, 8>(op, y, x, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_apply_cc(const tp_op_s* op, void* y, const void* x, cudaStream_t s) {
  switch (op->prec) {
    case TP_FP64: return launch_cc_t<double, double>(op, y, x, s);
    case TP_FP32: return launch_cc_t<float, float>(op, y, x, s);
    case TP_FP16: return launch_cc_t<__half, float>(op, y, x, s);
    case TP_BF16: return launch_cc_t<__nv_bfloat16, float>(op, y, x, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace tp
