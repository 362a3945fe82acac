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
// Work layout: n^2 threads per cell, CPB cells per block. In each
// contraction phase a thread owns one line of the cell along the contracted
// direction (x, then y, then z), so every 1D-matrix coefficient is the same
// for the whole warp: the matrices are a __grid_constant__ kernel parameter
// and enter the FMAs as constant-bank operands. Lines move between phases
// through shared memory. TS = storage type of the vectors, TC = arithmetic
// type.
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

template <int N>
__host__ __device__ constexpr int cc_cells_per_block() { return (128 / (N * N)) > 0 ? 128 / (N * N) : 1; }

template <typename TC, int N>
__host__ __device__ constexpr size_t cc_smem_bytes() {
  return sizeof(TC) * cc_cells_per_block<N>() * (4 * N * N * N + 20 * N * N);
}

// Face f: 0 = x-, 1 = x+, 2 = y-, 3 = y+, 4 = z-, 5 = z+; face arrays 2f = alpha, 2f+1 = beta.
// Face-point order inside an array (slow, fast): x faces (l, j), y faces (l, i), z faces (j, i).
template <typename TS, typename TC, int N>
__global__ void __launch_bounds__(N * N * cc_cells_per_block<N>())
apply_cc_kernel(const TS* __restrict__ x, TS* __restrict__ y, const __grid_constant__ OpConst<TC> P,
                int nx, int ny, int nz, long long ncells) {
  constexpr int CPB = cc_cells_per_block<N>();
  constexpr int N2 = N * N, N3 = N * N * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TC* base = reinterpret_cast<TC*>(smem_raw);
  const int tid = threadIdx.x;
  const int cs = tid / N2, t = tid % N2;
  TC* sU = base + cs * N3;                   // u, later c1
  TC* sA = base + (CPB + cs) * N3;           // a = M_x u
  TC* sB = base + (2 * CPB + cs) * N3;       // b = L_x u + x faces
  TC* sC = base + (3 * CPB + cs) * N3;       // c2 = M_y a
  TC* sF = base + 4 * CPB * N3 + cs * 12 * N2;                // raw face arrays (12), later z arrays final
  TC* sT = base + 4 * CPB * N3 + CPB * 12 * N2 + cs * 8 * N2;  // y/z face arrays after M_x

  const long long cell = (long long)blockIdx.x * CPB + cs;
  const bool valid = cell < ncells;
  const int cx = valid ? (int)(cell % nx) : 0;
  const int cy = valid ? (int)((cell / nx) % ny) : 0;
  const int cz = valid ? (int)(cell / ((long long)nx * ny)) : 0;
  const TS* xc = x + (valid ? cell : 0) * N3;

  // ---- gather u (coalesced) and the raw traces of the six faces at face point t = (p, q)
#pragma unroll
  for (int l = 0; l < N; ++l) sU[l * N2 + t] = valid ? load_as<TS, TC>(xc + l * N2 + t) : TC(0);
  {
    const int p = t / N, q = t % N;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int co = d == 0 ? cx : (d == 1 ? cy : cz);
      const int ncd = d == 0 ? nx : (d == 1 ? ny : nz);
      const long long std_ = d == 0 ? 1LL : (d == 1 ? (long long)nx : (long long)nx * ny);
      const int off = d == 0 ? p * N2 + q * N : (d == 1 ? p * N2 + q : p * N + q);
      const int step = d == 0 ? 1 : (d == 1 ? N : N2);
      const TC g = P.gamma[d], hh = P.half_inv_h[d];
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        const bool nb = valid && (side ? (co < ncd - 1) : (co > 0));
        const TS* src = (nb ? xc + (side ? std_ : -std_) * N3 : xc) + off;
        TC w[N];
#pragma unroll
        for (int m = 0; m < N; ++m) w[m] = valid ? load_as<TS, TC>(src + m * step) : TC(0);
        // value trace s and derivative trace sd of the line at the face
        const TC s = (side == nb) ? w[0] : w[N - 1];
        TC sd = TC(0);
        if (side == nb) {
#pragma unroll
          for (int m = 0; m < N; ++m) sd = fma(P.d0[m], w[m], sd);
        } else {
#pragma unroll
          for (int m = 0; m < N; ++m) sd = fma(P.d1[m], w[m], sd);
        }
        TC alpha, beta;
        if (nb) {
          alpha = side ? fma(-g, s, -hh * sd) : fma(-g, s, hh * sd);
          beta = side ? hh * s : -hh * s;
        } else {
          alpha = side ? -hh * sd : hh * sd;
          beta = side ? -hh * s : hh * s;
        }
        sF[(4 * d + 2 * side) * N2 + t] = alpha;
        sF[(4 * d + 2 * side + 1) * N2 + t] = beta;
      }
    }
  }
  __syncthreads();

  // ---- M_x along the fast index of the y- and z-face arrays (8 arrays x N rows)
  for (int w = t; w < 8 * N; w += N2) {
    const int q = w / N, r = w % N;
    TC row[N];
#pragma unroll
    for (int m = 0; m < N; ++m) row[m] = sF[(4 + q) * N2 + r * N + m];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      TC s = TC(0);
#pragma unroll
      for (int m = 0; m < N; ++m) s = fma(P.M[0][i * kMaxN + m], row[m], s);
      sT[q * N2 + r * N + i] = s;
    }
  }
  __syncthreads();

  // ---- x contraction on x-line (l, j): a = M_x u, b = L_x u + x-face terms
  {
    const int l = t / N, j = t % N;
    TC u[N];
#pragma unroll
    for (int m = 0; m < N; ++m) u[m] = sU[l * N2 + j * N + m];
    const TC am = sF[0 * N2 + t], bm = sF[1 * N2 + t], ap = sF[2 * N2 + t], bp = sF[3 * N2 + t];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      TC sa = TC(0), sb = TC(0);
#pragma unroll
      for (int m = 0; m < N; ++m) {
        sa = fma(P.M[0][i * kMaxN + m], u[m], sa);
        sb = fma(P.L[0][i * kMaxN + m], u[m], sb);
      }
      sb = fma(P.d1[i], bp, sb);
      sb = fma(P.d0[i], bm, sb);
      if (i == N - 1) sb += ap;
      if (i == 0) sb += am;
      sA[l * N2 + j * N + i] = sa;
      sB[l * N2 + j * N + i] = sb;
    }
  }
  // ---- M_y along the slow index of the z-face arrays (4 arrays x N columns)
  for (int w = t; w < 4 * N; w += N2) {
    const int q = w / N, i = w % N;
    TC col[N];
#pragma unroll
    for (int pp = 0; pp < N; ++pp) col[pp] = sT[(4 + q) * N2 + pp * N + i];
#pragma unroll
    for (int j = 0; j < N; ++j) {
      TC s = TC(0);
#pragma unroll
      for (int pp = 0; pp < N; ++pp) s = fma(P.M[1][j * kMaxN + pp], col[pp], s);
      sF[(8 + q) * N2 + j * N + i] = s;
    }
  }
  __syncthreads();

  // ---- y contraction on y-line (l, i): c1 = M_y b + L_y a + y-face terms, c2 = M_y a
  {
    const int l = t / N, i = t % N;
    TC a[N], b[N];
#pragma unroll
    for (int pp = 0; pp < N; ++pp) {
      a[pp] = sA[l * N2 + pp * N + i];
      b[pp] = sB[l * N2 + pp * N + i];
    }
    const TC am = sT[0 * N2 + t], bm = sT[1 * N2 + t], ap = sT[2 * N2 + t], bp = sT[3 * N2 + t];
#pragma unroll
    for (int j = 0; j < N; ++j) {
      TC s1 = TC(0), s2 = TC(0);
#pragma unroll
      for (int pp = 0; pp < N; ++pp) {
        s1 = fma(P.M[1][j * kMaxN + pp], b[pp], s1);
        s1 = fma(P.L[1][j * kMaxN + pp], a[pp], s1);
        s2 = fma(P.M[1][j * kMaxN + pp], a[pp], s2);
      }
      s1 = fma(P.d1[j], bp, s1);
      s1 = fma(P.d0[j], bm, s1);
      if (j == N - 1) s1 += ap;
      if (j == 0) s1 += am;
      sU[l * N2 + j * N + i] = s1;
      sC[l * N2 + j * N + i] = s2;
    }
  }
  __syncthreads();

  // ---- z contraction on z-line (j, i) = t: v = M_z c1 + L_z c2 + z-face terms; scatter
  if (valid) {
    TC c1[N], c2[N];
#pragma unroll
    for (int pp = 0; pp < N; ++pp) {
      c1[pp] = sU[pp * N2 + t];
      c2[pp] = sC[pp * N2 + t];
    }
    const TC am = sF[8 * N2 + t], bm = sF[9 * N2 + t], ap = sF[10 * N2 + t], bp = sF[11 * N2 + t];
    TS* yc = y + cell * N3;
#pragma unroll
    for (int l = 0; l < N; ++l) {
      TC s = TC(0);
#pragma unroll
      for (int pp = 0; pp < N; ++pp) {
        s = fma(P.M[2][l * kMaxN + pp], c1[pp], s);
        s = fma(P.L[2][l * kMaxN + pp], c2[pp], s);
      }
      s = fma(P.d1[l], bp, s);
      s = fma(P.d0[l], bm, s);
      if (l == N - 1) s += ap;
      if (l == 0) s += am;
      store_as<TS, TC>(yc + l * N2 + t, s);
    }
  }
}

template <typename TS, typename TC, int N>
static cudaError_t launch_cc_n(const tp_op_s* op, void* y, const void* x, cudaStream_t s) {
  constexpr int CPB = cc_cells_per_block<N>();
  constexpr size_t smem = cc_smem_bytes<TC, N>();
  const long long blocks = (op->ncells + CPB - 1) / CPB;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  const OpConst<TC>& P = *static_cast<const OpConst<TC>*>(op->hconst(sizeof(TC)));
  apply_cc_kernel<TS, TC, N><<<(unsigned)blocks, N * N * CPB, smem, s>>>(
      static_cast<const TS*>(x), static_cast<TS*>(y), P, op->mesh.nx, op->mesh.ny, op->mesh.nz, op->ncells);
  return cudaGetLastError();
}

template <typename TS, typename TC, int N>
static cudaError_t prepare_cc_n() {
  return cudaFuncSetAttribute(apply_cc_kernel<TS, TC, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)cc_smem_bytes<TC, N>());
}

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
  switch (op->prec) {
    case TP_FP64: return prepare_cc_t<double, double>(op->n);
    case TP_FP32: return prepare_cc_t<float, float>(op->n);
    case TP_FP16: return prepare_cc_t<__half, float>(op->n);
    case TP_BF16: return prepare_cc_t<__nv_bfloat16, float>(op->n);
  }
  return cudaErrorInvalidValue;
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
