// Sum-factorized SIPG Laplace apply on the FMA pipes ("CUDA-core" kernel).
//
// Sec. 2.1, Eq. (9): with the global 1D factors (M block diagonal, L block
// tridiagonal with the face terms) the operator is
//   A = L_z(x)M_y(x)M_x + M_z(x)L_y(x)M_x + M_z(x)M_y(x)L_x
//     = (M_z(x)M_y(x)M_x) * [ (M^-1 L)_x + (M^-1 L)_y + (M^-1 L)_z ],
// the same matrix written with one mass tensor on the left. Evaluated this
// way a cell needs six n x n contractions instead of seven, and the face
// terms need no tangential mass (they enter before the mass tensor):
//   w = sum_d (M_d^-1 L_d) u  along each direction d (three contractions),
//   v = M_z M_y M_x w          (three contractions).
// M^-1 L is block tridiagonal like L. Its diagonal block G = M^-1 L_int is
// the same for every cell; its neighbour blocks and the boundary-face
// corrections are rank 2 along the normal, because Gauss-Lobatto value traces
// are unit vectors (v0 = e_0, v1 = e_{n-1}):
//   high neighbour:  s = w_0,     sd = d0.w  ->  s*P1 + sd*P2
//   low neighbour:   s = w_{n-1}, sd = d1.w  ->  s*Q1 + sd*Q2
//   high boundary:   s = u_{n-1}, sd = d1.u  ->  s*B1 + sd*B2   (own line u)
//   low boundary:    s = u_0,     sd = d0.u  ->  s*C1 + sd*C2
// with P1 = M^-1(-g v1 + d1/2h), P2 = -M^-1 v1/2h, Q1 = M^-1(-g v0 - d0/2h),
// Q2 = M^-1 v0/2h, B1 = -M^-1 d1/2h, B2 = -M^-1 v1/2h, C1 = M^-1 d0/2h,
// C2 = M^-1 v0/2h (g the penalty, h the cell width normal to the face).
//
// Work layout: n^2 threads per cell, CPB cells per block (the tile shape: CPB is
// 128/n^2 halved, kept or doubled, picked per operator by the autotuner in tp_api.cu). In every phase a
// thread owns one line of its cell along the direction being contracted, so
// all threads of a warp apply the same 1D coefficients at the same time: the
// 1D data is a __grid_constant__ kernel parameter and the coefficients are
// constant-bank operands of the FMAs. The x-neighbour rows of the x-faces come from the block's own
// shared cell tensors where the neighbour is one of the block's cells (cells of a block are
// consecutive along x). Phases: (A) x- and y-lines of
// w_x = G_x u + x faces and w_y = G_y u + y faces; (B) z-lines: w = w_x + w_y
// + G_z u + z faces, then M_z w in registers; (C) y-lines: M_y; (D) x-lines:
// M_x and the store; given a vector b the store is the residual b - A x instead (the smoother's
// residuals without a separate pass). TS = storage type of the vectors, TC = arithmetic type.
//
// Degrees above 7 (8 < n <= 16, FP64 and FP32): one cell per block (n^2 threads) and three cell
// buffers instead of four (M_z w overwrites u: in phase B every thread reads and writes its own
// z-line only). The cell tensors are padded to a row pitch of n + 1 there and for FP32
// arithmetic at every n, so that the x-line phases, whose threads read rows n values apart, hit
// distinct shared-memory banks (the FP32 kernels are bound by shared-memory and L1 throughput;
// the FP64 ones by the FP64 pipe, and keep the unpadded layout).
//
// Instantiated in apply_cc.cu (n <= 8) and apply_cc_high.cu (8 < n <= 16).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "apply_common.cuh"

namespace tp {

// cells per block of tile-shape variant V (0: half, 1: the default 128/n^2, 2: double)
template <int N, int V>
__host__ __device__ constexpr int cc_cells_per_block() {
  return V == 0 ? ((128 / (N * N)) / 2 > 0 ? (128 / (N * N)) / 2 : 1)
                : (V == 1 ? ((128 / (N * N)) > 0 ? 128 / (N * N) : 1) : 2 * ((128 / (N * N)) > 0 ? 128 / (N * N) : 1));
}

// Row pitch of the shared cell tensors (element (l, j, i) at (l*N + j)*R + i) and the number
// of cell buffers; the operator constants' row pitch.
template <typename TC, int N> __host__ __device__ constexpr int cc_pitch() {
  return (N > kMaxN || sizeof(TC) == 4) ? N + 1 : N;
}
// FP64 arithmetic accumulates the y-lines into the x-line buffer (one more barrier, one buffer and
// one FP64 addition per DoF fewer: the FP64 pipe bounds that kernel); other types keep a separate
// y-line buffer (their kernels are bound by shared-memory instructions, which the merge would add).
template <typename TC> __host__ __device__ constexpr bool cc_merge_xy() { return sizeof(TC) == 8; }
template <typename TC, int N> __host__ __device__ constexpr int cc_buffers() {
  return (N > kMaxN ? 3 : 4) - (cc_merge_xy<TC>() ? 1 : 0);
}
template <typename TC, int N> using CcConst = OpConst<TC, (N > kMaxN ? kMaxNHigh : kMaxN)>;

template <typename TC, int N, int V>
__host__ __device__ constexpr size_t cc_smem_bytes() {
  return sizeof(TC) * cc_cells_per_block<N, V>() * cc_buffers<TC, N>() * N * N * cc_pitch<TC, N>();
}

// out = A in for a centrosymmetric A through its even-odd halves (AE, AO of OpConst), H = n/2
// rounded down: e_m = in[m] + in[n-1-m], o_m = in[m] - in[n-1-m] for m < H; ev_i = AE e,
// od_i = AO o; out[i] = ev_i + od_i, out[n-1-i] = ev_i - od_i. For odd n the middle node is
// its own mirror image: e_H = in[H] enters ev through the column AE[i][H] = A[i][H], no od term
// involves it, and the middle row is out[H] = AE[H] e. About n^2/2 + 2n operations instead of n^2.
template <typename TC, int N, int S>
__device__ __forceinline__ void contract_eo(TC (&out)[N], const TC (&AE)[S / 2][S / 2], const TC (&AO)[S / 2][S / 2],
                                            const TC (&in)[N]) {
  constexpr int H = N / 2, HE = (N + 1) / 2;  // odd and even halves' lengths
  TC e[HE], o[H];
#pragma unroll
  for (int m = 0; m < H; ++m) {
    e[m] = in[m] + in[N - 1 - m];
    o[m] = in[m] - in[N - 1 - m];
  }
  if constexpr (HE > H) e[H] = in[H];
#pragma unroll
  for (int i = 0; i < H; ++i) {
    TC ev = AE[i][0] * e[0], od = AO[i][0] * o[0];
#pragma unroll
    for (int m = 1; m < H; ++m) {
      ev = fma(AE[i][m], e[m], ev);
      od = fma(AO[i][m], o[m], od);
    }
    if constexpr (HE > H) ev = fma(AE[i][H], e[H], ev);
    out[i] = ev + od;
    out[N - 1 - i] = ev - od;
  }
  if constexpr (HE > H) {
    TC mid = AE[H][0] * e[0];
#pragma unroll
    for (int m = 1; m < HE; ++m) mid = fma(AE[H][m], e[m], mid);
    out[H] = mid;
  }
}

template <typename TC, int N, int S>
__device__ __forceinline__ void contract(TC (&out)[N], const TC* __restrict__ A, const TC (&in)[N]) {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    TC s = A[i * S] * in[0];
#pragma unroll
    for (int m = 1; m < N; ++m) s = fma(A[i * S + m], in[m], s);
    out[i] = s;
  }
}

// out = (M or G)_d in: the even-odd form for n >= 5 when the matrices are centrosymmetric
// (always on the symmetric Gauss-Lobatto element; checked on the host), the plain form otherwise
// (for n <= 4 the even-odd form saves no instruction).
template <typename TC, int N>
__device__ __forceinline__ void contract_d(TC (&out)[N], const CcConst<TC, N>& P, bool mass, int d,
                                           const TC (&in)[N]) {
  constexpr int S = CcConst<TC, N>::S;
  if constexpr (N >= 5) {
    if (P.centro) {
      if (mass)
        contract_eo<TC, N, S>(out, P.ME[d], P.MO[d], in);
      else
        contract_eo<TC, N, S>(out, P.GE[d], P.GO[d], in);
      return;
    }
  }
  contract<TC, N, S>(out, mass ? P.M[d] : P.G[d], in);
}

// Shared-memory row helpers of the vector layout (rows of N floats, 16-byte aligned)
// (16-byte chunk k of the row stored at chunk position k ^ sw: the swizzled layout below)
template <int N>
__device__ __forceinline__ void lds_row(float (&v)[N], const float* p, int sw = 0) {
#pragma unroll
  for (int k = 0; k < N / 4; ++k) {
    const float4 t = reinterpret_cast<const float4*>(p)[k ^ sw];
    v[4 * k] = t.x; v[4 * k + 1] = t.y; v[4 * k + 2] = t.z; v[4 * k + 3] = t.w;
  }
}
template <int N>
__device__ __forceinline__ void sts_row(float* p, const float (&v)[N], int sw = 0) {
#pragma unroll
  for (int k = 0; k < N / 4; ++k)
    reinterpret_cast<float4*>(p)[k ^ sw] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
}

// One x-row (N contiguous values) of a cell tensor in shared memory, as 16-byte loads in the
// float layout with unpadded rows (VX), else value by value.
template <typename TC, int N, bool VX>
__device__ __forceinline__ void x_row_shared(TC (&v)[N], const TC* p, int sw) {
  if constexpr (VX) {
    lds_row<N>(v, p, sw);
  } else {
#pragma unroll
    for (int m = 0; m < N; ++m) v[m] = p[m];
  }
}

// One x-row of a cell in global memory: 16-byte loads for FP32 vectors with n a multiple of 4
// (VG: the row starts 16-byte aligned), else value by value.
template <typename TS, typename TC, int N, bool VG>
__device__ __forceinline__ void x_row_global(TC (&v)[N], const TS* p) {
  if constexpr (VG) {
#pragma unroll
    for (int k = 0; k < N / 4; ++k) {
      const float4 t = __ldg(reinterpret_cast<const float4*>(p) + k);
      v[4 * k] = t.x; v[4 * k + 1] = t.y; v[4 * k + 2] = t.z; v[4 * k + 3] = t.w;
    }
  } else {
#pragma unroll
    for (int m = 0; m < N; ++m) v[m] = load_as<TS, TC>(p + m);
  }
}

template <typename TS, typename TC, int N, int V, bool RES>
__global__ void __launch_bounds__(N * N * cc_cells_per_block<N, V>())
apply_cc_kernel(const TS* __restrict__ x, TS* __restrict__ y, const TS* __restrict__ b,
                const __grid_constant__ CcConst<TC, N> P, int nx, int ny, int nz, long long c_begin, long long c_end) {
  constexpr int CPB = cc_cells_per_block<N, V>();
  constexpr int N2 = N * N, N3 = N * N * N;
  // Layout of a shared cell tensor: element (l, j, i) at l * PL + j * RP + i. FP32 arithmetic with
  // n = 4, 8, 16 keeps rows unpadded and 16-byte aligned (x-lines move as float4) and pads each
  // plane by n instead (PL = n(n + 1)), which keeps the y- and z-line phases free of bank
  // conflicts; otherwise rows are padded to cc_pitch.
  constexpr bool VX = sizeof(TC) == 4 && (N == 4 || N == 8 || N == 16);
  constexpr bool VG = VX && sizeof(TS) == 4;  // the global x-rows move as float4 as well
  // n = 8 with FP32 arithmetic (SW): the row (l, j) is stored at row position r = j ^ l of plane l,
  // its two 16-byte chunks swapped when r >= 4, so that the x-rows (16-byte accesses), the y-lines
  // and the z-lines (scalar accesses) of the half cell a warp holds all fall in distinct banks (the
  // padded layout leaves the x-rows 2-way). For n = 4 the same permutation (with the cells 16 banks
  // apart) also removes the x-row conflicts, but measured slower (the extra index arithmetic of the
  // y- and z-lines costs more than the conflicts), so n = 4 keeps the padded planes.
  constexpr bool SW = VX && N == 8;
  constexpr int RP = VX ? N : cc_pitch<TC, N>(), PL = SW ? N * N : (VX ? N * (N + 1) : N * RP);
  // pitch of the shared cell tensors (the allocation of cc_smem_bytes)
  constexpr int B = N * N * cc_pitch<TC, N>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TC* base = reinterpret_cast<TC*>(smem_raw);
  const int tid = threadIdx.x;
  const int cs = tid / N2, t = tid % N2, p = t / N, q = t % N;
  constexpr bool MXY = cc_merge_xy<TC>();
  TC* sU = base + cs * B;                   // u
  TC* sX = base + (CPB + cs) * B;           // w_x (with MXY: w_x + w_y), later M_y M_z w
  TC* sY = MXY ? sX : base + (2 * CPB + cs) * B;  // w_y
  TC* sZ = N > kMaxN ? sU : base + ((MXY ? 2 : 3) * CPB + cs) * B;  // M_z w
  auto ix = [](int l, int j, int i) {
    if constexpr (SW) {
      const int r = (j ^ l) & (N - 1);
      return l * PL + r * RP + ((((i >> 2) ^ ((r >> 2) & (N / 4 - 1)))) << 2) + (i & 3);
    } else {
      return l * PL + j * RP + i;
    }
  };
  // start of the stored row (l, j) and its chunk permutation
  auto rowp = [](int l, int j) { return SW ? l * PL + ((j ^ l) & (N - 1)) * RP : l * PL + j * RP; };
  auto rsw = [](int l, int j) { return SW ? ((((j ^ l) & (N - 1)) >> 2) & (N / 4 - 1)) : 0; };

  const long long cell = c_begin + (long long)blockIdx.x * CPB + cs;  // cells [c_begin, c_end) of the mesh
  const bool valid = cell < c_end;
  const int cx = valid ? (int)(cell % nx) : 0;
  const int cy = valid ? (int)((cell / nx) % ny) : 0;
  const int cz = valid ? (int)(cell / ((long long)nx * ny)) : 0;
  const TS* xc = x + (valid ? cell : 0) * N3;
  const long long sy = (long long)nx * N3, sz = (long long)nx * ny * N3;

  // ---- gather u (coalesced: by columns of the cell, or by x-rows of float4)
  if constexpr (VG) {
    TC r[N];
    if (valid) {
#pragma unroll
      for (int k = 0; k < N / 4; ++k) {
        const float4 v4 = __ldg(reinterpret_cast<const float4*>(xc + p * N2 + q * N) + k);
        r[4 * k] = v4.x; r[4 * k + 1] = v4.y; r[4 * k + 2] = v4.z; r[4 * k + 3] = v4.w;
      }
    } else {
#pragma unroll
      for (int i = 0; i < N; ++i) r[i] = TC(0);
    }
    sts_row<N>(sU + rowp(p, q), r, rsw(p, q));
  } else {
#pragma unroll
    for (int l = 0; l < N; ++l) sU[ix(l, p, q)] = valid ? load_as<TS, TC>(xc + l * N2 + t) : TC(0);
  }
  __syncthreads();

  // ---- (A) x-line (l=p, j=q) and y-line (l=p, i=q)
  {
    TC u[N], w[N];
    if constexpr (VX) {
      lds_row<N>(u, sU + rowp(p, q), rsw(p, q));
    } else {
#pragma unroll
      for (int m = 0; m < N; ++m) u[m] = sU[ix(p, q, m)];
    }
    contract_d<TC, N>(w, P, false, 0, u);
    if (valid) {
      // the x-neighbours' rows: from this block's shared cell tensors where the neighbour cell is
      // one of the block's (all but the block's first and last cell), else from global memory
      TC wl[N], wh[N];
      const bool hl = cx > 0, hh = cx < nx - 1;
      if (hl) {
        if (cs > 0) {
          x_row_shared<TC, N, VX>(wl, base + (cs - 1) * B + rowp(p, q), rsw(p, q));
        } else {
          x_row_global<TS, TC, N, VG>(wl, xc - N3 + p * N2 + q * N);
        }
      }
      if (hh) {
        if (cs + 1 < CPB && cell + 1 < c_end) {
          x_row_shared<TC, N, VX>(wh, base + (cs + 1) * B + rowp(p, q), rsw(p, q));
        } else {
          x_row_global<TS, TC, N, VG>(wh, xc + N3 + p * N2 + q * N);
        }
      }
      add_faces_lines<TC, N>(w, u, wl, hl, wh, hh, P, 0);
    }
    if constexpr (VX) {
      sts_row<N>(sX + rowp(p, q), w, rsw(p, q));
    } else {
#pragma unroll
      for (int i = 0; i < N; ++i) sX[ix(p, q, i)] = w[i];
    }
    if constexpr (MXY) __syncthreads();  // the y-lines add into the x-lines' buffer
#pragma unroll
    for (int m = 0; m < N; ++m) u[m] = sU[ix(p, m, q)];
    contract_d<TC, N>(w, P, false, 1, u);
    if (valid) {
      const TS* lo = cy > 0 ? xc - sy + p * N2 + q : nullptr;
      const TS* hi = cy < ny - 1 ? xc + sy + p * N2 + q : nullptr;
      add_faces<TS, TC, N>(w, u, lo, hi, N, P, 1);
    }
    if constexpr (MXY) {
#pragma unroll
      for (int j = 0; j < N; ++j) sX[ix(p, j, q)] += w[j];
    } else {
#pragma unroll
      for (int j = 0; j < N; ++j) sY[ix(p, j, q)] = w[j];
    }
  }
  __syncthreads();

  // ---- (B) z-line (j=p, i=q): w = w_x + w_y + G_z u + z faces; then M_z w
  {
    TC u[N], w[N], v[N];
#pragma unroll
    for (int m = 0; m < N; ++m) u[m] = sU[ix(m, p, q)];
    contract_d<TC, N>(w, P, false, 2, u);
    if (valid) {
      const TS* lo = cz > 0 ? xc - sz + t : nullptr;
      const TS* hi = cz < nz - 1 ? xc + sz + t : nullptr;
      add_faces<TS, TC, N>(w, u, lo, hi, N2, P, 2);
    }
    if constexpr (MXY) {
#pragma unroll
      for (int l = 0; l < N; ++l) w[l] += sX[ix(l, p, q)];
    } else {
#pragma unroll
      for (int l = 0; l < N; ++l) w[l] += sX[ix(l, p, q)] + sY[ix(l, p, q)];
    }
    contract_d<TC, N>(v, P, true, 2, w);
#pragma unroll
    for (int l = 0; l < N; ++l) sZ[ix(l, p, q)] = v[l];
  }
  __syncthreads();

  // ---- (C) y-line (l=p, i=q): M_y
  {
    TC w[N], v[N];
#pragma unroll
    for (int m = 0; m < N; ++m) w[m] = sZ[ix(p, m, q)];
    contract_d<TC, N>(v, P, true, 1, w);
#pragma unroll
    for (int j = 0; j < N; ++j) sX[ix(p, j, q)] = v[j];
  }
  __syncthreads();

  // ---- (D) x-line (l=p, j=q): M_x and scatter (y = A x, or y = b - A x when b is given)
  if (valid) {
    TC w[N], v[N];
    if constexpr (VX) {
      lds_row<N>(w, sX + rowp(p, q), rsw(p, q));
    } else {
#pragma unroll
      for (int m = 0; m < N; ++m) w[m] = sX[ix(p, q, m)];
    }
    contract_d<TC, N>(v, P, true, 0, w);
    TS* yc = y + cell * N3 + p * N2 + q * N;
    if constexpr (VG) {
      if constexpr (RES) {
#pragma unroll
        for (int k = 0; k < N / 4; ++k) {
          const float4 b4 = __ldg(reinterpret_cast<const float4*>(b + cell * N3 + p * N2 + q * N) + k);
          v[4 * k] = b4.x - v[4 * k]; v[4 * k + 1] = b4.y - v[4 * k + 1];
          v[4 * k + 2] = b4.z - v[4 * k + 2]; v[4 * k + 3] = b4.w - v[4 * k + 3];
        }
      }
#pragma unroll
      for (int k = 0; k < N / 4; ++k)
        reinterpret_cast<float4*>(yc)[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
    } else if constexpr (RES) {
      const TS* bc = b + cell * N3 + p * N2 + q * N;
#pragma unroll
      for (int i = 0; i < N; ++i) store_as<TS, TC>(yc + i, load_as<TS, TC>(bc + i) - v[i]);
    } else {
#pragma unroll
      for (int i = 0; i < N; ++i) store_as<TS, TC>(yc + i, v[i]);
    }
  }
}

template <typename TS, typename TC, int N, int V, bool RES>
static cudaError_t launch_cc_v(const tp_op_s* op, void* y, const void* x, long long c0, long long c1, cudaStream_t s,
                               const void* b) {
  constexpr int CPB = cc_cells_per_block<N, V>();
  constexpr size_t smem = cc_smem_bytes<TC, N, V>();
  const long long blocks = (c1 - c0 + CPB - 1) / CPB;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  if (blocks <= 0) return cudaSuccess;
  const CcConst<TC, N>& P = *static_cast<const CcConst<TC, N>*>(
      N > kMaxN ? op->hconst_high(sizeof(TC)) : op->hconst(sizeof(TC)));
  apply_cc_kernel<TS, TC, N, V, RES><<<(unsigned)blocks, N * N * CPB, smem, s>>>(
      static_cast<const TS*>(x), static_cast<TS*>(y), static_cast<const TS*>(b), P, op->mesh.nx, op->mesh.ny,
      op->mesh.nz, c0, c1);
  return cudaGetLastError();
}

// Launch of the tile variant the operator selected (n > 8: the one-cell tile only); the
// residual form b - A x (b not null) always takes the default tile.
template <typename TS, typename TC, int N>
static cudaError_t launch_cc_n(const tp_op_s* op, void* y, const void* x, long long c0, long long c1, cudaStream_t s,
                               const void* b) {
  if (b) return launch_cc_v<TS, TC, N, 1, true>(op, y, x, c0, c1, s, b);
  if constexpr (N > kMaxN) {
    return launch_cc_v<TS, TC, N, 1, false>(op, y, x, c0, c1, s, b);
  } else {
    switch (op->tile_variant) {
      case 0: return launch_cc_v<TS, TC, N, 0, false>(op, y, x, c0, c1, s, b);
      case 2: return launch_cc_v<TS, TC, N, 2, false>(op, y, x, c0, c1, s, b);
    }
    return launch_cc_v<TS, TC, N, 1, false>(op, y, x, c0, c1, s, b);
  }
}

template <typename TS, typename TC, int N, int V, bool RES>
static cudaError_t prepare_cc_v() {
  return cudaFuncSetAttribute(apply_cc_kernel<TS, TC, N, V, RES>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)cc_smem_bytes<TC, N, V>());
}

// Sets the dynamic shared-memory limit of every tile variant of degree N, and of the residual
// form, on the current device.
template <typename TS, typename TC, int N>
static cudaError_t prepare_cc_n() {
  cudaError_t e = prepare_cc_v<TS, TC, N, 1, true>();
  if constexpr (N > kMaxN) {
    if (e == cudaSuccess) e = prepare_cc_v<TS, TC, N, 1, false>();
  } else {
    if (e == cudaSuccess) e = prepare_cc_v<TS, TC, N, 0, false>();
    if (e == cudaSuccess) e = prepare_cc_v<TS, TC, N, 1, false>();
    if (e == cudaSuccess) e = prepare_cc_v<TS, TC, N, 2, false>();
  }
  return e;
}

}  // namespace tp
