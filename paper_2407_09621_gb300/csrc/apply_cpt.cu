// Sum-factorized SIPG Laplace apply on the FMA pipes with FP32 arithmetic for n = k + 1 = 2:
// one thread per cell.
//
// The operator is the inverse-mass form of Eq. (9) used by the CUDA-core kernel (apply_cc.cuh):
//   v = (M_z (x) M_y (x) M_x) w,   w = sum_d (M_d^-1 L_d) u  (+ the rank-2 face terms),
// with the same 1D constants (G = M^-1 L_int, the end derivatives d0, d1 and the face expansion
// vectors E of OpConst). One thread keeps the cell's u and w in registers and does all six
// contractions and the face terms there: no shared-memory transposes between the line phases and
// no barriers. The line-per-thread kernel moves every value through shared memory five times and is
// bound by the L1/shared-memory unit; here L1 carries only the global rows: the cell's own rows and,
// per face, the rows of the neighbour cell whose lines cross the face (whole x-rows; x-neighbours
// are the adjacent threads' own cells, mostly L1 hits).
//
// Measured against the line-per-thread kernel (FP32 vectors, ~2^25 DoFs): n = 2, 40 registers,
// 273 against 177 GDoF/s; n = 3, 72 registers, 116 against 189; n = 4, 156 registers, 124 against
// 239 (at 12 warps per SM the global-load latency of the face rows is exposed). So the library uses
// it at n = 2 only; the code is written for any n whose cell fits the registers.
//
// Face terms of direction d for a line with own values u[] and accumulator acc[] (as in
// add_faces_lines): a high neighbour line wh adds E[d][0] wh[0] + E[d][1] (d0 . wh), a low one wl
// adds E[d][2] wl[n-1] + E[d][3] (d1 . wl); at the boundary the own line gives E[d][4] u[n-1] +
// E[d][5] (d1 . u) (high) and E[d][6] u[0] + E[d][7] (d0 . u) (low).
#include "apply_common.cuh"

namespace tp {

namespace {

template <int N>
using CptConst = OpConst<float, kMaxN>;

__device__ __forceinline__ float load_cvt(float v) { return v; }
__device__ __forceinline__ float load_cvt(__half v) { return __half2float(v); }
__device__ __forceinline__ float load_cvt(__nv_bfloat16 v) { return __bfloat162float(v); }

// One x-row (N consecutive values) of a cell as FP32: 16-byte loads for FP32 n = 4, 8-byte loads
// for FP32 n = 2 and FP16/BF16 n = 4, 4-byte loads for FP16/BF16 n = 2, value by value for n = 3
// (rows of 3 values are not aligned beyond the element).
template <typename TS, int N>
__device__ __forceinline__ void ld_row(float (&v)[N], const TS* p) {
  if constexpr (std::is_same<TS, float>::value && N == 4) {
    const float4 t = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  } else if constexpr (std::is_same<TS, float>::value && N == 2) {
    const float2 t = __ldg(reinterpret_cast<const float2*>(p));
    v[0] = t.x; v[1] = t.y;
  } else if constexpr (!std::is_same<TS, float>::value && (N == 4 || N == 2)) {
    using V = typename std::conditional<N == 4, uint2, unsigned>::type;
    const V t = __ldg(reinterpret_cast<const V*>(p));
    const TS* h = reinterpret_cast<const TS*>(&t);
#pragma unroll
    for (int m = 0; m < N; ++m) v[m] = load_cvt(h[m]);
  } else {
#pragma unroll
    for (int m = 0; m < N; ++m) v[m] = load_as<TS, float>(p + m);
  }
}

template <typename TS, int N>
__device__ __forceinline__ void st_row(TS* p, const float (&v)[N]) {
  if constexpr (std::is_same<TS, float>::value && N == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else if constexpr (std::is_same<TS, float>::value && N == 2) {
    *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
  } else if constexpr (!std::is_same<TS, float>::value && (N == 4 || N == 2)) {
    using V = typename std::conditional<N == 4, uint2, unsigned>::type;
    V t;
    TS* h = reinterpret_cast<TS*>(&t);
#pragma unroll
    for (int m = 0; m < N; ++m) store_as<TS, float>(h + m, v[m]);
    *reinterpret_cast<V*>(p) = t;
  } else {
#pragma unroll
    for (int m = 0; m < N; ++m) store_as<TS, float>(p + m, v[m]);
  }
}

// A whole cell of N^3 values as FP32: 16-byte loads for FP32 storage when the cell is a multiple of
// 16 bytes (n = 2: 32 bytes), else row by row (FP16/BF16 storage measured ~5 % slower whole).
template <typename TS, int N>
__device__ __forceinline__ void ld_cell(float (&v)[N * N * N], const TS* p) {
  constexpr int B = N * N * N * (int)sizeof(TS);
  if constexpr (B % 16 == 0 && sizeof(TS) == 4) {
    constexpr int W = 16 / (int)sizeof(TS);  // values per 16-byte load
#pragma unroll
    for (int k = 0; k < B / 16; ++k) {
      const uint4 t = __ldg(reinterpret_cast<const uint4*>(p) + k);
      const TS* h = reinterpret_cast<const TS*>(&t);
#pragma unroll
      for (int m = 0; m < W; ++m) v[k * W + m] = load_cvt(h[m]);
    }
  } else {
#pragma unroll
    for (int r = 0; r < N * N; ++r) {
      float row[N];
      ld_row<TS, N>(row, p + r * N);
#pragma unroll
      for (int i = 0; i < N; ++i) v[r * N + i] = row[i];
    }
  }
}
template <typename TS, int N>
__device__ __forceinline__ void st_cell(TS* p, const float (&v)[N * N * N]) {
  constexpr int B = N * N * N * (int)sizeof(TS);
  if constexpr (B % 16 == 0 && sizeof(TS) == 4) {
    constexpr int W = 16 / (int)sizeof(TS);
#pragma unroll
    for (int k = 0; k < B / 16; ++k) {
      uint4 t;
      TS* h = reinterpret_cast<TS*>(&t);
#pragma unroll
      for (int m = 0; m < W; ++m) store_as<TS, float>(h + m, v[k * W + m]);
      reinterpret_cast<uint4*>(p)[k] = t;
    }
  } else {
#pragma unroll
    for (int r = 0; r < N * N; ++r) {
      float row[N];
#pragma unroll
      for (int i = 0; i < N; ++i) row[i] = v[r * N + i];
      st_row<TS, N>(p + r * N, row);
    }
  }
}

// Element (l, j, i) of a cell tensor in registers.
template <int N>
__device__ __forceinline__ constexpr int id3(int l, int j, int i) { return (l * N + j) * N + i; }

// acc[i] += sum_m A[i][m] in[m] for the N x N matrix A (row pitch S)
template <int N, int S>
__device__ __forceinline__ void mac(float (&acc)[N], const float* __restrict__ A, const float (&in)[N]) {
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int m = 0; m < N; ++m) acc[i] = fmaf(A[i * S + m], in[m], acc[i]);
}

// Direction d (0: x, 1: y, 2: z) of w += (M^-1 L)_d u with its two faces. For the lines of
// direction d the kernel walks the cell in slabs: a slab is the N lines that one set of N
// neighbour rows serves (d = 0: one x-row per line; d = 1: the rows (l, 0..N-1) of plane l hold
// the y-lines (l, i); d = 2: the rows (0..N-1, j) hold the z-lines (j, i)).
template <typename TS, int N, int d>
__device__ __forceinline__ void dir_terms(float (&w)[N * N * N], const float (&u)[N * N * N], const TS* lo,
                                          const TS* hi, const CptConst<N>& P) {
  constexpr int S = CptConst<N>::S, N2 = N * N;
  // element of line t (0..N-1) of slab s, node m along d
  auto at = [](int s, int t, int m) {
    return d == 0 ? id3<N>(s / N, s % N, m) : (d == 1 ? id3<N>(s, m, t) : id3<N>(m, s, t));
  };
  // row r (0..N-1) of slab s: its offset in a cell (the row holds node r of the slab's N lines along d)
  auto row = [](int s, int r) { return d == 1 ? id3<N>(s, r, 0) : id3<N>(r, s, 0); };
  constexpr int slabs = d == 0 ? N2 : N;
  // FP32 cells of at most 16 values are read whole (16-byte loads) instead of row by row: at n = 2
  // that halves the load instructions of this L1-bound kernel (273 -> 385 GDoF/s at 160^3)
  constexpr bool WHOLE = N * N * N <= 16 && sizeof(TS) == 4;
  float cl[WHOLE ? N * N * N : 1], ch[WHOLE ? N * N * N : 1];
  if constexpr (WHOLE) {
    if (lo) ld_cell<TS, N>(cl, lo);
    if (hi) ld_cell<TS, N>(ch, hi);
  }
#pragma unroll
  for (int s = 0; s < slabs; ++s) {
    // the slab's lines: own values and the interior contraction
#pragma unroll
    for (int t = 0; t < (d == 0 ? 1 : N); ++t) {
      float ul[N], acc[N];
#pragma unroll
      for (int m = 0; m < N; ++m) {
        ul[m] = u[at(s, t, m)];
        acc[m] = 0.f;
      }
      mac<N, S>(acc, P.G[d], ul);
      // boundary faces from the own line
      if (!hi) {
        float sd = 0.f;
#pragma unroll
        for (int m = 0; m < N; ++m) sd = fmaf(P.d1[m], ul[m], sd);
#pragma unroll
        for (int i = 0; i < N; ++i) acc[i] = fmaf(P.E[d][4][i], ul[N - 1], fmaf(P.E[d][5][i], sd, acc[i]));
      }
      if (!lo) {
        float sd = 0.f;
#pragma unroll
        for (int m = 0; m < N; ++m) sd = fmaf(P.d0[m], ul[m], sd);
#pragma unroll
        for (int i = 0; i < N; ++i) acc[i] = fmaf(P.E[d][6][i], ul[0], fmaf(P.E[d][7][i], sd, acc[i]));
      }
#pragma unroll
      for (int m = 0; m < N; ++m) w[at(s, t, m)] += acc[m];
    }
    // neighbour faces: the N rows of the slab in the neighbour cell; for d = 0 the slab is one
    // x-row, which is the line itself
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const TS* nb = side ? hi : lo;
      if (!nb) continue;
      float r[N][N];  // r[q][t]: node q along d of line t
      if constexpr (WHOLE) {
        const float(&c)[WHOLE ? N * N * N : 1] = side ? ch : cl;
#pragma unroll
        for (int q = 0; q < N; ++q)
#pragma unroll
          for (int t = 0; t < (d == 0 ? 1 : N); ++t) r[q][t] = c[d == 0 ? id3<N>(s / N, s % N, q) : row(s, q) + t];
      } else if (d == 0) {
        float v[N];
        ld_row<TS, N>(v, nb + id3<N>(s / N, s % N, 0));
#pragma unroll
        for (int q = 0; q < N; ++q) r[q][0] = v[q];
      } else {
#pragma unroll
        for (int q = 0; q < N; ++q) ld_row<TS, N>(r[q], nb + row(s, q));
      }
#pragma unroll
      for (int t = 0; t < (d == 0 ? 1 : N); ++t) {
        float sd = 0.f, sv;
        if (side) {  // high neighbour: its node 0 is at the face
#pragma unroll
          for (int q = 0; q < N; ++q) sd = fmaf(P.d0[q], r[q][t], sd);
          sv = r[0][t];
#pragma unroll
          for (int i = 0; i < N; ++i) {
            float& wi = w[at(s, t, i)];
            wi = fmaf(P.E[d][0][i], sv, fmaf(P.E[d][1][i], sd, wi));
          }
        } else {  // low neighbour: its node N-1 is at the face
#pragma unroll
          for (int q = 0; q < N; ++q) sd = fmaf(P.d1[q], r[q][t], sd);
          sv = r[N - 1][t];
#pragma unroll
          for (int i = 0; i < N; ++i) {
            float& wi = w[at(s, t, i)];
            wi = fmaf(P.E[d][2][i], sv, fmaf(P.E[d][3][i], sd, wi));
          }
        }
      }
    }
  }
}

// v = M_d w along direction d, in place
template <int N, int d>
__device__ __forceinline__ void mass_dir(float (&w)[N * N * N], const CptConst<N>& P) {
  constexpr int S = CptConst<N>::S;
#pragma unroll
  for (int a = 0; a < N; ++a)
#pragma unroll
    for (int c = 0; c < N; ++c) {
      float in[N], out[N];
#pragma unroll
      for (int m = 0; m < N; ++m) {
        in[m] = w[d == 0 ? id3<N>(a, c, m) : (d == 1 ? id3<N>(a, m, c) : id3<N>(m, a, c))];
        out[m] = 0.f;
      }
      mac<N, S>(out, P.M[d], in);
#pragma unroll
      for (int m = 0; m < N; ++m) w[d == 0 ? id3<N>(a, c, m) : (d == 1 ? id3<N>(a, m, c) : id3<N>(m, a, c))] = out[m];
    }
}

template <typename TS, int N, bool RES>
__global__ void __launch_bounds__(128) apply_cpt_kernel(const TS* __restrict__ x, TS* __restrict__ y,
                                                        const TS* __restrict__ b, const __grid_constant__ CptConst<N> P,
                                                        int nx, int ny, int nz, long long c_begin, long long c_end) {
  constexpr int N3 = N * N * N;
  const long long cell = c_begin + (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= c_end) return;
  const int cx = (int)(cell % nx), cy = (int)((cell / nx) % ny), cz = (int)(cell / ((long long)nx * ny));
  const TS* xc = x + cell * N3;
  const long long sy = (long long)nx * N3, sz = (long long)nx * ny * N3;
  float u[N3], w[N3];
  ld_cell<TS, N>(u, xc);
#pragma unroll
  for (int e = 0; e < N3; ++e) w[e] = 0.f;
  dir_terms<TS, N, 0>(w, u, cx > 0 ? xc - N3 : nullptr, cx < nx - 1 ? xc + N3 : nullptr, P);
  dir_terms<TS, N, 1>(w, u, cy > 0 ? xc - sy : nullptr, cy < ny - 1 ? xc + sy : nullptr, P);
  dir_terms<TS, N, 2>(w, u, cz > 0 ? xc - sz : nullptr, cz < nz - 1 ? xc + sz : nullptr, P);
  mass_dir<N, 0>(w, P);
  mass_dir<N, 1>(w, P);
  mass_dir<N, 2>(w, P);
  if constexpr (RES) {
    float bv[N3];
    ld_cell<TS, N>(bv, b + cell * N3);
#pragma unroll
    for (int e = 0; e < N3; ++e) w[e] = bv[e] - w[e];
  }
  st_cell<TS, N>(y + cell * N3, w);
}

template <typename TS, int N>
cudaError_t launch_cpt_n(const tp_op_s* op, void* y, const void* x, long long c0, long long c1, cudaStream_t s,
                         const void* b) {
  const long long blocks = (c1 - c0 + 127) / 128;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  if (blocks <= 0) return cudaSuccess;
  const CptConst<N>& P = *static_cast<const CptConst<N>*>(op->hconst(sizeof(float)));
  if (b)
    apply_cpt_kernel<TS, N, true><<<(unsigned)blocks, 128, 0, s>>>(
        static_cast<const TS*>(x), static_cast<TS*>(y), static_cast<const TS*>(b), P, op->mesh.nx, op->mesh.ny,
        op->mesh.nz, c0, c1);
  else
    apply_cpt_kernel<TS, N, false><<<(unsigned)blocks, 128, 0, s>>>(
        static_cast<const TS*>(x), static_cast<TS*>(y), nullptr, P, op->mesh.nx, op->mesh.ny, op->mesh.nz, c0, c1);
  return cudaGetLastError();
}

template <typename TS>
cudaError_t launch_cpt_t(const tp_op_s* op, void* y, const void* x, long long c0, long long c1, cudaStream_t s,
                         const void* b) {
  if (op->n == 2) return launch_cpt_n<TS, 2>(op, y, x, c0, c1, s, b);
  return cudaErrorInvalidValue;
}

}  // namespace

// Output rows of cells [c0, c1) with one thread per cell (FP32, FP16 and BF16 vectors, n = 2);
// y = A x, or y = b - A x when b is not null.
cudaError_t launch_apply_cpt_range(const tp_op_s* op, void* y, const void* x, long long c0, long long c1,
                                   cudaStream_t s, const void* b) {
  switch (op->prec) {
    case TP_FP32: return launch_cpt_t<float>(op, y, x, c0, c1, s, b);
    case TP_FP16: return launch_cpt_t<__half>(op, y, x, c0, c1, s, b);
    case TP_BF16: return launch_cpt_t<__nv_bfloat16>(op, y, x, c0, c1, s, b);
    default: break;
  }
  return cudaErrorInvalidValue;
}

}  // namespace tp
