// Vertex-patch multiplicative Schwarz smoother (Sec. 7.1, after Cui et al. 2024 and Witte et
// al. 2021): the local solves of one colour of patches.
//
// A vertex patch is the 2 x 2 x 2 block of cells around an interior vertex v (1 <= v_d <= nc_d
// - 1), P = 2n nodes per direction. On a Cartesian mesh the restriction of Eq. (9) to a patch
// is again a Kronecker sum, of the 1D factors restricted to the patch's two cells:
//   A_P = L_z (x) M_y (x) M_x + M_z (x) L_y (x) M_x + M_z (x) M_y (x) L_x   (P x P factors),
// so with the 1D generalized eigenpairs L S = M S diag(lam), S^T M S = I, the local solve is
// exact fast diagonalization:
//   A_P^{-1} r = (S_z (x) S_y (x) S_x) diag(1 / (lam_x + lam_y + lam_z)) (S_z (x) S_y (x) S_x)^T r,
// six P x P contractions and one scaling per patch DoF. The 1D patch factors depend only on
// whether the patch's left / right cell touches the boundary (type t = [v == 1] + 2 [v == nc - 1]),
// so each level holds 3 x 4 eigenbases, computed on the host in FP64.
//
// The colour of a patch is the parity of its vertex; patches of one colour share no DoF, so one
// thread block per patch adds its correction x_P += A_P^{-1} r_P without atomics. The sweep
// over colours, with the residual r = b - A x formed before each colour, is in mg.cu.
//
// Work layout: P^2 / 2 threads per patch; in every phase a thread owns two lines of the patch
// tensor along the contracted direction (rows padded to P + 1 against bank conflicts). Phases: S_x^T,
// S_y^T, then along z S_z^T, the scaling and S_z, then S_y and S_x; the patch tensor is read from
// r and added to x cell by cell, so that a warp's accesses are contiguous.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <type_traits>
#include <vector>

#include "apply_common.cuh"
#include "tp_internal.h"

namespace tp {

tp_status cuda_status(int err, const char* what);

namespace {

constexpr int kMaxP = 2 * kMaxN;  // patch nodes per direction (k <= 7)

struct VPDims {
  int nx, ny, nz;
  int first[3];  // vertex of the colour's first patch per direction (1 or 2)
};

// patches of parity p along a direction with nc cells: vertices p, p + 2, ... in [1, nc - 1]
__host__ __device__ inline int vp_count(int p, int nc) { return p ? nc / 2 : (nc - 1) / 2; }

// Widest vector type that tiles a row of P values: the basis rows are read with one wide
// shared-memory load per W coefficients (the kernel is bound by load instructions otherwise).
template <typename T, int P> struct RowVec { using V = float2; };
template <int P> struct RowVec<float, P> { using V = typename std::conditional<P % 4 == 0, float4, float2>::type; };
template <int P> struct RowVec<double, P> { using V = double2; };

// Two dot products of one basis row with two lines: each wide load of the row serves both.
template <typename T, int P>
__device__ __forceinline__ void dot_row2(const T* __restrict__ row, const T (&a)[P], const T (&b)[P], T& sa, T& sb) {
  using V = typename RowVec<T, P>::V;
  constexpr int W = sizeof(V) / sizeof(T);
  const V* rv = reinterpret_cast<const V*>(row);
  sa = T(0);
  sb = T(0);
#pragma unroll
  for (int m = 0; m < P / W; ++m) {
    const V c = rv[m];
    const T* cc = reinterpret_cast<const T*>(&c);
#pragma unroll
    for (int w = 0; w < W; ++w) {
      sa = fma(cc[w], a[m * W + w], sa);
      sb = fma(cc[w], b[m * W + w], sb);
    }
  }
}

// The bases and eigenvalues of interior patches (boundary type 0 in every direction: on fine levels
// nearly every patch), passed as a kernel parameter: their entries become constant-bank operands of
// the FMAs, so an interior patch loads no table into shared memory and reads no basis row from it.
// An interior patch's 1D factors are mirror-symmetric about the patch vertex, so its eigenvectors
// are even or odd (computed as such, in the even and odd subspaces): H = P/2 of each. In the
// kernel's eigen coordinates the even ones come first. E[d][m * H + c] is component m < H of even
// eigenvector c (component P-1-m is the same), O[d][m * H + c] that of odd eigenvector c (component
// P-1-m is its negative), lam[d] the eigenvalues in the same order. A contraction then costs P^2/2
// multiply-adds instead of P^2 (as the even-odd form of the CUDA-core kernel's 1D matrices), and the
// parameter holds half the entries. Measured on the FP32 vertex-patch V-cycle, against full bases in
// the parameter for P <= 8 and shared-memory bases above: k = 2 6.51 -> 6.21 ms (96^3), k = 3
// 19.41 -> 18.92 ms (128^3), k = 5 14.93 -> 14.14 ms (54^3), k = 7 7.84 -> 7.33 ms (40^3). The FP64
// kernel, bound by the FP64 pipe, measured slower with full bases in the parameter and keeps the
// shared-memory path: the path serves FP32 arithmetic, and the other instantiations take an empty
// parameter.
template <typename T, int P>
struct VPInterior {
  T E[3][(P / 2) * (P / 2)];
  T O[3][(P / 2) * (P / 2)];
  T lam[3][P];
};
struct VPNone {
  int unused;
};
template <typename T, int P>
__host__ __device__ constexpr bool vp_const_interior() { return sizeof(T) == 4 && P <= 16; }
template <typename T, int P>
using VPArg = typename std::conditional<vp_const_interior<T, P>(), VPInterior<T, P>, VPNone>::type;

// S^T applied to two lines in the even/odd eigenbasis (E, O from the kernel parameter): outputs in
// eigen coordinates, the even ones first
template <typename T, int P>
__device__ __forceinline__ void eo_fwd2(const T* E, const T* O, const T (&a)[P], const T (&b)[P], T (&ya)[P],
                                        T (&yb)[P]) {
  constexpr int H = P / 2;
  T ea[H], oa[H], eb[H], ob[H];
#pragma unroll
  for (int m = 0; m < H; ++m) {
    ea[m] = a[m] + a[P - 1 - m];
    oa[m] = a[m] - a[P - 1 - m];
    eb[m] = b[m] + b[P - 1 - m];
    ob[m] = b[m] - b[P - 1 - m];
  }
#pragma unroll
  for (int c = 0; c < H; ++c) {
    T se = T(0), so = T(0), te = T(0), to = T(0);
#pragma unroll
    for (int m = 0; m < H; ++m) {
      se = fma(E[m * H + c], ea[m], se);
      te = fma(E[m * H + c], eb[m], te);
      so = fma(O[m * H + c], oa[m], so);
      to = fma(O[m * H + c], ob[m], to);
    }
    ya[c] = se;
    yb[c] = te;
    ya[H + c] = so;
    yb[H + c] = to;
  }
}
// S applied to two lines given in eigen coordinates (even first): node values
template <typename T, int P>
__device__ __forceinline__ void eo_inv2(const T* E, const T* O, const T (&a)[P], const T (&b)[P], T (&ya)[P],
                                        T (&yb)[P]) {
  constexpr int H = P / 2;
#pragma unroll
  for (int X = 0; X < H; ++X) {
    T se = T(0), so = T(0), te = T(0), to = T(0);
#pragma unroll
    for (int c = 0; c < H; ++c) {
      se = fma(E[X * H + c], a[c], se);
      te = fma(E[X * H + c], b[c], te);
      so = fma(O[X * H + c], a[H + c], so);
      to = fma(O[X * H + c], b[H + c], to);
    }
    ya[X] = se + so;
    ya[P - 1 - X] = se - so;
    yb[X] = te + to;
    yb[P - 1 - X] = te - to;
  }
}

// dynamic shared memory of the patch kernel: two padded patch tensors, six P x P bases (S^T and S
// per direction), 3P eigenvalues
template <typename T, int N>
constexpr size_t vp_smem_bytes() {
  return sizeof(T) * (2 * (2 * N) * (2 * N) * (2 * N + 1) + 6 * (2 * N) * (2 * N) + 3 * (2 * N));
}

// FP32 vectors at n = 4 (k = 3) with 16-byte aligned x and r: global accesses by whole cell rows
// (one 16-byte load or store per row, four rows per thread) instead of single values. A warp's rows
// are two x-adjacent cells (512 contiguous bytes), and the shared stores of its rows' values hit 32
// distinct banks, where the value-by-value scatter met two-way conflicts.
template <typename TS, int N>
__host__ __device__ constexpr bool vp_rows() { return std::is_same<TS, float>::value && N == 4; }

// P^2 / 2 threads per patch; in every phase a thread owns two lines of the contracted direction,
// lines p0 and p0 + P/2 of the outer index, so that each basis row it loads serves two lines.
// TS: storage type of x and r; T: arithmetic type (FP32 for FP16/BF16 storage) of the tables and
// of every operation. ROWS: the row-wise global accesses above (only where vp_rows holds).
template <typename TS, typename T, int N, bool ROWS>
__global__ void __launch_bounds__(2 * N * N)
vp_patch_kernel(TS* __restrict__ x, const TS* __restrict__ r, const T* __restrict__ Stab, const T* __restrict__ Ltab,
                VPDims D, const __grid_constant__ VPArg<T, 2 * N> C) {
  constexpr int P = 2 * N, R = P + 1, N3 = N * N * N, H = P / 2, NT = P * H;
  extern __shared__ __align__(16) unsigned char vp_smem[];
  T* bufA = reinterpret_cast<T*>(vp_smem);
  T* bufB = bufA + P * P * R;
  T (*sF)[P * P] = reinterpret_cast<T (*)[P * P]>(bufB + P * P * R);  // sF[d][a * P + m] = S_d[m][a]
  T (*sB)[P * P] = sF + 3;                                               // sB[d][X * P + a] = S_d[X][a]
  T (*sL)[P] = reinterpret_cast<T (*)[P]>(bufB + P * P * R + 6 * P * P);
  const int tid = threadIdx.x, p0 = tid / P, p1 = p0 + H, q = tid % P;
  const int vx = D.first[0] + 2 * (int)blockIdx.x, vy = D.first[1] + 2 * (int)blockIdx.y;
  const int vz = D.first[2] + 2 * (int)blockIdx.z;
  const int t[3] = {(vx == 1 ? 1 : 0) + (vx == D.nx - 1 ? 2 : 0), (vy == 1 ? 1 : 0) + (vy == D.ny - 1 ? 2 : 0),
                    (vz == 1 ? 1 : 0) + (vz == D.nz - 1 ? 2 : 0)};
  constexpr bool kConst = vp_const_interior<T, 2 * N>();
  const bool interior = kConst && (t[0] | t[1] | t[2]) == 0;  // block-uniform
  if (!interior) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int e = tid + h * NT, X = e / P, a = e % P;
        const T v = Stab[(size_t)(d * 4 + t[d]) * kMaxP * kMaxP + X * kMaxP + a];  // S_d[X][a]
        sB[d][X * P + a] = v;
        sF[d][a * P + X] = v;
      }
      if (tid < P) sL[d][tid] = Ltab[(d * 4 + t[d]) * kMaxP + tid];
    }
  }
  // The patch's cells are (v - 1 + lx, v - 1 + ly, v - 1 + lz), lx, ly, lz in {0, 1}. Global
  // accesses walk the patch cell by cell (e = lc * n^3 + node: a warp reads contiguous values of
  // one cell) and map each value to its patch coordinates (Z, Y, X).
  const long long c0 = ((long long)(vz - 1) * D.ny + (vy - 1)) * D.nx + (vx - 1);
  auto gaddr = [&](int e) {
    const int lc = e / N3;
    return (c0 + ((long long)(lc >> 2) * D.ny + ((lc >> 1) & 1)) * D.nx + (lc & 1)) * N3 + e % N3;
  };
  auto saddr = [&](int e) {
    const int lc = e / N3, node = e % N3;
    const int X = (lc & 1) * N + node % N, Y = ((lc >> 1) & 1) * N + (node / N) % N, Z = (lc >> 2) * N + node / (N * N);
    return (Z * P + Y) * R + X;
  };
  // Row-wise form: row tid + NT * i of the patch (4 per thread) is row rr = tid % N^2 (nodes
  // rr * N .. rr * N + N - 1) of local cell lc = 2 i + tid / N^2.
  static_assert(!ROWS || (vp_rows<TS, N>() && NT == 2 * N * N), "row-wise accesses: FP32 vectors, n = 4");
  auto grow = [&](int i) {
    const int lc = 2 * i + tid / (N * N);
    return (c0 + ((long long)(lc >> 2) * D.ny + ((lc >> 1) & 1)) * D.nx + (lc & 1)) * N3 + (tid % (N * N)) * N;
  };
  auto srow = [&](int i) {
    const int lc = 2 * i + tid / (N * N), rr = tid % (N * N);
    return (((lc >> 2) * N + rr / N) * P + ((lc >> 1) & 1) * N + rr % N) * R + (lc & 1) * N;
  };
  if constexpr (ROWS) {
    float4 v[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = __ldg(reinterpret_cast<const float4*>(r + grow(i)));
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      T* d = bufA + srow(i);
      d[0] = v[i].x;
      d[1] = v[i].y;
      d[2] = v[i].z;
      d[3] = v[i].w;
    }
  } else {
    T v[2 * P];  // all loads in flight before the shared stores
#pragma unroll
    for (int j = 0; j < 2 * P; ++j) v[j] = load_as<TS, T>(r + gaddr(tid + j * NT));
#pragma unroll
    for (int j = 0; j < 2 * P; ++j) bufA[saddr(tid + j * NT)] = v[j];
  }
  __syncthreads();
  if constexpr (!kConst) {
    (void)C;
  }
  if (interior) {
    // the same six phases with the bases and eigenvalues from the kernel parameter
    if constexpr (kConst) {
    T i0[P], i1[P], y0[P], y1[P];
    // S_x^T along x-lines (Z = p, Y = q): bufA -> bufB
#pragma unroll
    for (int m = 0; m < P; ++m) {
      i0[m] = bufA[(p0 * P + q) * R + m];
      i1[m] = bufA[(p1 * P + q) * R + m];
    }
    eo_fwd2<T, P>(C.E[0], C.O[0], i0, i1, y0, y1);
#pragma unroll
    for (int a = 0; a < P; ++a) {
      bufB[(p0 * P + q) * R + a] = y0[a];
      bufB[(p1 * P + q) * R + a] = y1[a];
    }
    __syncthreads();
    // S_y^T along y-lines (Z = p, a = q): bufB -> bufA
#pragma unroll
    for (int m = 0; m < P; ++m) {
      i0[m] = bufB[(p0 * P + m) * R + q];
      i1[m] = bufB[(p1 * P + m) * R + q];
    }
    eo_fwd2<T, P>(C.E[1], C.O[1], i0, i1, y0, y1);
#pragma unroll
    for (int b = 0; b < P; ++b) {
      bufA[(p0 * P + b) * R + q] = y0[b];
      bufA[(p1 * P + b) * R + q] = y1[b];
    }
    __syncthreads();
    // z-lines (b = p, a = q): S_z^T, the scaling, S_z, in registers (a thread owns its z-lines)
#pragma unroll
    for (int m = 0; m < P; ++m) {
      i0[m] = bufA[(m * P + p0) * R + q];
      i1[m] = bufA[(m * P + p1) * R + q];
    }
    eo_fwd2<T, P>(C.E[2], C.O[2], i0, i1, y0, y1);
    {
      const T l0 = C.lam[0][q] + C.lam[1][p0], l1 = C.lam[0][q] + C.lam[1][p1];
#pragma unroll
      for (int c = 0; c < P; ++c) {
        y0[c] = y0[c] / (l0 + C.lam[2][c]);
        y1[c] = y1[c] / (l1 + C.lam[2][c]);
      }
    }
    eo_inv2<T, P>(C.E[2], C.O[2], y0, y1, i0, i1);
#pragma unroll
    for (int Z = 0; Z < P; ++Z) {
      bufA[(Z * P + p0) * R + q] = i0[Z];
      bufA[(Z * P + p1) * R + q] = i1[Z];
    }
    __syncthreads();
    // S_y along y-lines (Z = p, a = q): bufA -> bufB
#pragma unroll
    for (int b = 0; b < P; ++b) {
      i0[b] = bufA[(p0 * P + b) * R + q];
      i1[b] = bufA[(p1 * P + b) * R + q];
    }
    eo_inv2<T, P>(C.E[1], C.O[1], i0, i1, y0, y1);
#pragma unroll
    for (int Y = 0; Y < P; ++Y) {
      bufB[(p0 * P + Y) * R + q] = y0[Y];
      bufB[(p1 * P + Y) * R + q] = y1[Y];
    }
    __syncthreads();
    // S_x along x-lines (Z = p, Y = q): bufB -> bufA
#pragma unroll
    for (int a = 0; a < P; ++a) {
      i0[a] = bufB[(p0 * P + q) * R + a];
      i1[a] = bufB[(p1 * P + q) * R + a];
    }
    eo_inv2<T, P>(C.E[0], C.O[0], i0, i1, y0, y1);
#pragma unroll
    for (int X = 0; X < P; ++X) {
      bufA[(p0 * P + q) * R + X] = y0[X];
      bufA[(p1 * P + q) * R + X] = y1[X];
    }
    __syncthreads();
    }
  } else {
    // Two lines of the patch tensor in registers, contracted per output node o with a basis row:
    // sum_m S[m][o] in[m] (S^T applied, rows of sF) or sum_m S[o][m] in[m] (S applied, rows of sB);
    // each output goes straight to shared memory.
    T i0[P], i1[P], s0, s1;
    // S_x^T along x-lines (Z = p, Y = q): bufA -> bufB
  #pragma unroll
    for (int m = 0; m < P; ++m) {
      i0[m] = bufA[(p0 * P + q) * R + m];
      i1[m] = bufA[(p1 * P + q) * R + m];
    }
  #pragma unroll 2
    for (int a = 0; a < P; ++a) {
      dot_row2<T, P>(sF[0] + a * P, i0, i1, s0, s1);
      bufB[(p0 * P + q) * R + a] = s0;
      bufB[(p1 * P + q) * R + a] = s1;
    }
    __syncthreads();
    // S_y^T along y-lines (Z = p, a = q): bufB -> bufA
  #pragma unroll
    for (int m = 0; m < P; ++m) {
      i0[m] = bufB[(p0 * P + m) * R + q];
      i1[m] = bufB[(p1 * P + m) * R + q];
    }
  #pragma unroll 2
    for (int b = 0; b < P; ++b) {
      dot_row2<T, P>(sF[1] + b * P, i0, i1, s0, s1);
      bufA[(p0 * P + b) * R + q] = s0;
      bufA[(p1 * P + b) * R + q] = s1;
    }
    __syncthreads();
    // z-lines (b = p, a = q): S_z^T and the eigenvalue scaling into bufB, then S_z back into bufA.
    // A thread reads and writes only its own z-lines here, so no barrier is needed in between.
  #pragma unroll
    for (int m = 0; m < P; ++m) {
      i0[m] = bufA[(m * P + p0) * R + q];
      i1[m] = bufA[(m * P + p1) * R + q];
    }
    {
      const T l0 = sL[0][q] + sL[1][p0], l1 = sL[0][q] + sL[1][p1];
  #pragma unroll 2
      for (int c = 0; c < P; ++c) {
        dot_row2<T, P>(sF[2] + c * P, i0, i1, s0, s1);
        bufB[(c * P + p0) * R + q] = s0 / (l0 + sL[2][c]);
        bufB[(c * P + p1) * R + q] = s1 / (l1 + sL[2][c]);
      }
    }
  #pragma unroll
    for (int c = 0; c < P; ++c) {
      i0[c] = bufB[(c * P + p0) * R + q];
      i1[c] = bufB[(c * P + p1) * R + q];
    }
  #pragma unroll 2
    for (int Z = 0; Z < P; ++Z) {
      dot_row2<T, P>(sB[2] + Z * P, i0, i1, s0, s1);
      bufA[(Z * P + p0) * R + q] = s0;
      bufA[(Z * P + p1) * R + q] = s1;
    }
    __syncthreads();
    // S_y along y-lines (Z = p, a = q): bufA -> bufB
  #pragma unroll
    for (int b = 0; b < P; ++b) {
      i0[b] = bufA[(p0 * P + b) * R + q];
      i1[b] = bufA[(p1 * P + b) * R + q];
    }
  #pragma unroll 2
    for (int Y = 0; Y < P; ++Y) {
      dot_row2<T, P>(sB[1] + Y * P, i0, i1, s0, s1);
      bufB[(p0 * P + Y) * R + q] = s0;
      bufB[(p1 * P + Y) * R + q] = s1;
    }
    __syncthreads();
    // S_x along x-lines (Z = p, Y = q): bufB -> bufA
  #pragma unroll
    for (int a = 0; a < P; ++a) {
      i0[a] = bufB[(p0 * P + q) * R + a];
      i1[a] = bufB[(p1 * P + q) * R + a];
    }
  #pragma unroll 2
    for (int X = 0; X < P; ++X) {
      dot_row2<T, P>(sB[0] + X * P, i0, i1, s0, s1);
      bufA[(p0 * P + q) * R + X] = s0;
      bufA[(p1 * P + q) * R + X] = s1;
    }
    __syncthreads();
  }
  // x_P += the correction, cell by cell like the gather
  if constexpr (ROWS) {
    float4 v[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = *reinterpret_cast<const float4*>(x + grow(i));
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const T* c = bufA + srow(i);
      v[i].x += c[0];
      v[i].y += c[1];
      v[i].z += c[2];
      v[i].w += c[3];
      *reinterpret_cast<float4*>(x + grow(i)) = v[i];
    }
  } else {
    T v[2 * P];
#pragma unroll
    for (int j = 0; j < 2 * P; ++j) v[j] = static_cast<T>(x[gaddr(tid + j * NT)]);
#pragma unroll
    for (int j = 0; j < 2 * P; ++j) store_as<TS, T>(x + gaddr(tid + j * NT), v[j] + bufA[saddr(tid + j * NT)]);
  }
}

template <typename T, int P>
VPArg<T, P> vp_arg(const void* C) {
  if constexpr (vp_const_interior<T, P>()) {
    return *static_cast<const VPInterior<T, P>*>(C);
  } else {
    return VPNone{0};
  }
}

template <typename TS, typename T, int N>
cudaError_t launch_colour(int colour, const int nc[3], void* x, const void* r, const void* S, const void* L,
                          const void* Cint, cudaStream_t s) {
  const int par[3] = {colour & 1, (colour >> 1) & 1, (colour >> 2) & 1};
  const dim3 grid(vp_count(par[0], nc[0]), vp_count(par[1], nc[1]), vp_count(par[2], nc[2]));
  if (grid.x == 0 || grid.y == 0 || grid.z == 0) return cudaSuccess;
  if (grid.y > 65535 || grid.z > 65535) return cudaErrorInvalidConfiguration;
  VPDims D{nc[0], nc[1], nc[2], {par[0] ? 1 : 2, par[1] ? 1 : 2, par[2] ? 1 : 2}};
  if constexpr (vp_rows<TS, N>()) {
    if ((((uintptr_t)x | (uintptr_t)r) & 15) == 0) {
      vp_patch_kernel<TS, T, N, true><<<grid, 2 * N * N, vp_smem_bytes<T, N>(), s>>>(
          static_cast<TS*>(x), static_cast<const TS*>(r), static_cast<const T*>(S), static_cast<const T*>(L), D,
          vp_arg<T, 2 * N>(Cint));
      return cudaGetLastError();
    }
  }
  vp_patch_kernel<TS, T, N, false><<<grid, 2 * N * N, vp_smem_bytes<T, N>(), s>>>(
      static_cast<TS*>(x), static_cast<const TS*>(r), static_cast<const T*>(S), static_cast<const T*>(L), D,
      vp_arg<T, 2 * N>(Cint));
  return cudaGetLastError();
}

template <typename TS, typename T, int N>
cudaError_t prepare_colour() {
  cudaError_t e = cudaFuncSetAttribute(vp_patch_kernel<TS, T, N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)vp_smem_bytes<T, N>());
  if constexpr (vp_rows<TS, N>()) {
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(vp_patch_kernel<TS, T, N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)vp_smem_bytes<T, N>());
  }
  return e;
}

template <typename TS, typename T>
cudaError_t prepare_t(int n) {
  switch (n) {
    case 2: return prepare_colour<TS, T, 2>();
    case 3: return prepare_colour<TS, T, 3>();
    case 4: return prepare_colour<TS, T, 4>();
    case 5: return prepare_colour<TS, T, 5>();
    case 6: return prepare_colour<TS, T, 6>();
    case 7: return prepare_colour<TS, T, 7>();
    case 8: return prepare_colour<TS, T, 8>();
  }
  return cudaErrorInvalidValue;
}

template <typename TS, typename T>
cudaError_t launch_colour_t(int n, int colour, const int nc[3], void* x, const void* r, const void* S, const void* L,
                            const void* C, cudaStream_t s) {
  switch (n) {
    case 2: return launch_colour<TS, T, 2>(colour, nc, x, r, S, L, C, s);
    case 3: return launch_colour<TS, T, 3>(colour, nc, x, r, S, L, C, s);
    case 4: return launch_colour<TS, T, 4>(colour, nc, x, r, S, L, C, s);
    case 5: return launch_colour<TS, T, 5>(colour, nc, x, r, S, L, C, s);
    case 6: return launch_colour<TS, T, 6>(colour, nc, x, r, S, L, C, s);
    case 7: return launch_colour<TS, T, 7>(colour, nc, x, r, S, L, C, s);
    case 8: return launch_colour<TS, T, 8>(colour, nc, x, r, S, L, C, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

// true if colour c (vertex parities c & 1, c >> 1 & 1, c >> 2 & 1) has a patch on the mesh
bool vp_colour_nonempty(const int nc[3], int c) {
  return vp_count(c & 1, nc[0]) > 0 && vp_count((c >> 1) & 1, nc[1]) > 0 && vp_count((c >> 2) & 1, nc[2]) > 0;
}

// x_P += A_P^{-1} r_P for every patch of colour c (FP64 or FP32 vectors, or FP16/BF16 storage with
// FP32 arithmetic; every nc >= 2).
cudaError_t vp_colour(tp_precision prec, int n, const int nc[3], int colour, void* x, const void* r, const void* S,
                      const void* L, const void* C, cudaStream_t s) {
  switch (prec) {
    case TP_FP64: return launch_colour_t<double, double>(n, colour, nc, x, r, S, L, C, s);
    case TP_FP32: return launch_colour_t<float, float>(n, colour, nc, x, r, S, L, C, s);
    case TP_FP16: return launch_colour_t<__half, float>(n, colour, nc, x, r, S, L, C, s);
    case TP_BF16: return launch_colour_t<__nv_bfloat16, float>(n, colour, nc, x, r, S, L, C, s);
  }
  return cudaErrorInvalidValue;
}

namespace {

// the interior bases and eigenvalues of a level as the kernel parameter's bytes, from the even and
// odd half-bases EO[d] (2 H x H: even then odd, [m * H + c]) and their eigenvalues LEO[d] (even then odd)
template <typename T, int P>
void fill_interior(std::vector<unsigned char>& out, const std::vector<double> (&EO)[3], const std::vector<double> (&LEO)[3]) {
  constexpr int H = P / 2;
  VPInterior<T, P> c{};
  for (int d = 0; d < 3; ++d) {
    if (EO[d].empty()) continue;  // no interior vertex in this direction: no patch takes the tables
    for (int e = 0; e < H * H; ++e) {
      c.E[d][e] = (T)EO[d][e];
      c.O[d][e] = (T)EO[d][H * H + e];
    }
    for (int a = 0; a < P; ++a) c.lam[d][a] = (T)LEO[d][a];
  }
  out.assign(reinterpret_cast<const unsigned char*>(&c), reinterpret_cast<const unsigned char*>(&c) + sizeof(c));
}

template <typename T>
void fill_interior_t(int n, std::vector<unsigned char>& out, const std::vector<double> (&EO)[3],
                     const std::vector<double> (&LEO)[3]) {
  switch (n) {
    case 2: fill_interior<T, 4>(out, EO, LEO); break;
    case 3: fill_interior<T, 6>(out, EO, LEO); break;
    case 4: fill_interior<T, 8>(out, EO, LEO); break;
    case 5: fill_interior<T, 10>(out, EO, LEO); break;
    case 6: fill_interior<T, 12>(out, EO, LEO); break;
    case 7: fill_interior<T, 14>(out, EO, LEO); break;
    case 8: fill_interior<T, 16>(out, EO, LEO); break;
  }
}

// The eigenpairs of a mirror-symmetric P x P pencil (Mp, Lp) in its even and odd subspaces (basis
// vectors (e_m +- e_{P-1-m}) / sqrt(2), m < H): EO = [even half-components, odd half-components]
// (component m < H of the full eigenvector, each H x H as [m * H + c]), LEO = [even eigenvalues,
// odd eigenvalues]. The full vectors are M-orthonormal like those of gen_eig. False if the pencil is
// not mirror-symmetric or a reduced mass matrix is not positive definite.
bool split_even_odd(int P, const std::vector<double>& Mp, const std::vector<double>& Lp, std::vector<double>& EO,
                    std::vector<double>& LEO) {
  const int H = P / 2;
  double big = 0.0, asym = 0.0;
  for (int i = 0; i < P; ++i)
    for (int j = 0; j < P; ++j) {
      big = std::fmax(big, std::fabs(Lp[(size_t)i * P + j]) + std::fabs(Mp[(size_t)i * P + j]));
      asym = std::fmax(asym, std::fabs(Lp[(size_t)i * P + j] - Lp[(size_t)(P - 1 - i) * P + P - 1 - j]) +
                                 std::fabs(Mp[(size_t)i * P + j] - Mp[(size_t)(P - 1 - i) * P + P - 1 - j]));
    }
  if (asym > 1e-12 * big) return false;  // not mirror-symmetric: no even/odd eigenvectors
  EO.assign((size_t)2 * H * H, 0.0);
  LEO.assign((size_t)P, 0.0);
  for (int par = 0; par < 2; ++par) {
    const double sg = par ? -1.0 : 1.0;
    std::vector<double> Mr((size_t)H * H), Lr((size_t)H * H), lv, V;
    for (int i = 0; i < H; ++i)
      for (int j = 0; j < H; ++j) {
        const int ri = P - 1 - i, rj = P - 1 - j;
        Mr[(size_t)i * H + j] = 0.5 * (Mp[(size_t)i * P + j] + sg * Mp[(size_t)i * P + rj] + sg * Mp[(size_t)ri * P + j] +
                                       Mp[(size_t)ri * P + rj]);
        Lr[(size_t)i * H + j] = 0.5 * (Lp[(size_t)i * P + j] + sg * Lp[(size_t)i * P + rj] + sg * Lp[(size_t)ri * P + j] +
                                       Lp[(size_t)ri * P + rj]);
      }
    if (!gen_eig(H, Mr, Lr, lv, V)) return false;
    for (int m = 0; m < H; ++m)
      for (int c = 0; c < H; ++c) EO[(size_t)par * H * H + m * H + c] = V[(size_t)m * H + c] / std::sqrt(2.0);
    for (int c = 0; c < H; ++c) LEO[(size_t)par * H + c] = lv[c];
  }
  return true;
}

}  // namespace

// Eigenbases of the 1D patch factors of one level, uploaded in the arithmetic precision (FP64 for
// FP64 vectors, FP32 otherwise):
// S[(d*4 + t)][X * kMaxP + a] = component X of eigenvector a, L[(d*4 + t)][a] = its eigenvalue,
// for direction d and boundary type t. A mesh of min(nc, 4) cells with the level's h has every
// type of the level at its vertices 1 .. min(nc, 4) - 1. C_out: the interior (type 0) bases and
// eigenvalues as the bytes of the kernel's VPInterior parameter (zeros in a direction without
// interior vertices, where no patch takes them).
tp_status vp_tables(const tp_op_s* op, const int nc[3], tp_precision prec, void** S_out, void** L_out,
                    std::vector<unsigned char>* C_out) {
  const int n = op->n, P = 2 * n;
  std::vector<double> S((size_t)12 * kMaxP * kMaxP, 0.0), lam((size_t)12 * kMaxP, 0.0);
  std::vector<double> EO[3], LEO[3];  // interior patches: even/odd half-bases (kernel parameter)
  for (int d = 0; d < 3; ++d) {
    if (nc[d] < 2) { set_error("vertex-patch smoother: fewer than two cells in a direction"); return TP_ERR_UNSUPPORTED; }
    const int m = nc[d] >= 4 ? 4 : nc[d];
    std::vector<double> M, L;
    global_1d(op->ref, op->dir[d], m, M, L);
    const int N1 = m * n;
    for (int v = 1; v <= m - 1; ++v) {
      const int t = (v == 1 ? 1 : 0) + (v == m - 1 ? 2 : 0);
      std::vector<double> Mp((size_t)P * P), Lp((size_t)P * P), lv, V;
      for (int i = 0; i < P; ++i)
        for (int j = 0; j < P; ++j) {
          Mp[(size_t)i * P + j] = M[(size_t)((v - 1) * n + i) * N1 + (v - 1) * n + j];
          Lp[(size_t)i * P + j] = L[(size_t)((v - 1) * n + i) * N1 + (v - 1) * n + j];
        }
      if (!gen_eig(P, Mp, Lp, lv, V)) {
        set_error("vertex-patch smoother: patch mass matrix not positive definite");
        return TP_ERR_INVALID_ARG;
      }
      for (int X = 0; X < P; ++X)
        for (int a = 0; a < P; ++a) S[(size_t)(d * 4 + t) * kMaxP * kMaxP + X * kMaxP + a] = V[(size_t)X * P + a];
      for (int a = 0; a < P; ++a) lam[(size_t)(d * 4 + t) * kMaxP + a] = lv[a];
      if (t == 0 && !split_even_odd(P, Mp, Lp, EO[d], LEO[d])) {
        set_error("vertex-patch smoother: interior patch not mirror-symmetric or not positive definite");
        return TP_ERR_INVALID_ARG;
      }
    }
  }
  const size_t eb = prec == TP_FP64 ? 8 : 4;
  if (eb == 8) fill_interior_t<double>(n, *C_out, EO, LEO);
  else fill_interior_t<float>(n, *C_out, EO, LEO);
  std::vector<unsigned char> hS(S.size() * eb), hL(lam.size() * eb);
  for (size_t i = 0; i < S.size(); ++i) {
    if (eb == 8) reinterpret_cast<double*>(hS.data())[i] = S[i];
    else reinterpret_cast<float*>(hS.data())[i] = (float)S[i];
  }
  for (size_t i = 0; i < lam.size(); ++i) {
    if (eb == 8) reinterpret_cast<double*>(hL.data())[i] = lam[i];
    else reinterpret_cast<float*>(hL.data())[i] = (float)lam[i];
  }
  *S_out = *L_out = nullptr;
  const cudaError_t pe = prec == TP_FP64   ? prepare_t<double, double>(n)
                        : prec == TP_FP32 ? prepare_t<float, float>(n)
                        : prec == TP_FP16 ? prepare_t<__half, float>(n)
                                          : prepare_t<__nv_bfloat16, float>(n);
  tp_status st = cuda_status(pe, "vertex-patch kernel set-up");
  if (st == TP_OK) st = cuda_status(cudaMalloc(S_out, hS.size()), "vertex-patch tables");
  if (st == TP_OK) st = cuda_status(cudaMalloc(L_out, hL.size()), "vertex-patch tables");
  if (st == TP_OK) st = cuda_status(cudaMemcpy(*S_out, hS.data(), hS.size(), cudaMemcpyHostToDevice), "cudaMemcpy");
  if (st == TP_OK) st = cuda_status(cudaMemcpy(*L_out, hL.data(), hL.size(), cudaMemcpyHostToDevice), "cudaMemcpy");
  return st;
}

}  // namespace tp
