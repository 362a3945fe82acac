// Patch-wise SIPG apply over vertex patches (Sec. 2.1): the paper's form of the operator
// evaluation, on the FMA pipes (FP64 and FP32 vectors, k <= 7).
//
// A vertex patch is the 2 x 2 x 2 block of cells around an interior vertex v (1 <= v_d <= nc_d - 1),
// P = 2n nodes per direction. Its local operator is the Kronecker sum of Eq. (9),
//   A_P = L_z (x) M_y (x) M_x + M_z (x) L_y (x) M_x + M_z (x) M_y (x) L_x,
// with P x P 1D factors that carry a share of the cell integrals and the face integrals of the
// patch. In 1D the patch around v holds cells a = v - 1 and b = v; the face at v belongs to it,
// the boundary faces to the first and last patch, and a cell integral is split between the two
// patches that hold the cell (weight 1/2; weight 1 for the first and last cell). With the face
// terms of a cell on the left (F_l) and right (F_r) of a face and the full boundary faces B_0, B_1:
//   M_p = diag(w_a h Mhat, w_b h Mhat),
//   L_p = [ w_a Khat/h + F_l + [a = 0] B_0     L^{ab}                                ]
//         [ L^{ba}                            w_b Khat/h + F_r + [b = nc - 1] B_1   ]
//   F_l = g v1 v1^T - (v1 d1^T + d1 v1^T)/(2h),  F_r = g v0 v0^T + (v0 d0^T + d0 v0^T)/(2h),
//   L^{ab} = -g v1 v0^T - v1 d0^T/(2h) + d1 v0^T/(2h),  L^{ba} = (L^{ab})^T,
//   B_0 = g v0 v0^T + (v0 d0^T + d0 v0^T)/h,  B_1 = g v1 v1^T - (v1 d1^T + d1 v1^T)/h.
// Summed over the 1D patches these give the global 1D M and L, and since 3D vertex patches are
// products of 1D ones, the sum over 3D patches of E_P^T A_P E_P is A itself: the same operator as
// the cell-wise kernels, with every cell evaluated in up to eight patches.
//
// The factors depend only on the patch's boundary type per direction, t = [v = 1] + 2 [v = nc - 1],
// so the operator holds 3 x 4 pairs (M_p, L_p), computed on the host in FP64.
//
// One thread block per patch, P^2 threads; in each phase a thread owns one line of the patch
// tensor along the contracted direction (rows padded to P + 1 against bank conflicts):
//   (1) x-lines:  a = M_x u, b = L_x u
//   (2) y-lines:  c = M_y a, d = L_y a + M_y b
//   (3) z-lines:  y_P = L_z c + M_z d
// seven P x P contractions per patch line, 224 n + 8 flops per DoF in all (the paper's patch-wise
// count of Table 4 with N = P). Patches of one colour (vertex parity) share no cell, so the
// colours run as eight launches that add y_P into y without atomics, after y is cleared.
#include <cuda_runtime.h>

#include <vector>

#include "tp_internal.h"

namespace tp {

tp_status cuda_status(int err, const char* what);

namespace {

constexpr int kMaxP = 2 * kMaxN;

struct PwDims {
  int nx, ny, nz;
  int first[3];  // vertex of the colour's first patch per direction (1 or 2)
};

// patches of parity p along a direction with nc cells: vertices p, p + 2, ... in [1, nc - 1]
inline int pw_count(int p, int nc) { return p ? nc / 2 : (nc - 1) / 2; }

template <typename T, int N>
constexpr size_t pw_smem_bytes() {
  return sizeof(T) * (3 * (2 * N) * (2 * N) * (2 * N + 1) + 6 * (2 * N) * (2 * N));
}

// row i of A times a line (A row-major P x P in shared memory, read as uniform broadcasts)
template <typename T, int P>
__device__ __forceinline__ T pw_row(const T* __restrict__ A, int i, const T (&in)[P], T acc) {
#pragma unroll
  for (int m = 0; m < P; ++m) acc = fma(A[i * P + m], in[m], acc);
  return acc;
}

template <typename T, int N>
__global__ void __launch_bounds__(4 * N * N)
pw_patch_kernel(T* __restrict__ y, const T* __restrict__ x, const T* __restrict__ tab, PwDims D) {
  constexpr int P = 2 * N, R = P + 1, N3 = N * N * N, PP = P * P;
  extern __shared__ __align__(16) unsigned char pw_smem[];
  T* sU = reinterpret_cast<T*>(pw_smem);  // u, later y_P
  T* sA = sU + P * P * R;                  // a, later c
  T* sB = sA + P * P * R;                  // b, later d
  T* sM = sB + P * P * R;                  // [d][0] = M_p, [d][1] = L_p of direction d
  const int tid = threadIdx.x, p = tid / P, q = tid % P;
  const int vx = D.first[0] + 2 * (int)blockIdx.x, vy = D.first[1] + 2 * (int)blockIdx.y;
  const int vz = D.first[2] + 2 * (int)blockIdx.z;
  {
    const int t[3] = {(vx == 1 ? 1 : 0) + (vx == D.nx - 1 ? 2 : 0), (vy == 1 ? 1 : 0) + (vy == D.ny - 1 ? 2 : 0),
                      (vz == 1 ? 1 : 0) + (vz == D.nz - 1 ? 2 : 0)};
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int w = 0; w < 2; ++w)  // tab[((d * 4 + t) * 2 + w)][i * kMaxP + j]
        sM[(d * 2 + w) * PP + tid] = tab[(size_t)((d * 4 + t[d]) * 2 + w) * kMaxP * kMaxP + p * kMaxP + q];
  }
  // the patch's cells are (v - 1 + lx, v - 1 + ly, v - 1 + lz), lx, ly, lz in {0, 1}; global
  // accesses walk the patch cell by cell (e = lc * n^3 + node), so a warp touches contiguous values
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
  for (int e = tid; e < 8 * N3; e += PP) sU[saddr(e)] = x[gaddr(e)];
  __syncthreads();
  const T* Mx = sM;
  const T* Lx = sM + PP;
  const T* My = sM + 2 * PP;
  const T* Ly = sM + 3 * PP;
  const T* Mz = sM + 4 * PP;
  const T* Lz = sM + 5 * PP;
  {  // (1) x-line (Z = p, Y = q): a = M_x u, b = L_x u, each output row stored as computed
    T u[P];
#pragma unroll
    for (int m = 0; m < P; ++m) u[m] = sU[(p * P + q) * R + m];
#pragma unroll
    for (int i = 0; i < P; ++i) {
      sA[(p * P + q) * R + i] = pw_row<T, P>(Mx, i, u, T(0));
      sB[(p * P + q) * R + i] = pw_row<T, P>(Lx, i, u, T(0));
    }
  }
  __syncthreads();
  {  // (2) y-line (Z = p, X = q): c = M_y a, d = L_y a + M_y b (in place: the line is this thread's)
    T a[P], b[P];
#pragma unroll
    for (int m = 0; m < P; ++m) {
      a[m] = sA[(p * P + m) * R + q];
      b[m] = sB[(p * P + m) * R + q];
    }
#pragma unroll
    for (int j = 0; j < P; ++j) {
      sA[(p * P + j) * R + q] = pw_row<T, P>(My, j, a, T(0));
      sB[(p * P + j) * R + q] = pw_row<T, P>(My, j, b, pw_row<T, P>(Ly, j, a, T(0)));
    }
  }
  __syncthreads();
  {  // (3) z-line (Y = p, X = q): y_P = L_z c + M_z d
    T c[P], d[P];
#pragma unroll
    for (int m = 0; m < P; ++m) {
      c[m] = sA[(m * P + p) * R + q];
      d[m] = sB[(m * P + p) * R + q];
    }
#pragma unroll
    for (int l = 0; l < P; ++l) sU[(l * P + p) * R + q] = pw_row<T, P>(Mz, l, d, pw_row<T, P>(Lz, l, c, T(0)));
  }
  __syncthreads();
  for (int e = tid; e < 8 * N3; e += PP) {
    const long long g = gaddr(e);
    y[g] += sU[saddr(e)];
  }
}

template <typename T, int N>
cudaError_t pw_launch_n(const tp_op_s* op, void* y, const void* x, cudaStream_t s) {
  const int nc[3] = {op->mesh.nx, op->mesh.ny, op->mesh.nz};
  constexpr size_t smem = pw_smem_bytes<T, N>();
  cudaError_t e = cudaMemsetAsync(y, 0, (size_t)op->ndofs * sizeof(T), s);
  for (int colour = 0; colour < 8 && e == cudaSuccess; ++colour) {
    PwDims D{nc[0], nc[1], nc[2], {}};
    unsigned g[3];
    bool empty = false;
    for (int d = 0; d < 3; ++d) {
      const int par = (colour >> d) & 1;
      D.first[d] = par ? 1 : 2;
      const int cnt = pw_count(par, nc[d]);
      empty = empty || cnt <= 0;
      g[d] = (unsigned)(cnt > 0 ? cnt : 1);
    }
    if (empty) continue;
    pw_patch_kernel<T, N><<<dim3(g[0], g[1], g[2]), 4 * N * N, smem, s>>>(
        static_cast<T*>(y), static_cast<const T*>(x), static_cast<const T*>(op->pw_mats), D);
    e = cudaGetLastError();
  }
  return e;
}

template <typename T>
cudaError_t pw_launch_t(const tp_op_s* op, void* y, const void* x, cudaStream_t s) {
  switch (op->n) {
    case 2: return pw_launch_n<T, 2>(op, y, x, s);
    case 3: return pw_launch_n<T, 3>(op, y, x, s);
    case 4: return pw_launch_n<T, 4>(op, y, x, s);
    case 5: return pw_launch_n<T, 5>(op, y, x, s);
    case 6: return pw_launch_n<T, 6>(op, y, x, s);
    case 7: return pw_launch_n<T, 7>(op, y, x, s);
    case 8: return pw_launch_n<T, 8>(op, y, x, s);
  }
  return cudaErrorInvalidValue;
}

template <typename T, int N>
cudaError_t pw_prepare_n() {
  return cudaFuncSetAttribute(pw_patch_kernel<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)pw_smem_bytes<T, N>());
}

template <typename T>
cudaError_t pw_prepare_t(int n) {
  switch (n) {
    case 2: return pw_prepare_n<T, 2>();
    case 3: return pw_prepare_n<T, 3>();
    case 4: return pw_prepare_n<T, 4>();
    case 5: return pw_prepare_n<T, 5>();
    case 6: return pw_prepare_n<T, 6>();
    case 7: return pw_prepare_n<T, 7>();
    case 8: return pw_prepare_n<T, 8>();
  }
  return cudaErrorInvalidValue;
}

}  // namespace

// The 1D patch factors (M_p, L_p) of direction d and boundary type t (see the file header), P x P
// row-major, into M and L.
void pw_factors(const tp_op_s* op, int d, int t, std::vector<double>& M, std::vector<double>& L) {
  const int n = op->n, P = 2 * n;
  const Ref1D& r = op->ref;
  const double h = op->dir[d].h, g = op->dir[d].gamma, hh = 0.5 / h;
  const double wa = (t & 1) ? 1.0 : 0.5, wb = (t & 2) ? 1.0 : 0.5;
  M.assign((size_t)P * P, 0.0);
  L.assign((size_t)P * P, 0.0);
  auto v0 = [&](int i) { return i == 0 ? 1.0 : 0.0; };
  auto v1 = [&](int i) { return i == n - 1 ? 1.0 : 0.0; };
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      const double fl = g * v1(i) * v1(j) - (v1(i) * r.d1[j] + r.d1[i] * v1(j)) * hh;
      const double fr = g * v0(i) * v0(j) + (v0(i) * r.d0[j] + r.d0[i] * v0(j)) * hh;
      const double b0 = g * v0(i) * v0(j) + (v0(i) * r.d0[j] + r.d0[i] * v0(j)) * (2.0 * hh);
      const double b1 = g * v1(i) * v1(j) - (v1(i) * r.d1[j] + r.d1[i] * v1(j)) * (2.0 * hh);
      const double lab = -g * v1(i) * v0(j) - v1(i) * r.d0[j] * hh + r.d1[i] * v0(j) * hh;
      M[(size_t)i * P + j] = wa * h * r.Mhat[i * n + j];
      M[(size_t)(n + i) * P + n + j] = wb * h * r.Mhat[i * n + j];
      L[(size_t)i * P + j] = wa * r.Khat[i * n + j] / h + fl + ((t & 1) ? b0 : 0.0);
      L[(size_t)(n + i) * P + n + j] = wb * r.Khat[i * n + j] / h + fr + ((t & 2) ? b1 : 0.0);
      L[(size_t)i * P + n + j] = lab;
      L[(size_t)(n + j) * P + i] = lab;
    }
}

// Uploads the 3 x 4 factor pairs in the vectors' precision: tab[((d * 4 + t) * 2 + w)][i * kMaxP + j],
// w = 0 for M_p and 1 for L_p; sets the kernel's shared-memory limit on the current device.
tp_status prepare_apply_patch(tp_op_s* op) {
  const int n = op->n, P = 2 * n;
  if (op->mesh.nx < 2 || op->mesh.ny < 2 || op->mesh.nz < 2) {
    set_error("patch-wise apply: vertex patches need at least two cells per direction");
    return TP_ERR_UNSUPPORTED;
  }
  std::vector<double> tab((size_t)24 * kMaxP * kMaxP, 0.0), M, L;
  for (int d = 0; d < 3; ++d)
    for (int t = 0; t < 4; ++t) {
      pw_factors(op, d, t, M, L);
      for (int i = 0; i < P; ++i)
        for (int j = 0; j < P; ++j) {
          tab[(size_t)((d * 4 + t) * 2 + 0) * kMaxP * kMaxP + i * kMaxP + j] = M[(size_t)i * P + j];
          tab[(size_t)((d * 4 + t) * 2 + 1) * kMaxP * kMaxP + i * kMaxP + j] = L[(size_t)i * P + j];
        }
    }
  const bool f64 = op->prec == TP_FP64;
  std::vector<float> tf;
  if (!f64) tf.assign(tab.begin(), tab.end());
  const size_t bytes = tab.size() * (f64 ? sizeof(double) : sizeof(float));
  tp_status st = cuda_status(f64 ? pw_prepare_t<double>(n) : pw_prepare_t<float>(n), "patch-wise apply set-up");
  if (st == TP_OK) st = cuda_status(cudaMalloc(&op->pw_mats, bytes), "patch-wise apply tables");
  if (st == TP_OK)
    st = cuda_status(cudaMemcpy(op->pw_mats, f64 ? (const void*)tab.data() : (const void*)tf.data(), bytes,
                                cudaMemcpyHostToDevice),
                     "patch-wise apply tables");
  return st;
}

cudaError_t launch_apply_patch(const tp_op_s* op, void* y, const void* x, cudaStream_t s) {
  if (op->prec == TP_FP64) return pw_launch_t<double>(op, y, x, s);
  if (op->prec == TP_FP32) return pw_launch_t<float>(op, y, x, s);
  return cudaErrorInvalidValue;
}

}  // namespace tp
