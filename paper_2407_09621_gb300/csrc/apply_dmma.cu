// FP64 tensor-core (DMMA) SIPG apply for k = 3 and k = 7: the six n x n contractions of the
// inverse-mass form (apply_cc.cu)
//   w = sum_d (M_d^-1 L_d) u + face terms,   v = (M_z (x) M_y (x) M_x) w
// run as `mma.sync.m8n8k4.f64` products, the rank-2 face terms on the FMA pipe.
//
// A contraction along direction d maps the n^2 lines of a cell (rows) times the 1D matrix
// (Sec. 3: a small dense GEMM per tensor direction): D[line][i] = sum_m U[line][m] G[i][m], in
// groups of 8 lines (M = 8), K = 4 input nodes per step, N = 8 output nodes (for n = 4 the upper
// four columns are zero and are dropped). Each thread keeps its B fragments (the 1D matrices)
// in registers for the whole kernel; A fragments are read from the cell tensor in shared
// memory, which holds u, w and one temporary per cell. One warp per cell, no block-wide
// barriers. The shared cell tensors are padded against bank conflicts (the concern of Sec. 4.1,
// met here by padding rather than an XOR permutation): element (l, j, i) sits at l*PL + j*RP + i
// with RP = 4, PL = 20 for n = 4 and RP = 12, PL = 100 for n = 8. A half-warp's A fragment touches
// 4 lines x 4 nodes; with these pitches (2 RP and 2 PL are 8 or 24 modulo the 32 banks) its 16
// doubles fall in 16 distinct bank pairs for lines along x, y and z. For n = 4 every fragment load
// and store is then conflict-free (the unpadded layout: 4-way along z); for n = 8 the fragment
// stores of even and odd nodes stay 2-way (unpadded: up to 4-way), half the wavefronts in all.
//
// On this part DMMA and DFMA issue to the same FP64 pipe (DMMA measured at 1.05 TFLOP/s, DFMA
// at 1.19-1.25), so this kernel is the tensor-core comparator of the FP64 apply, not its
// fastest form.
#include "apply_common.cuh"

namespace tp {

namespace dmma {

// cells (warps) per block of tile-shape variant V: half, default (4 for n = 8, 8 for n = 4), double
template <int N, int V>
__host__ __device__ constexpr int cells_per_block() { return (N == 8 ? 4 : 8) * (V == 0 ? 1 : (V == 1 ? 2 : 4)) / 2; }

// pitches of the padded shared cell tensor: row (RP) and plane (PL); its size in doubles
template <int N> __host__ __device__ constexpr int rp() { return N == 8 ? 12 : N; }
template <int N> __host__ __device__ constexpr int pl() { return N == 8 ? 100 : N * N + 4; }
template <int N> __host__ __device__ constexpr int cell_pad() { return N * pl<N>(); }

template <int N, int V>
__host__ __device__ constexpr size_t smem_bytes() { return sizeof(double) * 3 * cell_pad<N>() * cells_per_block<N, V>(); }

// Offset of node m of line r along direction D, in the padded shared layout (PAD) or the
// canonical global layout (l*N + j)*N + i: D = 0 (x): r = l*N + j; D = 1 (y): r = l*N + i;
// D = 2 (z): r = j*N + i.
template <int N, int D, bool PAD>
__device__ __forceinline__ int off(int r, int m) {
  constexpr int R = PAD ? rp<N>() : N, L = PAD ? pl<N>() : N * N;
  if (D == 0) return (r / N) * L + (r % N) * R + m;
  if (D == 1) return (r / N) * L + m * R + (r % N);
  return m * L + (r / N) * R + (r % N);
}

__device__ __forceinline__ void mma_f64(double& d0, double& d1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(d0), "+d"(d1)
               : "d"(a), "d"(b));
}

// dst[line][i] (+)= sum_m src[line][m] A[i][m] along direction D for all N^2 lines of one cell.
// bf[ks] is this lane's B fragment A[lane/4][4 ks + lane%4] (0 for rows >= N).
// src: a padded shared cell tensor; dst: padded shared (GDST false) or the cell in global memory.
template <int N, int D, bool ACC, bool GDST = false>
__device__ __forceinline__ void contract_dmma(double* dst, const double* src, const double (&bf)[N / 4], int lane) {
  constexpr int G = N * N / 8;
  const int rr = lane >> 2, cc = lane & 3, i0 = 2 * cc;
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const int r = g * 8 + rr;
    double c0 = 0.0, c1 = 0.0;
    if (ACC && i0 < N) {
      c0 = dst[off<N, D, !GDST>(r, i0)];
      c1 = dst[off<N, D, !GDST>(r, i0 + 1)];
    }
#pragma unroll
    for (int ks = 0; ks < N / 4; ++ks) mma_f64(c0, c1, src[off<N, D, true>(r, ks * 4 + cc)], bf[ks]);
    if (i0 < N) {
      dst[off<N, D, !GDST>(r, i0)] = c0;
      dst[off<N, D, !GDST>(r, i0 + 1)] = c1;
    }
  }
}

// Face terms of direction D for the lines this lane owns, added into sW.
template <int N, int D>
__device__ __forceinline__ void faces_dmma(double* sW, const double* sU, const double* xc, bool has_lo, bool has_hi,
                                           long long nb, const OpConst<double>& P, int lane) {
  constexpr int step = D == 0 ? 1 : (D == 1 ? N : N * N);
  for (int r = lane; r < N * N; r += 32) {
    double u[N], acc[N];
#pragma unroll
    for (int m = 0; m < N; ++m) {
      u[m] = sU[off<N, D, true>(r, m)];
      acc[m] = 0.0;
    }
    const double* own = xc + off<N, D, false>(r, 0);
    add_faces<double, double, N>(acc, u, has_lo ? own - nb : nullptr, has_hi ? own + nb : nullptr, step, P, D);
#pragma unroll
    for (int m = 0; m < N; ++m) sW[off<N, D, true>(r, m)] += acc[m];
  }
}

template <int N, int V>
__global__ void __launch_bounds__(32 * cells_per_block<N, V>())
apply_dmma_kernel(const double* __restrict__ x, double* __restrict__ y, const __grid_constant__ OpConst<double> P,
                  int nx, int ny, int nz, long long c_begin, long long c_end) {
  constexpr int CPB = cells_per_block<N, V>(), N3 = N * N * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int C = cell_pad<N>();
  double* sU = reinterpret_cast<double*>(smem_raw) + warp * 3 * C;
  double* sW = sU + C;
  double* sT = sW + C;
  const long long cell = c_begin + (long long)blockIdx.x * CPB + warp;  // cells [c_begin, c_end)
  if (cell >= c_end) return;  // whole warp; the kernel has no block-wide barrier
  const int cx = (int)(cell % nx), cy = (int)((cell / nx) % ny), cz = (int)(cell / ((long long)nx * ny));
  const double* xc = x + cell * N3;

  // B fragments of the six 1D matrices: lane holds A[lane/4][4 ks + lane%4]
  double bG[3][N / 4], bM[3][N / 4];
  {
    const int io = lane >> 2, mk = lane & 3;
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int ks = 0; ks < N / 4; ++ks) {
        bG[d][ks] = io < N ? P.G[d][io * kMaxN + ks * 4 + mk] : 0.0;
        bM[d][ks] = io < N ? P.M[d][io * kMaxN + ks * 4 + mk] : 0.0;
      }
  }
  for (int e = lane; e < N3; e += 32) sU[(e / (N * N)) * pl<N>() + ((e / N) % N) * rp<N>() + e % N] = __ldg(xc + e);
  __syncwarp();

  // w = G_x u + G_y u + G_z u on the tensor cores
  contract_dmma<N, 0, false>(sW, sU, bG[0], lane);
  __syncwarp();
  contract_dmma<N, 1, true>(sW, sU, bG[1], lane);
  __syncwarp();
  contract_dmma<N, 2, true>(sW, sU, bG[2], lane);
  __syncwarp();
  // + the face terms of the six faces (FMA pipe)
  faces_dmma<N, 0>(sW, sU, xc, cx > 0, cx < nx - 1, N3, P, lane);
  __syncwarp();
  faces_dmma<N, 1>(sW, sU, xc, cy > 0, cy < ny - 1, (long long)nx * N3, P, lane);
  __syncwarp();
  faces_dmma<N, 2>(sW, sU, xc, cz > 0, cz < nz - 1, (long long)nx * ny * N3, P, lane);
  __syncwarp();
  // v = M_x M_y M_z w, the last contraction stored straight to y
  contract_dmma<N, 2, false>(sT, sW, bM[2], lane);
  __syncwarp();
  contract_dmma<N, 1, false>(sW, sT, bM[1], lane);
  __syncwarp();
  contract_dmma<N, 0, false, true>(y + cell * N3, sW, bM[0], lane);
}

template <int N, int V>
static cudaError_t launch_v(const tp_op_s* op, void* y, const void* x, long long c0, long long c1, cudaStream_t s) {
  constexpr int CPB = cells_per_block<N, V>();
  const long long blocks = (c1 - c0 + CPB - 1) / CPB;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  if (blocks <= 0) return cudaSuccess;
  apply_dmma_kernel<N, V><<<(unsigned)blocks, 32 * CPB, smem_bytes<N, V>(), s>>>(
      static_cast<const double*>(x), static_cast<double*>(y), op->c64, op->mesh.nx, op->mesh.ny, op->mesh.nz, c0, c1);
  return cudaGetLastError();
}

template <int N>
static cudaError_t launch_n(const tp_op_s* op, void* y, const void* x, long long c0, long long c1, cudaStream_t s) {
  switch (op->tile_variant) {
    case 0: return launch_v<N, 0>(op, y, x, c0, c1, s);
    case 2: return launch_v<N, 2>(op, y, x, c0, c1, s);
  }
  return launch_v<N, 1>(op, y, x, c0, c1, s);
}

template <int N>
static cudaError_t prepare_n() {
  cudaError_t e = cudaFuncSetAttribute(apply_dmma_kernel<N, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem_bytes<N, 0>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(apply_dmma_kernel<N, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_bytes<N, 1>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(apply_dmma_kernel<N, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_bytes<N, 2>());
  return e;
}

}  // namespace dmma

bool dmma_supported(const tp_op_s* op) { return op->prec == TP_FP64 && (op->n == 4 || op->n == 8); }

int dmma_tile_cells(int n, int v) { return (n == 8 ? 4 : 8) * (v == 0 ? 1 : (v == 1 ? 2 : 4)) / 2; }

cudaError_t prepare_apply_dmma(const tp_op_s* op) {
  if (op->n == 4) return dmma::prepare_n<4>();
  if (op->n == 8) return dmma::prepare_n<8>();
  return cudaErrorInvalidValue;
}

// Output rows of cells [c0, c1) only.
cudaError_t launch_apply_dmma_range(const tp_op_s* op, void* y, const void* x, long long c0, long long c1,
                                    cudaStream_t s) {
  if (op->n == 4) return dmma::launch_n<4>(op, y, x, c0, c1, s);
  if (op->n == 8) return dmma::launch_n<8>(op, y, x, c0, c1, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_apply_dmma(const tp_op_s* op, void* y, const void* x, cudaStream_t s) {
  return launch_apply_dmma_range(op, y, x, 0, op->ncells, s);
}

}  // namespace tp
