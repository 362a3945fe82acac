// Internal declarations of libtp (not part of the C ABI).
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/tp.h"

namespace tp {

constexpr int kMaxN = 8;       // n = k + 1 <= 8 (k <= 7): every kernel family and the multigrid
constexpr int kMaxNHigh = 16;  // n <= 16 (k <= 15): the CUDA-core apply in FP64 and FP32 only

// 1D reference data of the Gauss-Lobatto Lagrange basis on [0, 1] (Sec. 2).
struct Ref1D {
  int k = 0, n = 0;
  std::vector<double> nodes;  // n Gauss-Lobatto points, ascending
  std::vector<double> Mhat;   // n*n, int phi_i phi_j (row-major, [i*n + j])
  std::vector<double> Khat;   // n*n, int phi_i' phi_j'
  std::vector<double> d0, d1; // phi_i'(0), phi_i'(1)
};

Ref1D make_ref1d(int k);
void gauss_legendre(int q, std::vector<double>& x, std::vector<double>& w);  // on [0, 1]
// Lagrange basis values (rows = points) of the Gauss-Lobatto nodes at points x.
std::vector<double> lagrange_eval(const std::vector<double>& nodes, const std::vector<double>& x);

// Per-direction 1D operator data for a uniform mesh (Sec. 2.1, Eq. (9)).
// M = h Mhat; L = interior diagonal block of the 1D SIPG stiffness
//   Khat/h + g(v1 v1^T + v0 v0^T) - (v1 d1^T + d1 v1^T)/(2h) + (v0 d0^T + d0 v0^T)/(2h).
struct Dir1D {
  double h = 0, gamma = 0;
  std::vector<double> M, L;  // n*n row-major
};

Dir1D make_dir1d(const Ref1D& r, double h, int penalty_mode);
void global_1d(const Ref1D& r, const Dir1D& d, int nc, std::vector<double>& M, std::vector<double>& L);
// inverse of a small dense n x n row-major matrix (Gauss-Jordan, partial pivoting)
std::vector<double> invert(int n, const std::vector<double>& A);
bool gen_eig(int N, const std::vector<double>& M, const std::vector<double>& L, std::vector<double>& lam,
             std::vector<double>& V);

// 1D operator data of the apply kernel, templated on the compute type and on the
// row pitch NM of its matrices (kMaxN for n <= 8, kMaxNHigh above). Passed by value
// as a __grid_constant__ kernel parameter (5.5 KB for double at NM = 8, 22 KB at 16),
// so the coefficients are read from the constant bank. Per direction d: M = h M-hat,
// G = M^-1 L_int, and the face expansion vectors E[d][0..7] = P1, P2, Q1, Q2, B1, B2,
// C1, C2 (see apply_cc.cuh).
template <typename T, int NM = kMaxN>
struct OpConst {
  static constexpr int S = NM;  // row pitch of M and G: entry (i, j) at [i * S + j]
  T M[3][NM * NM];
  T G[3][NM * NM];
  T d0[NM], d1[NM];
  T E[3][8][NM];
  // Even-odd halves of the centrosymmetric M and G (A[n-1-i][n-1-m] = A[i][m], the reference
  // element and the Gauss-Lobatto nodes being symmetric about 1/2), for i, m < H = floor(n/2):
  // AE[i][m] = (A[i][m] + A[i][n-1-m]) / 2 and AO[i][m] = (A[i][m] - A[i][n-1-m]) / 2; for odd n
  // also the middle column and row AE[i][H] = A[i][H], AE[H][m] = A[H][m] (i, m <= H).
  T ME[3][NM / 2][NM / 2], MO[3][NM / 2][NM / 2];
  T GE[3][NM / 2][NM / 2], GO[3][NM / 2][NM / 2];
  int centro;  // 1 if every M and G above is centrosymmetric (to 1e-12 relative)
};

// Kernel parameters of the Blackwell tensor-core apply (apply_umma.cu).
struct UmmaParams {
  int nx, ny, nz;
  long long ncells;
  float out_scale;  // 1 / (power-of-two scale of the stored block matrices)
  float lo_scale;   // scale of the low-part products (1: they share the accumulator)
  int tiles[3];     // tiles of 8 x 16 x 1 cells along x, y, z
  int seg;          // tiles per z-segment of a tile column (one work unit)
  long long units;  // work units: tile columns x z-segments
  unsigned long long wait_ns;  // limit of every bounded wait on the pipeline barriers (1 s by default)
  int test_withhold;           // failure-injection tests only: CTA 0 skips its first input-tile copy
  // boundary-face corrections, FP32: per direction d the mass matrix M_d (n = 4, row-major), the basis
  // derivatives at the ends, and 1/(2 h_d)
  float fM[3][16];
  float fd0[4], fd1[4];
  float fhh[3];
};

void set_error(const char* fmt, ...);
tp_status cuda_status(int err, const char* what);

}  // namespace tp

struct tp_mesh_s {
  int nx, ny, nz;
  double lx, ly, lz;
};

struct tp_op_s {
  tp_mesh_s mesh;
  int k, n;
  tp_precision prec;
  tp_op_opts opts;
  long long ncells, ndofs;
  tp::OpConst<double> c64;    // host copies of the kernel-parameter constants (n <= 8)
  tp::OpConst<float> c32;
  tp::OpConst<double, tp::kMaxNHigh> c64h;  // the same for 8 < n <= 16
  tp::OpConst<float, tp::kMaxNHigh> c32h;
  int device = 0;
  void* tc_mats = nullptr;    // tensor kernel operand matrices (device)
  int tc_blocks_per_sm = 1, sm_count = 1;
  int tile_variant = 1;         // CUDA-core / DMMA tile shape: 0 half, 1 default, 2 double cells per block
  bool use_umma = false;        // tensor kernel runs on tcgen05 (k = 3, FP16/BF16 vectors)
  void* umma_mats = nullptr;    // its seven block matrices (and low parts) on the device
  int* umma_err = nullptr;      // device error code of its bounded waits (0 = none)
  void* pw_mats = nullptr;      // patch-wise kernel: its 3 x 4 pairs of 1D patch factors (device)
  tp::UmmaParams umma_params;
  const void* hconst(size_t tc_bytes) const { return tc_bytes == 8 ? (const void*)&c64 : (const void*)&c32; }
  const void* hconst_high(size_t tc_bytes) const { return tc_bytes == 8 ? (const void*)&c64h : (const void*)&c32h; }
  // host-buffer path (tp_apply_host): library-owned staging, and the streams and events of its
  // copy/compute pipeline (created on first use)
  void* hx = nullptr; void* hy = nullptr;
  size_t hbytes = 0;
  void* hpipe = nullptr;
  tp::Ref1D ref;
  tp::Dir1D dir[3];
};
