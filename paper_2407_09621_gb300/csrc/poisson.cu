// Right-hand side and L2 error of the manufactured Poisson problems (Sec. 7.2).
//
// u = sum_m a_m sin(p_m pi x) sin(q_m pi y) sin(r_m pi z) on the box, so
// f = -Laplace u = sum_m a_m pi^2 (p^2/lx^2 + q^2/ly^2 + r^2/lz^2) ... with the
// sine arguments scaled to the box lengths (p pi x / lx); on the unit cube
// the single mode (1, 1, 1, 1) is the problem of Sec. 7.2. u vanishes on the
// boundary (g = 0), so the load vector is b_a = int f phi_a: separable per
// mode, a tensor product of 1D load vectors (30-point Gauss per cell, host).
// The L2 error || u_h - u || uses per-cell tensor Gauss quadrature with k+4
// points per direction, sum-factorized evaluation of u_h, FP64 throughout.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "tp_internal.h"

namespace tp {

tp_status cuda_status(int err, const char* what);
int stream_blocks(long long n);

constexpr int kMaxModes = 16;
constexpr int kMaxQ = kMaxN + 3;  // k + 4 points

struct RhsDims {
  int n, nx, ny, nz, nmodes;
  double coef[kMaxModes];
};

__global__ void rhs_kernel(double* __restrict__ b, const double* __restrict__ bx, const double* __restrict__ by,
                           const double* __restrict__ bz, RhsDims D, long long ndofs) {
  const int n = D.n, N1x = D.nx * n, N1y = D.ny * n, N1z = D.nz * n;
  const long long n3 = (long long)n * n * n;
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < ndofs; g += (long long)gridDim.x * blockDim.x) {
    const long long cell = g / n3;
    const int loc = (int)(g % n3), i = loc % n, j = (loc / n) % n, l = loc / (n * n);
    const int cx = (int)(cell % D.nx), cy = (int)((cell / D.nx) % D.ny), cz = (int)(cell / ((long long)D.nx * D.ny));
    double s = 0.0;
    for (int m = 0; m < D.nmodes; ++m)
      s += D.coef[m] * bx[(size_t)m * N1x + cx * n + i] * by[(size_t)m * N1y + cy * n + j] *
           bz[(size_t)m * N1z + cz * n + l];
    b[g] = s;
  }
}

struct L2Params {
  int n, q, nx, ny, nz, nmodes;
  double h[3];
  double E[kMaxQ * kMaxN];  // E[p*n + i] = phi_i(xq_p)
  double xq[kMaxQ], wq[kMaxQ];
  double a[kMaxModes];
  int p[kMaxModes][3];
  double len[3];
};

// one block per cell: sum-factorized evaluation of u_h at q^3 points, squared error, block partial
__global__ void __launch_bounds__(256) l2_kernel(const double* __restrict__ u, const __grid_constant__ L2Params P,
                                                 double* __restrict__ partial) {
  __shared__ double su[kMaxN * kMaxN * kMaxN];
  __shared__ double t1[kMaxN * kMaxN * kMaxQ];
  __shared__ double t2[kMaxN * kMaxQ * kMaxQ];
  __shared__ double red[8];
  const int n = P.n, q = P.q, n3 = n * n * n;
  const long long cell = blockIdx.x;
  const int cx = (int)(cell % P.nx), cy = (int)((cell / P.nx) % P.ny), cz = (int)(cell / ((long long)P.nx * P.ny));
  for (int e = threadIdx.x; e < n3; e += blockDim.x) su[e] = u[cell * n3 + e];
  __syncthreads();
  for (int e = threadIdx.x; e < n * n * q; e += blockDim.x) {  // t1[l][j][px]
    const int px = e % q, j = (e / q) % n, l = e / (q * n);
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += P.E[px * n + i] * su[(l * n + j) * n + i];
    t1[e] = s;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n * q * q; e += blockDim.x) {  // t2[l][py][px]
    const int px = e % q, py = (e / q) % q, l = e / (q * q);
    double s = 0.0;
    for (int j = 0; j < n; ++j) s += P.E[py * n + j] * t1[(l * n + j) * q + px];
    t2[e] = s;
  }
  __syncthreads();
  double acc = 0.0;
  for (int e = threadIdx.x; e < q * q * q; e += blockDim.x) {
    const int px = e % q, py = (e / q) % q, pz = e / (q * q);
    double uh = 0.0;
    for (int l = 0; l < n; ++l) uh += P.E[pz * n + l] * t2[(l * q + py) * q + px];
    const double x = (cx + P.xq[px]) * P.h[0], y = (cy + P.xq[py]) * P.h[1], z = (cz + P.xq[pz]) * P.h[2];
    double ue = 0.0;
    for (int m = 0; m < P.nmodes; ++m)
      ue += P.a[m] * sin(P.p[m][0] * M_PI * x / P.len[0]) * sin(P.p[m][1] * M_PI * y / P.len[1]) *
            sin(P.p[m][2] * M_PI * z / P.len[2]);
    const double d = uh - ue;
    acc += P.wq[px] * P.wq[py] * P.wq[pz] * d * d;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) s += red[w];
    partial[blockIdx.x] = s * P.h[0] * P.h[1] * P.h[2];
  }
}

__global__ void sum_kernel(const double* __restrict__ v, long long n, double* __restrict__ out) {
  __shared__ double red[32];
  double s = 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) s += v[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) t += red[w];
    *out = t;
  }
}

static std::vector<double> load_1d(const tp_op_s* op, int d, int mode, double len) {
  const int n = op->n, nc = d == 0 ? op->mesh.nx : (d == 1 ? op->mesh.ny : op->mesh.nz);
  const double h = op->dir[d].h;
  std::vector<double> xq, wq;
  gauss_legendre(30, xq, wq);
  std::vector<double> V = lagrange_eval(op->ref.nodes, xq);
  std::vector<double> b((size_t)nc * n, 0.0);
  for (int c = 0; c < nc; ++c)
    for (int qq = 0; qq < 30; ++qq) {
      const double f = std::sin(mode * M_PI * (c + xq[qq]) * h / len);
      for (int i = 0; i < n; ++i) b[(size_t)c * n + i] += h * wq[qq] * f * V[qq * n + i];
    }
  return b;
}

static tp_status check_modes(int nmodes, const double* a, const int* pqr, const char* who) {
  if (nmodes < 1 || nmodes > kMaxModes || !a || !pqr) {
    set_error("%s: need 1..%d modes with coefficient and wave-number arrays", who, kMaxModes);
    return TP_ERR_INVALID_ARG;
  }
  for (int m = 0; m < 3 * nmodes; ++m)
    if (pqr[m] < 1) { set_error("%s: wave numbers must be >= 1", who); return TP_ERR_INVALID_ARG; }
  return TP_OK;
}

}  // namespace tp

using namespace tp;

extern "C" tp_status tp_rhs_sines(tp_op op, double* b, int nmodes, const double* a, const int* pqr, void* stream) {
  if (!op || !b) { set_error("tp_rhs_sines: NULL argument"); return TP_ERR_INVALID_ARG; }
  tp_status st = check_modes(nmodes, a, pqr, "tp_rhs_sines");
  if (st != TP_OK) return st;
  const double len[3] = {op->mesh.lx, op->mesh.ly, op->mesh.lz};
  const int N1[3] = {op->mesh.nx * op->n, op->mesh.ny * op->n, op->mesh.nz * op->n};
  std::vector<double> hb[3];
  RhsDims D;
  memset(&D, 0, sizeof(D));
  D.n = op->n; D.nx = op->mesh.nx; D.ny = op->mesh.ny; D.nz = op->mesh.nz; D.nmodes = nmodes;
  for (int m = 0; m < nmodes; ++m) {
    const double kk = M_PI * M_PI * (pqr[3 * m] * pqr[3 * m] / (len[0] * len[0]) +
                                     pqr[3 * m + 1] * pqr[3 * m + 1] / (len[1] * len[1]) +
                                     pqr[3 * m + 2] * pqr[3 * m + 2] / (len[2] * len[2]));
    D.coef[m] = a[m] * kk;
    for (int d = 0; d < 3; ++d) {
      std::vector<double> v = load_1d(op, d, pqr[3 * m + d], len[d]);
      hb[d].insert(hb[d].end(), v.begin(), v.end());
    }
  }
  double* dv[3] = {nullptr, nullptr, nullptr};
  cudaStream_t s = (cudaStream_t)stream;
  for (int d = 0; d < 3 && st == TP_OK; ++d) {
    st = cuda_status(cudaMalloc(&dv[d], sizeof(double) * nmodes * N1[d]), "tp_rhs_sines");
    if (st == TP_OK)
      st = cuda_status(cudaMemcpyAsync(dv[d], hb[d].data(), sizeof(double) * nmodes * N1[d], cudaMemcpyHostToDevice, s),
                       "tp_rhs_sines");
  }
  if (st == TP_OK) {
    rhs_kernel<<<stream_blocks(op->ndofs), 256, 0, s>>>(b, dv[0], dv[1], dv[2], D, op->ndofs);
    st = cuda_status(cudaGetLastError(), "tp_rhs_sines");
  }
  if (st == TP_OK) st = cuda_status(cudaStreamSynchronize(s), "tp_rhs_sines");
  for (int d = 0; d < 3; ++d)
    if (dv[d]) cudaFree(dv[d]);
  return st;
}

extern "C" tp_status tp_l2_error_sines(tp_op op, const double* u, int nmodes, const double* a, const int* pqr,
                                       double* err, void* stream) {
  if (!op || !u || !err) { set_error("tp_l2_error_sines: NULL argument"); return TP_ERR_INVALID_ARG; }
  tp_status st = check_modes(nmodes, a, pqr, "tp_l2_error_sines");
  if (st != TP_OK) return st;
  if (op->ncells > 0x7fffffffLL) { set_error("tp_l2_error_sines: too many cells"); return TP_ERR_INVALID_ARG; }
  if (op->n > kMaxN) {
    set_error("tp_l2_error_sines: degree k=%d above %d is not supported", op->k, kMaxN - 1);
    return TP_ERR_UNSUPPORTED;
  }
  L2Params P;
  memset(&P, 0, sizeof(P));
  P.n = op->n;
  P.q = op->k + 4;
  P.nx = op->mesh.nx; P.ny = op->mesh.ny; P.nz = op->mesh.nz;
  P.nmodes = nmodes;
  for (int d = 0; d < 3; ++d) P.h[d] = op->dir[d].h;
  P.len[0] = op->mesh.lx; P.len[1] = op->mesh.ly; P.len[2] = op->mesh.lz;
  std::vector<double> xq, wq;
  gauss_legendre(P.q, xq, wq);
  std::vector<double> E = lagrange_eval(op->ref.nodes, xq);
  for (int p = 0; p < P.q; ++p) {
    P.xq[p] = xq[p];
    P.wq[p] = wq[p];
    for (int i = 0; i < P.n; ++i) P.E[p * P.n + i] = E[p * P.n + i];
  }
  for (int m = 0; m < nmodes; ++m) {
    P.a[m] = a[m];
    for (int d = 0; d < 3; ++d) P.p[m][d] = pqr[3 * m + d];
  }
  double* partial = nullptr;
  double* dout = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  st = cuda_status(cudaMalloc(&partial, sizeof(double) * (op->ncells + 1)), "tp_l2_error_sines");
  if (st == TP_OK) {
    dout = partial + op->ncells;
    l2_kernel<<<(unsigned)op->ncells, 256, 0, s>>>(u, P, partial);
    sum_kernel<<<1, 1024, 0, s>>>(partial, op->ncells, dout);
    double h = 0.0;
    st = cuda_status(cudaGetLastError(), "tp_l2_error_sines");
    if (st == TP_OK) st = cuda_status(cudaMemcpyAsync(&h, dout, sizeof(double), cudaMemcpyDeviceToHost, s), "tp_l2_error_sines");
    if (st == TP_OK) st = cuda_status(cudaStreamSynchronize(s), "tp_l2_error_sines");
    if (st == TP_OK) *err = std::sqrt(h);
  }
  if (partial) cudaFree(partial);
  return st;
}
