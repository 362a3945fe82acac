// Geometric multigrid V-cycle (Algorithm 2, Sec. 7.1) for the SIPG operator.
//
// Levels: uniform coarsening by 2 in every direction, same degree k, the
// operator rediscretized on each level (Sec. 2 with that level's h).
// Smoother: Chebyshev semi-iteration of the given degree on D^{-1} A with
// D = diag(A) evaluated from the Kronecker form of Eq. (9), or the paper's
// multiplicative vertex-patch Schwarz smoother (patch solves in schwarz.cu;
// the sweep over the eight colours here). Transfer: prolongation is the
// exact embedding of the coarse DG space (coarse basis evaluated at the fine
// nodes, a Kronecker product of 1D n x n matrices per child), restriction
// its transpose; both sum-factorized. Coarse solve: exact, in FP64, by fast
// diagonalization with the 1D generalized eigenpairs L V = M V Lambda.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <array>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "tp_internal.h"
#include "tp_vec.h"

namespace tp {

tp_status cuda_status(int err, const char* what);
cudaError_t launch_apply(const tp_op_s* op, void* y, const void* x, cudaStream_t s);
cudaError_t launch_residual(const tp_op_s* op, void* r, const void* b, const void* x, cudaStream_t s);
size_t elem_bytes(tp_precision p);
// vertex-patch smoother (schwarz.cu)
bool vp_colour_nonempty(const int nc[3], int c);
cudaError_t vp_colour(tp_precision prec, int n, const int nc[3], int colour, void* x, const void* r, const void* S,
                      const void* L, const void* C, cudaStream_t s);
tp_status vp_tables(const tp_op_s* op, const int nc[3], tp_precision prec, void** S_out, void** L_out,
                    std::vector<unsigned char>* C_out);

// Division of n < 2^31 by an invariant d >= 1 with one multiply-high (Granlund and Montgomery,
// "Division by invariant integers using multiplication", 1994): with l = ceil(log2 d) and
// m = floor(2^32 (2^l - d) / d) + 1, floor(n / d) = (umulhi(n, m) + n) >> l.
struct FastDiv {
  uint32_t d = 1, m = 1, l = 0;
};

inline FastDiv make_fastdiv(uint32_t d) {
  FastDiv f;
  f.d = d;
  f.l = 0;
  while ((1ull << f.l) < d) ++f.l;
  f.m = (uint32_t)((((1ull << 32) * ((1ull << f.l) - d)) / d) + 1);
  return f;
}

__device__ __forceinline__ uint32_t fast_div(uint32_t n, const FastDiv& f) {
  return (__umulhi(n, f.m) + n) >> f.l;
}

template <typename T>
struct JacobiParams {
  T Md[3][kMaxN], Ld[3][kMaxN];  // diagonals of the 1D mass and interior stiffness blocks
  T lo[3], hi[3];                // boundary corrections of L's diagonal at node 0 / node n-1
  int nx, ny, nz;
  FastDiv dx, dy;                // division by nx and by ny (cells < 2^31)
};

template <typename T>
struct TransferParams {
  T P[2][kMaxN * kMaxN];  // P[c][i*kMaxN + j] = phi_j((c + x_i)/2)
};

// Arithmetic type of a storage type: FP16/BF16 vectors are computed on in FP32.
template <typename TS> struct Arith { using T = TS; };
template <> struct Arith<__half> { using T = float; };
template <> struct Arith<__nv_bfloat16> { using T = float; };
template <typename TS> using arith_t = typename Arith<TS>::T;

template <typename TS>
__device__ __forceinline__ arith_t<TS> ld(const TS* p) { return (arith_t<TS>)(*p); }
template <typename TS>
__device__ __forceinline__ void st(TS* p, arith_t<TS> v) { *p = (TS)v; }

// 1/d. In FP64 a division costs many instructions of the slow FP64 pipe; instead the FP32
// reciprocal seeds two Newton-Raphson steps r <- r + r(1 - d r) (each doubles the correct bits:
// 24 -> 48 -> full precision).
__device__ __forceinline__ float recip(float d) { return 1.0f / d; }
__device__ __forceinline__ double recip(double d) {
  double r = (double)(1.0f / (float)d);
  r = fma(r, fma(-d, r, 1.0), r);
  r = fma(r, fma(-d, r, 1.0), r);
  return r;
}

// D^{-1} at DoF (cell, l, j, i)
template <typename T, int N>
__device__ __forceinline__ T jacobi_inv(const JacobiParams<T>& J, long long idx) {
  constexpr int N3 = N * N * N;
  const uint32_t cell = (uint32_t)(idx / N3);
  const int loc = (int)(idx - (long long)cell * N3);
  const int i = loc % N, j = (loc / N) % N, l = loc / (N * N);
  const uint32_t q = fast_div(cell, J.dx), cz_ = fast_div(q, J.dy);
  const int cx = (int)(cell - q * (uint32_t)J.nx), cy = (int)(q - cz_ * (uint32_t)J.ny), cz = (int)cz_;
  T lx = J.Ld[0][i], ly = J.Ld[1][j], lz = J.Ld[2][l];
  if (cx == 0 && i == 0) lx += J.lo[0];
  if (cx == J.nx - 1 && i == N - 1) lx += J.hi[0];
  if (cy == 0 && j == 0) ly += J.lo[1];
  if (cy == J.ny - 1 && j == N - 1) ly += J.hi[1];
  if (cz == 0 && l == 0) lz += J.lo[2];
  if (cz == J.nz - 1 && l == N - 1) lz += J.hi[2];
  const T mx = J.Md[0][i], my = J.Md[1][j], mz = J.Md[2][l];
  return recip(lz * my * mx + mz * ly * mx + mz * my * lx);
}

// Chebyshev update: if t: r -= t;  d = c1*d + c2*D^{-1} r (c1 == 0: d is not read);  x = (x_zero ? 0 : x) + d
template <typename TS, int N, typename T = arith_t<TS>>
__global__ void cheb_update_kernel(long long n, const __grid_constant__ JacobiParams<T> J, TS* __restrict__ x,
                                   TS* __restrict__ r, TS* __restrict__ d, const TS* __restrict__ t, T c1, T c2,
                                   int x_zero) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    T ri = ld(r + i);
    if (t) {
      ri -= ld(t + i);
      st(r + i, ri);
    }
    T di = c2 * jacobi_inv<T, N>(J, i) * ri;
    if (c1 != T(0)) di = fma(c1, ld(d + i), di);
    st(d + i, di);
    st(x + i, x_zero ? di : ld(x + i) + di);
  }
}

// Vectorized Chebyshev update for cells whose n^3 entries split into 16-byte groups: each thread
// handles VW = 16 / sizeof(TS) consecutive entries of one cell with 16-byte loads and stores (more
// bytes in flight per thread than the scalar form). D^{-1} of an interior cell is a per-block
// shared table over the n^3 local positions; cells on the mesh boundary evaluate the Kronecker
// diagonal with the boundary corrections from shared copies of the 1D diagonals.
template <typename TS, int N, typename T = arith_t<TS>>
__global__ void __launch_bounds__(256) cheb_update_vec_kernel(long long ngroups, const __grid_constant__ JacobiParams<T> J,
                                                              TS* __restrict__ x, TS* __restrict__ r,
                                                              TS* __restrict__ d, const TS* __restrict__ t, T c1,
                                                              T c2, int x_zero) {
  constexpr int N3 = N * N * N, VW = 16 / (int)sizeof(TS), GPC = N3 / VW;
  __shared__ T dint[N3];
  __shared__ T sM[3][N], sL[3][N], slo[3], shi[3];
  for (int e = threadIdx.x; e < N3; e += blockDim.x) {
    const int i = e % N, j = (e / N) % N, l = e / (N * N);
    dint[e] = recip(J.Ld[2][l] * J.Md[1][j] * J.Md[0][i] + J.Md[2][l] * J.Ld[1][j] * J.Md[0][i] +
                    J.Md[2][l] * J.Md[1][j] * J.Ld[0][i]);
  }
  if (threadIdx.x < 3 * N) {
    const int dd = threadIdx.x / N, m = threadIdx.x % N;
    sM[dd][m] = J.Md[dd][m];
    sL[dd][m] = J.Ld[dd][m];
  }
  if (threadIdx.x < 3) {
    slo[threadIdx.x] = J.lo[threadIdx.x];
    shi[threadIdx.x] = J.hi[threadIdx.x];
  }
  __syncthreads();
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < ngroups; g += (long long)gridDim.x * blockDim.x) {
    const uint32_t cell = (uint32_t)(g / GPC);
    const int loc0 = (int)(g - (long long)cell * GPC) * VW;
    const uint32_t q = fast_div(cell, J.dx), cz_ = fast_div(q, J.dy);
    const int cx = (int)(cell - q * (uint32_t)J.nx), cy = (int)(q - cz_ * (uint32_t)J.ny), cz = (int)cz_;
    const bool bnd = cx == 0 || cx == J.nx - 1 || cy == 0 || cy == J.ny - 1 || cz == 0 || cz == J.nz - 1;
    uint4 vr = reinterpret_cast<const uint4*>(r)[g], vx = make_uint4(0u, 0u, 0u, 0u), vd = make_uint4(0u, 0u, 0u, 0u);
    if (!x_zero) vx = reinterpret_cast<const uint4*>(x)[g];
    if (c1 != T(0)) vd = reinterpret_cast<const uint4*>(d)[g];
    uint4 vt = make_uint4(0u, 0u, 0u, 0u);
    if (t) vt = reinterpret_cast<const uint4*>(t)[g];
    TS* pr = reinterpret_cast<TS*>(&vr);
    TS* px = reinterpret_cast<TS*>(&vx);
    TS* pd = reinterpret_cast<TS*>(&vd);
    const TS* pt = reinterpret_cast<const TS*>(&vt);
#pragma unroll
    for (int v = 0; v < VW; ++v) {
      const int loc = loc0 + v;
      T dinv = dint[loc];
      if (bnd) {
        const int i = loc % N, j = (loc / N) % N, l = loc / (N * N);
        T lx = sL[0][i], ly = sL[1][j], lz = sL[2][l];
        if (cx == 0 && i == 0) lx += slo[0];
        if (cx == J.nx - 1 && i == N - 1) lx += shi[0];
        if (cy == 0 && j == 0) ly += slo[1];
        if (cy == J.ny - 1 && j == N - 1) ly += shi[1];
        if (cz == 0 && l == 0) lz += slo[2];
        if (cz == J.nz - 1 && l == N - 1) lz += shi[2];
        dinv = recip(lz * sM[1][j] * sM[0][i] + sM[2][l] * ly * sM[0][i] + sM[2][l] * sM[1][j] * lx);
      }
      T ri = (T)pr[v];
      if (t) ri -= (T)pt[v];
      T di = c2 * dinv * ri;
      if (c1 != T(0)) di = fma(c1, (T)pd[v], di);
      pr[v] = (TS)ri;
      pd[v] = (TS)di;
      px[v] = (TS)(x_zero ? di : (T)px[v] + di);
    }
    if (t) reinterpret_cast<uint4*>(r)[g] = vr;
    reinterpret_cast<uint4*>(d)[g] = vd;
    reinterpret_cast<uint4*>(x)[g] = vx;
  }
}

// y = s * D^{-1} t (inv = 1) or y = s * D t (inv = 0)
template <typename TS, int N, typename T = arith_t<TS>>
__global__ void dinv_kernel(long long n, const __grid_constant__ JacobiParams<T> J, TS* __restrict__ y,
                            const TS* __restrict__ t, T s, int inv) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const T di = jacobi_inv<T, N>(J, i);
    st(y + i, inv ? s * di * ld(t + i) : s * ld(t + i) / di);
  }
}

// xf += P xc : one block per coarse cell, thread (l, j, i); children in turn.
template <typename TS, int N, typename T = arith_t<TS>>
__global__ void __launch_bounds__(N * N * N) prolong_add_kernel(TS* __restrict__ xf, const TS* __restrict__ xc,
                                                                const __grid_constant__ TransferParams<T> P, int ncx,
                                                                int ncy, int ncz) {
  constexpr int N2 = N * N, N3 = N2 * N;
  __shared__ T u[N3], t1[N3], t2[N3];
  const long long C = blockIdx.x;
  const int tid = threadIdx.x, i = tid % N, j = (tid / N) % N, l = tid / N2;
  const int cx = (int)(C % ncx), cy = (int)((C / ncx) % ncy), cz = (int)(C / ((long long)ncx * ncy));
  u[tid] = ld(xc + C * N3 + tid);
  __syncthreads();
  for (int b = 0; b < 8; ++b) {
    const int bx = b & 1, by = (b >> 1) & 1, bz = b >> 2;
    T s = 0;
#pragma unroll
    for (int m = 0; m < N; ++m) s = fma(P.P[bx][i * kMaxN + m], u[l * N2 + j * N + m], s);
    t1[tid] = s;
    __syncthreads();
    s = 0;
#pragma unroll
    for (int m = 0; m < N; ++m) s = fma(P.P[by][j * kMaxN + m], t1[l * N2 + m * N + i], s);
    t2[tid] = s;
    __syncthreads();
    s = 0;
#pragma unroll
    for (int m = 0; m < N; ++m) s = fma(P.P[bz][l * kMaxN + m], t2[m * N2 + j * N + i], s);
    const long long F = ((long long)(2 * cz + bz) * (2 * ncy) + (2 * cy + by)) * (2LL * ncx) + (2 * cx + bx);
    st(xf + F * N3 + tid, ld(xf + F * N3 + tid) + s);
    __syncthreads();
  }
}

// xc = P^T rf : one block per coarse cell, sum over the eight children.
template <typename TS, int N, typename T = arith_t<TS>>
__global__ void __launch_bounds__(N * N * N) restrict_kernel(TS* __restrict__ xc, const TS* __restrict__ rf,
                                                             const __grid_constant__ TransferParams<T> P, int ncx,
                                                             int ncy, int ncz) {
  constexpr int N2 = N * N, N3 = N2 * N;
  __shared__ T u[N3], t1[N3], t2[N3];
  const long long C = blockIdx.x;
  const int tid = threadIdx.x, i = tid % N, j = (tid / N) % N, l = tid / N2;
  const int cx = (int)(C % ncx), cy = (int)((C / ncx) % ncy), cz = (int)(C / ((long long)ncx * ncy));
  T acc = 0;
  for (int b = 0; b < 8; ++b) {
    const int bx = b & 1, by = (b >> 1) & 1, bz = b >> 2;
    const long long F = ((long long)(2 * cz + bz) * (2 * ncy) + (2 * cy + by)) * (2LL * ncx) + (2 * cx + bx);
    u[tid] = ld(rf + F * N3 + tid);
    __syncthreads();
    T s = 0;
#pragma unroll
    for (int m = 0; m < N; ++m) s = fma(P.P[bx][m * kMaxN + i], u[l * N2 + j * N + m], s);
    t1[tid] = s;
    __syncthreads();
    s = 0;
#pragma unroll
    for (int m = 0; m < N; ++m) s = fma(P.P[by][m * kMaxN + j], t1[l * N2 + m * N + i], s);
    t2[tid] = s;
    __syncthreads();
    s = 0;
#pragma unroll
    for (int m = 0; m < N; ++m) s = fma(P.P[bz][m * kMaxN + l], t2[m * N2 + j * N + i], s);
    acc += s;
    __syncthreads();
  }
  st(xc + C * N3 + tid, acc);
}

// ---- coarse solve by fast diagonalization (FP64), on a lexicographic N1z x N1y x N1x tensor
struct FDDims {
  int n, nx, ny, nz;     // nodes per direction, cells
  int N1[3];             // nx*n, ny*n, nz*n
};

template <typename T>
__global__ void fd_gather(const T* __restrict__ b, double* __restrict__ lex, FDDims D, double scale) {
  const long long tot = (long long)D.N1[0] * D.N1[1] * D.N1[2];
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int gx = (int)(e % D.N1[0]), gy = (int)((e / D.N1[0]) % D.N1[1]), gz = (int)(e / ((long long)D.N1[0] * D.N1[1]));
    const long long cell = ((long long)(gz / D.n) * D.ny + gy / D.n) * D.nx + gx / D.n;
    const int loc = ((gz % D.n) * D.n + gy % D.n) * D.n + gx % D.n;
    lex[e] = scale * (double)ld(b + cell * D.n * D.n * D.n + loc);
  }
}

template <typename T>
__global__ void fd_scatter(const double* __restrict__ lex, T* __restrict__ x, FDDims D, double scale) {
  const long long tot = (long long)D.N1[0] * D.N1[1] * D.N1[2];
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int gx = (int)(e % D.N1[0]), gy = (int)((e / D.N1[0]) % D.N1[1]), gz = (int)(e / ((long long)D.N1[0] * D.N1[1]));
    const long long cell = ((long long)(gz / D.n) * D.ny + gy / D.n) * D.nx + gx / D.n;
    const int loc = ((gz % D.n) * D.n + gy % D.n) * D.n + gx % D.n;
    st(x + cell * D.n * D.n * D.n + loc, (arith_t<T>)(scale * lex[e]));
  }
}

// out = W applied along `axis` (0 = x fastest, 2 = z): out[..a..] = sum_m W(m, a) in[..m..],
// W(m, a) = V[m*N + a] (transpose == 0, i.e. V^T applied) or V[a*N + m] (transpose == 1, V applied).
__global__ void fd_contract(const double* __restrict__ in, double* __restrict__ out, const double* __restrict__ V,
                            FDDims D, int axis, int transpose) {
  const long long tot = (long long)D.N1[0] * D.N1[1] * D.N1[2];
  const int N = D.N1[axis];
  const long long stride = axis == 0 ? 1 : (axis == 1 ? D.N1[0] : (long long)D.N1[0] * D.N1[1]);
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int a = (int)((e / stride) % N);
    const long long base = e - (long long)a * stride;
    double s = 0.0;
    for (int m = 0; m < N; ++m) {
      const double w = transpose ? V[(size_t)a * N + m] : V[(size_t)m * N + a];
      s = fma(w, in[base + m * stride], s);
    }
    out[e] = s;
  }
}

__global__ void fd_divide(double* __restrict__ t, const double* __restrict__ lx, const double* __restrict__ ly,
                          const double* __restrict__ lz, FDDims D) {
  const long long tot = (long long)D.N1[0] * D.N1[1] * D.N1[2];
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int gx = (int)(e % D.N1[0]), gy = (int)((e / D.N1[0]) % D.N1[1]), gz = (int)(e / ((long long)D.N1[0] * D.N1[1]));
    t[e] /= lx[gx] + ly[gy] + lz[gz];
  }
}

// deterministic pseudo-random start vector in [-1, 1] (power iteration)
template <typename T>
__global__ void hash_fill(long long n, T* __restrict__ x, unsigned seed) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    unsigned long long z = (unsigned long long)i * 0x9E3779B97F4A7C15ULL + seed;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    st(x + i, (arith_t<T>)((double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0));
  }
}

}  // namespace tp

// ------------------------------------------------------------------ host side
struct tp_mg_level {
  int nc[3];
  tp_op_s* op = nullptr;  // owned
  long long ndofs = 0;
  void *x = nullptr, *b = nullptr, *r = nullptr, *d = nullptr, *t = nullptr;
  double lmax = 0.0;
  void *vpS = nullptr, *vpL = nullptr;  // vertex-patch smoother: 1D patch eigenbases and eigenvalues
  std::vector<unsigned char> vpC;       // and the interior ones as the patch kernel's parameter
  tp::JacobiParams<double> j64;
  tp::JacobiParams<float> j32;
};

struct tp_mg_s {
  int k = 0, n = 0;
  tp_precision prec = TP_FP32;  // storage/arithmetic of the V-cycle vectors
  tp_mg_opts opts;
  std::vector<tp_mg_level> lv;  // 0 = coarsest
  tp::TransferParams<double> p64;
  tp::TransferParams<float> p32;
  tp::FDDims fd;
  double *fdV[3] = {nullptr, nullptr, nullptr}, *fdL[3] = {nullptr, nullptr, nullptr};
  double *fdT0 = nullptr, *fdT1 = nullptr;
  double* partial = nullptr;  // reduction scratch
  double* dots = nullptr;     // device results of reductions
};

namespace tp {

static int grid_for(long long n) { return stream_blocks(n); }

template <typename T>
static const JacobiParams<T>& jparams(const tp_mg_level& L);
template <>
const JacobiParams<double>& jparams<double>(const tp_mg_level& L) { return L.j64; }
template <>
const JacobiParams<float>& jparams<float>(const tp_mg_level& L) { return L.j32; }

template <typename T>
static const TransferParams<T>& tparams(const tp_mg_s* mg);
template <>
const TransferParams<double>& tparams<double>(const tp_mg_s* mg) { return mg->p64; }
template <>
const TransferParams<float>& tparams<float>(const tp_mg_s* mg) { return mg->p32; }

template <typename T, int N>
static cudaError_t cheb_update_n(const tp_mg_level& L, void* x, void* r, void* d, const void* t, double c1, double c2,
                                 int x_zero, cudaStream_t s) {
  using A = arith_t<T>;
  constexpr int VW = 16 / (int)sizeof(T);
  const bool aligned = !(((uintptr_t)x | (uintptr_t)r | (uintptr_t)d | (uintptr_t)t) & 15);
  if ((N * N * N) % VW == 0 && aligned) {
    const long long groups = L.ndofs / VW;
    cheb_update_vec_kernel<T, N><<<grid_for(groups), 256, 0, s>>>(groups, jparams<A>(L), (T*)x, (T*)r, (T*)d,
                                                                  (const T*)t, (A)c1, (A)c2, x_zero);
  } else {
    cheb_update_kernel<T, N><<<grid_for(L.ndofs), 256, 0, s>>>(L.ndofs, jparams<A>(L), (T*)x, (T*)r, (T*)d,
                                                               (const T*)t, (A)c1, (A)c2, x_zero);
  }
  return cudaGetLastError();
}

template <typename T, int N>
static cudaError_t dinv_n(const tp_mg_level& L, void* y, const void* t, double sc, int inv, cudaStream_t s) {
  dinv_kernel<T, N><<<grid_for(L.ndofs), 256, 0, s>>>(L.ndofs, jparams<arith_t<T>>(L), (T*)y, (const T*)t,
                                                      (arith_t<T>)sc, inv);
  return cudaGetLastError();
}

template <typename T, int N>
static cudaError_t prolong_n(const tp_mg_s* mg, int l, void* xf, const void* xc, cudaStream_t s) {
  const tp_mg_level& C = mg->lv[l - 1];
  const long long nc = (long long)C.nc[0] * C.nc[1] * C.nc[2];
  prolong_add_kernel<T, N><<<(unsigned)nc, N * N * N, 0, s>>>((T*)xf, (const T*)xc, tparams<arith_t<T>>(mg), C.nc[0], C.nc[1],
                                                              C.nc[2]);
  return cudaGetLastError();
}

template <typename T, int N>
static cudaError_t restrict_n(const tp_mg_s* mg, int l, void* xc, const void* rf, cudaStream_t s) {
  const tp_mg_level& C = mg->lv[l - 1];
  const long long nc = (long long)C.nc[0] * C.nc[1] * C.nc[2];
  restrict_kernel<T, N><<<(unsigned)nc, N * N * N, 0, s>>>((T*)xc, (const T*)rf, tparams<arith_t<T>>(mg), C.nc[0], C.nc[1],
                                                           C.nc[2]);
  return cudaGetLastError();
}

#define TP_DISPATCH_N(n, CALL) \
  switch (n) {                 \
    case 2: return CALL(2);    \
    case 3: return CALL(3);    \
    case 4: return CALL(4);    \
    case 5: return CALL(5);    \
    case 6: return CALL(6);    \
    case 7: return CALL(7);    \
    case 8: return CALL(8);    \
  }                            \
  return cudaErrorInvalidValue;

// storage type of the V-cycle vectors
#define TP_DISPATCH_PREC(prec, CALL)                      \
  switch (prec) {                                         \
    case TP_FP64: { using T = double; CALL; }             \
    case TP_FP32: { using T = float; CALL; }              \
    case TP_FP16: { using T = __half; CALL; }             \
    case TP_BF16: { using T = __nv_bfloat16; CALL; }      \
  }                                                       \
  return cudaErrorInvalidValue;

static cudaError_t cheb_update(const tp_mg_s* mg, const tp_mg_level& L, void* x, void* r, void* d, const void* t,
                               double c1, double c2, int x_zero, cudaStream_t s) {
#define CU(N) cheb_update_n<T, N>(L, x, r, d, t, c1, c2, x_zero, s)
  TP_DISPATCH_PREC(mg->prec, TP_DISPATCH_N(mg->n, CU))
#undef CU
}

static cudaError_t dinv(const tp_mg_s* mg, const tp_mg_level& L, void* y, const void* t, double sc, int inv,
                        cudaStream_t s) {
#define DI(N) dinv_n<T, N>(L, y, t, sc, inv, s)
  TP_DISPATCH_PREC(mg->prec, TP_DISPATCH_N(mg->n, DI))
#undef DI
}

cudaError_t mg_prolong_add(const tp_mg_s* mg, int l, void* xf, const void* xc, cudaStream_t s) {
#define PR(N) prolong_n<T, N>(mg, l, xf, xc, s)
  TP_DISPATCH_PREC(mg->prec, TP_DISPATCH_N(mg->n, PR))
#undef PR
}

cudaError_t mg_restrict(const tp_mg_s* mg, int l, void* xc, const void* rf, cudaStream_t s) {
#define RE(N) restrict_n<T, N>(mg, l, xc, rf, s)
  TP_DISPATCH_PREC(mg->prec, TP_DISPATCH_N(mg->n, RE))
#undef RE
}

static long long fd_total(const FDDims& D) { return (long long)D.N1[0] * D.N1[1] * D.N1[2]; }

cudaError_t mg_coarse_solve(const tp_mg_s* mg, void* x, const void* b, cudaStream_t s) {
  const FDDims& D = mg->fd;
  const long long tot = fd_total(D);
  const int g = grid_for(tot);
  switch (mg->prec) {
    case TP_FP64: fd_gather<double><<<g, 256, 0, s>>>((const double*)b, mg->fdT0, D, 1.0); break;
    case TP_FP32: fd_gather<float><<<g, 256, 0, s>>>((const float*)b, mg->fdT0, D, 1.0); break;
    case TP_FP16: fd_gather<__half><<<g, 256, 0, s>>>((const __half*)b, mg->fdT0, D, 1.0); break;
    case TP_BF16: fd_gather<__nv_bfloat16><<<g, 256, 0, s>>>((const __nv_bfloat16*)b, mg->fdT0, D, 1.0); break;
  }
  double *a = mg->fdT0, *c = mg->fdT1;
  for (int ax = 0; ax < 3; ++ax) {
    fd_contract<<<g, 256, 0, s>>>(a, c, mg->fdV[ax], D, ax, 0);
    double* tmp = a; a = c; c = tmp;
  }
  fd_divide<<<g, 256, 0, s>>>(a, mg->fdL[0], mg->fdL[1], mg->fdL[2], D);
  for (int ax = 0; ax < 3; ++ax) {
    fd_contract<<<g, 256, 0, s>>>(a, c, mg->fdV[ax], D, ax, 1);
    double* tmp = a; a = c; c = tmp;
  }
  switch (mg->prec) {
    case TP_FP64: fd_scatter<double><<<g, 256, 0, s>>>(a, (double*)x, D, 1.0); break;
    case TP_FP32: fd_scatter<float><<<g, 256, 0, s>>>(a, (float*)x, D, 1.0); break;
    case TP_FP16: fd_scatter<__half><<<g, 256, 0, s>>>(a, (__half*)x, D, 1.0); break;
    case TP_BF16: fd_scatter<__nv_bfloat16><<<g, 256, 0, s>>>(a, (__nv_bfloat16*)x, D, 1.0); break;
  }
  return cudaGetLastError();
}

// r = b - t
template <typename T>
static cudaError_t sub_t(long long n, void* r, const void* b, const void* t, cudaStream_t s) {
  const double c[2] = {1.0, -1.0};
  const T* v[2] = {(const T*)b, (const T*)t};
  return multi_axpy<T>(n, (T*)r, 0.0, v, c, 2, s);
}

// r = b - A x: fused into the CUDA-core apply's store, else A x into the scratch t and a
// difference pass
static cudaError_t residual(const tp_mg_s* mg, const tp_mg_level& L, void* r, const void* b, const void* x, void* t,
                            cudaStream_t s) {
  if (L.op->opts.kernel == TP_KERNEL_CUDA_CORE) return launch_residual(L.op, r, b, x, s);
  cudaError_t e = launch_apply(L.op, t, x, s);
  if (e != cudaSuccess) return e;
  TP_DISPATCH_PREC(mg->prec, return sub_t<T>(L.ndofs, r, b, t, s))
}

// One vertex-patch Schwarz sweep on level l: for each colour (ascending, or descending when
// `post`) r = b - A x, then x_P += A_P^{-1} r_P on the colour's patches. With x_zero, x is
// cleared and the first colour takes r = b.
static cudaError_t smooth_vertex_patch(const tp_mg_s* mg, int l, void* x, const void* b, int x_zero, int post,
                                       cudaStream_t s) {
  const tp_mg_level& L = mg->lv[l];
  cudaError_t e = cudaSuccess;
  if (x_zero) e = cudaMemsetAsync(x, 0, L.ndofs * elem_bytes(mg->prec), s);
  bool zero = x_zero != 0;
  for (int i = 0; i < 8 && e == cudaSuccess; ++i) {
    const int c = post ? 7 - i : i;
    if (!vp_colour_nonempty(L.nc, c)) continue;
    const void* r = b;
    if (!zero) {
      e = residual(mg, L, L.r, b, x, L.t, s);
      r = L.r;
    }
    zero = false;
    if (e == cudaSuccess) e = vp_colour(mg->prec, mg->n, L.nc, c, x, r, L.vpS, L.vpL, L.vpC.data(), s);
  }
  return e;
}

// Smoothing step on level l from x (x_zero: x is taken as 0 and not read): `degree`
// Chebyshev-Jacobi steps, or one vertex-patch sweep (colours descending when `post`).
cudaError_t mg_smooth(const tp_mg_s* mg, int l, void* x, const void* b, int x_zero, cudaStream_t s, int post = 0) {
  if (mg->opts.smoother == TP_SMOOTHER_VERTEX_PATCH) return smooth_vertex_patch(mg, l, x, b, x_zero, post, s);
  const tp_mg_level& L = mg->lv[l];
  const double lmax = L.lmax, lmin = lmax / mg->opts.ratio;
  const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin), sigma = theta / delta;
  double rho = 1.0 / sigma;
  cudaError_t e;
  if (x_zero) {
    e = cudaMemcpyAsync(L.r, b, L.ndofs * elem_bytes(mg->prec), cudaMemcpyDeviceToDevice, s);
  } else {
    e = residual(mg, L, L.r, b, x, L.t, s);
  }
  if (e != cudaSuccess) return e;
  e = cheb_update(mg, L, x, L.r, L.d, nullptr, 0.0, 1.0 / theta, x_zero, s);
  for (int it = 1; it < mg->opts.degree && e == cudaSuccess; ++it) {
    e = launch_apply(L.op, L.t, L.d, s);
    if (e != cudaSuccess) break;
    const double rho_new = 1.0 / (2.0 * sigma - rho);
    e = cheb_update(mg, L, x, L.r, L.d, L.t, rho_new * rho, 2.0 * rho_new / delta, 0, s);
    rho = rho_new;
  }
  return e;
}

cudaError_t mg_vcycle(const tp_mg_s* mg, int l, void* x, const void* b, int x_zero, cudaStream_t s) {
  if (l == 0) return mg_coarse_solve(mg, x, b, s);
  const tp_mg_level& L = mg->lv[l];
  const tp_mg_level& C = mg->lv[l - 1];
  cudaError_t e = mg_smooth(mg, l, x, b, x_zero, s);
  if (e == cudaSuccess) e = residual(mg, L, L.r, b, x, L.t, s);
  if (e == cudaSuccess) e = mg_restrict(mg, l, C.b, L.r, s);
  if (e == cudaSuccess) e = mg_vcycle(mg, l - 1, C.x, C.b, 1, s);
  if (e == cudaSuccess) e = mg_prolong_add(mg, l, x, C.x, s);
  if (e == cudaSuccess) e = mg_smooth(mg, l, x, b, 0, s, 1);
  return e;
}

template <typename T>
static tp_status estimate_lmax_t(tp_mg_s* mg, int l, int iters, cudaStream_t s, double* out) {
  tp_mg_level& L = mg->lv[l];
  hash_fill<T><<<grid_for(L.ndofs), 256, 0, s>>>(L.ndofs, (T*)L.d, 12345u + l);
  double rho = 0.0, h[2];
  // L.d = x, L.t = A x, L.r = D x then D^{-1} A x
  for (int it = 0; it < iters; ++it) {
    cudaError_t e = launch_apply(L.op, L.t, L.d, s);
    if (e == cudaSuccess) e = dinv(mg, L, L.r, L.d, 1.0, 0, s);
    if (e == cudaSuccess) {
      const T* v[2] = {(const T*)L.t, (const T*)L.r};
      e = multi_dot<T>(L.ndofs, (const T*)L.d, v, 2, mg->partial, mg->dots, s);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, mg->dots, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e, "tp_mg_create: eigenvalue estimate");
    rho = h[0] / h[1];
    if (!std::isfinite(rho) || !(h[1] > 0)) {
      set_error("tp_mg_create: eigenvalue estimate broke down on level %d", l);
      return TP_ERR_NONFINITE;
    }
    // x <- D^{-1} A x, normalised
    e = dinv(mg, L, L.r, L.t, 1.0, 1, s);
    double nn = 0.0;
    if (e == cudaSuccess) {
      const T* v[1] = {(const T*)L.r};
      e = multi_dot<T>(L.ndofs, (const T*)L.r, v, 1, mg->partial, mg->dots, s);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&nn, mg->dots, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e, "tp_mg_create: eigenvalue estimate");
    if (!(nn > 0) || !std::isfinite(nn)) {
      set_error("tp_mg_create: eigenvalue estimate broke down on level %d", l);
      return TP_ERR_NONFINITE;
    }
    const double c[1] = {1.0 / std::sqrt(nn)};
    const T* v[1] = {(const T*)L.r};
    e = multi_axpy<T>(L.ndofs, (T*)L.d, 0.0, v, c, 1, s);
    if (e != cudaSuccess) return cuda_status(e, "tp_mg_create: eigenvalue estimate");
  }
  *out = rho;
  return TP_OK;
}

// lmax(D^{-1}A) on level l: power iteration x <- D^{-1}A x / |.| from a fixed
// pseudo-random start; the estimate is the generalized Rayleigh quotient
// (x, A x) / (x, D x) of the last iterate, which never exceeds lmax.
static tp_status estimate_lmax(tp_mg_s* mg, int l, int iters, cudaStream_t s, double* out) {
  switch (mg->prec) {
    case TP_FP64: return estimate_lmax_t<double>(mg, l, iters, s, out);
    case TP_FP32: return estimate_lmax_t<float>(mg, l, iters, s, out);
    case TP_FP16: return estimate_lmax_t<__half>(mg, l, iters, s, out);
    case TP_BF16: return estimate_lmax_t<__nv_bfloat16>(mg, l, iters, s, out);
  }
  set_error("tp_mg_create: unknown precision");
  return TP_ERR_INVALID_ARG;
}

int mg_finest_level(const tp_mg_s* mg) { return (int)mg->lv.size() - 1; }
tp_precision mg_precision(const tp_mg_s* mg) { return mg->prec; }
long long mg_finest_ndofs(const tp_mg_s* mg) { return mg->lv.back().ndofs; }

}  // namespace tp

using namespace tp;

static void free_level(tp_mg_level& L, bool own_xb) {
  if (L.op) tp_op_destroy(L.op);
  if (own_xb) {
    if (L.x) cudaFree(L.x);
    if (L.b) cudaFree(L.b);
  }
  if (L.r) cudaFree(L.r);
  if (L.d) cudaFree(L.d);
  if (L.t) cudaFree(L.t);
  if (L.vpS) cudaFree(L.vpS);
  if (L.vpL) cudaFree(L.vpL);
  L = tp_mg_level();
}

extern "C" {

tp_status tp_mg_destroy(tp_mg mg) {
  if (!mg) return TP_OK;
  for (size_t l = 0; l < mg->lv.size(); ++l) free_level(mg->lv[l], l + 1 < mg->lv.size());
  for (int d = 0; d < 3; ++d) {
    if (mg->fdV[d]) cudaFree(mg->fdV[d]);
    if (mg->fdL[d]) cudaFree(mg->fdL[d]);
  }
  if (mg->fdT0) cudaFree(mg->fdT0);
  if (mg->fdT1) cudaFree(mg->fdT1);
  if (mg->partial) cudaFree(mg->partial);
  if (mg->dots) cudaFree(mg->dots);
  delete mg;
  return TP_OK;
}

tp_status tp_mg_create(tp_mg* out, tp_op finest, const tp_mg_opts* opts) {
  if (!out) { set_error("tp_mg_create: out is NULL"); return TP_ERR_INVALID_ARG; }
  *out = nullptr;
  if (!finest) { set_error("tp_mg_create: operator is NULL"); return TP_ERR_INVALID_ARG; }
  if (finest->n > kMaxN) {
    set_error("tp_mg_create: degree k=%d above %d (the transfer and smoother kernels take n <= %d)", finest->k,
              kMaxN - 1, kMaxN);
    return TP_ERR_UNSUPPORTED;
  }
  if (finest->ncells >= (1LL << 31)) {
    set_error("tp_mg_create: meshes of 2^31 cells or more are not supported");
    return TP_ERR_UNSUPPORTED;
  }
  tp_mg_opts o{3, 15.0, 1.1, 0.0, 4, TP_FP32, 20, TP_KERNEL_CUDA_CORE, 0, TP_FP16, TP_SMOOTHER_CHEBYSHEV};
  if (opts) o = *opts;
  if (o.smoother != TP_SMOOTHER_CHEBYSHEV && o.smoother != TP_SMOOTHER_VERTEX_PATCH) {
    set_error("tp_mg_create: smoother must be TP_SMOOTHER_CHEBYSHEV or TP_SMOOTHER_VERTEX_PATCH");
    return TP_ERR_INVALID_ARG;
  }
  if (o.kernel == TP_KERNEL_PATCH) {
    set_error("tp_mg_create: the level operators take the CUDA-core or tensor kernels, not the patch-wise one");
    return TP_ERR_UNSUPPORTED;
  }
  if (o.degree < 1 || o.degree > 16 || !(o.ratio > 1.0) || !(o.safety > 0) || o.coarse_cells < 1 ||
      (o.precision != TP_FP64 && o.precision != TP_FP32 && o.precision != TP_FP16 && o.precision != TP_BF16) ||
      o.power_iters < 1 || o.lmax < 0) {
    set_error("tp_mg_create: invalid options (degree 1..16, ratio > 1, safety > 0, coarse_cells >= 1, "
              "precision FP64, FP32, FP16 or BF16, power_iters >= 1, lmax >= 0)");
    return TP_ERR_INVALID_ARG;
  }
  tp_mg_s* mg = new (std::nothrow) tp_mg_s();
  if (!mg) { set_error("tp_mg_create: out of host memory"); return TP_ERR_OOM; }
  mg->k = finest->k;
  mg->n = finest->n;
  mg->prec = (tp_precision)o.precision;
  mg->opts = o;
  // level sizes: halve every direction while all are even and any exceeds coarse_cells
  std::vector<std::array<int, 3>> sizes;
  std::array<int, 3> cur = {finest->mesh.nx, finest->mesh.ny, finest->mesh.nz};
  sizes.push_back(cur);
  while ((cur[0] > o.coarse_cells || cur[1] > o.coarse_cells || cur[2] > o.coarse_cells) && cur[0] % 2 == 0 &&
         cur[1] % 2 == 0 && cur[2] % 2 == 0) {
    cur = {cur[0] / 2, cur[1] / 2, cur[2] / 2};
    sizes.push_back(cur);
  }
  const int nl = (int)sizes.size();
  if (nl > TP_MAX_LEVELS) {
    delete mg;
    set_error("tp_mg_create: more than %d levels", TP_MAX_LEVELS);
    return TP_ERR_INVALID_ARG;
  }
  mg->lv.resize(nl);
  const size_t eb = elem_bytes(mg->prec);
  tp_status st = TP_OK;
  tp_op_opts oo{finest->opts.penalty, o.kernel, o.ec, o.tc_type, finest->opts.autotune};
  for (int l = 0; l < nl && st == TP_OK; ++l) {
    tp_mg_level& L = mg->lv[l];
    const auto& sz = sizes[nl - 1 - l];
    L.nc[0] = sz[0]; L.nc[1] = sz[1]; L.nc[2] = sz[2];
    tp_mesh_s m{sz[0], sz[1], sz[2], finest->mesh.lx, finest->mesh.ly, finest->mesh.lz};
    tp_op_opts lo = oo;
    if (lo.kernel == TP_KERNEL_TENSOR && (mg->prec == TP_FP64 || mg->k < 2 || mg->k > 3)) lo.kernel = TP_KERNEL_CUDA_CORE;
    if (lo.kernel != TP_KERNEL_TENSOR) lo.ec = 0;
    st = tp_dg_laplace_create(&L.op, &m, mg->k, mg->prec, &lo);
    if (st != TP_OK) break;
    L.ndofs = L.op->ndofs;
    const size_t bytes = (size_t)L.ndofs * eb;
    if (l + 1 < nl) {
      st = cuda_status(cudaMalloc(&L.x, bytes), "tp_mg_create: level vectors");
      if (st == TP_OK) st = cuda_status(cudaMalloc(&L.b, bytes), "tp_mg_create: level vectors");
    }
    if (st == TP_OK) st = cuda_status(cudaMalloc(&L.r, bytes), "tp_mg_create: level vectors");
    if (st == TP_OK) st = cuda_status(cudaMalloc(&L.d, bytes), "tp_mg_create: level vectors");
    if (st == TP_OK) st = cuda_status(cudaMalloc(&L.t, bytes), "tp_mg_create: level vectors");
    // Jacobi diagonal data
    if (st == TP_OK) {
      memset(&L.j64, 0, sizeof(L.j64));
      for (int d = 0; d < 3; ++d) {
        const Dir1D& dd = L.op->dir[d];
        for (int i = 0; i < mg->n; ++i) {
          L.j64.Md[d][i] = dd.M[i * mg->n + i];
          L.j64.Ld[d][i] = dd.L[i * mg->n + i];
        }
        L.j64.lo[d] = L.op->ref.d0[0] / dd.h;
        L.j64.hi[d] = -L.op->ref.d1[mg->n - 1] / dd.h;
      }
      L.j64.nx = sz[0]; L.j64.ny = sz[1]; L.j64.nz = sz[2];
      L.j32.nx = sz[0]; L.j32.ny = sz[1]; L.j32.nz = sz[2];
      L.j64.dx = L.j32.dx = make_fastdiv((uint32_t)sz[0]);
      L.j64.dy = L.j32.dy = make_fastdiv((uint32_t)sz[1]);
      for (int d = 0; d < 3; ++d) {
        for (int i = 0; i < kMaxN; ++i) { L.j32.Md[d][i] = (float)L.j64.Md[d][i]; L.j32.Ld[d][i] = (float)L.j64.Ld[d][i]; }
        L.j32.lo[d] = (float)L.j64.lo[d];
        L.j32.hi[d] = (float)L.j64.hi[d];
      }
    }
  }
  // transfer matrices
  if (st == TP_OK) {
    memset(&mg->p64, 0, sizeof(mg->p64));
    const Ref1D& r = mg->lv.back().op->ref;
    for (int c = 0; c < 2; ++c) {
      std::vector<double> xs(mg->n);
      for (int i = 0; i < mg->n; ++i) xs[i] = 0.5 * (c + r.nodes[i]);
      std::vector<double> V = lagrange_eval(r.nodes, xs);
      for (int i = 0; i < mg->n; ++i)
        for (int j = 0; j < mg->n; ++j) {
          mg->p64.P[c][i * kMaxN + j] = V[i * mg->n + j];
          mg->p32.P[c][i * kMaxN + j] = (float)V[i * mg->n + j];
        }
    }
  }
  // coarse fast diagonalization
  if (st == TP_OK) {
    tp_mg_level& C = mg->lv[0];
    mg->fd.n = mg->n;
    mg->fd.nx = C.nc[0]; mg->fd.ny = C.nc[1]; mg->fd.nz = C.nc[2];
    for (int d = 0; d < 3 && st == TP_OK; ++d) {
      const int N1 = C.nc[d] * mg->n;
      mg->fd.N1[d] = N1;
      std::vector<double> M, L, lam, V;
      global_1d(C.op->ref, C.op->dir[d], C.nc[d], M, L);
      if (!gen_eig(N1, M, L, lam, V)) { set_error("tp_mg_create: coarse mass matrix not positive definite"); st = TP_ERR_INVALID_ARG; break; }
      st = cuda_status(cudaMalloc(&mg->fdV[d], sizeof(double) * N1 * N1), "tp_mg_create: coarse solve");
      if (st == TP_OK) st = cuda_status(cudaMalloc(&mg->fdL[d], sizeof(double) * N1), "tp_mg_create: coarse solve");
      if (st == TP_OK) st = cuda_status(cudaMemcpy(mg->fdV[d], V.data(), sizeof(double) * N1 * N1, cudaMemcpyHostToDevice), "cudaMemcpy");
      if (st == TP_OK) st = cuda_status(cudaMemcpy(mg->fdL[d], lam.data(), sizeof(double) * N1, cudaMemcpyHostToDevice), "cudaMemcpy");
    }
    const long long tot = fd_total(mg->fd);
    if (st == TP_OK) st = cuda_status(cudaMalloc(&mg->fdT0, sizeof(double) * tot), "tp_mg_create: coarse solve");
    if (st == TP_OK) st = cuda_status(cudaMalloc(&mg->fdT1, sizeof(double) * tot), "tp_mg_create: coarse solve");
  }
  if (st == TP_OK) st = cuda_status(cudaMalloc(&mg->partial, sizeof(double) * (kMaxMulti + 1) * dot_blocks(mg->lv.back().ndofs)), "tp_mg_create: scratch");
  if (st == TP_OK) st = cuda_status(cudaMalloc(&mg->dots, sizeof(double) * kMaxMulti), "tp_mg_create: scratch");
  // vertex-patch eigenbases of every smoothed level (each has >= 2 cells per direction: it is at
  // least twice the coarsest level)
  for (int l = 1; l < nl && st == TP_OK && o.smoother == TP_SMOOTHER_VERTEX_PATCH; ++l)
    st = vp_tables(mg->lv[l].op, mg->lv[l].nc, mg->prec, &mg->lv[l].vpS, &mg->lv[l].vpL, &mg->lv[l].vpC);
  // smoother eigenvalue bounds
  for (int l = 1; l < nl && st == TP_OK && o.smoother == TP_SMOOTHER_CHEBYSHEV; ++l) {
    if (o.lmax > 0) {
      mg->lv[l].lmax = o.lmax;
    } else {
      double est = 0.0;
      st = estimate_lmax(mg, l, o.power_iters, 0, &est);
      mg->lv[l].lmax = o.safety * est;
    }
  }
  if (st == TP_OK) st = cuda_status(cudaDeviceSynchronize(), "tp_mg_create");
  if (st != TP_OK) {
    tp_mg_destroy(mg);
    return st;
  }
  *out = mg;
  return TP_OK;
}

tp_status tp_mg_get_info(tp_mg mg, tp_mg_info_t* info) {
  if (!mg || !info) { set_error("tp_mg_get_info: NULL argument"); return TP_ERR_INVALID_ARG; }
  memset(info, 0, sizeof(*info));
  info->levels = (int)mg->lv.size();
  info->precision = mg->prec;
  for (int l = 0; l < info->levels && l < TP_MAX_LEVELS; ++l) {
    info->cells[l][0] = mg->lv[l].nc[0];
    info->cells[l][1] = mg->lv[l].nc[1];
    info->cells[l][2] = mg->lv[l].nc[2];
    info->ndofs[l] = mg->lv[l].ndofs;
    info->lmax[l] = mg->lv[l].lmax;
  }
  return TP_OK;
}

tp_status tp_mg_level_op(tp_mg mg, int level, tp_op* op) {
  if (!mg || !op || level < 0 || level >= (int)mg->lv.size()) { set_error("tp_mg_level_op: bad argument"); return TP_ERR_INVALID_ARG; }
  *op = mg->lv[level].op;
  return TP_OK;
}

static tp_status check_level(tp_mg mg, int level, const void* a, const void* b, const char* who, int min_level) {
  if (!mg || !a || !b) { set_error("%s: NULL argument", who); return TP_ERR_INVALID_ARG; }
  if (level < min_level || level >= (int)mg->lv.size()) { set_error("%s: level %d out of range", who, level); return TP_ERR_INVALID_ARG; }
  if (((uintptr_t)a & 15) || ((uintptr_t)b & 15)) { set_error("%s: vectors must be 16-byte aligned", who); return TP_ERR_INVALID_ARG; }
  return TP_OK;
}

tp_status tp_vcycle(tp_mg mg, void* x, const void* b, void* stream) {
  tp_status st = check_level(mg, (int)(mg ? mg->lv.size() - 1 : 0), x, b, "tp_vcycle", 0);
  if (st != TP_OK) return st;
  return cuda_status(mg_vcycle(mg, (int)mg->lv.size() - 1, x, b, 0, (cudaStream_t)stream), "tp_vcycle");
}

tp_status tp_mg_smooth(tp_mg mg, int level, void* x, const void* b, void* stream) {
  tp_status st = check_level(mg, level, x, b, "tp_mg_smooth", 1);
  if (st != TP_OK) return st;
  return cuda_status(mg_smooth(mg, level, x, b, 0, (cudaStream_t)stream), "tp_mg_smooth");
}

tp_status tp_mg_restrict(tp_mg mg, int level, void* coarse, const void* fine, void* stream) {
  tp_status st = check_level(mg, level, coarse, fine, "tp_mg_restrict", 1);
  if (st != TP_OK) return st;
  return cuda_status(mg_restrict(mg, level, coarse, fine, (cudaStream_t)stream), "tp_mg_restrict");
}

tp_status tp_mg_prolongate_add(tp_mg mg, int level, void* fine, const void* coarse, void* stream) {
  tp_status st = check_level(mg, level, fine, coarse, "tp_mg_prolongate_add", 1);
  if (st != TP_OK) return st;
  return cuda_status(mg_prolong_add(mg, level, fine, coarse, (cudaStream_t)stream), "tp_mg_prolongate_add");
}

tp_status tp_mg_coarse_solve(tp_mg mg, void* x, const void* b, void* stream) {
  tp_status st = check_level(mg, 0, x, b, "tp_mg_coarse_solve", 0);
  if (st != TP_OK) return st;
  return cuda_status(mg_coarse_solve(mg, x, b, (cudaStream_t)stream), "tp_mg_coarse_solve");
}

}  // extern "C"
