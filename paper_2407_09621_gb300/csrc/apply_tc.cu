// Tensor-core SIPG apply for degrees k = 2, 3 (n <= 4), mma.sync m16n8k16 with
// FP32 accumulation (Sec. 3.2 / Sec. 5: half-precision operands, single-
// precision accumulator; Algorithm 1 error correction optional).
//
// Inverse-mass form of Eq. (9) (see apply_cc.cu): v = M3 w, w = K3 u + faces,
// with K3 = G_z(+)G_y(+)G_x (the three M^-1 L_int contractions as one 64 x 64
// matrix) and M3 = M_z(x)M_y(x)M_x, cells padded to 4 x 4 x 4 = 64 entries.
// With 64 entries per cell the two cell products are plain GEMMs whose row
// index is the cell: W (cells x 64) = U (cells x 64) K3^T and V = W M3^T. The
// cell-major vector layout is already the row-major A operand, so no reshaping
// is needed; the paper's per-direction reshapes (Sec. 4.1) disappear. The face
// terms (rank 2 along each normal, see apply_cc.cu) are added to W in FP32 on
// the FMA pipes from neighbour tiles staged in shared memory.
//
// Block: 128 threads (4 warps), a tile of 64 consecutive cells; warp w owns
// cells 16w..16w+15 in both GEMMs. Shared memory: the two 64 x 64 operand
// matrices (and their low parts with EC), the A operand (72-half rows, so
// ldmatrix rows of 16 bytes hit distinct banks), W in FP32, the raw own tile
// with one halo cell on each side (x faces) and a staging area for the y and
// z neighbour tiles (the tiles at cell offsets -+nx and -+nx*ny).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <type_traits>
#include <cstring>
#include <vector>

#include "tp_internal.h"

namespace tp {

constexpr int kTcCells = 64;  // cells per block
constexpr int kTcRow = 72;    // halves per A/B row in shared memory (64 + 8 padding)
constexpr int kTcWRow = 68;   // floats per W row

template <typename TO>
struct OpTraits;
template <>
struct OpTraits<__half> {
  static __device__ __forceinline__ __half from(float v) { return __float2half_rn(v); }
  static __device__ __forceinline__ float to(__half v) { return __half2float(v); }
};
template <>
struct OpTraits<__nv_bfloat16> {
  static __device__ __forceinline__ __nv_bfloat16 from(float v) { return __float2bfloat16_rn(v); }
  static __device__ __forceinline__ float to(__nv_bfloat16 v) { return __bfloat162float(v); }
};

template <typename TS>
__device__ __forceinline__ float ld_f32(const TS* p) { return (float)*p; }
template <>
__device__ __forceinline__ float ld_f32<__half>(const __half* p) { return __half2float(*p); }
template <>
__device__ __forceinline__ float ld_f32<__nv_bfloat16>(const __nv_bfloat16* p) { return __bfloat162float(*p); }
template <typename TS>
__device__ __forceinline__ float ldg_f32(const TS* p) { return (float)__ldg(p); }
template <>
__device__ __forceinline__ float ldg_f32<__half>(const __half* p) { return __half2float(__ldg(p)); }
template <>
__device__ __forceinline__ float ldg_f32<__nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat162float(__ldg(p));
}
template <typename TS>
__device__ __forceinline__ TS from_f32(float v) { return (TS)v; }
template <>
__device__ __forceinline__ __half from_f32<__half>(float v) { return __float2half_rn(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 from_f32<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}

template <typename TO>
__device__ __forceinline__ void mma16816(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1);
template <>
__device__ __forceinline__ void mma16816<__half>(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
               "{%0,%1,%2,%3};\n"
               : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
               : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
template <>
__device__ __forceinline__ void mma16816<__nv_bfloat16>(float (&c)[4], const uint32_t (&a)[4], uint32_t b0,
                                                        uint32_t b1) {
  asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
               "{%0,%1,%2,%3};\n"
               : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
               : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// acc (16 cells x 64) = A_rows (16 x 64, shared, row stride kTcRow) * B^T, B stored [out][in].
// With EC: main = Ah Bh, corr = Al Bh (has_al: the A operand is refined) + Ah Bl (has_bl: the
// matrix is refined); Algorithm 1 refines both.
template <typename TO, bool EC>
__device__ __forceinline__ void tile_gemm(float (&acc)[8][4], float (&cor)[8][4], const TO* Ah, const TO* Al,
                                          bool has_al, const TO* Bh, const TO* Bl, bool has_bl, int lane) {
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
#pragma unroll
    for (int e = 0; e < 4; ++e) { acc[nt][e] = 0.f; cor[nt][e] = 0.f; }
  const int mi = lane >> 3, r = lane & 7;
  // A: matrices (rows 0-7,k0), (rows 8-15,k0), (rows 0-7,k8), (rows 8-15,k8)
  const int arow = r + (mi & 1) * 8, acol = (mi >> 1) * 8;
  // B (x4 = two n-tiles): (n 0-7,k0), (n 0-7,k8), (n 8-15,k0), (n 8-15,k8)
  const int brow = r + (mi >> 1) * 8, bcol = (mi & 1) * 8;
#pragma unroll
  for (int ks = 0; ks < 4; ++ks) {
    uint32_t ah[4], al[4] = {0u, 0u, 0u, 0u};
    ldsm_x4(smem_u32(Ah + arow * kTcRow + ks * 16 + acol), ah[0], ah[1], ah[2], ah[3]);
    if (EC && has_al) ldsm_x4(smem_u32(Al + arow * kTcRow + ks * 16 + acol), al[0], al[1], al[2], al[3]);
#pragma unroll
    for (int np = 0; np < 4; ++np) {
      uint32_t b[4];
      ldsm_x4(smem_u32(Bh + (np * 16 + brow) * kTcRow + ks * 16 + bcol), b[0], b[1], b[2], b[3]);
      mma16816<TO>(acc[2 * np], ah, b[0], b[1]);
      mma16816<TO>(acc[2 * np + 1], ah, b[2], b[3]);
      if (EC) {
        if (has_bl) {
          uint32_t bl[4];
          ldsm_x4(smem_u32(Bl + (np * 16 + brow) * kTcRow + ks * 16 + bcol), bl[0], bl[1], bl[2], bl[3]);
          mma16816<TO>(cor[2 * np], ah, bl[0], bl[1]);
          mma16816<TO>(cor[2 * np + 1], ah, bl[2], bl[3]);
        }
        if (has_al) {
          mma16816<TO>(cor[2 * np], al, b[0], b[1]);
          mma16816<TO>(cor[2 * np + 1], al, b[2], b[3]);
        }
      }
    }
  }
}

// writes acc (+ cor * 2^-s) of warp rows [16w, 16w+16) into W (FP32)
template <bool EC>
__device__ __forceinline__ void store_acc(float* sW, const float (&acc)[8][4], const float (&cor)[8][4], int w,
                                          int lane, float inv_scale, const float* rowmul) {
  const int g = lane >> 2, t = lane & 3;
  const float m0 = rowmul[16 * w + g], m1 = rowmul[16 * w + g + 8];
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const int col = nt * 8 + 2 * t;
    float v0 = acc[nt][0], v1 = acc[nt][1], v2 = acc[nt][2], v3 = acc[nt][3];
    if (EC) {
      v0 = fmaf(cor[nt][0], inv_scale, v0);
      v1 = fmaf(cor[nt][1], inv_scale, v1);
      v2 = fmaf(cor[nt][2], inv_scale, v2);
      v3 = fmaf(cor[nt][3], inv_scale, v3);
    }
    sW[(16 * w + g) * kTcWRow + col] = v0 * m0;
    sW[(16 * w + g) * kTcWRow + col + 1] = v1 * m0;
    sW[(16 * w + g + 8) * kTcWRow + col] = v2 * m1;
    sW[(16 * w + g + 8) * kTcWRow + col + 1] = v3 * m1;
  }
}

// Power of two 2^e >= max |v| over a cell row (1 for an all-zero row): the row is divided by it
// before rounding to the operand type, so FP16 never overflows and the rounding error is
// relative to the row's largest entry; the exact power is reapplied in the FP32 epilogue.
__device__ __forceinline__ float row_pow2(float amax) {
  if (!(amax > 0.f)) return 1.f;
  int e;
  frexpf(amax, &e);  // amax = f * 2^e, f in [0.5, 1)
  return ldexpf(1.f, e);
}

// rounds v to the operand type; with EC also stores the scaled residual
template <typename TO, bool EC>
__device__ __forceinline__ void split_store(TO* hi, TO* lo, int idx, float v, float scale) {
  const TO h = OpTraits<TO>::from(v);
  hi[idx] = h;
  if (EC) lo[idx] = OpTraits<TO>::from((v - OpTraits<TO>::to(h)) * scale);
}

struct TcDims {
  int nx, ny, nz;
  long long ncells;
  float scale, inv_scale;  // 2^s and 2^-s of Algorithm 1
  float k3_inv, m3_inv;    // the operand matrices are stored times powers of two k3, m3
  int refine_vec, refine_mat;  // error-correction mode (both 1: Algorithm 1)
};

// Copies cells [first, first + count) of x into dst (zeros outside [0, ncells)),
// with 16-byte vectors when the cell size allows it.
template <typename TS, int N>
__device__ __forceinline__ void stage_cells(TS* dst, const TS* __restrict__ x, long long first, int count,
                                            long long ncells, int tid) {
  constexpr int N3 = N * N * N;
  constexpr int CB = N3 * (int)sizeof(TS);  // bytes per cell
  if (CB % 16 == 0) {
    constexpr int CH = CB / 16;  // 16-byte chunks per cell
    const uint4* src = reinterpret_cast<const uint4*>(x);
    uint4* d = reinterpret_cast<uint4*>(dst);
    for (int e = tid; e < count * CH; e += 128) {
      const long long cell = first + e / CH;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (cell >= 0 && cell < ncells) v = __ldg(src + cell * CH + e % CH);
      d[e] = v;
    }
  } else {
    for (int e = tid; e < count * N3; e += 128) {
      const long long cell = first + e / N3;
      dst[e] = (cell >= 0 && cell < ncells) ? __ldg(x + cell * N3 + e % N3) : from_f32<TS>(0.f);
    }
  }
}

template <typename TS, typename TO, int N, bool EC>
__global__ void __launch_bounds__(128) apply_tc_kernel(const TS* __restrict__ x, TS* __restrict__ y,
                                                      const TO* __restrict__ mats,
                                                      const __grid_constant__ OpConst<float> P, TcDims D) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int MAT = 64 * kTcRow;  // halves per operand matrix in shared memory
  constexpr int N2 = N * N, N3 = N2 * N;
  TO* sK = reinterpret_cast<TO*>(smem_raw);      // K3 (hi), then K3 lo, M3 hi, M3 lo
  TO* sM = sK + (EC ? 2 : 1) * MAT;
  TO* sAh = sK + (EC ? 4 : 2) * MAT;
  TO* sAl = sAh + MAT;  // only with EC
  float* sW = reinterpret_cast<float*>(sAh + (EC ? 2 : 1) * MAT);
  // raw tiles: own with one halo cell each side (66 cells), then y-, y+, z-, z+ (64 cells each)
  float* sRow = sW + kTcCells * kTcWRow;  // per-row multipliers of the current GEMM output
  TS* sR = reinterpret_cast<TS*>(sRow + kTcCells);
  TS* sNb[4] = {sR + (kTcCells + 2) * N3, sR + (2 * kTcCells + 2) * N3, sR + (3 * kTcCells + 2) * N3,
                sR + (4 * kTcCells + 2) * N3};

  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const long long sy = D.nx, sz = (long long)D.nx * D.ny;

  // ---- operand matrices (global, [K3h | K3l | M3h | M3l] or [K3h | M3h], each 64 x 64) -> shared
  {
    constexpr int nm = EC ? 4 : 2;
    for (int e = tid; e < nm * 64 * 8; e += 128) {  // 16-byte chunks
      const int m = e / 512, rem = e % 512, row = rem / 8, ch = rem % 8;
      const uint4 v = __ldg(reinterpret_cast<const uint4*>(mats + (size_t)m * 4096 + row * 64) + ch);
      *reinterpret_cast<uint4*>(sK + m * MAT + row * kTcRow + ch * 8) = v;
    }
  }
  const long long ntiles = (D.ncells + kTcCells - 1) / kTcCells;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
  const long long c0 = tile * kTcCells;
  // ---- all raw tiles in one phase
  stage_cells<TS, N>(sR, x, c0 - 1, kTcCells + 2, D.ncells, tid);
  stage_cells<TS, N>(sNb[0], x, c0 - sy, kTcCells, D.ncells, tid);
  stage_cells<TS, N>(sNb[1], x, c0 + sy, kTcCells, D.ncells, tid);
  stage_cells<TS, N>(sNb[2], x, c0 - sz, kTcCells, D.ncells, tid);
  stage_cells<TS, N>(sNb[3], x, c0 + sz, kTcCells, D.ncells, tid);
  __syncthreads();
  // ---- A operand (padded to 4^3), row-scaled, with optional split; 2 threads per cell row
  {
    const int c = tid >> 1, p0 = (tid & 1) * 32;
    float v[32], amax = 0.f;
#pragma unroll
    for (int q = 0; q < 32; ++q) {
      const int p = p0 + q, i = p & 3, j = (p >> 2) & 3, l = p >> 4;
      v[q] = (i < N && j < N && l < N) ? ld_f32<TS>(sR + (c + 1) * N3 + (l * N + j) * N + i) : 0.f;
      amax = fmaxf(amax, fabsf(v[q]));
    }
    amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, 1));
    const float rs = row_pow2(amax), inv = 1.f / rs;
#pragma unroll
    for (int q = 0; q < 32; ++q) split_store<TO, EC>(sAh, sAl, c * kTcRow + p0 + q, v[q] * inv, D.scale);
    if ((tid & 1) == 0) sRow[c] = rs * D.k3_inv;
  }
  __syncthreads();

  float acc[8][4], cor[8][4];
  // ---- W = U K3^T
  tile_gemm<TO, EC>(acc, cor, sAh + 16 * w * kTcRow, sAl + 16 * w * kTcRow, EC && sizeof(TS) == 4 && D.refine_vec,
                    sK, sK + MAT, D.refine_mat != 0, lane);
  store_acc<EC>(sW, acc, cor, w, lane, D.inv_scale, sRow);
  __syncthreads();

  // ---- faces, one direction at a time; tasks = (cell, line) along the normal
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const TS* nb_lo = d == 0 ? sR : sNb[2 * d - 2];               // cell c's low neighbour at index c
    const TS* nb_hi = d == 0 ? sR + 2 * N3 : sNb[2 * d - 1];      // cell c's high neighbour at index c
    constexpr int dummy = 0;
    (void)dummy;
    const int lstep = d == 0 ? 1 : (d == 1 ? N : N2);  // stride of the line inside a cell
    const int pstep = d == 0 ? 1 : (d == 1 ? 4 : 16);  // stride along the line in the padded W row
    for (int task = tid; task < kTcCells * N2; task += 128) {
      const int c = task / N2, a = (task % N2) / N, b = task % N;
      const long long cell = c0 + c;
      if (cell >= D.ncells) continue;
      int co, ncd;
      if (d == 0) { co = (int)(cell % D.nx); ncd = D.nx; }
      else if (d == 1) { co = (int)((cell / D.nx) % D.ny); ncd = D.ny; }
      else { co = (int)(cell / ((long long)D.nx * D.ny)); ncd = D.nz; }
      int off, pofs;
      if (d == 0) { off = (a * N + b) * N; pofs = a * 16 + b * 4; }        // (l=a, j=b)
      else if (d == 1) { off = a * N2 + b; pofs = a * 16 + b; }           // (l=a, i=b)
      else { off = a * N + b; pofs = a * 4 + b; }                         // (j=a, i=b)
      const TS* own = sR + (c + 1) * N3 + off;
      const TS* lo = nb_lo + c * N3 + off;
      const TS* hi = nb_hi + c * N3 + off;
      float u[N], wv[N], add[N];
#pragma unroll
      for (int m = 0; m < N; ++m) { u[m] = ld_f32<TS>(own + m * lstep); add[m] = 0.f; }
      if (co < ncd - 1) {
        float sd = 0.f;
#pragma unroll
        for (int m = 0; m < N; ++m) { wv[m] = ld_f32<TS>(hi + m * lstep); sd = fmaf(P.d0[m], wv[m], sd); }
#pragma unroll
        for (int i = 0; i < N; ++i) add[i] = fmaf(P.E[d][0][i], wv[0], fmaf(P.E[d][1][i], sd, add[i]));
      } else {
        float sd = 0.f;
#pragma unroll
        for (int m = 0; m < N; ++m) sd = fmaf(P.d1[m], u[m], sd);
#pragma unroll
        for (int i = 0; i < N; ++i) add[i] = fmaf(P.E[d][4][i], u[N - 1], fmaf(P.E[d][5][i], sd, add[i]));
      }
      if (co > 0) {
        float sd = 0.f;
#pragma unroll
        for (int m = 0; m < N; ++m) { wv[m] = ld_f32<TS>(lo + m * lstep); sd = fmaf(P.d1[m], wv[m], sd); }
#pragma unroll
        for (int i = 0; i < N; ++i) add[i] = fmaf(P.E[d][2][i], wv[N - 1], fmaf(P.E[d][3][i], sd, add[i]));
      } else {
        float sd = 0.f;
#pragma unroll
        for (int m = 0; m < N; ++m) sd = fmaf(P.d0[m], u[m], sd);
#pragma unroll
        for (int i = 0; i < N; ++i) add[i] = fmaf(P.E[d][6][i], u[0], fmaf(P.E[d][7][i], sd, add[i]));
      }
#pragma unroll
      for (int i = 0; i < N; ++i) sW[c * kTcWRow + pofs + i * pstep] += add[i];
    }
    __syncthreads();
  }

  // ---- W -> A operand, row-scaled (split with EC)
  {
    const int c = tid >> 1, p0 = (tid & 1) * 32;
    float amax = 0.f;
#pragma unroll
    for (int q = 0; q < 32; ++q) amax = fmaxf(amax, fabsf(sW[c * kTcWRow + p0 + q]));
    amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, 1));
    const float rs = row_pow2(amax), inv = 1.f / rs;
#pragma unroll
    for (int q = 0; q < 32; ++q) split_store<TO, EC>(sAh, sAl, c * kTcRow + p0 + q, sW[c * kTcWRow + p0 + q] * inv, D.scale);
    __syncthreads();  // every row scale is read before sRow is overwritten
    if ((tid & 1) == 0) sRow[c] = rs * D.m3_inv;
  }
  __syncthreads();

  // ---- V = W M3^T
  tile_gemm<TO, EC>(acc, cor, sAh + 16 * w * kTcRow, sAl + 16 * w * kTcRow, EC && D.refine_vec, sM, sM + MAT,
                    D.refine_mat != 0, lane);
  store_acc<EC>(sW, acc, cor, w, lane, D.inv_scale, sRow);
  __syncthreads();

  // ---- coalesced write-out of the N^3 real entries of every cell
  const int ncell_tile = (int)((D.ncells - c0) < kTcCells ? (D.ncells - c0) : kTcCells);
  for (int e = tid; e < ncell_tile * N3; e += 128) {
    const int c = e / N3, r = e % N3, i = r % N, j = (r / N) % N, l = r / N2;
    y[c0 * N3 + e] = from_f32<TS>(sW[c * kTcWRow + l * 16 + j * 4 + i]);
  }
  __syncthreads();  // the next tile overwrites the staged data
  }  // tile loop
}

template <typename TS, typename TO, int N, bool EC>
static size_t tc_smem_bytes() {
  const size_t mats = (EC ? 4 : 2) * 64 * kTcRow * sizeof(TO);
  const size_t a = (EC ? 2 : 1) * 64 * kTcRow * sizeof(TO);
  const size_t wbytes = (kTcCells * kTcWRow + kTcCells) * sizeof(float);
  const size_t raw = (size_t)(5 * kTcCells + 2) * N * N * N * sizeof(TS);
  return mats + a + wbytes + ((raw + 15) & ~(size_t)15);
}

// host: build K3 and M3 (64 x 64, padded), split into the operand type, upload
template <typename TO>
static TO host_round(float v);
template <>
__half host_round<__half>(float v) { return __float2half_rn(v); }
template <>
__nv_bfloat16 host_round<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <typename TO>
static float host_widen(TO v);
template <>
float host_widen<__half>(__half v) { return __half2float(v); }
template <>
float host_widen<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

// Operand scaling: G_d = M_d^-1 L_d grows as 1/h^2 and M3 shrinks as h^3, out of the FP16 range.
// Each matrix is stored times the power of two that brings its largest entry into [32, 64) (K3)
// or [0.5, 1) (M3); with unit-scaled rows every product then stays far below the FP16 maximum.
static double pow2_to(double amax, double target) {
  int e;
  std::frexp(amax / target, &e);
  return std::ldexp(1.0, -e);
}
static void tc_scales(const tp_op_s* op, double& sk, double& sm) {
  double kmax = 0.0, mmax = 0.0;
  for (int d = 0; d < 3; ++d)
    for (int e = 0; e < kMaxN * kMaxN; ++e) {
      kmax = std::fmax(kmax, std::fabs(op->c64.G[d][e]));
      mmax = std::fmax(mmax, std::fabs(op->c64.M[d][e]));
    }
  sk = pow2_to(3.0 * kmax, 64.0);
  sm = pow2_to(mmax * mmax * mmax, 1.0);
}

template <typename TO>
static std::vector<TO> build_mats(const tp_op_s* op, bool ec, float scale) {
  const int n = op->n;
  double sw, sm;
  tc_scales(op, sw, sm);
  std::vector<double> K3(64 * 64, 0.0), M3(64 * 64, 0.0);
  auto G = [&](int d, int a, int b) { return op->c64.G[d][a * kMaxN + b]; };
  auto M = [&](int d, int a, int b) { return op->c64.M[d][a * kMaxN + b]; };
  for (int l = 0; l < n; ++l)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        const int r = l * 16 + j * 4 + i;
        for (int l2 = 0; l2 < n; ++l2)
          for (int j2 = 0; j2 < n; ++j2)
            for (int i2 = 0; i2 < n; ++i2) {
              const int c = l2 * 16 + j2 * 4 + i2;
              double k = 0.0;
              if (j == j2 && i == i2) k += G(2, l, l2);
              if (l == l2 && i == i2) k += G(1, j, j2);
              if (l == l2 && j == j2) k += G(0, i, i2);
              K3[r * 64 + c] = sw * k;
              M3[r * 64 + c] = sm * M(2, l, l2) * M(1, j, j2) * M(0, i, i2);
            }
      }
  std::vector<TO> out((ec ? 4 : 2) * 4096);
  auto put = [&](const std::vector<double>& A, int slot_h, int slot_l) {
    for (int e = 0; e < 4096; ++e) {
      const float v = (float)A[e];
      const TO h = host_round<TO>(v);
      out[(size_t)slot_h * 4096 + e] = h;
      if (slot_l >= 0) out[(size_t)slot_l * 4096 + e] = host_round<TO>((v - host_widen<TO>(h)) * scale);
    }
  };
  if (ec) {
    put(K3, 0, 1);
    put(M3, 2, 3);
  } else {
    put(K3, 0, -1);
    put(M3, 1, -1);
  }
  return out;
}

static int tc_type_of(const tp_op_s* op) {
  if (op->prec == TP_FP16 || op->prec == TP_BF16) return op->prec;
  return op->opts.tc_type;
}

template <typename TS, typename TO, int N, bool EC>
static cudaError_t launch_tc_t(const tp_op_s* op, void* y, const void* x, cudaStream_t s) {
  TcDims D;
  D.nx = op->mesh.nx; D.ny = op->mesh.ny; D.nz = op->mesh.nz;
  D.ncells = op->ncells;
  const float sc = std::is_same<TO, __half>::value ? 2048.f : 256.f;
  D.scale = sc;
  D.inv_scale = 1.f / sc;
  double sk, sm;
  tc_scales(op, sk, sm);
  D.k3_inv = (float)(1.0 / sk);
  D.m3_inv = (float)(1.0 / sm);
  // error-correction mode: 1 both operands (Algorithm 1), 2 the matrix only, 3 the vector only
  D.refine_vec = op->opts.ec == 1 || op->opts.ec == 3;
  D.refine_mat = op->opts.ec == 1 || op->opts.ec == 2;
  // persistent blocks: every block copies the operand matrices once and walks over tiles
  const long long tiles = (op->ncells + kTcCells - 1) / kTcCells;
  const long long cap = (long long)op->tc_blocks_per_sm * op->sm_count;
  const long long blocks = tiles < cap ? tiles : cap;
  apply_tc_kernel<TS, TO, N, EC><<<(unsigned)blocks, 128, tc_smem_bytes<TS, TO, N, EC>(), s>>>(
      static_cast<const TS*>(x), static_cast<TS*>(y), static_cast<const TO*>(op->tc_mats), op->c32, D);
  return cudaGetLastError();
}

template <typename TS, typename TO, int N, bool EC>
static cudaError_t prepare_tc_t(const tp_op_s* op) {
  tp_op_s* o = const_cast<tp_op_s*>(op);
  cudaError_t e = cudaFuncSetAttribute(apply_tc_kernel<TS, TO, N, EC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)tc_smem_bytes<TS, TO, N, EC>());
  if (e != cudaSuccess) return e;
  int per_sm = 0, sms = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, apply_tc_kernel<TS, TO, N, EC>, 128,
                                                    tc_smem_bytes<TS, TO, N, EC>());
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, op->device);
  if (e != cudaSuccess) return e;
  o->tc_blocks_per_sm = per_sm > 0 ? per_sm : 1;
  o->sm_count = sms > 0 ? sms : 1;
  return cudaSuccess;
}

template <typename TS, typename TO, int N>
static cudaError_t dispatch_n(const tp_op_s* op, void* y, const void* x, cudaStream_t s, bool prepare) {
  if (op->opts.ec) return prepare ? prepare_tc_t<TS, TO, N, true>(op) : launch_tc_t<TS, TO, N, true>(op, y, x, s);
  return prepare ? prepare_tc_t<TS, TO, N, false>(op) : launch_tc_t<TS, TO, N, false>(op, y, x, s);
}

template <typename TS, typename TO>
static cudaError_t dispatch_ec(const tp_op_s* op, void* y, const void* x, cudaStream_t s, bool prepare) {
  if (op->n == 3) return dispatch_n<TS, TO, 3>(op, y, x, s, prepare);
  if (op->n == 4) return dispatch_n<TS, TO, 4>(op, y, x, s, prepare);
  return cudaErrorInvalidValue;
}

static cudaError_t dispatch(const tp_op_s* op, void* y, const void* x, cudaStream_t s, bool prepare) {
  const int tt = tc_type_of(op);
  switch (op->prec) {
    case TP_FP16: return dispatch_ec<__half, __half>(op, y, x, s, prepare);
    case TP_BF16: return dispatch_ec<__nv_bfloat16, __nv_bfloat16>(op, y, x, s, prepare);
    case TP_FP32:
      return tt == TP_BF16 ? dispatch_ec<float, __nv_bfloat16>(op, y, x, s, prepare)
                           : dispatch_ec<float, __half>(op, y, x, s, prepare);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_apply_tc(const tp_op_s* op, void* y, const void* x, cudaStream_t s) {
  return dispatch(op, y, x, s, false);
}

// Builds and uploads the operand matrices (owned by the operator) and sets the
// kernel's shared-memory limit on the current device.
cudaError_t prepare_apply_tc(tp_op_s* op) {
  const bool ec = op->opts.ec != 0;
  const int tt = tc_type_of(op);
  const float sc = tt == TP_BF16 ? 256.f : 2048.f;
  size_t bytes = (ec ? 4 : 2) * 4096 * 2;
  cudaError_t e = cudaMalloc(&op->tc_mats, bytes);
  if (e != cudaSuccess) return e;
  if (tt == TP_BF16) {
    std::vector<__nv_bfloat16> m = build_mats<__nv_bfloat16>(op, ec, sc);
    e = cudaMemcpy(op->tc_mats, m.data(), bytes, cudaMemcpyHostToDevice);
  } else {
    std::vector<__half> m = build_mats<__half>(op, ec, sc);
    e = cudaMemcpy(op->tc_mats, m.data(), bytes, cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) return e;
  return dispatch(op, nullptr, nullptr, 0, true);
}

}  // namespace tp
