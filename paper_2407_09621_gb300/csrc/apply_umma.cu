// Blackwell tensor-core SIPG apply for k = 3 with FP16/BF16 vectors: TMA + tcgen05.mma + TMEM.
//
// With n = 4 a cell has 64 DoFs, and the operator of Sec. 2, Eq. (2) restricted to the rows of a
// cell is seven dense 64 x 64 blocks: the interior diagonal block
//   A_cc = L_z(x)M_y(x)M_x + M_z(x)L_y(x)M_x + M_z(x)M_y(x)L_x   (Eq. (9), L the interior block)
// and one block per face neighbour, e.g. A_{c,c+x} = M_z(x)M_y(x)L^{c,c+1}_x. So
//   v_c = sum over the seven blocks b of A_b u_{nb_b(c)},
// a GEMM whose rows are cells: D (cells x 64) = sum_b U_b (cells x 64) A_b^T, each U_b the input
// tile shifted by the neighbour's cell offset (+-1, +-nx, +-nx*ny). The cell-major layout makes
// every U_b a plain 128-byte-per-row tile that TMA loads directly (rows outside the mesh are
// zero-filled). A boundary face is handled with a ghost neighbour: the missing neighbour's row is
// replaced by a line-wise linear map of the cell's own row (two nonzero layers along the normal),
// chosen so that A_{c,nb} ghost = (boundary-face term - interior-face term) of the diagonal:
//   high side: w_0 = -u_{n-1},  w_1 = (d1.u + (2 g h) u_{n-1} + d0[0] u_{n-1}) / d0[1]
//   low side:  w_{n-1} = -u_0,  w_{n-2} = (d0.u - (2 g h) u_0 + d1[n-1] u_0) / d1[n-2]
// (g the penalty, h the cell width, d0/d1 the basis derivatives at the ends). Every cell then
// uses the same seven blocks.
//
// One CTA per SM, persistent over tiles of 128 cells, warp-specialized so that loads, products
// and stores of consecutive tiles overlap:
//   warp 0      TMA producer: streams the seven input tiles of every output tile through a ring
//               of 16 KB shared-memory slots (zero fill outside the mesh);
//   warp 1      MMA issuer: per slot four tcgen05.mma (M = 128, N = 64, K = 16) into one of two
//               TMEM accumulators, then tcgen05.commit releases the slot;
//   warps 2-5   ghost patches: for tiles that hold boundary cells, read the own tile's rows and
//               write the ghost rows into the neighbour slots before the MMA reads them;
//   warps 6-9   epilogue: tcgen05.ld of the finished accumulator (one cell row per thread),
//               scale, round to the storage type and store.
// Algorithm 1 error correction splits each block matrix into a high part and the rounded
// remainder; both products accumulate into the same FP32 accumulator. The input vector is
// already in the operand type, so only the matrix needs the split (two products instead of
// three), and because the matrices are normalized by a power of two (largest entry in
// [32, 64)) the remainder needs no 2^s scaling: remainders below the FP16 normal range lose at
// most 2^-25 in absolute value against entries of order 32.
// Every wait is bounded: on a timeout the kernel records an error code, the other roles stop at
// their next wait, in-flight copies and products are drained (bounded) and TMEM is released.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <type_traits>
#include <vector>

#include "../../include/tp_test.h"
#include "tp_internal.h"

namespace tp {

namespace umma {

constexpr int kRows = 128;            // cells per tile (UMMA M)
constexpr int kTileBytes = kRows * 128;
constexpr int kMatBytes = 64 * 128;   // one 64 x 64 16-bit block matrix
constexpr int kThreads = 320;         // warp 0 TMA, warp 1 MMA, warps 2-5 patches, warps 6-9 epilogue
constexpr int kWaitLimit = 1 << 22;

using Params = UmmaParams;

template <bool EC>
__host__ __device__ constexpr int nmat() { return EC ? 14 : 7; }
// ring slots that fit beside the block matrices in 227 KB of shared memory
template <bool EC>
__host__ __device__ constexpr int nslots() { return EC ? 7 : 10; }
template <bool EC>
__host__ __device__ constexpr size_t smem_bytes() {
  return 1024 + (size_t)nmat<EC>() * kMatBytes + (size_t)nslots<EC>() * kTileBytes + 8 * (3 * nslots<EC>() + 5) + 16;
}

__device__ __forceinline__ uint32_t s2u(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;\n" : "=l"(t));
  return t;
}

// Bounded wait (at most limit_ns, one second by default, and at most kWaitLimit polls) for the
// phase of `bar` with the given parity. Gives up early when another role has raised the abort
// flag; on its own timeout it raises the flag and records `code`.
__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity, volatile int* abort, int* err, int code,
                                         uint64_t limit_ns) {
  if (try_wait(bar, parity)) return true;
  const uint64_t t0 = now_ns();
  for (int it = 0; it < kWaitLimit; ++it) {
    if (try_wait(bar, parity)) return true;
    if ((it & 31) == 31) {
      if (*abort) return false;
      if (now_ns() - t0 > limit_ns) break;
      __nanosleep(64);
    }
  }
  *abort = 1;
  atomicExch(err, code);
  return false;
}

// Bounded wait that ignores the abort flag (draining work already issued).
__device__ __forceinline__ void drain_bar(uint32_t bar, uint32_t parity, int* err, int code) {
  const uint64_t t0 = now_ns();
  for (int it = 0; it < kWaitLimit; ++it) {
    if (try_wait(bar, parity)) return;
    if ((it & 31) == 31) {
      if (now_ns() - t0 > 1000000000ull) break;
      __nanosleep(64);
    }
  }
  atomicExch(err, code);
}

__device__ __forceinline__ void arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}

// UMMA shared-memory descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes apart
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// byte offset of 16-byte chunk c of row r in a 128-byte-swizzled tile (1024-byte aligned base)
__device__ __forceinline__ int sw_off(int r, int c) { return r * 128 + ((c ^ (r & 7)) << 4); }

template <typename TO>
__device__ __forceinline__ float to_f(TO v);
template <>
__device__ __forceinline__ float to_f<__half>(__half v) { return __half2float(v); }
template <>
__device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <typename TO>
__device__ __forceinline__ TO from_f(float v);
template <>
__device__ __forceinline__ __half from_f<__half>(float v) { return __float2half_rn(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

#define TP_LD32(r, base, ta)                                                                               \
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15," \
               "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"              \
               : "=r"(r[base + 0]), "=r"(r[base + 1]), "=r"(r[base + 2]), "=r"(r[base + 3]),             \
                 "=r"(r[base + 4]), "=r"(r[base + 5]), "=r"(r[base + 6]), "=r"(r[base + 7]),             \
                 "=r"(r[base + 8]), "=r"(r[base + 9]), "=r"(r[base + 10]), "=r"(r[base + 11]),           \
                 "=r"(r[base + 12]), "=r"(r[base + 13]), "=r"(r[base + 14]), "=r"(r[base + 15]),         \
                 "=r"(r[base + 16]), "=r"(r[base + 17]), "=r"(r[base + 18]), "=r"(r[base + 19]),         \
                 "=r"(r[base + 20]), "=r"(r[base + 21]), "=r"(r[base + 22]), "=r"(r[base + 23]),         \
                 "=r"(r[base + 24]), "=r"(r[base + 25]), "=r"(r[base + 26]), "=r"(r[base + 27]),         \
                 "=r"(r[base + 28]), "=r"(r[base + 29]), "=r"(r[base + 30]), "=r"(r[base + 31])          \
               : "r"(ta))

// Ghost row for direction d and side (1 = high, 0 = low) from the own row u (64 values, index
// (l*4 + j)*4 + i), written into the swizzled tile row r.
template <typename TO>
__device__ __forceinline__ void write_ghost(unsigned char* tile, int r, const float (&u)[64], int d, int side,
                                            const Params& P) {
  float w[64];
#pragma unroll
  for (int e = 0; e < 64; ++e) w[e] = 0.f;
  const int stride = d == 0 ? 1 : (d == 1 ? 4 : 16);
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      // line start for tangential indices (a, b)
      const int s0 = d == 0 ? (a * 16 + b * 4) : (d == 1 ? (a * 16 + b) : (a * 4 + b));
      if (side) {
        float t = 0.f;
#pragma unroll
        for (int m = 0; m < 4; ++m) t = fmaf(P.gh[d][m], u[s0 + m * stride], t);
        w[s0] = -u[s0 + 3 * stride];
        w[s0 + stride] = t;
      } else {
        float t = 0.f;
#pragma unroll
        for (int m = 0; m < 4; ++m) t = fmaf(P.gl[d][m], u[s0 + m * stride], t);
        w[s0 + 3 * stride] = -u[s0];
        w[s0 + 2 * stride] = t;
      }
    }
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    uint4 v;
    TO* h = reinterpret_cast<TO*>(&v);
#pragma unroll
    for (int q = 0; q < 8; ++q) h[q] = from_f<TO>(w[c * 8 + q]);
    *reinterpret_cast<uint4*>(tile + sw_off(r, c)) = v;
  }
}

// Which of the seven input tiles of the tile starting at cell c0 need ghost patches: bit b
// (1..6 = x-, x+, y-, y+, z-, z+) if a cell of the tile lies on that side of the mesh, bit 0 if
// any does (the patch warps then also read the own tile).
__device__ __forceinline__ uint32_t tile_bmask(long long c0, const Params& P) {
  const long long c1 = (c0 + kRows < P.ncells ? c0 + kRows : P.ncells) - 1;
  const long long nx = P.nx, ny = P.ny, nxy = nx * ny;
  uint32_t m = 0;
  if ((c1 / nx) * nx >= c0) m |= 1u << 1;                 // cx == 0
  if (((c1 + 1) / nx) * nx >= c0 + 1) m |= 1u << 2;       // cx == nx-1
  const long long q0 = c0 / nx, q1 = c1 / nx;             // rows of cells along y (all slabs)
  if ((q1 / ny) * ny >= q0) m |= 1u << 3;                 // cy == 0
  if (((q1 + 1) / ny) * ny >= q0 + 1) m |= 1u << 4;       // cy == ny-1
  if (c0 < nxy) m |= 1u << 5;                             // cz == 0
  if (c1 >= (long long)(P.nz - 1) * nxy) m |= 1u << 6;    // cz == nz-1
  return m ? (m | 1u) : 0u;
}

template <typename TO, bool EC>
__global__ void __launch_bounds__(kThreads, 1)
apply_umma_kernel(const __grid_constant__ CUtensorMap tmx, TO* __restrict__ y, const TO* __restrict__ mats,
                  const __grid_constant__ Params P, int* __restrict__ err) {
  constexpr int NMAT = nmat<EC>(), S = nslots<EC>();
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sB = base;                      // NMAT block matrices, [out n][in k], swizzled
  unsigned char* sA = base + NMAT * kMatBytes;   // S input-tile slots
  uint64_t* bars = reinterpret_cast<uint64_t*>(sA + S * kTileBytes);
  // full[S] (TMA landed), ready[S] (ghost rows written), empty[S] (MMAs done with the slot),
  // accf[2] (accumulator complete), acce[2] (accumulator read), drain
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 3 * S + 5);
  volatile int* abort = reinterpret_cast<volatile int*>(tslot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t bar0 = s2u(bars);
  auto full = [&](int s) { return bar0 + 8u * s; };
  auto ready = [&](int s) { return bar0 + 8u * (S + s); };
  auto empty = [&](int s) { return bar0 + 8u * (2 * S + s); };
  auto accf = [&](int a) { return bar0 + 8u * (3 * S + a); };
  auto acce = [&](int a) { return bar0 + 8u * (3 * S + 2 + a); };
  const uint32_t drain = bar0 + 8u * (3 * S + 4);

  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(full(s)));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;\n" ::"r"(ready(s)));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(empty(s)));
    }
    for (int a = 0; a < 2; ++a) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(accf(a)));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;\n" ::"r"(acce(a)));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(drain));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    *abort = 0;
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(s2u(tslot)), "r"(128));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  // block matrices -> shared, swizzled
  for (int e = tid; e < NMAT * 64 * 8; e += kThreads) {
    const int m = e >> 9, n = (e >> 3) & 63, c = e & 7;
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(mats + ((size_t)m * 64 + n) * 64) + c);
    *reinterpret_cast<uint4*>(sB + m * kMatBytes + sw_off(n, c)) = v;
  }
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tslot;
  const long long ntiles = (P.ncells + kRows - 1) / kRows;
  const long long sy = P.nx, sz = (long long)P.nx * P.ny;

  if (warp == 0) {
    // ---------------------------------------------------------------- TMA producer
    if (lane == 0) {
      const long long offs[7] = {0, -1, 1, -sy, sy, -sz, sz};
      int slot = 0;
      uint32_t ph = 0, issued = 0, iph = 0;  // per-slot: issued at least once, parity of the last issue
      bool ok = true;
      for (long long t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        for (int b = 0; b < 7; ++b) {
          if (!(ok = wait_bar(empty(slot), ph ^ 1u, abort, err, 1, P.wait_ns))) break;
          if (P.test_withhold && blockIdx.x == 0 && t == 0 && b == 0) {
            // failure-injection tests: this slot never fills, so the waits on it run out
            if (++slot == S) { slot = 0; ph ^= 1u; }
            continue;
          }
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(full(slot)), "r"(kTileBytes)
                       : "memory");
          const int row = (int)(t * kRows + offs[b]);  // may be negative or past the end: zero fill
          asm volatile(
              "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n"
              ::"r"(s2u(sA + slot * kTileBytes)), "l"((uint64_t)&tmx), "r"(0), "r"(row), "r"(full(slot))
              : "memory");
          issued |= 1u << slot;
          iph = (iph & ~(1u << slot)) | (ph << slot);
          if (++slot == S) { slot = 0; ph ^= 1u; }
        }
      }
      // let every copy in flight land before the CTA can leave
      for (int s = 0; s < S; ++s)
        if (issued >> s & 1u) drain_bar(full(s), (iph >> s) & 1u, err, 5);
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      const uint32_t fmt = std::is_same<TO, __nv_bfloat16>::value ? 1u : 0u;
      // D F32, A/B F16 (0) or BF16 (1), both K-major, N = 64, M = 128
      const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);
      int slot = 0, it = 0;
      uint32_t ph = 0, rdy = 0;  // rdy: per-slot parity of the ready barriers (used only when patched)
      bool ok = true;
      for (long long t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++it) {
        const int a = it & 1;
        if (!(ok = wait_bar(acce(a), ((it >> 1) & 1) ^ 1u, abort, err, 2, P.wait_ns))) break;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const uint32_t bm = tile_bmask(t * kRows, P);
        const uint32_t dt = tmem + 64u * a;
        for (int b = 0; b < 7; ++b) {
          if (bm >> b & 1u) {
            ok = wait_bar(ready(slot), (rdy >> slot) & 1u, abort, err, 3, P.wait_ns);
            rdy ^= 1u << slot;
          } else {
            ok = wait_bar(full(slot), ph, abort, err, 3, P.wait_ns);
          }
          if (!ok) break;
          asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {
            const uint64_t ad = sw128_desc(s2u(sA + slot * kTileBytes) + ks * 32);
            const uint64_t bd = sw128_desc(s2u(sB + b * kMatBytes) + ks * 32);
            const uint32_t acc = (b | ks) != 0;
            asm volatile("{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                         ::"r"(dt), "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
            if (EC) {
              const uint64_t bl = sw128_desc(s2u(sB + (7 + b) * kMatBytes) + ks * 32);
              asm volatile("{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                           ::"r"(dt), "l"(ad), "l"(bl), "r"(idesc), "r"(1u));
            }
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(empty(slot))
                       : "memory");
          if (++slot == S) { slot = 0; ph ^= 1u; }
        }
        if (!ok) break;
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(accf(a))
                     : "memory");
      }
      // every product issued so far has finished before TMEM is released
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(drain)
                   : "memory");
      drain_bar(drain, 0, err, 6);
    }
  } else if (warp < 6) {
    // ---------------------------------------------------------------- ghost patches
    const int row = tid - 64;
    int slot = 0;
    uint32_t ph = 0;
    bool ok = true;
    for (long long t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      const uint32_t bm = tile_bmask(t * kRows, P);
      if (!bm) {
        slot += 7;
        while (slot >= S) { slot -= S; ph ^= 1u; }
        continue;
      }
      const long long cell = t * kRows + row;
      bool bnd[6] = {false, false, false, false, false, false};
      if (cell < P.ncells) {
        const int cx = (int)(cell % P.nx), cy = (int)((cell / P.nx) % P.ny), cz = (int)(cell / sz);
        bnd[0] = cx == 0; bnd[1] = cx == P.nx - 1;
        bnd[2] = cy == 0; bnd[3] = cy == P.ny - 1;
        bnd[4] = cz == 0; bnd[5] = cz == P.nz - 1;
      }
      const bool any = bnd[0] | bnd[1] | bnd[2] | bnd[3] | bnd[4] | bnd[5];
      float u[64];
      if (!(ok = wait_bar(full(slot), ph, abort, err, 4, P.wait_ns))) break;
      if (any) {
        const unsigned char* own = sA + slot * kTileBytes;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const uint4 v = *reinterpret_cast<const uint4*>(own + sw_off(row, c));
          const TO* h = reinterpret_cast<const TO*>(&v);
#pragma unroll
          for (int q = 0; q < 8; ++q) u[c * 8 + q] = to_f<TO>(h[q]);
        }
      }
      arrive(ready(slot));
      if (++slot == S) { slot = 0; ph ^= 1u; }
#pragma unroll
      for (int b = 1; b < 7; ++b) {
        if (bm >> b & 1u) {
          if (!(ok = wait_bar(full(slot), ph, abort, err, 4, P.wait_ns))) break;
          if (bnd[b - 1]) write_ghost<TO>(sA + slot * kTileBytes, row, u, (b - 1) >> 1, (b - 1) & 1, P);
          asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
          arrive(ready(slot));
        }
        if (++slot == S) { slot = 0; ph ^= 1u; }
      }
    }
  } else {
    // ---------------------------------------------------------------- epilogue
    const int q4 = warp & 3;  // this warp may read TMEM lanes 32*q4 .. 32*q4+31
    const int row = 32 * q4 + lane;
    int it = 0;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
      const int a = it & 1;
      // warp-uniform decision: the TMEM loads below are .sync.aligned
      if (!__all_sync(0xffffffffu, wait_bar(accf(a), (it >> 1) & 1, abort, err, 7, P.wait_ns))) break;
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      uint32_t r[64];
      const uint32_t ta = tmem + ((uint32_t)(32 * q4) << 16) + 64u * a;
      TP_LD32(r, 0, ta);
      TP_LD32(r, 32, ta + 32);
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      arrive(acce(a));
      const long long cell = t * kRows + row;
      if (cell < P.ncells) {
        uint4* dst = reinterpret_cast<uint4*>(y + cell * 64);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          uint4 o;
          TO* h = reinterpret_cast<TO*>(&o);
#pragma unroll
          for (int q = 0; q < 8; ++q) h[q] = from_f<TO>(__uint_as_float(r[c * 8 + q]) * P.out_scale);
          dst[c] = o;
        }
      }
    }
  }
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(128));
  }
}

}  // namespace umma

// ------------------------------------------------------------------ host side

static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

template <typename TO>
static TO host_to(float v);
template <>
__half host_to<__half>(float v) { return __float2half_rn(v); }
template <>
__nv_bfloat16 host_to<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <typename TO>
static float host_from(TO v);
template <>
float host_from<__half>(__half v) { return __half2float(v); }
template <>
float host_from<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

// The seven 64 x 64 blocks [b][out (l,j,i)][in (l',j',i')] in the original Kronecker form of Eq. (9):
// b = 0 the interior diagonal block, 1..6 the x-, x+, y-, y+, z-, z+ neighbour blocks.
static std::vector<double> umma_blocks(const tp_op_s* op) {
  const int n = 4;
  const Ref1D& R = op->ref;
  std::vector<double> B(7 * 4096, 0.0);
  auto Mv = [&](int d, int a, int b) { return op->dir[d].M[a * n + b]; };
  auto Lv = [&](int d, int a, int b) { return op->dir[d].L[a * n + b]; };
  // L^{c,c+1}[i][j] = -g v1_i v0_j - v1_i d0_j/(2h) + d1_i v0_j/(2h); L^{c,c-1}[i][j] = L^{c,c+1}[j][i]
  auto Lp = [&](int d, int i, int j) {
    const double g = op->dir[d].gamma, hh = 0.5 / op->dir[d].h;
    const double v1i = i == n - 1, v0j = j == 0;
    return -g * v1i * v0j - v1i * R.d0[j] * hh + R.d1[i] * v0j * hh;
  };
  for (int l = 0; l < n; ++l)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i)
        for (int l2 = 0; l2 < n; ++l2)
          for (int j2 = 0; j2 < n; ++j2)
            for (int i2 = 0; i2 < n; ++i2) {
              const int r = (l * n + j) * n + i, c = (l2 * n + j2) * n + i2;
              const double mz = Mv(2, l, l2), my = Mv(1, j, j2), mx = Mv(0, i, i2);
              B[0 * 4096 + r * 64 + c] = Lv(2, l, l2) * my * mx + mz * Lv(1, j, j2) * mx + mz * my * Lv(0, i, i2);
              B[1 * 4096 + r * 64 + c] = mz * my * Lp(0, i2, i);
              B[2 * 4096 + r * 64 + c] = mz * my * Lp(0, i, i2);
              B[3 * 4096 + r * 64 + c] = mz * Lp(1, j2, j) * mx;
              B[4 * 4096 + r * 64 + c] = mz * Lp(1, j, j2) * mx;
              B[5 * 4096 + r * 64 + c] = Lp(2, l2, l) * my * mx;
              B[6 * 4096 + r * 64 + c] = Lp(2, l, l2) * my * mx;
            }
  return B;
}

template <typename TO, bool EC>
static cudaError_t umma_prepare_t(tp_op_s* op) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return cudaErrorNotSupported;
  std::vector<double> B = umma_blocks(op);
  double amax = 0.0;
  for (double v : B) amax = std::fmax(amax, std::fabs(v));
  int e2;
  std::frexp(amax / 32.0, &e2);
  const double sc = std::ldexp(1.0, -e2);  // largest stored entry in [32, 64)
  // Algorithm 1 split of the (normalized) block matrices: high part and rounded remainder
  std::vector<TO> hm((EC ? 14 : 7) * 4096);
  for (int e = 0; e < 7 * 4096; ++e) {
    const double v = B[e] * sc;
    const TO h = host_to<TO>((float)v);
    hm[e] = h;
    if (EC) hm[7 * 4096 + e] = host_to<TO>((float)(v - (double)host_from<TO>(h)));
  }
  cudaError_t err = cudaMalloc(&op->umma_mats, hm.size() * sizeof(TO));
  if (err == cudaSuccess) err = cudaMemcpy(op->umma_mats, hm.data(), hm.size() * sizeof(TO), cudaMemcpyHostToDevice);
  if (err == cudaSuccess) err = cudaMalloc(&op->umma_err, sizeof(int));
  if (err == cudaSuccess) err = cudaMemset(op->umma_err, 0, sizeof(int));
  if (err != cudaSuccess) return err;
  umma::Params& P = op->umma_params;
  memset(&P, 0, sizeof(P));
  P.nx = op->mesh.nx; P.ny = op->mesh.ny; P.nz = op->mesh.nz;
  P.ncells = op->ncells;
  P.out_scale = (float)(1.0 / sc);
  P.lo_scale = 1.0f;
  P.wait_ns = 1000000000ull;
  P.test_withhold = 0;
  const Ref1D& R = op->ref;
  for (int d = 0; d < 3; ++d) {
    const double g2h = 2.0 * op->dir[d].gamma * op->dir[d].h;
    for (int m = 0; m < 4; ++m) {
      const double e3 = m == 3, e0 = m == 0;
      P.gh[d][m] = (float)((R.d1[m] + g2h * e3 + R.d0[0] * e3) / R.d0[1]);
      P.gl[d][m] = (float)((R.d0[m] - g2h * e0 + R.d1[3] * e0) / R.d1[2]);
    }
  }
  int sms = 0;
  err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, op->device);
  if (err != cudaSuccess) return err;
  op->sm_count = sms > 0 ? sms : 1;
  return cudaFuncSetAttribute(umma::apply_umma_kernel<TO, EC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)umma::smem_bytes<EC>());
}

template <typename TO, bool EC>
static cudaError_t umma_launch_t(const tp_op_s* op, void* y, const void* x, cudaStream_t s) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return cudaErrorNotSupported;
  CUtensorMap tm;
  cuuint64_t dims[2] = {64, (cuuint64_t)op->ncells};
  cuuint64_t strides[1] = {128};
  cuuint32_t box[2] = {64, (cuuint32_t)umma::kRows}, estr[2] = {1, 1};
  const CUtensorMapDataType dt =
      std::is_same<TO, __half>::value ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  if (enc(&tm, dt, 2, const_cast<void*>(x), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
          CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
      CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  const long long tiles = (op->ncells + umma::kRows - 1) / umma::kRows;
  const int grid = (int)(tiles < op->sm_count ? tiles : op->sm_count);
  umma::apply_umma_kernel<TO, EC><<<grid, umma::kThreads, umma::smem_bytes<EC>(), s>>>(
      tm, static_cast<TO*>(y), static_cast<const TO*>(op->umma_mats), op->umma_params, op->umma_err);
  return cudaGetLastError();
}

// TMA row coordinates (cell index + neighbour offset) must fit in int32.
bool umma_supported(const tp_op_s* op) {
  const long long reach = op->ncells + (long long)op->mesh.nx * op->mesh.ny + umma::kRows;
  return op->n == 4 && (op->prec == TP_FP16 || op->prec == TP_BF16) && reach < (1LL << 31);
}

cudaError_t prepare_apply_umma(tp_op_s* op) {
  const bool ec = op->opts.ec != 0 || op->prec == TP_BF16;
  if (op->prec == TP_FP16) return ec ? umma_prepare_t<__half, true>(op) : umma_prepare_t<__half, false>(op);
  return umma_prepare_t<__nv_bfloat16, true>(op);
}

cudaError_t launch_apply_umma(const tp_op_s* op, void* y, const void* x, cudaStream_t s) {
  const bool ec = op->opts.ec != 0 || op->prec == TP_BF16;
  if (op->prec == TP_FP16) return ec ? umma_launch_t<__half, true>(op, y, x, s) : umma_launch_t<__half, false>(op, y, x, s);
  return umma_launch_t<__nv_bfloat16, true>(op, y, x, s);
}

}  // namespace tp

extern "C" tp_status tp_test_set_wait_fault(tp_op op, int withhold_first_copy, double wait_limit_s) {
  using namespace tp;
  if (!op) { set_error("tp_test_set_wait_fault: NULL op"); return TP_ERR_INVALID_ARG; }
  if (!(wait_limit_s >= 0.0) || wait_limit_s > 60.0) {
    set_error("tp_test_set_wait_fault: wait limit must be in [0, 60] seconds");
    return TP_ERR_INVALID_ARG;
  }
  if (!op->use_umma || op->opts.kernel != TP_KERNEL_TENSOR) {
    set_error("tp_test_set_wait_fault: the operator does not run the tcgen05 apply");
    return TP_ERR_UNSUPPORTED;
  }
  op->umma_params.test_withhold = withhold_first_copy ? 1 : 0;
  op->umma_params.wait_ns = wait_limit_s > 0.0 ? (unsigned long long)(wait_limit_s * 1e9) : 1000000000ull;
  return TP_OK;
}
