// Blackwell tensor-core SIPG apply for k = 3 with FP16/BF16 vectors: TMA + tcgen05.mma + TMEM.
//
// With n = 4 a cell has 64 DoFs, and the operator of Sec. 2, Eq. (2) restricted to the rows of a
// cell is seven dense 64 x 64 blocks: the interior diagonal block
//   A_cc = L_z(x)M_y(x)M_x + M_z(x)L_y(x)M_x + M_z(x)M_y(x)L_x   (Eq. (9), L the interior block)
// and one block per face neighbour, e.g. A_{c,c+x} = M_z(x)M_y(x)L^{c,c+1}_x. So
//   v_c = sum over the seven blocks b of A_b u_{nb_b(c)},
// a GEMM whose rows are cells: D (cells x 64) = sum_b U_b (cells x 64) A_b^T, each U_b the input
// rows of the tile's cells shifted by one cell along one axis. A tile is a plane patch of 8 x 16 x 1
// cells (128 rows, the UMMA M); TMA loads it through 4D tensor maps over (64 values, nx, ny, nz),
// one 128-byte row per cell, cells outside the mesh arriving as zeros. A missing neighbour
// therefore contributes nothing, and every cell is first computed with the interior diagonal
// block. A boundary cell differs from that only by its boundary faces: the 1D block of a cell on
// the low (high) end of direction d is L + dL_0 (L + dL_1) with the rank-2
//   dL_0 = (v0 d0^T + d0 v0^T)/(2h),  dL_1 = -(v1 d1^T + d1 v1^T)/(2h),
// so a second, small kernel adds (M (x) M (x) dL) u_c for each boundary face of each boundary
// cell on the FMA pipes (rank 2 along the normal, the mass tensor along the two tangents), one
// thread per boundary cell.
//
// Loads per tile, instead of seven: a window box of 8 x 18 x 1 cells holds the tile's own rows and
// those of its y-neighbours at row offsets 8, 0 and 16 (multiples of the 8-row swizzle atom, so each
// is a plain operand), and two boxes shifted by one cell along x hold the x-neighbours. The z-terms
// need no load: a CTA walks a z-segment of one tile column, and the own rows of tile z are also the
// z+ neighbour rows of tile z - 1 and the z- neighbour rows of tile z + 1, so their products go into
// those tiles' accumulators. A segment [z0, z1) loads the own rows of tiles z0 - 1 and z1 as halos.
// That is 52 KB per tile from L2 instead of 112 KB, and the ring of 18 KB slots looks about three
// tiles ahead.
//
// Issue rate, measured on this part: one thread issues a tcgen05.mma (M = 128, K = 16) only every
// ~112 cycles, whatever N (64 .. 192) and wherever A sits (shared memory or TMEM), while the
// tensor pipe finishes an N = 64 product in ~36 cycles when four warps issue. With seven 64 x 64
// blocks (28 products) per tile a single issuer sets the pace, so two warps issue into separate
// TMEM accumulators that the epilogue adds, and the own rows take one product for three blocks:
// the z+, own and z- blocks sit side by side in shared memory and the accumulators of tiles
// z - 1, z and z + 1 in adjacent TMEM columns (N = 192; split in two where the rotation of four
// accumulators wraps).
//
// One CTA per SM, persistent over work units (a tile column's z-segment), warp-specialized so
// that loads, products and stores of consecutive tiles overlap:
//   warp 0      TMA producer: streams the boxes of every tile through the slot ring (and asks L2
//               to prefetch the window boxes a few tiles ahead);
//   warp 1      MMA issuer A: the own rows (z+, own and z- blocks) and, without error correction,
//               the y- rows, into accumulator set A (TMEM columns 0-255), four tcgen05.mma per
//               operand (K = 16 each);
//   warp 10     MMA issuer B: the y+ rows and the two x-neighbour boxes (with error correction
//               also the y- rows), into set B (256-511);
//               each issuer's tcgen05.commit releases the slots it read, and a tile's accumulators
//               go to the epilogue when both issuers have committed them;
//   warps 2-9   epilogue, two groups of four warps taking alternate tiles: tcgen05.ld of both
//               accumulators of a finished tile (one cell row per thread), add them, zero set A's
//               (its products all accumulate; set B's first product overwrites), scale, round to
//               the storage type and store the rows of cells inside the mesh.
// Algorithm 1 error correction splits each block matrix into a high part and the rounded
// remainder. For the own rows both products accumulate into the same FP32 accumulator; for each
// shifted operand the high part and the remainder sit side by side in shared memory and one
// N = 128 product (as costly to issue as one N = 64 product, and reading the operand once) writes
// two adjacent accumulators that the epilogue adds. The input vector is
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

constexpr int kRows = 128;            // cells per tile (UMMA M): 8 x 16 x 1
constexpr int kBX = 8, kBY = 16;
constexpr int kTileBytes = kRows * 128;            // one tile box
constexpr int kWinBytes = (kRows + 2 * kBX) * 128; // the window box: the tile with a y-halo row each side
constexpr int kSlotBytes = kWinBytes;
constexpr int kMatBytes = 64 * 128;   // one 64 x 64 16-bit block matrix
constexpr int kThreads = 352;         // warp 0 TMA, warps 1 and 10 MMA, warps 2-9 epilogue (two groups of four)
constexpr int kPrefetch = 4;          // tiles ahead whose window box the producer prefetches into L2
constexpr int kAcc = 4;               // TMEM accumulators of 64 columns per issuer (all 512 columns)
constexpr int kWaitLimit = 1 << 22;

using Params = UmmaParams;

template <bool EC>
__host__ __device__ constexpr int nmat() { return EC ? 14 : 7; }
// Output staging: without error correction each epilogue warp writes its 32 rows (4 KB, 8 x 4
// cells) into shared memory and stores them with one TMA box; with it, the products bound the
// kernel and the ring needs the room, so rows are stored from registers.
template <bool EC>
__host__ __device__ constexpr int stage_bytes() { return EC ? 0 : 8 * 4096; }
// ring slots that fit beside the block matrices in 227 KB of shared memory (at most 32: per-slot bits)
template <bool EC>
__host__ __device__ constexpr int nslots() {
  return (232448 - 2048 - nmat<EC>() * kMatBytes - stage_bytes<EC>()) / kSlotBytes < 32
             ? (232448 - 2048 - nmat<EC>() * kMatBytes - stage_bytes<EC>()) / kSlotBytes
             : 32;
}
template <bool EC>
__host__ __device__ constexpr size_t smem_bytes() {
  return 1024 + (size_t)nmat<EC>() * kMatBytes + (size_t)nslots<EC>() * kSlotBytes + stage_bytes<EC>() +
         8 * (2 * nslots<EC>() + 2 * kAcc + 1) + 16;
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

// 32 columns of zeros into this warp's 32 TMEM lanes
#define TP_ST32Z(ta)                                                                                       \
  asm volatile("tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1," \
               "%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};\n" ::"r"(ta), "r"(0u)                      \
               : "memory")

// Shared-memory position of block matrix b (own, x-, x+, y-, y+, z-, z+; lo = 1: its Algorithm 1
// remainder). The z+, own and z- blocks sit side by side (in that order), so one product with
// N = 192 applies all three to the own rows; their remainders follow them. With error correction
// each of the four shifted blocks is followed by its remainder, so one product with N = 128 applies
// both, into two adjacent accumulators that the epilogue adds.
template <bool EC>
__device__ __forceinline__ int mat_pos(int b, int lo) {
  if (b == 6 || b == 0 || b == 5) return (b == 6 ? 0 : (b == 0 ? 1 : 2)) + (EC && lo ? 3 : 0);
  return EC ? 6 + 2 * (b - 1) + lo : b + 2;
}

// Boundary-face correction of one cell in FP32: o += s hh (M_t1 (x) M_t2 (x) (e_end beta^T + beta e_end^T)) u
// for the face of direction D on side SIDE (0: low, beta = d0, end 0, s = +1; 1: high, beta = d1,
// end 3, s = -1). Node (t1, t2, m) of the line along D at tangential indices (t1, t2): D = 0
// (t1, t2, m) = (z, y, x), D = 1 (z, x, y), D = 2 (y, x, z); the tangential masses are M_z, M_y
// (D = 0), M_z, M_x (D = 1), M_y, M_x (D = 2). All indices are compile-time (registers).
template <int D, int SIDE>
__device__ __forceinline__ void add_face(float (&o)[64], const float (&u)[64], const Params& P) {
  constexpr int END = SIDE ? 3 : 0;
  auto node = [](int t1, int t2, int m) {
    return D == 0 ? (t1 * 4 + t2) * 4 + m : (D == 1 ? (t1 * 4 + m) * 4 + t2 : (m * 4 + t1) * 4 + t2);
  };
  const float* beta = SIDE ? P.fd1 : P.fd0;
  const float* M1 = P.fM[D == 2 ? 1 : 2];
  const float* M2 = P.fM[D == 0 ? 1 : 0];
  float sa[16], sb[16], ta[16], tb[16];
#pragma unroll
  for (int a = 0; a < 16; ++a) {
    float acc = 0.f;
#pragma unroll
    for (int m = 0; m < 4; ++m) acc = fmaf(beta[m], u[node(a >> 2, a & 3, m)], acc);
    sa[a] = acc;
    sb[a] = u[node(a >> 2, a & 3, END)];
  }
  // T = S M2^T, then W = M1 T (the tangential mass tensor applied to S)
#pragma unroll
  for (int t1 = 0; t1 < 4; ++t1)
#pragma unroll
    for (int t2 = 0; t2 < 4; ++t2) {
      float xa = 0.f, xb = 0.f;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        xa = fmaf(sa[t1 * 4 + b], M2[t2 * 4 + b], xa);
        xb = fmaf(sb[t1 * 4 + b], M2[t2 * 4 + b], xb);
      }
      ta[t1 * 4 + t2] = xa;
      tb[t1 * 4 + t2] = xb;
    }
  const float sg = SIDE ? -P.fhh[D] : P.fhh[D];
#pragma unroll
  for (int t1 = 0; t1 < 4; ++t1)
#pragma unroll
    for (int t2 = 0; t2 < 4; ++t2) {
      float wa = 0.f, wb = 0.f;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        wa = fmaf(M1[t1 * 4 + b], ta[b * 4 + t2], wa);
        wb = fmaf(M1[t1 * 4 + b], tb[b * 4 + t2], wb);
      }
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const float add = (m == END ? wa : 0.f) + beta[m] * wb;
        o[node(t1, t2, m)] = fmaf(sg, add, o[node(t1, t2, m)]);
      }
    }
}

// Work unit u: tile column (tx, ty) and its z-segment [z0, z1).
struct Unit {
  int x0, y0, z0, z1;
};
__device__ __forceinline__ Unit unit_of(long long u, const Params& P) {
  const long long cols = (long long)P.tiles[0] * P.tiles[1];
  const long long col = u % cols, sg = u / cols;
  Unit w;
  w.x0 = (int)(col % P.tiles[0]) * kBX;
  w.y0 = (int)(col / P.tiles[0]) * kBY;
  w.z0 = (int)sg * P.seg;
  w.z1 = min(w.z0 + P.seg, P.nz);
  return w;
}

template <typename TO, bool EC>
__global__ void __launch_bounds__(kThreads, 1)
apply_umma_kernel(const __grid_constant__ CUtensorMap tmw, const __grid_constant__ CUtensorMap tmt,
                  const __grid_constant__ CUtensorMap tmy, const TO* __restrict__ x, TO* __restrict__ y, const TO* __restrict__ mats,
                  const __grid_constant__ Params P, int* __restrict__ err) {
  constexpr int NMAT = nmat<EC>(), S = nslots<EC>();
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sB = base;                      // NMAT block matrices, [out n][in k], swizzled
  unsigned char* sA = base + NMAT * kMatBytes;   // S slots of kSlotBytes
  unsigned char* sY = sA + S * kSlotBytes;       // output staging, 4 KB per epilogue warp
  uint64_t* bars = reinterpret_cast<uint64_t*>(sY + stage_bytes<EC>());
  // full[S] (TMA landed), empty[S] (MMAs done with the slot), accf[kAcc] (accumulator complete),
  // acce[kAcc] (accumulator read and zeroed), drain
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 2 * S + 2 * kAcc + 1);
  volatile int* abort = reinterpret_cast<volatile int*>(tslot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t bar0 = s2u(bars);
  auto full = [&](int s) { return bar0 + 8u * s; };
  auto empty = [&](int s) { return bar0 + 8u * (S + s); };
  auto accf = [&](int a) { return bar0 + 8u * (2 * S + a); };
  auto acce = [&](int a) { return bar0 + 8u * (2 * S + kAcc + a); };
  const uint32_t drain = bar0 + 8u * (2 * S + 2 * kAcc);

  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(full(s)));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 2;\n" ::"r"(empty(s)));  // both issuers
    }
    for (int a = 0; a < kAcc; ++a) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 2;\n" ::"r"(accf(a)));  // both issuers
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;\n" ::"r"(acce(a)));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 2;\n" ::"r"(drain));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    *abort = 0;
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(s2u(tslot)), "r"(128 * kAcc));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  // block matrices -> shared, swizzled, at their positions (the error-correction remainders as a
  // second set of seven)
  for (int e = tid; e < NMAT * 64 * 8; e += kThreads) {
    const int m = e >> 9, n = (e >> 3) & 63, c = e & 7;
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(mats + ((size_t)m * 64 + n) * 64) + c);
    *reinterpret_cast<uint4*>(sB + mat_pos<EC>(m % 7, m / 7) * kMatBytes + sw_off(n, c)) = v;
  }
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tslot;
  // every product of issuer A accumulates, so its accumulators start at zero (and the epilogue
  // zeroes each one again after reading it)
  if (warp >= 2 && warp < 10) {
    const uint32_t t0 = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(((warp - 2) >> 2) * 32 * kAcc);
#pragma unroll
    for (int c = 0; c < kAcc; ++c) TP_ST32Z(t0 + 32u * c);
    asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");

  if (warp == 0) {
    // ---------------------------------------------------------------- TMA producer
    if (lane == 0) {
      int slot = 0;
      uint32_t ph = 0, issued = 0, iph = 0;  // per-slot: issued at least once, parity of the last issue
      bool ok = true, first = true;
      // one box into the next slot; boxes may start one cell outside the mesh (zeros arrive)
      auto load = [&](const CUtensorMap* tm, int bytes, int cx, int cy, int cz) -> bool {
        if (!wait_bar(empty(slot), ph ^ 1u, abort, err, 1, P.wait_ns)) return false;
        if (P.test_withhold && blockIdx.x == 0 && first) {
          // failure-injection tests: this slot never fills, so the waits on it run out
          first = false;
          if (++slot == S) { slot = 0; ph ^= 1u; }
          return true;
        }
        first = false;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(full(slot)), "r"(bytes)
                     : "memory");
        asm volatile(
            "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];\n"
            ::"r"(s2u(sA + slot * kSlotBytes)), "l"((uint64_t)tm), "r"(0), "r"(cx), "r"(cy), "r"(cz), "r"(full(slot))
            : "memory");
        issued |= 1u << slot;
        iph = (iph & ~(1u << slot)) | (ph << slot);
        if (++slot == S) { slot = 0; ph ^= 1u; }
        return true;
      };
      for (long long u = blockIdx.x; u < P.units && ok; u += gridDim.x) {
        const Unit w = unit_of(u, P);
        // first touches of the column come from DRAM: ask L2 for the first window boxes early
        for (int z = w.z0; z < w.z1 && z < w.z0 + kPrefetch; ++z)
          asm volatile("cp.async.bulk.prefetch.tensor.4d.L2.global [%0, {%1, %2, %3, %4}];\n"
                       ::"l"((uint64_t)&tmw), "r"(0), "r"(w.x0), "r"(w.y0 - 1), "r"(z) : "memory");
        if (w.z0 > 0) ok = load(&tmt, kTileBytes, w.x0, w.y0, w.z0 - 1);
        for (int z = w.z0; z < w.z1 && ok; ++z) {
          if (z + kPrefetch < w.z1)
            asm volatile("cp.async.bulk.prefetch.tensor.4d.L2.global [%0, {%1, %2, %3, %4}];\n"
                         ::"l"((uint64_t)&tmw), "r"(0), "r"(w.x0), "r"(w.y0 - 1), "r"(z + kPrefetch) : "memory");
          ok = load(&tmw, kWinBytes, w.x0, w.y0 - 1, z) && load(&tmt, kTileBytes, w.x0 - 1, w.y0, z) &&
               load(&tmt, kTileBytes, w.x0 + 1, w.y0, z);
        }
        if (ok && w.z1 < P.nz) ok = load(&tmt, kTileBytes, w.x0, w.y0, w.z1);
      }
      // let every copy in flight land before the CTA can leave
      for (int s = 0; s < S; ++s)
        if (issued >> s & 1u) drain_bar(full(s), (iph >> s) & 1u, err, 5);
    }
  } else if (warp == 1 || warp == 10) {
    // ---------------------------------------------------------------- MMA issuers
    // One thread issues a tcgen05.mma only every ~110 cycles on this part, so two warps issue:
    // A (warp 1) the own rows (z+, own and z- blocks in one product) into TMEM columns
    // [0, 64 kAcc), and without error correction also the y- rows; B (warp 10) the other shifted
    // operands into columns [64 kAcc, 128 kAcc): the y+ rows and the two x-neighbour boxes, and with
    // error correction also the y- rows, each as one N = 128 product (high part and remainder into
    // two adjacent accumulators, two tiles' worth rotating) instead of two N = 64 products. The
    // epilogue adds a tile's accumulators. Both issuers walk the whole slot ring in order: each
    // waits for every slot to fill and releases every slot (a slot is refilled after both released
    // it), passing over the slots it does not read.
    if (lane == 0) {
      const bool RA = warp == 1;
      const uint32_t fmt = std::is_same<TO, __nv_bfloat16>::value ? 1u : 0u;
      // D F32, A/B F16 (0) or BF16 (1), both K-major, M = 128; N = 64 per block in the product
      const uint32_t idesc0 = (1u << 4) | (fmt << 7) | (fmt << 10) | ((128u >> 4) << 24);
      const uint32_t tset = tmem + (RA ? 0u : 64u * kAcc);
      int slot = 0;
      uint32_t ph = 0;
      bool ok = true;
      long long g = 0;  // running index of this CTA's tiles; accumulator g % kAcc
      // A: accumulators of tiles gt .. gt + nb - 1 (+)= rows at `a_addr` times the nb blocks from
      // shared position `pos` on (transposed), and with error correction their remainders (from
      // pos + 3); a run of accumulators that wraps past the last one of the set is split in two
      auto mma = [&](long long gt, uint32_t a_addr, int pos, int nb) {
        while (nb > 0) {
          const int a0 = (int)(gt % kAcc), c = min(nb, kAcc - a0);
          const uint32_t dt = tset + 64u * (uint32_t)a0;
          const uint32_t idesc = idesc0 | ((64u * (uint32_t)c >> 3) << 17);
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {
            const uint64_t ad = sw128_desc(a_addr + ks * 32);
            const uint64_t bd = sw128_desc(s2u(sB + pos * kMatBytes) + ks * 32);
            asm volatile("tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, 1;\n"
                         ::"r"(dt), "l"(ad), "l"(bd), "r"(idesc));
            if (EC) {
              const uint64_t bl = sw128_desc(s2u(sB + (pos + 3) * kMatBytes) + ks * 32);
              asm volatile("tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, 1;\n"
                           ::"r"(dt), "l"(ad), "l"(bl), "r"(idesc));
            }
          }
          gt += c;
          pos += c;
          nb -= c;
        }
      };
      // B: the accumulator of tile gt (+)= rows at `a_addr` times shifted block b (with error
      // correction: its high part and remainder, N = 128, into two adjacent accumulators);
      // `init`: the first product of the tile
      auto mmaB = [&](long long gt, uint32_t a_addr, int b, bool init) {
        const uint32_t dt = EC ? tset + 128u * (uint32_t)(gt & 1) : tset + 64u * (uint32_t)(gt % kAcc);
        const uint32_t idesc = idesc0 | (((EC ? 128u : 64u) >> 3) << 17);
        const uint32_t bb = s2u(sB + mat_pos<EC>(b, 0) * kMatBytes);
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
          const uint64_t ad = sw128_desc(a_addr + ks * 32);
          const uint64_t bd = sw128_desc(bb + ks * 32);
          const uint32_t acc = (init && ks == 0) ? 0u : 1u;
          asm volatile("{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                       ::"r"(dt), "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
        }
      };
      // wait until the epilogue has read the previous tile held by accumulator gt % kAcc
      auto acquire = [&](long long gt) -> bool {
        if (!wait_bar(acce((int)(gt % kAcc)), (uint32_t)((gt / kAcc) & 1) ^ 1u, abort, err, 2, P.wait_ns)) return false;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        return true;
      };
      auto take = [&]() -> uint32_t {  // wait for the next slot; its shared address
        if (!wait_bar(full(slot), ph, abort, err, 3, P.wait_ns)) return 0u;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        return s2u(sA + slot * kSlotBytes);
      };
      auto release = [&]() {  // once the products issued so far are done
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(empty(slot))
                     : "memory");
        if (++slot == S) { slot = 0; ph ^= 1u; }
      };
      auto pass = [&]() -> bool {  // a slot this issuer does not read: release it once it is full
        if (!wait_bar(full(slot), ph, abort, err, 3, P.wait_ns)) return false;
        arrive(empty(slot));
        if (++slot == S) { slot = 0; ph ^= 1u; }
        return true;
      };
      auto finish = [&](long long gt) {
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                     ::"r"(accf((int)(gt % kAcc))) : "memory");
      };
      for (long long u = blockIdx.x; u < P.units && ok; u += gridDim.x) {
        const Unit w = unit_of(u, P);
        const long long g0 = g;
        bool held = false;  // A: the accumulator of the current tile is acquired already
        if (w.z0 > 0) {  // halo below: the z- neighbour rows of tile z0
          if (RA) {
            uint32_t a;
            if (!(ok = acquire(g0)) || !(a = take())) { ok = false; break; }
            mma(g0, a, mat_pos<EC>(5, 0), 1);
            release();
            held = true;
          } else if (!(ok = pass())) {
            break;
          }
        }
        for (int z = w.z0; z < w.z1 && ok; ++z) {
          const long long gz = g0 + (z - w.z0);
          uint32_t a;
          if (!(a = take())) { ok = false; break; }
          // the window: y- rows at offset 0, own rows at kBX, y+ rows at 2 kBX (rows of 128 bytes)
          if (RA) {
            if (!held && !(ok = acquire(gz))) break;
            if (z + 1 < w.z1 && !(ok = acquire(gz + 1))) break;
            // the own rows are also the z+ neighbour rows of tile z - 1 (its last product from A)
            // and the z- neighbour rows of tile z + 1: one product applies the z+, own and z- blocks
            // to them, over the tiles of this segment among z - 1, z, z + 1
            const int lo = z > w.z0 ? -1 : 0, hi = z + 1 < w.z1 ? 1 : 0;
            mma(gz + lo, a + kBX * 128, 1 + lo, hi - lo + 1);
            if (lo < 0) finish(gz - 1);
            if (!EC) mma(gz, a, mat_pos<EC>(3, 0), 1);
            release();
            if (!(ok = pass() && pass())) break;  // the x-neighbour boxes
            held = true;  // tile z + 1 was acquired above (or does not exist in this segment)
          } else {
            // set B rotates kAcc accumulators of 64 columns, or with error correction two pairs of
            // 64: wait for the epilogue to have read tile gz - kAcc (gz - 2)
            if (!(ok = acquire(EC ? gz + kAcc - 2 : gz))) break;
            if (EC) mmaB(gz, a, 3, true);
            mmaB(gz, a + 2 * kBX * 128, 4, !EC);
            release();
            if (!(a = take())) { ok = false; break; }
            mmaB(gz, a, 1, false);
            release();
            if (!(a = take())) { ok = false; break; }
            mmaB(gz, a, 2, false);
            release();
            finish(gz);
          }
        }
        if (!ok) break;
        const long long glast = g0 + (w.z1 - w.z0) - 1;
        if (w.z1 < P.nz) {  // halo above: the z+ neighbour rows of the last tile
          if (RA) {
            uint32_t a;
            if (!(a = take())) { ok = false; break; }
            mma(glast, a, mat_pos<EC>(6, 0), 1);
            release();
          } else if (!(ok = pass())) {
            break;
          }
        }
        if (RA) finish(glast);
        g = glast + 1;
      }
      // every product issued so far has finished before TMEM is released
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(drain)
                   : "memory");
      drain_bar(drain, 0, err, 6);
    }
  } else {
    // ---------------------------------------------------------------- epilogue
    const int q4 = warp & 3;  // this warp may read TMEM lanes 32*q4 .. 32*q4+31
    const int grp = (warp - 2) >> 2;  // group 0 takes the even tiles, group 1 the odd ones
    const int row = 32 * q4 + lane;
    long long g = 0;
    bool ok = true;
    for (long long u = blockIdx.x; u < P.units && ok; u += gridDim.x) {
      const Unit w = unit_of(u, P);
      for (int z = w.z0; z < w.z1; ++z, ++g) {
        if ((int)(g & 1) != grp) continue;
        const int a = (int)(g % kAcc);
        // warp-uniform decision: the TMEM loads below are .sync.aligned
        if (!__all_sync(0xffffffffu, wait_bar(accf(a), (uint32_t)((g / kAcc) & 1), abort, err, 7, P.wait_ns))) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        uint32_t r[64], rb[32];
        const uint32_t ta = tmem + ((uint32_t)(32 * q4) << 16) + 64u * (uint32_t)a;
        // set B: the tile's accumulator, or with error correction its high-part and remainder pair
        const uint32_t tb = EC ? tmem + ((uint32_t)(32 * q4) << 16) + 64u * kAcc + 128u * (uint32_t)(g & 1)
                               : ta + 64u * kAcc;
#pragma unroll
        for (int h = 0; h < 2; ++h) {  // the issuers' accumulators, 32 columns at a time
          TP_LD32(r, 32 * h, ta + 32 * h);
          TP_LD32(rb, 0, tb + 32 * h);
          asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
          for (int q = 0; q < 32; ++q) r[32 * h + q] = __float_as_uint(__uint_as_float(r[32 * h + q]) + __uint_as_float(rb[q]));
          if (EC) {
            TP_LD32(rb, 0, tb + 64 + 32 * h);
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
            for (int q = 0; q < 32; ++q)
              r[32 * h + q] = __float_as_uint(__uint_as_float(r[32 * h + q]) + __uint_as_float(rb[q]));
          }
        }
        TP_ST32Z(ta);
        TP_ST32Z(ta + 32);
        asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        arrive(acce(a));
        if (stage_bytes<EC>() > 0) {
          // this warp's 32 rows are the 8 x 4 cells at (w.x0, w.y0 + 4 q4, z): swizzled into its
          // staging buffer (conflict-free), then one TMA store; cells outside the mesh are clipped
          const uint32_t sb = s2u(sY + (warp - 2) * 4096);
          if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");  // buffer read out
          __syncwarp();
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            uint4 ov;
            TO* h = reinterpret_cast<TO*>(&ov);
#pragma unroll
            for (int q = 0; q < 8; ++q) h[q] = from_f<TO>(__uint_as_float(r[c * 8 + q]) * P.out_scale);
            asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};\n" ::"r"(sb + (uint32_t)sw_off(lane, c)), "r"(ov.x),
                         "r"(ov.y), "r"(ov.z), "r"(ov.w)
                         : "memory");
          }
          asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
          __syncwarp();
          if (lane == 0 && w.y0 + 4 * q4 < P.ny) {
            asm volatile(
                "cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%1, %2, %3, %4}], [%5];\n"
                ::"l"((uint64_t)&tmy), "r"(0), "r"(w.x0), "r"(w.y0 + 4 * q4), "r"(z), "r"(sb)
                : "memory");
            asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
          }
        } else {
          const int cx = w.x0 + (row & (kBX - 1)), cy = w.y0 + row / kBX;
          if (cx < P.nx && cy < P.ny) {
            uint4* dst = reinterpret_cast<uint4*>(y + (((long long)z * P.ny + cy) * P.nx + cx) * 64);
#pragma unroll
            for (int c = 0; c < 8; ++c) {
              uint4 ov;
              TO* h = reinterpret_cast<TO*>(&ov);
#pragma unroll
              for (int q = 0; q < 8; ++q) h[q] = from_f<TO>(__uint_as_float(r[c * 8 + q]) * P.out_scale);
              dst[c] = ov;
            }
          }
        }
      }
    }
    // the staged stores have landed before the kernel ends (the boundary kernel reads them next)
    if (stage_bytes<EC>() > 0 && lane == 0) asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");
  }
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(128 * kAcc));
  }
}

// Boundary-face corrections, one thread per boundary cell, after the apply: the cells of the six
// boundary faces are enumerated face by face (x-, x+, y-, y+, z-, z+); a cell on several faces is
// handled by the thread of the first of them, which adds the corrections of all its faces (FP32)
// to the stored row and rounds it again.
template <typename TO>
__global__ void __launch_bounds__(128) umma_fix_kernel(const TO* __restrict__ x, TO* __restrict__ y,
                                                       const __grid_constant__ Params P) {
  const long long fx = (long long)P.ny * P.nz, fy = (long long)P.nx * P.nz, fz = (long long)P.nx * P.ny;
  long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= 2 * (fx + fy + fz)) return;
  int f, cx, cy, cz;
  if (b < 2 * fx) {
    f = (int)(b / fx);
    const long long i = b % fx;
    cx = f ? P.nx - 1 : 0; cy = (int)(i % P.ny); cz = (int)(i / P.ny);
  } else if ((b -= 2 * fx) < 2 * fy) {
    f = 2 + (int)(b / fy);
    const long long i = b % fy;
    cy = f == 3 ? P.ny - 1 : 0; cx = (int)(i % P.nx); cz = (int)(i / P.nx);
  } else {
    b -= 2 * fy;
    f = 4 + (int)(b / fz);
    const long long i = b % fz;
    cz = f == 5 ? P.nz - 1 : 0; cx = (int)(i % P.nx); cy = (int)(i / P.nx);
  }
  const bool on[6] = {cx == 0, cx == P.nx - 1, cy == 0, cy == P.ny - 1, cz == 0, cz == P.nz - 1};
  for (int g = 0; g < f; ++g)
    if (on[g]) return;  // the thread of an earlier face owns this cell
  const long long cell = ((long long)cz * P.ny + cy) * P.nx + cx;
  float u[64], o[64];
  const uint4* src = reinterpret_cast<const uint4*>(x + cell * 64);
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const uint4 v = __ldg(src + c);
    const TO* h = reinterpret_cast<const TO*>(&v);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      u[c * 8 + q] = to_f<TO>(h[q]);
      o[c * 8 + q] = 0.f;
    }
  }
  if (on[0]) add_face<0, 0>(o, u, P);
  if (on[1]) add_face<0, 1>(o, u, P);
  if (on[2]) add_face<1, 0>(o, u, P);
  if (on[3]) add_face<1, 1>(o, u, P);
  if (on[4]) add_face<2, 0>(o, u, P);
  if (on[5]) add_face<2, 1>(o, u, P);
  uint4* dst = reinterpret_cast<uint4*>(y + cell * 64);
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    uint4 v = dst[c];
    TO* h = reinterpret_cast<TO*>(&v);
#pragma unroll
    for (int q = 0; q < 8; ++q) h[q] = from_f<TO>(to_f<TO>(h[q]) + o[c * 8 + q]);
    dst[c] = v;
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

static void umma_schedule(int nx, int ny, int nz, int sms, umma::Params& P);

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
  for (int d = 0; d < 3; ++d) {
    for (int e = 0; e < 16; ++e) P.fM[d][e] = (float)op->dir[d].M[e];
    P.fhh[d] = (float)(0.5 / op->dir[d].h);
  }
  for (int m = 0; m < 4; ++m) {
    P.fd0[m] = (float)op->ref.d0[m];
    P.fd1[m] = (float)op->ref.d1[m];
  }
  int sms = 0;
  err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, op->device);
  if (err != cudaSuccess) return err;
  op->sm_count = sms > 0 ? sms : 1;
  umma_schedule(op->mesh.nx, op->mesh.ny, op->mesh.nz, op->sm_count, P);
  return cudaFuncSetAttribute(umma::apply_umma_kernel<TO, EC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)umma::smem_bytes<EC>());
}

// Tiles of 8 x 16 x 1 cells; work units are z-segments of tile columns. The segment length is the
// one that minimizes the busiest CTA's work: its units times (tiles per unit + the two halo boxes
// of an inner segment, about a third of a tile's loads each).
static void umma_schedule(int nx, int ny, int nz, int sms, umma::Params& P) {
  P.tiles[0] = (nx + umma::kBX - 1) / umma::kBX;
  P.tiles[1] = (ny + umma::kBY - 1) / umma::kBY;
  P.tiles[2] = nz;
  const long long cols = (long long)P.tiles[0] * P.tiles[1];
  double best = -1.0;
  for (int L = 1; L <= nz; ++L) {
    const long long segs = (nz + L - 1) / L, units = cols * segs;
    const long long per = (units + sms - 1) / sms;
    const double cost = (double)per * (L + (segs > 1 ? 0.7 : 0.0));
    if (best < 0.0 || cost < best - 1e-9) {
      best = cost;
      P.seg = L;
      P.units = units;
    }
  }
}

template <typename TO, bool EC>
static cudaError_t umma_launch_t(const tp_op_s* op, void* y, const void* x, cudaStream_t s) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return cudaErrorNotSupported;
  const umma::Params& P = op->umma_params;
  const CUtensorMapDataType dt =
      std::is_same<TO, __half>::value ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  // (64 values, nx, ny, nz), one 128-byte row per cell; boxes of 8 x 18 x 1 cells (the window: a
  // tile with a y-halo row on each side) and 8 x 16 x 1 cells (a tile)
  cuuint64_t dims[4] = {64, (cuuint64_t)op->mesh.nx, (cuuint64_t)op->mesh.ny, (cuuint64_t)op->mesh.nz};
  cuuint64_t strides[3] = {128, 128ull * op->mesh.nx, 128ull * op->mesh.nx * op->mesh.ny};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  cuuint32_t boxw[4] = {64, (cuuint32_t)umma::kBX, (cuuint32_t)(umma::kBY + 2), 1};
  cuuint32_t boxt[4] = {64, (cuuint32_t)umma::kBX, (cuuint32_t)umma::kBY, 1};
  cuuint32_t boxy[4] = {64, (cuuint32_t)umma::kBX, 4, 1};  // one epilogue warp's 32 output rows
  CUtensorMap tmw, tmt, tmy;
  if (enc(&tmw, dt, 4, const_cast<void*>(x), dims, strides, boxw, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
          CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
          CUDA_SUCCESS ||
      enc(&tmt, dt, 4, const_cast<void*>(x), dims, strides, boxt, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
          CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
          CUDA_SUCCESS ||
      enc(&tmy, dt, 4, y, dims, strides, boxy, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  const int grid = (int)(P.units < op->sm_count ? P.units : op->sm_count);
  umma::apply_umma_kernel<TO, EC><<<grid, umma::kThreads, umma::smem_bytes<EC>(), s>>>(
      tmw, tmt, tmy, static_cast<const TO*>(x), static_cast<TO*>(y), static_cast<const TO*>(op->umma_mats), P,
      op->umma_err);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long long slots = 2 * ((long long)P.ny * P.nz + (long long)P.nx * P.nz + (long long)P.nx * P.ny);
  const long long blocks = (slots + 127) / 128;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  umma::umma_fix_kernel<TO><<<(unsigned)blocks, 128, 0, s>>>(static_cast<const TO*>(x), static_cast<TO*>(y), P);
  return cudaGetLastError();
}

// the tcgen05 apply: k = 3 with FP16/BF16 vectors (per-axis TMA coordinates are int32: any mesh)
bool umma_supported(const tp_op_s* op) {
  return op->n == 4 && (op->prec == TP_FP16 || op->prec == TP_BF16);
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
