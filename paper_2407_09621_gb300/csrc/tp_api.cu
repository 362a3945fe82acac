// C-ABI entry points of libtp: handles, validation, error text, dispatch.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>

#include "tp_internal.h"

namespace tp {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

tp_status cuda_status(int err, const char* what) {
  if (err == cudaSuccess) return TP_OK;
  set_error("%s: %s", what, cudaGetErrorString((cudaError_t)err));
  return err == cudaErrorMemoryAllocation ? TP_ERR_OOM : TP_ERR_CUDA;
}

cudaError_t launch_apply_cc(const tp_op_s* op, void* y, const void* x, cudaStream_t s);
cudaError_t launch_apply_cc_range(const tp_op_s* op, void* y, const void* x, long long c0, long long c1,
                                  cudaStream_t s, const void* b);
cudaError_t launch_apply_dmma_range(const tp_op_s* op, void* y, const void* x, long long c0, long long c1,
                                    cudaStream_t s);
cudaError_t prepare_apply_cc(const tp_op_s* op);
cudaError_t launch_apply_tc(const tp_op_s* op, void* y, const void* x, cudaStream_t s);
cudaError_t prepare_apply_tc(tp_op_s* op);
bool umma_supported(const tp_op_s* op);
bool dmma_supported(const tp_op_s* op);
cudaError_t prepare_apply_dmma(const tp_op_s* op);
cudaError_t launch_apply_dmma(const tp_op_s* op, void* y, const void* x, cudaStream_t s);
cudaError_t prepare_apply_umma(tp_op_s* op);
cudaError_t launch_apply_umma(const tp_op_s* op, void* y, const void* x, cudaStream_t s);
tp_status prepare_apply_patch(tp_op_s* op);
cudaError_t launch_apply_patch(const tp_op_s* op, void* y, const void* x, cudaStream_t s);

// the apply kernel family chosen at creation
cudaError_t launch_apply(const tp_op_s* op, void* y, const void* x, cudaStream_t s) {
  if (op->opts.kernel == TP_KERNEL_PATCH) return launch_apply_patch(op, y, x, s);
  if (op->opts.kernel != TP_KERNEL_TENSOR) return launch_apply_cc(op, y, x, s);
  if (op->prec == TP_FP64) return launch_apply_dmma(op, y, x, s);
  return op->use_umma ? launch_apply_umma(op, y, x, s) : launch_apply_tc(op, y, x, s);
}

// r = b - A x in one pass where the CUDA-core kernel runs (its store takes b); other kernel
// families return cudaErrorNotSupported and the caller forms A x and the difference.
cudaError_t launch_residual(const tp_op_s* op, void* r, const void* b, const void* x, cudaStream_t s) {
  if (op->opts.kernel == TP_KERNEL_CUDA_CORE) return launch_apply_cc_range(op, r, x, 0, op->ncells, s, b);
  return cudaErrorNotSupported;
}

int cc_tile_cells(int n, int v);
bool cc_cell_per_thread(const tp_op_s* op);
int dmma_tile_cells(int n, int v);
size_t elem_bytes(tp_precision p);

// Autotuner of the apply's tile shape (cells per thread block of the CUDA-core and DMMA kernels:
// the default halved, kept or doubled). Each shape is timed with CUDA events on a proxy of the
// operator's mesh (same nx and ny, enough z-layers for about 128 MB per vector) after one
// warm-up launch; the fastest is kept. The per-cell arithmetic does not depend on the shape, so
// the choice changes no result. Tuning is best effort: if the proxy vectors cannot be
// allocated the default shape stays. Degrees above 7 have a single shape and are not tuned.
static tp_status autotune_apply(tp_op_s* op) {
  const bool dm = op->opts.kernel == TP_KERNEL_TENSOR && op->prec == TP_FP64;
  if (op->opts.kernel == TP_KERNEL_TENSOR && !dm) return TP_OK;  // tcgen05 / mma.sync: fixed tiles
  if (op->opts.kernel == TP_KERNEL_PATCH) return TP_OK;           // one patch per thread block
  if (op->n > kMaxN) return TP_OK;                                 // n > 8: one tile shape
  if (op->opts.kernel == TP_KERNEL_CUDA_CORE && cc_cell_per_thread(op)) return TP_OK;  // one shape
  if (op->opts.dword) return TP_OK;                                // double-word: one tile shape
  const long long eb = (long long)elem_bytes(op->prec);
  const long long n3 = (long long)op->n * op->n * op->n;
  const long long slab = (long long)op->mesh.nx * op->mesh.ny;
  long long nz = (128LL << 20) / (slab * n3 * eb);
  nz = nz < 1 ? 1 : (nz > op->mesh.nz ? op->mesh.nz : nz);
  tp_op_s proxy = *op;  // shares the constants; owns nothing
  proxy.hx = proxy.hy = nullptr;
  proxy.mesh.nz = (int)nz;
  proxy.ncells = slab * nz;
  proxy.ndofs = proxy.ncells * n3;
  const size_t bytes = (size_t)(proxy.ndofs * eb);
  void *x = nullptr, *y = nullptr;
  if (cudaMalloc(&x, bytes) != cudaSuccess || cudaMalloc(&y, bytes) != cudaSuccess) {
    if (x) cudaFree(x);
    cudaGetLastError();
    return TP_OK;
  }
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  tp_status st = cuda_status(cudaMemset(x, 0x3c, bytes), "autotune fill");
  if (st == TP_OK) st = cuda_status(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "autotune stream");
  if (st == TP_OK) st = cuda_status(cudaEventCreate(&e0), "autotune event");
  if (st == TP_OK) st = cuda_status(cudaEventCreate(&e1), "autotune event");
  float best = 0.f;
  int best_v = op->tile_variant;
  for (int v = 0; v < 3 && st == TP_OK; ++v) {
    proxy.tile_variant = v;
    st = cuda_status(launch_apply(&proxy, y, x, s), "autotune launch");
    if (st == TP_OK) st = cuda_status(cudaEventRecord(e0, s), "autotune event");
    for (int r = 0; r < 3 && st == TP_OK; ++r) st = cuda_status(launch_apply(&proxy, y, x, s), "autotune launch");
    if (st == TP_OK) st = cuda_status(cudaEventRecord(e1, s), "autotune event");
    if (st == TP_OK) st = cuda_status(cudaEventSynchronize(e1), "autotune sync");
    float ms = 0.f;
    if (st == TP_OK) st = cuda_status(cudaEventElapsedTime(&ms, e0, e1), "autotune timing");
    if (st == TP_OK && (v == 0 || ms < best)) {
      best = ms;
      best_v = v;
    }
  }
  if (st == TP_OK) op->tile_variant = best_v;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  cudaFree(x);
  cudaFree(y);
  return st;
}

// Tensor family: tcgen05 (TMA, TMEM) for k = 3 with FP16/BF16 vectors, mma.sync otherwise.
static cudaError_t prepare_tensor(tp_op_s* op) {
  if (op->prec == TP_FP64) return dmma_supported(op) ? prepare_apply_dmma(op) : cudaErrorInvalidValue;
  op->use_umma = umma_supported(op);
  return op->use_umma ? prepare_apply_umma(op) : prepare_apply_tc(op);
}

size_t elem_bytes(tp_precision p) {
  switch (p) {
    case TP_FP64: return 8;
    case TP_FP32: return 4;
    case TP_FP16: return 2;
    case TP_BF16: return 2;
  }
  return 0;
}

template <typename T, int NM>
static void fill_const(OpConst<T, NM>& c, const tp_op_s* op) {
  memset(&c, 0, sizeof(c));
  const int n = op->n;
  const std::vector<double>& d0 = op->ref.d0;
  const std::vector<double>& d1 = op->ref.d1;
  for (int d = 0; d < 3; ++d) {
    const Dir1D& D = op->dir[d];
    const std::vector<double> Minv = invert(n, D.M);
    const double g = D.gamma, hh = 0.5 / D.h;
    // M^-1 applied to the trace vectors: columns n-1 and 0 of M^-1 are M^-1 v1 and M^-1 v0
    std::vector<double> mv0(n), mv1(n), md0(n), md1(n);
    for (int i = 0; i < n; ++i) {
      mv0[i] = Minv[i * n + 0];
      mv1[i] = Minv[i * n + n - 1];
      md0[i] = md1[i] = 0.0;
      for (int m = 0; m < n; ++m) {
        md0[i] += Minv[i * n + m] * d0[m];
        md1[i] += Minv[i * n + m] * d1[m];
      }
    }
    for (int i = 0; i < n; ++i) {
      for (int j = 0; j < n; ++j) {
        double gij = 0.0;
        for (int m = 0; m < n; ++m) gij += Minv[i * n + m] * D.L[m * n + j];
        c.M[d][i * NM + j] = (T)D.M[i * n + j];
        c.G[d][i * NM + j] = (T)gij;
      }
      c.E[d][0][i] = (T)(-g * mv1[i] + hh * md1[i]);  // P1: high neighbour, value trace
      c.E[d][1][i] = (T)(-hh * mv1[i]);               // P2: high neighbour, derivative trace
      c.E[d][2][i] = (T)(-g * mv0[i] - hh * md0[i]);  // Q1: low neighbour, value trace
      c.E[d][3][i] = (T)(hh * mv0[i]);                // Q2: low neighbour, derivative trace
      c.E[d][4][i] = (T)(-hh * md1[i]);               // B1: high boundary, own value trace
      c.E[d][5][i] = (T)(-hh * mv1[i]);               // B2: high boundary, own derivative trace
      c.E[d][6][i] = (T)(hh * md0[i]);                // C1: low boundary, own value trace
      c.E[d][7][i] = (T)(hh * mv0[i]);                // C2: low boundary, own derivative trace
    }
  }
  for (int i = 0; i < n; ++i) {
    c.d0[i] = (T)d0[i];
    c.d1[i] = (T)d1[i];
  }
  // even-odd halves (used for n >= 5 when the matrices are centrosymmetric)
  bool centro = n >= 5;
  for (int d = 0; d < 3 && centro; ++d) {
    const Dir1D& D = op->dir[d];
    const std::vector<double> Minv = invert(n, D.M);
    std::vector<double> G(n * n, 0.0);
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j)
        for (int m = 0; m < n; ++m) G[i * n + j] += Minv[i * n + m] * D.L[m * n + j];
    double gmax = 0.0, mmax = 0.0;
    for (int e = 0; e < n * n; ++e) {
      gmax = std::max(gmax, std::fabs(G[e]));
      mmax = std::max(mmax, std::fabs(D.M[e]));
    }
    for (int i = 0; i < n && centro; ++i)
      for (int j = 0; j < n && centro; ++j) {
        const int r = (n - 1 - i) * n + (n - 1 - j);
        centro = std::fabs(G[i * n + j] - G[r]) <= 1e-12 * gmax && std::fabs(D.M[i * n + j] - D.M[r]) <= 1e-12 * mmax;
      }
    const int H = n / 2;
    for (int i = 0; i < H; ++i)
      for (int m = 0; m < H; ++m) {
        c.ME[d][i][m] = (T)(0.5 * (D.M[i * n + m] + D.M[i * n + n - 1 - m]));
        c.MO[d][i][m] = (T)(0.5 * (D.M[i * n + m] - D.M[i * n + n - 1 - m]));
        c.GE[d][i][m] = (T)(0.5 * (G[i * n + m] + G[i * n + n - 1 - m]));
        c.GO[d][i][m] = (T)(0.5 * (G[i * n + m] - G[i * n + n - 1 - m]));
      }
    if (n % 2 == 1) {  // the middle node: column H of the even half, and the middle row
      for (int i = 0; i <= H; ++i) {
        c.ME[d][i][H] = (T)D.M[i * n + H];
        c.GE[d][i][H] = (T)G[i * n + H];
        c.ME[d][H][i] = (T)D.M[H * n + i];
        c.GE[d][H][i] = (T)G[H * n + i];
      }
    }
  }
  c.centro = centro ? 1 : 0;
}

// Algorithmic flops per DoF of the sum-factorized apply in the inverse-mass form (FMA = 2
// flops): 6 n x n contractions (12n), 6 derivative traces (12), 6 faces x two dense expansion
// vectors (24), summing the three directions (2): 12n + 38. With the even-odd form of the
// contractions (n >= 5, centrosymmetric matrices) a line costs n^2/2 FMAs and 2n adds for even
// n, (n^2 + 1)/2 FMAs and 2(n - 1) adds for odd n: 6n + 50 (even) or 6n + 50 - 6/n (odd).
double apply_flops_per_dof(int n, bool even_odd) {
  const double line = !even_odd ? 2.0 * n * n : (n % 2 == 0 ? 1.0 * n * n + 2.0 * n : n * n + 1.0 + 2.0 * (n - 1));
  return 6.0 * line / n + 38.0;
}

}  // namespace tp

using namespace tp;

namespace {

// Copy/compute pipeline of tp_apply_host: the cells are cut into min(16, nz) ranges of whole
// z-slabs (meshes with at least kMinChunks z-layers); chunk i is copied in on `in`, applied on
// `comp` once chunks i-1..i+1 (its face neighbours) are resident, and copied out on `out`, so the
// three overlap (H2D and D2H use separate copy engines). More chunks shorten the unoverlapped
// first copy-in and last copy-out.
constexpr int kMinChunks = 8, kMaxChunks = 16;
struct HostPipe {
  cudaStream_t in = nullptr, comp = nullptr, out = nullptr;
  cudaEvent_t start = nullptr, done = nullptr, loaded[kMaxChunks] = {}, applied[kMaxChunks] = {};
};

void destroy_pipe(HostPipe* p) {
  if (!p) return;
  for (cudaStream_t s : {p->in, p->comp, p->out})
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : {p->start, p->done})
    if (e) cudaEventDestroy(e);
  for (int i = 0; i < kMaxChunks; ++i) {
    if (p->loaded[i]) cudaEventDestroy(p->loaded[i]);
    if (p->applied[i]) cudaEventDestroy(p->applied[i]);
  }
  delete p;
}

tp_status make_pipe(HostPipe** out) {
  HostPipe* p = new (std::nothrow) HostPipe();
  if (!p) { set_error("tp_apply_host: out of host memory"); return TP_ERR_OOM; }
  tp_status st = TP_OK;
  for (cudaStream_t* s : {&p->in, &p->comp, &p->out})
    if (st == TP_OK) st = cuda_status(cudaStreamCreateWithFlags(s, cudaStreamNonBlocking), "tp_apply_host streams");
  for (cudaEvent_t* e : {&p->start, &p->done})
    if (st == TP_OK) st = cuda_status(cudaEventCreateWithFlags(e, cudaEventDisableTiming), "tp_apply_host events");
  for (int i = 0; i < kMaxChunks && st == TP_OK; ++i) {
    st = cuda_status(cudaEventCreateWithFlags(&p->loaded[i], cudaEventDisableTiming), "tp_apply_host events");
    if (st == TP_OK)
      st = cuda_status(cudaEventCreateWithFlags(&p->applied[i], cudaEventDisableTiming), "tp_apply_host events");
  }
  if (st != TP_OK) {
    destroy_pipe(p);
    return st;
  }
  *out = p;
  return TP_OK;
}

// Pipelined host apply for the kernels that can restrict their output to a range of cells
// (CUDA-core and DMMA). Ordered after prior work on `s`, and `s` waits for its completion.
tp_status apply_host_pipelined(tp_op_s* op, void* y_host, const void* x_host, cudaStream_t s) {
  if (!op->hpipe) {
    HostPipe* p = nullptr;
    tp_status st = make_pipe(&p);
    if (st != TP_OK) return st;
    op->hpipe = p;
  }
  HostPipe& P = *static_cast<HostPipe*>(op->hpipe);
  const long long slab = (long long)op->mesh.nx * op->mesh.ny;
  const int nz = op->mesh.nz;
  const size_t cell_bytes = (size_t)(op->ndofs / op->ncells) * elem_bytes(op->prec);
  const int chunks = nz < kMaxChunks ? nz : kMaxChunks;
  auto z_at = [&](int i) { return (long long)nz * i / chunks; };  // chunk i = slabs [z_at(i), z_at(i+1))
  auto launch = [&](long long c0, long long c1, cudaStream_t st) {
    return op->opts.kernel == TP_KERNEL_TENSOR ? launch_apply_dmma_range(op, op->hy, op->hx, c0, c1, st)
                                               : launch_apply_cc_range(op, op->hy, op->hx, c0, c1, st, nullptr);
  };
  tp_status st = cuda_status(cudaEventRecord(P.start, s), "tp_apply_host");
  for (cudaStream_t q : {P.in, P.comp, P.out})
    if (st == TP_OK) st = cuda_status(cudaStreamWaitEvent(q, P.start, 0), "tp_apply_host");
  unsigned char* dx = static_cast<unsigned char*>(op->hx);
  unsigned char* dy = static_cast<unsigned char*>(op->hy);
  const unsigned char* hx = static_cast<const unsigned char*>(x_host);
  unsigned char* hy = static_cast<unsigned char*>(y_host);
  auto copy_in = [&](int i) {
    const size_t o = (size_t)(z_at(i) * slab) * cell_bytes, n = (size_t)((z_at(i + 1) - z_at(i)) * slab) * cell_bytes;
    tp_status r = cuda_status(cudaMemcpyAsync(dx + o, hx + o, n, cudaMemcpyHostToDevice, P.in), "tp_apply_host H2D");
    if (r == TP_OK) r = cuda_status(cudaEventRecord(P.loaded[i], P.in), "tp_apply_host");
    return r;
  };
  if (st == TP_OK) st = copy_in(0);
  for (int i = 0; i < chunks && st == TP_OK; ++i) {
    if (i + 1 < chunks) st = copy_in(i + 1);
    const int need = i + 1 < chunks ? i + 1 : i;  // the chunk above must be resident (face neighbours)
    if (st == TP_OK) st = cuda_status(cudaStreamWaitEvent(P.comp, P.loaded[need], 0), "tp_apply_host");
    if (st == TP_OK) st = cuda_status(launch(z_at(i) * slab, z_at(i + 1) * slab, P.comp), "tp_apply_host launch");
    if (st == TP_OK) st = cuda_status(cudaEventRecord(P.applied[i], P.comp), "tp_apply_host");
    if (st == TP_OK) st = cuda_status(cudaStreamWaitEvent(P.out, P.applied[i], 0), "tp_apply_host");
    if (st == TP_OK) {
      const size_t o = (size_t)(z_at(i) * slab) * cell_bytes;
      const size_t n = (size_t)((z_at(i + 1) - z_at(i)) * slab) * cell_bytes;
      st = cuda_status(cudaMemcpyAsync(hy + o, dy + o, n, cudaMemcpyDeviceToHost, P.out), "tp_apply_host D2H");
    }
  }
  if (st == TP_OK) st = cuda_status(cudaEventRecord(P.done, P.out), "tp_apply_host");
  if (st == TP_OK) st = cuda_status(cudaStreamWaitEvent(s, P.done, 0), "tp_apply_host");
  if (st == TP_OK) st = cuda_status(cudaStreamSynchronize(s), "tp_apply_host sync");
  return st;
}

}  // namespace

extern "C" {

const char* tp_last_error(void) { return g_err; }

tp_status tp_mesh_create(tp_mesh* out, int nx, int ny, int nz, double lx, double ly, double lz) {
  if (!out) { set_error("tp_mesh_create: out is NULL"); return TP_ERR_INVALID_ARG; }
  *out = nullptr;
  if (nx < 1 || ny < 1 || nz < 1) { set_error("tp_mesh_create: cell counts must be >= 1"); return TP_ERR_INVALID_ARG; }
  if (!(lx > 0) || !(ly > 0) || !(lz > 0)) { set_error("tp_mesh_create: lengths must be > 0"); return TP_ERR_INVALID_ARG; }
  const long long nc = (long long)nx * ny * nz;
  if (nc > (1LL << 53)) { set_error("tp_mesh_create: too many cells"); return TP_ERR_INVALID_ARG; }
  tp_mesh_s* m = new (std::nothrow) tp_mesh_s{nx, ny, nz, lx, ly, lz};
  if (!m) { set_error("tp_mesh_create: out of host memory"); return TP_ERR_OOM; }
  *out = m;
  return TP_OK;
}

tp_status tp_mesh_destroy(tp_mesh m) {
  delete m;
  return TP_OK;
}

tp_status tp_dg_laplace_create(tp_op* out, tp_mesh m, int k, tp_precision p, const tp_op_opts* opts) {
  if (!out) { set_error("tp_dg_laplace_create: out is NULL"); return TP_ERR_INVALID_ARG; }
  *out = nullptr;
  if (!m) { set_error("tp_dg_laplace_create: mesh is NULL"); return TP_ERR_INVALID_ARG; }
  if (k < 1 || k > kMaxNHigh - 1) {
    set_error("tp_dg_laplace_create: degree k=%d outside [1,%d]", k, kMaxNHigh - 1);
    return TP_ERR_INVALID_ARG;
  }
  if (p != TP_FP64 && p != TP_FP32 && p != TP_FP16 && p != TP_BF16) {
    set_error("tp_dg_laplace_create: unknown precision %d", (int)p);
    return TP_ERR_INVALID_ARG;
  }
  tp_op_opts o{TP_PENALTY_CONFIG, TP_KERNEL_AUTO, 0, TP_FP16, 0, 0};
  if (opts) o = *opts;
  if (o.penalty != TP_PENALTY_CONFIG && o.penalty != TP_PENALTY_PAPER) {
    set_error("tp_dg_laplace_create: unknown penalty mode %d", o.penalty);
    return TP_ERR_INVALID_ARG;
  }
  if (o.kernel < TP_KERNEL_AUTO || o.kernel > TP_KERNEL_PATCH) {
    set_error("tp_dg_laplace_create: unknown kernel family %d", o.kernel);
    return TP_ERR_INVALID_ARG;
  }
  if (o.tc_type != TP_FP16 && o.tc_type != TP_BF16) {
    set_error("tp_dg_laplace_create: tc_type must be TP_FP16 or TP_BF16");
    return TP_ERR_INVALID_ARG;
  }
  if (o.ec < 0 || o.ec > 3) {
    set_error("tp_dg_laplace_create: ec must be 0 (off), 1 (both operands), 2 (matrix) or 3 (vector)");
    return TP_ERR_INVALID_ARG;
  }
  if (o.dword != 0 && o.dword != 1) {
    set_error("tp_dg_laplace_create: dword must be 0 (FP64 arithmetic) or 1 (double-word FP32 arithmetic)");
    return TP_ERR_INVALID_ARG;
  }
  if (o.dword && (p != TP_FP64 || (o.kernel != TP_KERNEL_AUTO && o.kernel != TP_KERNEL_CUDA_CORE) || k + 1 > kMaxN)) {
    set_error("tp_dg_laplace_create: double-word arithmetic is for FP64 vectors on the CUDA-core kernel, k <= %d",
              kMaxN - 1);
    return TP_ERR_UNSUPPORTED;
  }
  const long long ncells = (long long)m->nx * m->ny * m->nz;
  if (o.kernel == TP_KERNEL_AUTO) {
    // The fastest family measured on GB300 for each precision: FP16/BF16 vectors at k = 3 run on
    // tcgen05 (faster than the CUDA-core kernel at every measured size); FP64 stays on DFMA (DMMA
    // shares the FP64 pipe and is slower) and FP32 on the CUDA-core kernel (the mma.sync path is
    // slower); everything else is CUDA-core.
    o.kernel = ((p == TP_FP16 || p == TP_BF16) && k == 3) ? TP_KERNEL_TENSOR : TP_KERNEL_CUDA_CORE;
  }
  if (o.kernel == TP_KERNEL_TENSOR && p == TP_FP64) {
    if (k != 3 && k != 7) {
      set_error("tp_dg_laplace_create: the FP64 tensor (DMMA) kernel supports k = 3 and k = 7");
      return TP_ERR_UNSUPPORTED;
    }
    if (o.ec) {
      set_error("tp_dg_laplace_create: error correction applies to half-precision operands, not FP64");
      return TP_ERR_UNSUPPORTED;
    }
  } else if (o.kernel == TP_KERNEL_TENSOR) {
    if (k < 2 || k > 3) {
      set_error("tp_dg_laplace_create: the half-precision tensor kernels support k = 2, 3");
      return TP_ERR_UNSUPPORTED;
    }
    if ((p == TP_FP16 || p == TP_BF16) && o.tc_type != (int)p) o.tc_type = p;
    // BF16 keeps 8 significand bits: without the split of Algorithm 1 the five roundings of the
    // tensor path (input, K3, W, M3, output) exceed the 5e-3 per-apply tolerance
    if (p == TP_BF16 && o.ec != 1 && o.ec != 2) o.ec = 1;
    // FP16/BF16 vectors are exact operands: refining "the vector" alone refines nothing
    if (p == TP_FP16 && o.ec == 3) o.ec = 0;
  } else if (o.ec) {
    set_error("tp_dg_laplace_create: error correction needs the tensor kernel");
    return TP_ERR_UNSUPPORTED;
  }
  if (o.kernel == TP_KERNEL_PATCH) {
    if ((p != TP_FP64 && p != TP_FP32) || k > kMaxN - 1) {
      set_error("tp_dg_laplace_create: the patch-wise kernel takes FP64 or FP32 vectors and k <= %d", kMaxN - 1);
      return TP_ERR_UNSUPPORTED;
    }
    if (m->nx < 2 || m->ny < 2 || m->nz < 2) {
      set_error("tp_dg_laplace_create: the patch-wise kernel needs at least two cells per direction");
      return TP_ERR_UNSUPPORTED;
    }
  }
  if (k + 1 > kMaxN && (o.kernel == TP_KERNEL_TENSOR || (p != TP_FP64 && p != TP_FP32))) {
    set_error("tp_dg_laplace_create: degrees above %d need the CUDA-core kernel and FP64 or FP32 vectors", kMaxN - 1);
    return TP_ERR_UNSUPPORTED;
  }
  const long long n3 = (long long)(k + 1) * (k + 1) * (k + 1);
  if (ncells > (1LL << 62) / n3) { set_error("tp_dg_laplace_create: DoF count overflows"); return TP_ERR_INVALID_ARG; }
  tp_op_s* op = new (std::nothrow) tp_op_s();
  if (!op) { set_error("tp_dg_laplace_create: out of host memory"); return TP_ERR_OOM; }
  op->mesh = *m;
  op->k = k;
  op->n = k + 1;
  op->prec = p;
  op->opts = o;
  op->ncells = ncells;
  op->ndofs = ncells * n3;
  op->ref = make_ref1d(k);
  const double hs[3] = {m->lx / m->nx, m->ly / m->ny, m->lz / m->nz};
  for (int d = 0; d < 3; ++d) op->dir[d] = make_dir1d(op->ref, hs[d], o.penalty);
  tp_status st = cuda_status(cudaGetDevice(&op->device), "cudaGetDevice");
  if (st != TP_OK) { delete op; return st; }
  if (op->n > kMaxN) {
    fill_const(op->c64h, op);
    fill_const(op->c32h, op);
  } else {
    fill_const(op->c64, op);
    fill_const(op->c32, op);
  }
  if (op->opts.kernel == TP_KERNEL_PATCH)
    st = prepare_apply_patch(op);
  else
    st = cuda_status(op->opts.kernel == TP_KERNEL_TENSOR ? prepare_tensor(op) : prepare_apply_cc(op),
                     "apply kernel set-up");
  if (st == TP_OK && op->opts.kernel == TP_KERNEL_CUDA_CORE && op->n <= kMaxN) {
    // small meshes (fewer cells than two default thread blocks per SM) take the half-size tile: twice
    // the blocks to spread over the SMs; the results do not depend on the tile shape
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, op->device) == cudaSuccess && sms > 0 &&
        op->ncells < 2LL * sms * cc_tile_cells(op->n, 1))
      op->tile_variant = 0;
  }
  if (st == TP_OK && o.autotune) st = autotune_apply(op);
  if (st != TP_OK) {
    tp_op_destroy(op);
    return st;
  }
  *out = op;
  return TP_OK;
}

tp_status tp_op_get_info(tp_op op, tp_op_info_t* info) {
  if (!op || !info) { set_error("tp_op_get_info: NULL argument"); return TP_ERR_INVALID_ARG; }
  info->ncells = op->ncells;
  info->ndofs = op->ndofs;
  info->k = op->k;
  info->n = op->n;
  info->precision = op->prec;
  info->kernel = op->opts.kernel;
  info->elem_bytes = elem_bytes(op->prec);
  // the CUDA-core kernel takes the even-odd path (the DMMA and tensor kernels do not)
  const int centro = op->n > kMaxN ? op->c64h.centro : op->c64.centro;
  const bool eo = op->opts.kernel == TP_KERNEL_CUDA_CORE && op->n >= 5 && centro;
  info->flops_per_dof = op->opts.kernel == TP_KERNEL_PATCH ? 224.0 * op->n + 8.0 : apply_flops_per_dof(op->n, eo);
  info->tensor_path = op->opts.kernel != TP_KERNEL_TENSOR ? 0 : (op->prec == TP_FP64 ? 3 : (op->use_umma ? 2 : 1));
  // FP32 vectors on the half-precision tensor paths: FP32 accuracy (1e-5 per apply) only with FP16
  // operands and both operands refined (Algorithm 1, ec = 1)
  info->approximate = op->prec == TP_FP32 && op->opts.kernel == TP_KERNEL_TENSOR &&
                      !(op->opts.tc_type == TP_FP16 && op->opts.ec == 1);
  info->dword = op->opts.dword;
  info->tile_cells = op->opts.kernel == TP_KERNEL_PATCH ? 8
                     : info->tensor_path == 0 ? (op->opts.kernel == TP_KERNEL_CUDA_CORE && cc_cell_per_thread(op)
                                                     ? 128
                                                     : cc_tile_cells(op->n, op->opts.dword ? 1 : op->tile_variant))
                     : info->tensor_path == 3 ? dmma_tile_cells(op->n, op->tile_variant)
                     : info->tensor_path == 2 ? 128 : 0;
  return TP_OK;
}

tp_status tp_op_check(tp_op op) {
  if (!op) { set_error("tp_op_check: NULL op"); return TP_ERR_INVALID_ARG; }
  tp_status st = cuda_status(cudaDeviceSynchronize(), "tp_op_check sync");
  if (st != TP_OK || !op->umma_err) return st;
  int code = 0;
  st = cuda_status(cudaMemcpy(&code, op->umma_err, sizeof(int), cudaMemcpyDeviceToHost), "tp_op_check read");
  if (st != TP_OK) return st;
  if (code == 0) return TP_OK;
  cudaMemset(op->umma_err, 0, sizeof(int));
  set_error("tp_op_check: a bounded wait of the tcgen05 apply gave up (code %d)", code);
  return TP_ERR_TIMEOUT;
}


tp_status tp_op_destroy(tp_op op) {
  if (!op) return TP_OK;
  if (op->hpipe) destroy_pipe(static_cast<HostPipe*>(op->hpipe));
  if (op->hx) cudaFree(op->hx);
  if (op->hy) cudaFree(op->hy);
  if (op->tc_mats) cudaFree(op->tc_mats);
  if (op->umma_mats) cudaFree(op->umma_mats);
  if (op->umma_err) cudaFree(op->umma_err);
  if (op->pw_mats) cudaFree(op->pw_mats);
  delete op;
  return TP_OK;
}

// The operator's constants, matrices and status word live on the device that was current at its
// creation; a launch with another device current would read memory that device never filled.
static tp_status check_device(tp_op op, const char* who) {
  int dev = -1;
  tp_status st = cuda_status(cudaGetDevice(&dev), "cudaGetDevice");
  if (st != TP_OK) return st;
  if (dev != op->device) {
    set_error("%s: device %d is current, the operator lives on device %d", who, dev, op->device);
    return TP_ERR_INVALID_ARG;
  }
  return TP_OK;
}

static tp_status check_vectors(tp_op op, const void* y, const void* x, const char* who) {
  if (!op) { set_error("%s: op is NULL", who); return TP_ERR_INVALID_ARG; }
  if (!x || !y) { set_error("%s: NULL vector", who); return TP_ERR_INVALID_ARG; }
  if (((uintptr_t)x & 15) || ((uintptr_t)y & 15)) { set_error("%s: vectors must be 16-byte aligned", who); return TP_ERR_INVALID_ARG; }
  const size_t bytes = (size_t)op->ndofs * elem_bytes(op->prec);
  const uintptr_t xa = (uintptr_t)x, ya = (uintptr_t)y;
  if (xa < ya + bytes && ya < xa + bytes) { set_error("%s: x and y overlap", who); return TP_ERR_INVALID_ARG; }
  return check_device(op, who);
}

tp_status tp_apply(tp_op op, void* y, const void* x, void* stream) {
  tp_status st = check_vectors(op, y, x, "tp_apply");
  if (st != TP_OK) return st;
  return cuda_status(launch_apply(op, y, x, (cudaStream_t)stream), "tp_apply launch");
}

tp_status tp_apply_host(tp_op op, void* y_host, const void* x_host, void* stream) {
  if (!op || !x_host || !y_host) { set_error("tp_apply_host: NULL argument"); return TP_ERR_INVALID_ARG; }
  const size_t bytes = (size_t)op->ndofs * elem_bytes(op->prec);
  const uintptr_t xa = (uintptr_t)x_host, ya = (uintptr_t)y_host;
  if (xa < ya + bytes && ya < xa + bytes) { set_error("tp_apply_host: x and y overlap"); return TP_ERR_INVALID_ARG; }
  tp_status dst = check_device(op, "tp_apply_host");
  if (dst != TP_OK) return dst;
  if (op->hbytes < bytes) {
    if (op->hx) cudaFree(op->hx);
    if (op->hy) cudaFree(op->hy);
    op->hx = op->hy = nullptr;
    op->hbytes = 0;
    tp_status st = cuda_status(cudaMalloc(&op->hx, bytes), "tp_apply_host staging");
    if (st == TP_OK) st = cuda_status(cudaMalloc(&op->hy, bytes), "tp_apply_host staging");
    if (st != TP_OK) return st;
    op->hbytes = bytes;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const bool ranged = op->opts.kernel == TP_KERNEL_CUDA_CORE || (op->opts.kernel == TP_KERNEL_TENSOR && op->prec == TP_FP64);
  if (ranged && op->mesh.nz >= kMinChunks) return apply_host_pipelined(op, y_host, x_host, s);
  tp_status st = cuda_status(cudaMemcpyAsync(op->hx, x_host, bytes, cudaMemcpyHostToDevice, s), "tp_apply_host H2D");
  if (st == TP_OK) st = cuda_status(launch_apply(op, op->hy, op->hx, s), "tp_apply_host launch");
  if (st == TP_OK) st = cuda_status(cudaMemcpyAsync(y_host, op->hy, bytes, cudaMemcpyDeviceToHost, s), "tp_apply_host D2H");
  if (st == TP_OK) st = cuda_status(cudaStreamSynchronize(s), "tp_apply_host sync");
  return st;
}

}  // extern "C"
