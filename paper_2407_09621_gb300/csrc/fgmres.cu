// Flexible GMRES (Saad 1993) with right preconditioning in FP64 on the GPU
// (Sec. 7.1: the outer iteration in double precision, the multigrid
// preconditioner in lower precision with conversion at its entry and exit).
//
// Arnoldi step j: z_j = M^{-1} v_j (one V-cycle, zero initial guess),
// w = A z_j (FP64 apply), classical Gram-Schmidt with one re-orthogonalization
// pass (two fused multi-dot/multi-axpy passes over V), v_{j+1} = w/||w||.
// The small Hessenberg least-squares problem is solved on the host with
// Givens rotations; its residual |g_{j+1}| is the convergence test.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

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
cudaError_t mg_vcycle(const tp_mg_s* mg, int l, void* x, const void* b, int x_zero, cudaStream_t s);
int mg_finest_level(const tp_mg_s* mg);
tp_precision mg_precision(const tp_mg_s* mg);
long long mg_finest_ndofs(const tp_mg_s* mg);
size_t elem_bytes(tp_precision p);
}  // namespace tp

struct tp_solver_s {
  tp_op_s* A = nullptr;
  tp_mg_s* mg = nullptr;
  int m = 30;
  long long n = 0;
  std::vector<double*> V, Z;
  double* w = nullptr;
  void* pb = nullptr;  // preconditioner input (mg precision)
  void* px = nullptr;  // preconditioner output
  double* partial = nullptr;
  double* dots = nullptr;
  int* flag = nullptr;  // device word of the zero test of the initial guess
  std::vector<double> history;
  int reorth = 0;  // second Gram-Schmidt passes in the last solve
  // the preconditioner V-cycle (fixed input pb, output px) captured once as a CUDA graph
  cudaGraphExec_t vcycle_graph = nullptr;
  bool graph_tried = false;
  int graph_launches = 0, direct_vcycles = 0;  // preconditioner applications of the current solve
};

using namespace tp;

static void solver_free(tp_solver_s* s) {
  for (double* p : s->V) if (p) cudaFree(p);
  for (double* p : s->Z) if (p) cudaFree(p);
  if (s->w) cudaFree(s->w);
  if (s->pb) cudaFree(s->pb);
  if (s->px) cudaFree(s->px);
  if (s->partial) cudaFree(s->partial);
  if (s->dots) cudaFree(s->dots);
  if (s->flag) cudaFree(s->flag);
  if (s->vcycle_graph) cudaGraphExecDestroy(s->vcycle_graph);
}

// Captures the V-cycle on a private stream (capture is not possible on the legacy default
// stream); returns false if capture is unavailable, in which case launches stay direct.
static bool capture_vcycle(tp_solver_s* s) {
  s->graph_tried = true;
  cudaStream_t cs;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return false;
  cudaGraph_t g = nullptr;
  bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  if (ok) {
    const cudaError_t e = tp::mg_vcycle(s->mg, tp::mg_finest_level(s->mg), s->px, s->pb, 1, cs);
    const cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    ok = e == cudaSuccess && e2 == cudaSuccess && g != nullptr;
  }
  if (ok) ok = cudaGraphInstantiate(&s->vcycle_graph, g, 0) == cudaSuccess;
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cs);
  cudaGetLastError();  // clear a failed capture
  if (!ok) s->vcycle_graph = nullptr;
  return ok;
}

static cudaError_t run_vcycle(tp_solver_s* s, cudaStream_t st) {
  if (!s->graph_tried) capture_vcycle(s);
  if (s->vcycle_graph) {
    ++s->graph_launches;
    return cudaGraphLaunch(s->vcycle_graph, st);
  }
  ++s->direct_vcycles;
  return tp::mg_vcycle(s->mg, tp::mg_finest_level(s->mg), s->px, s->pb, 1, st);
}

extern "C" {

tp_status tp_fgmres_create(tp_solver* out, tp_op A, tp_mg mg, int restart) {
  if (!out) { set_error("tp_fgmres_create: out is NULL"); return TP_ERR_INVALID_ARG; }
  *out = nullptr;
  if (!A || A->prec != TP_FP64) { set_error("tp_fgmres_create: A must be an FP64 operator"); return TP_ERR_INVALID_ARG; }
  if (restart < 1 || restart > 256) { set_error("tp_fgmres_create: restart must be in [1, 256]"); return TP_ERR_INVALID_ARG; }
  if (mg && mg_finest_ndofs(mg) != A->ndofs) { set_error("tp_fgmres_create: preconditioner size differs from A"); return TP_ERR_INVALID_ARG; }
  tp_solver_s* s = new (std::nothrow) tp_solver_s();
  if (!s) { set_error("tp_fgmres_create: out of host memory"); return TP_ERR_OOM; }
  s->A = A;
  s->mg = mg;
  s->m = restart;
  s->n = A->ndofs;
  const size_t bytes = sizeof(double) * (size_t)s->n;
  tp_status st = TP_OK;
  s->V.assign(restart + 1, nullptr);
  s->Z.assign(restart, nullptr);
  for (int i = 0; i <= restart && st == TP_OK; ++i) st = cuda_status(cudaMalloc(&s->V[i], bytes), "tp_fgmres_create: Krylov basis");
  for (int i = 0; i < restart && st == TP_OK; ++i) st = cuda_status(cudaMalloc(&s->Z[i], bytes), "tp_fgmres_create: flexible basis");
  if (st == TP_OK) st = cuda_status(cudaMalloc(&s->w, bytes), "tp_fgmres_create: work vector");
  if (st == TP_OK && mg) {
    const size_t pbytes = elem_bytes(mg_precision(mg)) * (size_t)s->n;
    st = cuda_status(cudaMalloc(&s->pb, pbytes), "tp_fgmres_create: preconditioner vectors");
    if (st == TP_OK) st = cuda_status(cudaMalloc(&s->px, pbytes), "tp_fgmres_create: preconditioner vectors");
  }
  if (st == TP_OK) st = cuda_status(cudaMalloc(&s->partial, sizeof(double) * (kMaxMulti + 1) * dot_blocks(s->n)), "tp_fgmres_create: scratch");
  if (st == TP_OK) st = cuda_status(cudaMalloc(&s->dots, sizeof(double) * 3 * (restart + 2)), "tp_fgmres_create: scratch");
  if (st == TP_OK) st = cuda_status(cudaMalloc(&s->flag, sizeof(int)), "tp_fgmres_create: scratch");
  if (st != TP_OK) {
    solver_free(s);
    delete s;
    return st;
  }
  *out = s;
  return TP_OK;
}

tp_status tp_solver_destroy(tp_solver s) {
  if (!s) return TP_OK;
  solver_free(s);
  delete s;
  return TP_OK;
}

}  // extern "C"

namespace {

// Scale of the FP16 V-cycle input relative to O(1) entries. The V-cycle approximates A^-1, whose
// gain on the smoothest mode is 1 / (lambda_1 m), lambda_1 ~ 3 pi^2 the smallest eigenvalue of
// (A, M (x) M (x) M) and m ~ hx hy hz / n^3 the mean row sum of the 3D mass matrix. The input is
// scaled by the largest power of two that keeps 8x that gain times O(1) entries below FP16's
// 65504, and by at most 1; smaller inputs would push the residuals into FP16's subnormal range.
double fp16_input_scale(const tp_op_s* A) {
  const double n3 = (double)A->n * A->n * A->n;
  const double pi = 3.14159265358979323846;
  const double gain = n3 / (3.0 * pi * pi * A->dir[0].h * A->dir[1].h * A->dir[2].h);
  const double s = 65504.0 / (8.0 * gain);
  return s >= 1.0 ? 1.0 : std::ldexp(1.0, (int)std::floor(std::log2(s)));
}

struct Ctx {
  tp_solver_s* s;
  cudaStream_t st;
};

cudaError_t dots_to_host(Ctx& c, const double* w, int nq, double* host) {
  std::vector<const double*> v(c.s->V.begin(), c.s->V.begin() + nq);
  cudaError_t e = multi_dot<double>(c.s->n, w, v.data(), nq, c.s->partial, c.s->dots, c.st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(host, c.s->dots, sizeof(double) * nq, cudaMemcpyDeviceToHost, c.st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.st);
  return e;
}

cudaError_t norm_to_host(Ctx& c, const double* w, double* out) {
  const double* v[1] = {w};
  cudaError_t e = multi_dot<double>(c.s->n, w, v, 1, c.s->partial, c.s->dots, c.st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, c.s->dots, sizeof(double), cudaMemcpyDeviceToHost, c.st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.st);
  if (e == cudaSuccess) *out = std::sqrt(*out);
  return e;
}

// out = b - A x (one pass where the operator's kernel stores the residual form itself), in FP64
// arithmetic: a double-word operator (tp_op_opts.dword) serves the Arnoldi products only
cudaError_t residual64(Ctx& c, double* out, const double* b, const double* x) {
  const tp_op_s* A = c.s->A;
  tp_op_s native;
  if (A->opts.dword) {
    native = *A;  // shares the constants and owns nothing
    native.opts.dword = 0;
    A = &native;
  }
  if (A->opts.kernel == TP_KERNEL_CUDA_CORE) return launch_residual(A, out, b, x, c.st);
  cudaError_t e = launch_apply(A, c.s->w, x, c.st);
  const double coef[2] = {1.0, -1.0};
  const double* v[2] = {b, c.s->w};
  if (e == cudaSuccess) e = multi_axpy<double>(c.s->n, out, 0.0, v, coef, 2, c.st);
  return e;
}

// *flag = 1 if any entry of x differs from zero (NaN included); every writer writes the same value.
__global__ void any_nonzero_kernel(const double* __restrict__ x, long long n, int* __restrict__ flag) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    if (!(x[i] == 0.0)) {
      *flag = 1;
      return;
    }
}

// r0 = b - A x0; a zero initial guess (the usual x0 = 0) gives r0 = b without an apply, exactly as
// the apply would (A 0 = 0 and b - 0 = b in floating point).
cudaError_t initial_residual(Ctx& c, double* out, const double* b, const double* x) {
  cudaError_t e = cudaMemsetAsync(c.s->flag, 0, sizeof(int), c.st);
  if (e == cudaSuccess) {
    any_nonzero_kernel<<<stream_blocks(c.s->n), 256, 0, c.st>>>(x, c.s->n, c.s->flag);
    e = cudaGetLastError();
  }
  int nz = 1;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&nz, c.s->flag, sizeof(int), cudaMemcpyDeviceToHost, c.st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.st);
  if (e != cudaSuccess) return e;
  if (nz) return residual64(c, out, b, x);
  return cudaMemcpyAsync(out, b, sizeof(double) * c.s->n, cudaMemcpyDeviceToDevice, c.st);
}

}  // namespace

extern "C" tp_status tp_fgmres_solve(tp_solver s, double* x, const double* b, double rtol, int maxit,
                                     tp_solve_info* info, void* stream) {
  if (info) memset(info, 0, sizeof(*info));
  if (!s || !x || !b) { set_error("tp_fgmres_solve: NULL argument"); return TP_ERR_INVALID_ARG; }
  if (((uintptr_t)x & 15) || ((uintptr_t)b & 15)) { set_error("tp_fgmres_solve: vectors must be 16-byte aligned"); return TP_ERR_INVALID_ARG; }
  if (!(rtol > 0) || maxit < 1) { set_error("tp_fgmres_solve: rtol must be > 0 and maxit >= 1"); return TP_ERR_INVALID_ARG; }
  Ctx c{s, (cudaStream_t)stream};
  const int m = s->m;
  const long long n = s->n;
  const double pscale = std::sqrt((double)n);  // v_j has unit norm: scale to O(1) entries for low precision
  s->history.clear();
  s->reorth = 0;
  s->graph_launches = s->direct_vcycles = 0;
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m), h(m + 2), h2(m + 2);
  auto Hij = [&](int i, int j) -> double& { return H[(size_t)i * m + j]; };
  int its = 0, restarts = 0, converged = 0;
  double beta0 = 0.0, rel = 1.0;
  cudaError_t e = initial_residual(c, s->V[0], b, x);
  if (e == cudaSuccess) e = norm_to_host(c, s->V[0], &beta0);
  if (e != cudaSuccess) return cuda_status(e, "tp_fgmres_solve");
  if (!std::isfinite(beta0)) { set_error("tp_fgmres_solve: non-finite initial residual"); return TP_ERR_NONFINITE; }
  s->history.push_back(1.0);
  tp_status status = TP_OK;
  if (beta0 == 0.0) converged = 1;
  double beta = beta0;
  while (!converged && its < maxit && status == TP_OK) {
    if (restarts > 0) {
      e = residual64(c, s->V[0], b, x);
      if (e == cudaSuccess) e = norm_to_host(c, s->V[0], &beta);
      if (e != cudaSuccess) { status = cuda_status(e, "tp_fgmres_solve"); break; }
      if (beta <= rtol * beta0) { converged = 1; break; }
    }
    {
      const double c1[1] = {1.0 / beta};
      const double* v[1] = {s->V[0]};
      e = multi_axpy<double>(n, s->V[0], 0.0, v, c1, 1, c.st);
    }
    std::fill(H.begin(), H.end(), 0.0);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int jend = 0;
    for (int j = 0; j < m && e == cudaSuccess; ++j) {
      // z_j = M^{-1} v_j
      if (s->mg) {
        const tp_precision mp = mg_precision(s->mg);
        // FP16 keeps FP32's precision over a range of only 2^-24..65504: the V-cycle's gain on
        // smooth components (up to 1/lambda_min(A)) must not overflow its output
        const double sc = mp == TP_FP16 ? pscale * fp16_input_scale(s->A) : pscale;
        switch (mp) {
          case TP_FP64:
            e = convert<double, double>(n, (double*)s->pb, s->V[j], sc, c.st);
            if (e == cudaSuccess) e = run_vcycle(s, c.st);
            if (e == cudaSuccess) e = convert<double, double>(n, s->Z[j], (const double*)s->px, 1.0 / sc, c.st);
            break;
          case TP_FP32:
            e = convert<float, double>(n, (float*)s->pb, s->V[j], sc, c.st);
            if (e == cudaSuccess) e = run_vcycle(s, c.st);
            if (e == cudaSuccess) e = convert<double, float>(n, s->Z[j], (const float*)s->px, 1.0 / sc, c.st);
            break;
          case TP_FP16:
            e = convert<__half, double>(n, (__half*)s->pb, s->V[j], sc, c.st);
            if (e == cudaSuccess) e = run_vcycle(s, c.st);
            if (e == cudaSuccess) e = convert<double, __half>(n, s->Z[j], (const __half*)s->px, 1.0 / sc, c.st);
            break;
          default:
            e = convert<__nv_bfloat16, double>(n, (__nv_bfloat16*)s->pb, s->V[j], sc, c.st);
            if (e == cudaSuccess) e = run_vcycle(s, c.st);
            if (e == cudaSuccess)
              e = convert<double, __nv_bfloat16>(n, s->Z[j], (const __nv_bfloat16*)s->px, 1.0 / sc, c.st);
            break;
        }
      } else {
        e = cudaMemcpyAsync(s->Z[j], s->V[j], sizeof(double) * n, cudaMemcpyDeviceToDevice, c.st);
      }
      if (e == cudaSuccess) e = launch_apply(s->A, s->w, s->Z[j], c.st);
      // classical Gram-Schmidt with one re-orthogonalization pass; the coefficients stay on the
      // device (h at dots[0..j], h2 at dots[m+1..], |w|^2 after pass 3), one host read per step:
      //   pass 1: h = V^T w;  pass 2: w -= V h, h2 = V^T w;  pass 3: w -= V h2, |w|^2;  v_{j+1} = w/|w|
      std::vector<const double*> vj(s->V.begin(), s->V.begin() + j + 1);
      double* d_h = s->dots;
      double* d_h2 = s->dots + (m + 1);
      double* d_n = s->dots + 2 * (m + 1);
      if (e == cudaSuccess) e = multi_dot<double>(n, s->w, vj.data(), j + 1, s->partial, d_h, c.st);
      if (e == cudaSuccess) e = multi_axpy_dot<double>(n, s->w, vj.data(), d_h, j + 1, 1, s->partial, d_h2, c.st);
      if (e == cudaSuccess) e = multi_axpy_dot<double>(n, s->w, vj.data(), d_h2, j + 1, 0, s->partial, d_n, c.st);
      if (e == cudaSuccess) e = scale_inv_sqrt<double>(n, s->V[j + 1], s->w, d_n + j + 1, c.st);
      std::vector<double> hostd(3 * (m + 2));
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(hostd.data(), s->dots, sizeof(double) * 3 * (m + 2), cudaMemcpyDeviceToHost, c.st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(c.st);
      if (e != cudaSuccess) break;
      ++s->reorth;
      for (int i = 0; i <= j; ++i) h[i] = hostd[i] + hostd[m + 1 + i];
      const double hn = std::sqrt(hostd[2 * (m + 1) + j + 1]);
      for (int i = 0; i <= j; ++i) Hij(i, j) = h[i];
      Hij(j + 1, j) = hn;
      bool finite = std::isfinite(hn);
      for (int i = 0; i <= j; ++i) finite = finite && std::isfinite(h[i]);
      if (!finite) {
        set_error("tp_fgmres_solve: non-finite value in the Arnoldi process (iteration %d)", its);
        status = TP_ERR_NONFINITE;
        break;
      }
      for (int i = 0; i < j; ++i) {
        const double t = cs[i] * Hij(i, j) + sn[i] * Hij(i + 1, j);
        Hij(i + 1, j) = -sn[i] * Hij(i, j) + cs[i] * Hij(i + 1, j);
        Hij(i, j) = t;
      }
      const double den = std::hypot(Hij(j, j), Hij(j + 1, j));
      cs[j] = den > 0 ? Hij(j, j) / den : 1.0;
      sn[j] = den > 0 ? Hij(j + 1, j) / den : 0.0;
      Hij(j, j) = den;
      Hij(j + 1, j) = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++its;
      jend = j + 1;
      rel = std::fabs(g[j + 1]) / beta0;
      s->history.push_back(rel);
      if (rel <= rtol) { converged = 1; break; }
      if (its >= maxit || hn == 0.0) break;
    }
    if (e != cudaSuccess) { status = cuda_status(e, "tp_fgmres_solve"); break; }
    if (status != TP_OK) break;
    for (int i = jend - 1; i >= 0; --i) {
      double sum = g[i];
      for (int k2 = i + 1; k2 < jend; ++k2) sum -= Hij(i, k2) * y[k2];
      y[i] = sum / Hij(i, i);
    }
    {
      std::vector<const double*> v(s->Z.begin(), s->Z.begin() + jend);
      e = multi_axpy<double>(n, x, 1.0, v.data(), y.data(), jend, c.st);
      if (e != cudaSuccess) { status = cuda_status(e, "tp_fgmres_solve"); break; }
    }
    if (!converged) ++restarts;
  }
  double true_rel = NAN;
  if (status == TP_OK || status == TP_ERR_NOT_CONVERGED) {
    double rn = 0.0;
    e = residual64(c, s->V[0], b, x);
    if (e == cudaSuccess) e = norm_to_host(c, s->V[0], &rn);
    if (e != cudaSuccess) status = cuda_status(e, "tp_fgmres_solve");
    true_rel = beta0 > 0 ? rn / beta0 : 0.0;
  }
  if (info) {
    info->iterations = its;
    info->restarts = restarts;
    info->converged = converged;
    info->rel_residual = rel;
    info->true_rel_residual = true_rel;
    info->history = s->history.data();
    info->history_len = (int)s->history.size();
    info->reorthogonalizations = s->reorth;
    info->vcycle_graph = s->graph_launches > 0 && s->direct_vcycles == 0;
  }
  if (status == TP_OK && !converged) {
    set_error("tp_fgmres_solve: not converged after %d iterations (relative residual %.3e)", its, rel);
    return TP_ERR_NOT_CONVERGED;
  }
  return status;
}

namespace tp {
long long solver_ndofs(const tp_solver_s* s) { return s->n; }
const void* solver_mg(const tp_solver_s* s) { return s->mg; }

// Captures the preconditioner's V-cycle graph ahead of the first solve (used by batched
// set-up so that capture happens outside the timed, multi-threaded solve phase).
void fgmres_prepare(tp_solver_s* s) {
  if (s && s->mg && !s->graph_tried) capture_vcycle(s);
}
}  // namespace tp
