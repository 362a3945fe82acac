// Batched Poisson solves of uneven sizes and degrees (the batching pattern of
// the solve of Sec. 7: many independent problems through one GPU).
//
// Every problem gets its own FP64 operator, multigrid hierarchy (low
// precision) and FGMRES solver at set-up; the solve phase runs the problems
// concurrently: `streams` host worker threads, each with its own non-blocking
// CUDA stream, take problems from a shared queue ordered by size (largest
// first, so the tail is made of small problems), and every preconditioner
// application is one launch of the V-cycle's captured CUDA graph. Small
// problems, which cannot fill the GPU on their own, overlap with each other.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "tp_internal.h"

namespace tp {
tp_status cuda_status(int err, const char* what);
void fgmres_prepare(tp_solver_s* s);
}  // namespace tp

using namespace tp;

namespace {

struct Item {
  tp_mesh mesh = nullptr;
  tp_op op = nullptr;
  tp_mg mg = nullptr;
  tp_solver solver = nullptr;
  double* b = nullptr;
  double* x = nullptr;
  bool own_x = false;
  long long ndofs = 0;
};

void release(Item& it) {
  if (it.solver) tp_solver_destroy(it.solver);
  if (it.mg) tp_mg_destroy(it.mg);
  if (it.op) tp_op_destroy(it.op);
  if (it.mesh) tp_mesh_destroy(it.mesh);
  if (it.b) cudaFree(it.b);
  if (it.own_x && it.x) cudaFree(it.x);
  it = Item();
}

}  // namespace

extern "C" tp_status tp_batch_solve(const tp_batch_problem* probs, int count, const tp_batch_opts* opts,
                                    tp_batch_result* results, double* total_seconds) {
  if (!probs || count < 1 || !results) {
    set_error("tp_batch_solve: need problems, count >= 1 and a results array");
    return TP_ERR_INVALID_ARG;
  }
  tp_batch_opts o{TP_FP32, TP_KERNEL_CUDA_CORE, 0, 30, 1e-10, 300, 8, 0};
  if (opts) o = *opts;
  if (o.streams < 1 || o.streams > 64 || o.restart < 1 || !(o.rtol > 0) || o.maxit < 1) {
    set_error("tp_batch_solve: invalid options (streams 1..64, restart >= 1, rtol > 0, maxit >= 1)");
    return TP_ERR_INVALID_ARG;
  }
  memset(results, 0, sizeof(tp_batch_result) * count);
  std::vector<Item> items(count);
  tp_status st = TP_OK;
  // ---- set-up (not timed)
  for (int i = 0; i < count && st == TP_OK; ++i) {
    const tp_batch_problem& p = probs[i];
    Item& it = items[i];
    st = tp_mesh_create(&it.mesh, p.nx, p.ny, p.nz, 1.0, 1.0, 1.0);
    const tp_op_opts oo{TP_PENALTY_CONFIG, TP_KERNEL_AUTO, 0, TP_FP16, o.autotune};
    if (st == TP_OK) st = tp_dg_laplace_create(&it.op, it.mesh, p.k, TP_FP64, &oo);
    if (st != TP_OK) break;
    it.ndofs = it.op->ndofs;
    tp_mg_opts mo{3, 15.0, 1.1, 0.0, 4, o.mg_precision, 20, o.kernel, o.ec, TP_FP16};
    st = tp_mg_create(&it.mg, it.op, &mo);
    if (st == TP_OK) st = tp_fgmres_create(&it.solver, it.op, it.mg, o.restart);
    if (st == TP_OK) st = cuda_status(cudaMalloc(&it.b, sizeof(double) * it.ndofs), "tp_batch_solve");
    if (st == TP_OK) {
      if (p.x) {
        it.x = p.x;
      } else {
        st = cuda_status(cudaMalloc(&it.x, sizeof(double) * it.ndofs), "tp_batch_solve");
        it.own_x = true;
      }
    }
    if (st == TP_OK) st = tp_rhs_sines(it.op, it.b, p.nmodes, p.a, p.pqr, nullptr);
    if (st == TP_OK) fgmres_prepare(it.solver);
  }
  if (st == TP_OK) st = cuda_status(cudaDeviceSynchronize(), "tp_batch_solve set-up");
  if (st != TP_OK) {
    for (Item& it : items) release(it);
    return st;
  }
  // ---- concurrent solves (timed)
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return items[a].ndofs > items[b].ndofs; });
  std::atomic<int> next{0};
  std::mutex err_mu;
  tp_status worker_status = TP_OK;
  char worker_err[512] = "";
  int device = 0;
  cudaGetDevice(&device);
  const int nthreads = std::min(o.streams, count);
  const auto t0 = std::chrono::steady_clock::now();
  auto worker = [&]() {
    cudaSetDevice(device);
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      std::lock_guard<std::mutex> lock(err_mu);
      worker_status = TP_ERR_CUDA;
      snprintf(worker_err, sizeof(worker_err), "tp_batch_solve: stream creation failed");
      return;
    }
    for (;;) {
      const int q = next.fetch_add(1);
      if (q >= count) break;
      const int i = order[q];
      Item& it = items[i];
      const auto ts = std::chrono::steady_clock::now();
      tp_solve_info info;
      tp_status r = cuda_status(cudaMemsetAsync(it.x, 0, sizeof(double) * it.ndofs, s), "tp_batch_solve");
      if (r == TP_OK) r = tp_fgmres_solve(it.solver, it.x, it.b, o.rtol, o.maxit, &info, s);
      const auto te = std::chrono::steady_clock::now();
      results[i].iterations = info.iterations;
      results[i].converged = info.converged;
      results[i].true_rel_residual = info.true_rel_residual;
      results[i].seconds = std::chrono::duration<double>(te - ts).count();
      results[i].status = r;
      if (r != TP_OK && r != TP_ERR_NOT_CONVERGED) {
        std::lock_guard<std::mutex> lock(err_mu);
        if (worker_status == TP_OK) {
          worker_status = r;
          snprintf(worker_err, sizeof(worker_err), "%s", tp_last_error());
        }
      }
    }
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  };
  std::vector<std::thread> pool;
  for (int t = 0; t < nthreads; ++t) pool.emplace_back(worker);
  for (std::thread& t : pool) t.join();
  const auto t1 = std::chrono::steady_clock::now();
  if (total_seconds) *total_seconds = std::chrono::duration<double>(t1 - t0).count();
  // ---- errors against the manufactured solutions (not timed)
  for (int i = 0; i < count && worker_status == TP_OK; ++i) {
    const tp_batch_problem& p = probs[i];
    tp_status r = tp_l2_error_sines(items[i].op, items[i].x, p.nmodes, p.a, p.pqr, &results[i].l2_error, nullptr);
    if (r != TP_OK) { worker_status = r; snprintf(worker_err, sizeof(worker_err), "%s", tp_last_error()); }
  }
  for (Item& it : items) release(it);
  if (worker_status != TP_OK) {
    set_error("%s", worker_err);
    return worker_status;
  }
  return TP_OK;
}
