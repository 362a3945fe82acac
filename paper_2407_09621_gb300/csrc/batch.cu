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
long long solver_ndofs(const tp_solver_s* s);
const void* solver_mg(const tp_solver_s* s);
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

namespace {

// One FGMRES solve per entry, run by `streams` host worker threads with one non-blocking CUDA stream
// each, taking entries from a shared queue ordered by size (largest first). zero_x: start from
// x = 0 (else the given x is the initial guess). Returns the first hard failure (not-converged
// solves only report it in their status).
tp_status run_concurrent(int count, tp_solver_s* const* solvers, double* const* x, const double* const* b,
                         const long long* ndofs, double rtol, int maxit, int streams, bool zero_x,
                         tp_solve_info* infos, tp_status* statuses, double* seconds, double* total_seconds) {
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return ndofs[a] > ndofs[c]; });
  std::atomic<int> next{0};
  std::mutex err_mu;
  tp_status worker_status = TP_OK;
  char worker_err[512] = "";
  int device = 0;
  cudaGetDevice(&device);
  const int nthreads = std::min(streams, count);
  const auto t0 = std::chrono::steady_clock::now();
  auto worker = [&]() {
    cudaSetDevice(device);
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      std::lock_guard<std::mutex> lock(err_mu);
      worker_status = TP_ERR_CUDA;
      snprintf(worker_err, sizeof(worker_err), "batched solve: stream creation failed");
      return;
    }
    for (;;) {
      const int q = next.fetch_add(1);
      if (q >= count) break;
      const int i = order[q];
      const auto ts = std::chrono::steady_clock::now();
      tp_solve_info info;
      memset(&info, 0, sizeof(info));
      tp_status r = zero_x ? cuda_status(cudaMemsetAsync(x[i], 0, sizeof(double) * ndofs[i], s), "batched solve")
                           : TP_OK;
      if (r == TP_OK) r = tp_fgmres_solve(solvers[i], x[i], b[i], rtol, maxit, &info, s);
      const auto te = std::chrono::steady_clock::now();
      if (infos) infos[i] = info;
      if (statuses) statuses[i] = r;
      if (seconds) seconds[i] = std::chrono::duration<double>(te - ts).count();
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
  if (worker_status != TP_OK) set_error("%s", worker_err);
  return worker_status;
}

}  // namespace

extern "C" tp_status tp_batch_solve(const tp_batch_problem* probs, int count, const tp_batch_opts* opts,
                                    tp_batch_result* results, double* total_seconds) {
  if (!probs || count < 1 || !results) {
    set_error("tp_batch_solve: need problems, count >= 1 and a results array");
    return TP_ERR_INVALID_ARG;
  }
  tp_batch_opts o{TP_FP32, TP_KERNEL_CUDA_CORE, 0, 30, 1e-10, 300, 8, 0, TP_SMOOTHER_CHEBYSHEV};
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
    tp_mg_opts mo{3, 15.0, 1.1, 0.0, 4, o.mg_precision, 20, o.kernel, o.ec, TP_FP16, o.smoother};
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
  std::vector<tp_solver_s*> sol(count);
  std::vector<double*> xs(count);
  std::vector<const double*> bs(count);
  std::vector<long long> nd(count);
  std::vector<tp_solve_info> infos(count);
  std::vector<tp_status> sts(count, TP_OK);
  std::vector<double> secs(count, 0.0);
  for (int i = 0; i < count; ++i) {
    sol[i] = items[i].solver;
    xs[i] = items[i].x;
    bs[i] = items[i].b;
    nd[i] = items[i].ndofs;
  }
  tp_status worker_status = run_concurrent(count, sol.data(), xs.data(), bs.data(), nd.data(), o.rtol, o.maxit,
                                           o.streams, true, infos.data(), sts.data(), secs.data(), total_seconds);
  char worker_err[512] = "";
  if (worker_status != TP_OK) snprintf(worker_err, sizeof(worker_err), "%s", tp_last_error());
  for (int i = 0; i < count; ++i) {
    results[i].iterations = infos[i].iterations;
    results[i].converged = infos[i].converged;
    results[i].true_rel_residual = infos[i].true_rel_residual;
    results[i].seconds = secs[i];
    results[i].status = sts[i];
  }
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

extern "C" tp_status tp_batch_solve_solvers(const tp_solver* solvers, double* const* x, const double* const* b,
                                            int count, const tp_batch_opts* opts, tp_solve_info* infos,
                                            tp_status* statuses, double* total_seconds) {
  if (!solvers || !x || !b || count < 1) {
    set_error("tp_batch_solve_solvers: need solvers, x and b arrays and count >= 1");
    return TP_ERR_INVALID_ARG;
  }
  tp_batch_opts o{TP_FP32, TP_KERNEL_CUDA_CORE, 0, 30, 1e-10, 300, 8, 0, TP_SMOOTHER_CHEBYSHEV};
  if (opts) o = *opts;
  if (o.streams < 1 || o.streams > 64 || !(o.rtol > 0) || o.maxit < 1) {
    set_error("tp_batch_solve_solvers: invalid options (streams 1..64, rtol > 0, maxit >= 1)");
    return TP_ERR_INVALID_ARG;
  }
  std::vector<long long> nd(count);
  for (int i = 0; i < count; ++i) {
    if (!solvers[i] || !x[i] || !b[i]) {
      set_error("tp_batch_solve_solvers: NULL solver or vector at entry %d", i);
      return TP_ERR_INVALID_ARG;
    }
    nd[i] = solver_ndofs(solvers[i]);
  }
  // solvers run concurrently: each must own its state (no solver or multigrid object twice)
  std::vector<const void*> owners;
  for (int i = 0; i < count; ++i) {
    owners.push_back(solvers[i]);
    if (solver_mg(solvers[i])) owners.push_back(solver_mg(solvers[i]));
  }
  std::sort(owners.begin(), owners.end());
  if (std::adjacent_find(owners.begin(), owners.end()) != owners.end()) {
    set_error("tp_batch_solve_solvers: a solver or multigrid object appears twice in the batch");
    return TP_ERR_INVALID_ARG;
  }
  for (int i = 0; i < count; ++i) fgmres_prepare(solvers[i]);
  tp_status st = cuda_status(cudaDeviceSynchronize(), "tp_batch_solve_solvers set-up");
  if (st != TP_OK) return st;
  return run_concurrent(count, const_cast<tp_solver_s* const*>(solvers), x, b, nd.data(), o.rtol, o.maxit, o.streams,
                        false, infos, statuses, nullptr, total_seconds);
}
