/*
 * CSR sparse matrix-vector product y = A x over the oracle's assembled SIPG
 * matrix (oracle/sipg.py assemble: Sec. 2, Eq. (2) summed into CSR), rows
 * split across OpenMP threads. TEST INFRASTRUCTURE: it times the oracle on
 * all host cores for the CPU baseline of the 8^3-cell apply; it computes
 * nothing the GPU path uses and shares no code with it.
 *
 * Plain definition: y_r = sum over p in [indptr[r], indptr[r+1]) of
 * data[p] * x[indices[p]], summed in index order, in double precision.
 */
#include <stdint.h>

#ifdef _OPENMP
#include <omp.h>
#endif

void oracle_csr_spmv(int64_t nrows, const int64_t* indptr, const int32_t* indices, const double* data,
                     const double* x, double* y, int threads) {
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel for schedule(static)
#endif
  for (int64_t r = 0; r < nrows; ++r) {
    double s = 0.0;
    for (int64_t p = indptr[r]; p < indptr[r + 1]; ++p) s += data[p] * x[indices[p]];
    y[r] = s;
  }
}

int oracle_csr_threads(void) {
#ifdef _OPENMP
  int t = 0;
#pragma omp parallel
  {
#pragma omp master
    t = omp_get_num_threads();
  }
  return t;
#else
  return 1;
#endif
}
