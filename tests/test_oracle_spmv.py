"""The C/OpenMP CSR SpMV used for the CPU baseline computes y = A x of the
oracle's assembled matrix: pinned against the dense product of the same
matrix and against SciPy, with one thread and with several."""
import numpy as np

from oracle.sipg import Mesh, assemble
from oracle.spmv import csr_arrays, csr_spmv_omp, omp_threads
from tp_synth import uniform_vector


def test_csr_spmv_matches_dense_product():
    A = assemble(Mesh(3, 2, 2), 2)
    x = uniform_vector(A.shape[0], seed=3)
    ref = A.toarray() @ x
    arr = csr_arrays(A)
    for threads in (1, 3, 0):
        y = csr_spmv_omp(arr, x, threads=threads)
        assert np.linalg.norm(y - ref) <= 1e-14 * np.linalg.norm(ref)
    assert np.array_equal(csr_spmv_omp(arr, x, threads=1), csr_spmv_omp(arr, x, threads=2))
    assert omp_threads() >= 1


def test_csr_spmv_matches_scipy_on_the_8cubed_workload():
    A = assemble(Mesh(8, 8, 8), 3)
    x = uniform_vector(A.shape[0], seed=0)
    y = csr_spmv_omp(csr_arrays(A), x)
    ref = A @ x
    assert np.linalg.norm(y - ref) <= 1e-14 * np.linalg.norm(ref)
