"""CPU FP64 oracle for the SIPG DG-Laplace operator and its multigrid/FGMRES solve.

TEST INFRASTRUCTURE ONLY. This package is a plain, slow, obviously-correct
restatement of what the GPU library computes, used to check it. Only the
test suite (``tests/``), ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import it. It shares no code with the CUDA library
(``paper_2407_09621_gb300``) and never imports it.

Modules (each function cites the passage of the paper it follows; section,
equation and algorithm numbers are those of the paper's LaTeX source):

* ``basis``   -- Gauss-Lobatto Lagrange basis, Gauss-Legendre quadrature (Sec. 2).
* ``sipg``    -- 1D element/face matrices, Kronecker assembly of the global
                 SIPG matrix (Sec. 2 Eq. (2); Sec. 2.1 Eq. (9)), block apply.
* ``brute``   -- brute-force 3D quadrature assembly of Eq. (2) on tiny meshes.
* ``solve``   -- exact discrete solve by fast diagonalization, right-hand
                 side and L2 error of the Poisson problem (Sec. 7.2).
* ``mg``      -- transfer operators, Chebyshev-Jacobi smoother, Algorithm 2
                 V-cycle and flexible GMRES (Sec. 7).
* ``schwarz`` -- vertex-patch multiplicative Schwarz smoother (Sec. 7.1).
* ``patchwise`` -- the operator evaluated patch by patch over vertex patches
                 (Sec. 2.1, Eq. (9) with 2(k+1)-point 1D patch factors).
* ``spmv``, ``spmv_omp.c`` -- CSR SpMV of the assembled matrix through SciPy
                 (one core) and plain C/OpenMP (all host cores), used only to
                 time the oracle for the CPU baseline.

The error correction of Algorithm 1 has no oracle function: its GPU results
are checked against the FP64 oracle's products directly.

Parity status of every function is stated in its module header.
"""
