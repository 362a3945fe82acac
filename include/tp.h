/*
 * libtp -- sum-factorized SIPG DG-Laplace operator on GB300 (sm_103a).
 *
 * C ABI of the library. Plain C types only: handles are opaque pointers,
 * vectors are raw pointers (device or host, as each call states), CUDA
 * streams are passed as `void*` holding a cudaStream_t (NULL = the legacy
 * default stream). No call throws; every call returns a tp_status and, on
 * failure, leaves a message for tp_last_error() (thread-local).
 *
 * Problem (Sec. 2 of "Acceleration of Tensor-Product Operations with Tensor
 * Cores"): -Laplace(u) = f in a box, u = 0 on its boundary (Eq. (1)),
 * discretized by the symmetric interior penalty method (Eq. (2), read with
 * jumps [[.]] where the printed form shows averages) with discontinuous
 * tensor-product polynomials of degree k on the Gauss-Lobatto points of a
 * uniform Cartesian hex mesh. On such a mesh the operator is the Kronecker
 * sum of Sec. 2.1, Eq. (9): A = L_z(x)M_y(x)M_x + M_z(x)L_y(x)M_x + M_z(x)M_y(x)L_x
 * with the 1D DG mass M and the 1D SIPG stiffness L (face terms included).
 *
 * Vector layout (every call): cell-major, n = k+1,
 *   g = ((cz*ny + cy)*nx + cx)*n^3 + (l*n + j)*n + i
 * where (i, j, l) are the x, y, z node indices of cell (cx, cy, cz); i is
 * fastest. Element type = the operator's precision (double, float, IEEE
 * half, bfloat16).
 */
#ifndef TP_H
#define TP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TP_OK = 0,
  TP_ERR_INVALID_ARG = 1,   /* bad handle, size, pointer, alignment or aliasing */
  TP_ERR_CUDA = 2,          /* a CUDA runtime call failed; see tp_last_error() */
  TP_ERR_OOM = 3,           /* a library-owned allocation failed */
  TP_ERR_NONFINITE = 4,     /* a NaN/Inf was detected where the call checks for it */
  TP_ERR_NOT_CONVERGED = 5, /* an iterative solve stopped without reaching its tolerance */
  TP_ERR_TIMEOUT = 6,       /* a bounded device-side wait gave up */
  TP_ERR_UNSUPPORTED = 7    /* valid request the library does not implement */
} tp_status;

typedef enum { TP_FP64 = 0, TP_FP32 = 1, TP_FP16 = 2, TP_BF16 = 3 } tp_precision;

/* Penalty of Eq. (2): (k+1)^2/h (default) or the paper's k(k+1)(1/h+ + 1/h-),
 * h the cell width normal to the face, on interior and boundary faces alike. */
typedef enum { TP_PENALTY_CONFIG = 0, TP_PENALTY_PAPER = 1 } tp_penalty;

/* Kernel family for tp_apply. AUTO picks, per precision and degree, the family
 * that measured fastest on GB300: the tcgen05 tensor kernel for FP16/BF16
 * vectors at k = 3, the CUDA-core kernel otherwise (FP64: the DFMA kernel beats DMMA,
 * which shares the FP64 pipe; FP32: the CUDA-core kernel beats mma.sync).
 * CUDA_CORE forces the FMA-pipe sum-factorization kernel (the paper's CUDA-core
 * comparator, App. A); TENSOR forces the tensor-core kernel. PATCH evaluates the
 * operator patch-wise, the paper's form (Sec. 2.1): over the vertex patches of
 * 2 x 2 x 2 cells, each patch applying the Kronecker sum of Eq. (9) with 1D
 * factors of size N = 2(k+1) that hold its share of the cell integrals (half of
 * an interior cell's, all of a first or last cell's) and the faces it owns (the
 * face at its vertex, and the boundary faces in the first and last patch), the
 * patch results summed over eight colours of disjoint patches. The sum is the
 * same operator; every DoF is computed in up to eight patches, 224(k+1) + 8
 * flops per DoF. FP64 and FP32 vectors, k <= 7, at least two cells per
 * direction; on the FMA pipes. */
typedef enum { TP_KERNEL_AUTO = 0, TP_KERNEL_CUDA_CORE = 1, TP_KERNEL_TENSOR = 2, TP_KERNEL_PATCH = 3 } tp_kernel;

typedef struct {
  int penalty;  /* tp_penalty */
  int kernel;   /* tp_kernel */
  int ec;       /* error-corrected half-precision products, tensor kernel only: 0 off, 1 both
                   operands split (Algorithm 1), 2 the operator matrices only, 3 the vector-side
                   operand only (the FP32 vector and the intermediate W; with FP16/BF16 vectors
                   the vector is exact, so 3 is 0 for FP16 and 1 for BF16, which always splits) */
  int tc_type;  /* operand type of the tensor kernel: TP_FP16 (default) or TP_BF16; for FP16/BF16
                   vectors it must equal the vector type */
  int autotune; /* 1: at creation, time the tile shapes of the apply kernel (CUDA-core and DMMA:
                   cells per thread block, the default halved, kept or doubled) on this device on a
                   proxy of the mesh (same nx, ny, about 128 MB per vector) and keep the fastest.
                   Results do not depend on the tile shape. 0 (default): the default shape, halved
                   for meshes with fewer cells than two default blocks per SM */
  int dword;    /* FP64 vectors on the CUDA-core kernel (k <= 7): 1 = double-word FP32 arithmetic:
                   every FP64 value is split on load into an unevaluated sum of two FP32 numbers
                   (about 48 significand bits) and the contractions and face terms run as
                   error-free FP32 transformations on the FMA pipe, the result joined back to FP64
                   on store. On GB300, whose FP64 pipe delivers ~1.25 TFLOP/s against ~75 for FP32,
                   this is ~3.5-4x the FP64 kernel's rate; the relative error per apply is ~1e-14
                   (FP64 arithmetic: ~1e-15), inside the 1e-12 FP64 tolerance. Inputs of magnitude
                   below 2^-126 are taken as 0, below 2^-74 with 24 significand bits, and above
                   2^127 are out of range. 0 (default): FP64 arithmetic on the DFMA pipe.
                   No tile autotuning with 1 (one tile shape) */
} tp_op_opts;

/* Tensor kernel (TP_KERNEL_TENSOR). With FP64 vectors (k = 3 and k = 7 only) the six 1D
 * contractions per cell run as `mma.sync.m8n8k4.f64` (DMMA) and the face terms on the FMA
 * pipe, FP64 throughout. For k = 3 with FP16/BF16 vectors it runs on the
 * Blackwell tensor cores (tcgen05.mma, operands staged by TMA, FP32 accumulators in
 * TMEM): each cell row of the output is the sum of seven dense 64 x 64 blocks of
 * Eq. (2)/(9) (the interior diagonal block and one per face neighbour) applied to
 * the cell's and its six neighbours' coefficients (zero outside the mesh), and a
 * second launch adds the rank-2 boundary-face corrections of boundary cells on
 * the FMA pipes in FP32 (so boundary entries are rounded to the storage type
 * twice); with ec = 1 (always for BF16) the blocks are split as in Algorithm 1. Otherwise `mma.sync` m16n8k16 with FP32 accumulation for
 * degrees k = 2, 3 (n <= 4, cells padded to 4^3): per cell W = K3 u with
 * K3 = G_z(+)G_y(+)G_x and V = (M_z(x)M_y(x)M_x) W as dense 64 x 64 products, the
 * rank-2 face terms added to W on the FMA pipes in FP32 between them. Vectors may
 * be FP16/BF16 (operands = storage) or FP32 (operands rounded to tc_type; with
 * ec = 1 every operand is split as in Algorithm 1: a = a_h + da*2^-s with
 * s = 11 for FP16 and 8 for BF16, and a*b = a_h b_h + (da b_h + a_h db)*2^-s).
 * BF16 vectors always use the split (8 significand bits are too few for the
 * 5e-3 per-apply tolerance otherwise).
 * FP32 vectors on the half-precision tensor paths reach FP32 accuracy (relative
 * l2 error <= 1e-5 per apply) only with FP16 operands and ec = 1. The other
 * combinations are APPROXIMATE operators (tp_op_info_t.approximate = 1): with
 * FP16 operands ec = 0 stays within 5e-3 and ec = 2 or 3 in between; with BF16
 * operands ec = 1 stays within 1e-4 and ec = 0 within 2e-2. */

typedef struct tp_mesh_s* tp_mesh;
typedef struct tp_op_s* tp_op;

typedef struct {
  long long ncells;       /* nx*ny*nz */
  long long ndofs;        /* ncells*(k+1)^3 */
  int k, n;               /* degree and nodes per direction */
  int precision;          /* tp_precision */
  int kernel;             /* tp_kernel family tp_apply will launch */
  size_t elem_bytes;      /* bytes per vector entry */
  double flops_per_dof;   /* algorithmic flops per DoF of one tp_apply (FMA = 2) */
  int tensor_path;        /* tensor kernel only: 1 = mma.sync f16/bf16, 2 = tcgen05 (TMA + TMEM),
                             3 = mma.sync f64 (DMMA); 0 for the CUDA-core and patch-wise kernels */
  int tile_cells;         /* cells per thread block (CUDA-core, DMMA; 8 for the patch-wise kernel: one
                             vertex patch) or per tile (tcgen05) of the apply launch; 0 for mma.sync */
  int approximate;        /* 1: FP32 vectors on a tensor path that does not reach FP32 accuracy
                             (see the tensor kernel note above); 0 otherwise */
  int dword;              /* 1: FP64 vectors in double-word FP32 arithmetic (tp_op_opts.dword) */
} tp_op_info_t;

/* Uniform Cartesian mesh of [0,lx]x[0,ly]x[0,lz] with nx*ny*nz cells
 * (Sec. 2: cells mapped from the reference cube [0,1]^3). Host-only object.
 * Errors: TP_ERR_INVALID_ARG if out is NULL, a count < 1, a length <= 0 or
 * the DoF count would overflow 2^62. */
tp_status tp_mesh_create(tp_mesh* out, int nx, int ny, int nz, double lx, double ly, double lz);
tp_status tp_mesh_destroy(tp_mesh m);

/* SIPG Laplace operator of degree k on mesh m, for vectors of precision p,
 * on the current CUDA device (Sec. 2, Eq. (2) and Sec. 2.1, Eq. (9)).
 * 1 <= k <= 15; degrees above 7 (n = k + 1 up to 16, the arbitrary-size
 * sweep of the paper's appendix) run on the CUDA-core kernel with FP64 or FP32
 * vectors only, and take no multigrid hierarchy and no tp_l2_error_sines.
 * opts may be NULL (config penalty, AUTO kernel, no EC).
 * The 1D matrices are computed on the host in FP64 and uploaded once; the
 * library owns that device memory until tp_op_destroy. The mesh may be
 * destroyed after this call. Errors: TP_ERR_INVALID_ARG (k, p, opts),
 * TP_ERR_OOM, TP_ERR_CUDA, TP_ERR_UNSUPPORTED (kernel family not built for p
 * and k, e.g. k > 7 with a tensor kernel or FP16/BF16 vectors). */
tp_status tp_dg_laplace_create(tp_op* out, tp_mesh m, int k, tp_precision p, const tp_op_opts* opts);
tp_status tp_op_get_info(tp_op op, tp_op_info_t* info);
tp_status tp_op_destroy(tp_op op);

/* y = A x: the matrix-free cell loop of Sec. 2.1 (gather, cell operation,
 * face operations, scatter) as one kernel launch, asynchronous on `stream`.
 * x and y are DEVICE pointers owned by the caller, ndofs entries of the
 * operator's precision in the layout above, 16-byte aligned, not
 * overlapping. The operator's device (current at its creation) must be the
 * current device. Errors: TP_ERR_INVALID_ARG (NULL/unaligned/overlapping
 * pointers, another device current), TP_ERR_CUDA (launch failure).
 * Ownership: nothing is retained. */
tp_status tp_apply(tp_op op, void* y, const void* x, void* stream);

/* y = A x with HOST vectors: copies x to a library-owned device buffer,
 * applies, copies y back, and synchronizes `stream` before returning.
 * Pinned host memory gives the fastest copies; pageable memory works.
 * The staging buffers (2*ndofs entries) are allocated on first use and kept
 * until tp_op_destroy. The operator's device must be current. Errors as
 * tp_apply, plus TP_ERR_OOM. */
tp_status tp_apply_host(tp_op op, void* y_host, const void* x_host, void* stream);

/* y = A x with HOST vectors, allocating no device memory. The paper has no
 * counterpart: this is for callers that cannot call cudaMalloc, such as a
 * process whose device memory is all handed out by its own fixed pool or
 * budget, or a caller that must not meet the allocator's latency or its
 * out-of-memory failure mid-run. Operator creation itself allocates nothing
 * on the device only for the CUDA-core kernel (TP_KERNEL_AUTO or
 * TP_KERNEL_CUDA_CORE resolving to it) with autotune = 0; the tensor kernels
 * allocate their operand matrices (mma.sync: 2 x 64 x 64 entries; tcgen05:
 * 7 or 14 blocks of 64 x 64 entries and one status word) and autotune = 1
 * allocates two proxy vectors of about 128 MB while it times the tile shapes.
 * Staging goes through one static device array of 2*TP_NOALLOC_MAX_BYTES
 * bytes (x half, y half) that every GPU loading the library holds until the
 * process exits. CUDA loads a library's device code lazily by default, so
 * the array is committed on a device by the first call on that device (or
 * when the library loads, with CUDA_MODULE_LOADING=EAGER): make that first
 * call before the caller's pool reserves the device's memory; if the array
 * cannot be placed, the call fails with TP_ERR_CUDA and a message saying so.
 * The first call on a device also looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and keeps it for the
 * process (the cached address does not survive cudaDeviceReset); make that
 * first call before any stream capture. Vectors larger than
 * TP_NOALLOC_MAX_BYTES bytes are rejected with TP_ERR_INVALID_ARG before any
 * GPU work, and so is a call made while another device than the operator's
 * is current. Every call shares the array: calls that overlap on the GPU
 * (other threads, other streams) race and must be serialized by the caller.
 * Each call overwrites both halves completely, so nothing carries over.
 * Synchronizes `stream` before returning. Errors as tp_apply_host (never
 * TP_ERR_OOM). */
#define TP_NOALLOC_MAX_BYTES (8 * 1024 * 1024)
tp_status tp_apply_host_noalloc(tp_op op, void* y_host, const void* x_host, void* stream);

/* Device status of the op's kernels. The tcgen05 apply (k = 3 with FP16/BF16
 * vectors on the tensor kernel) bounds every wait on its barriers; a wait that
 * gives up stores a nonzero code in a device word owned by the op and the
 * launch stops issuing work. This call synchronizes the device, reads and
 * clears that word, and returns TP_ERR_TIMEOUT (code in tp_last_error()) if it
 * was set, else TP_OK. Errors: TP_ERR_INVALID_ARG (NULL op), TP_ERR_CUDA. */
tp_status tp_op_check(tp_op op);


/* ------------------------------------------------------------------ multigrid
 * Geometric multigrid V-cycle of Algorithm 2 (Sec. 7.1) on the operator's box:
 * levels from uniform coarsening by 2 in every direction (while all cell
 * counts are even and one exceeds coarse_cells), the same degree and penalty
 * on every level, the operator rediscretized with that level's h.
 *  - smoother S_l, one of two (tp_mg_opts.smoother):
 *    TP_SMOOTHER_CHEBYSHEV (default): `degree` steps of Chebyshev iteration on
 *    D^{-1} A_l, D = diag(A_l), eigenvalue interval [lmax/ratio, lmax];
 *    TP_SMOOTHER_VERTEX_PATCH: the paper's multiplicative vertex-patch Schwarz
 *    smoother (Sec. 7.1): the 2x2x2-cell patches around interior vertices,
 *    coloured by vertex parity (8 colours, a colour's patches disjoint); per
 *    colour r = b - A_l x, then x_P += A_P^{-1} r_P on each of its patches,
 *    solved exactly by fast diagonalization of the patch's Kronecker-sum
 *    matrix. One sweep per smoothing step, colours ascending before and
 *    descending after the coarse correction (tp_mg_smooth: ascending); the
 *    patch solves compute in FP64 for FP64 vectors and in FP32 otherwise;
 *  - restriction I_down = P^T, prolongation I_up = P, the exact embedding of
 *    the coarse DG space into the fine one;
 *  - coarse solve A_0^{-1}: exact, in FP64, by fast diagonalization.
 * Vectors of the V-cycle have the multigrid precision: TP_FP64, TP_FP32, or
 * TP_FP16/TP_BF16 storage with FP32 arithmetic (the low-precision
 * preconditioners of Sec. 7.1; with TP_KERNEL_TENSOR and k = 3 the FP16/BF16
 * level operators run on tcgen05). Level 0 is the coarsest, level `levels-1`
 * the finest (the operator given at creation). FP16 spans only 2^-24..65504:
 * inside tp_fgmres_solve its V-cycle input is scaled by the largest power of
 * two (at most 1) that keeps the V-cycle's gain on the smoothest mode, about
 * n^3 / (3 pi^2 hx hy hz), from overflowing; BF16 has FP32's range. */
#define TP_MAX_LEVELS 16

#define TP_SMOOTHER_CHEBYSHEV 0
#define TP_SMOOTHER_VERTEX_PATCH 1

typedef struct tp_mg_s* tp_mg;

typedef struct {
  int degree;        /* Chebyshev degree per smoothing step (default 3) */
  double ratio;      /* lmax / lmin of the Chebyshev interval (default 15) */
  double safety;     /* factor applied to the estimated lmax (default 1.1) */
  double lmax;       /* > 0: use this bound on every level instead of estimating it */
  int coarse_cells;  /* stop coarsening once no direction has more cells (default 4) */
  int precision;     /* TP_FP64, TP_FP32 (default), TP_FP16 or TP_BF16 */
  int power_iters;   /* power iterations for the lmax estimate (default 20) */
  int kernel;        /* apply kernel of the level operators: TP_KERNEL_CUDA_CORE (default) or
                        TP_KERNEL_TENSOR (FP32/FP16/BF16 vectors, k = 2, 3; otherwise CUDA-core);
                        TP_KERNEL_PATCH is rejected (TP_ERR_UNSUPPORTED) */
  int ec;            /* tensor kernel with Algorithm 1 error correction */
  int tc_type;       /* tensor operand type: TP_FP16 (default) or TP_BF16 */
  int smoother;      /* TP_SMOOTHER_CHEBYSHEV (default) or TP_SMOOTHER_VERTEX_PATCH */
} tp_mg_opts;

typedef struct {
  int levels;
  int precision;
  int cells[TP_MAX_LEVELS][3];
  long long ndofs[TP_MAX_LEVELS];
  double lmax[TP_MAX_LEVELS];  /* smoother bound used on each level (0 on level 0) */
} tp_mg_info_t;

/* Builds the hierarchy below `finest` (which must outlive the hierarchy; its
 * mesh, degree and penalty are used, not its precision). opts may be NULL.
 * Allocates the level operators, vectors and scratch (owned until
 * tp_mg_destroy) and, unless opts->lmax > 0, estimates lmax(D^{-1}A_l) per
 * level by power iteration on the GPU (synchronizes the device).
 * The vertex-patch smoother estimates no lmax (lmax and ratio are unused).
 * Errors: TP_ERR_INVALID_ARG, TP_ERR_OOM, TP_ERR_CUDA, TP_ERR_NONFINITE,
 * TP_ERR_UNSUPPORTED (finest degree above 7; kernel TP_KERNEL_PATCH). */
tp_status tp_mg_create(tp_mg* out, tp_op finest, const tp_mg_opts* opts);
tp_status tp_mg_get_info(tp_mg mg, tp_mg_info_t* info);
/* Level operator (owned by the hierarchy; valid until tp_mg_destroy). */
tp_status tp_mg_level_op(tp_mg mg, int level, tp_op* op);
tp_status tp_mg_destroy(tp_mg mg);

/* One V-cycle (Algorithm 2) on the finest level: x <- Vcycle(A, x, b).
 * x (in/out, initial guess) and b are DEVICE vectors of the multigrid
 * precision and the finest level's size, 16-byte aligned. Asynchronous on
 * `stream`; uses the hierarchy's vectors, so calls on one hierarchy must not
 * overlap. */
tp_status tp_vcycle(tp_mg mg, void* x, const void* b, void* stream);
/* The steps of Algorithm 2 one at a time (same vector rules, level sizes):
 * smoothing x <- S_l(x, b) on level l >= 1; coarse = P^T fine (level l >= 1 is
 * the fine side); fine += P coarse; x = A_0^{-1} b on level 0. */
tp_status tp_mg_smooth(tp_mg mg, int level, void* x, const void* b, void* stream);
tp_status tp_mg_restrict(tp_mg mg, int level, void* coarse, const void* fine, void* stream);
tp_status tp_mg_prolongate_add(tp_mg mg, int level, void* fine, const void* coarse, void* stream);
tp_status tp_mg_coarse_solve(tp_mg mg, void* x, const void* b, void* stream);

/* ------------------------------------------------------------------ FGMRES
 * Flexible GMRES (Saad 1993) with right preconditioning, restarted every
 * `restart` iterations, in FP64 on the GPU (Sec. 7.1): Arnoldi vectors,
 * Gram-Schmidt orthogonalization (classical, with one re-orthogonalization
 * pass), the operator applications w = A z_j and the true residual at each
 * restart are FP64; the preconditioner is one V-cycle of `mg` in its own
 * precision with zero initial guess (the input is converted, scaled by
 * sqrt(ndofs), and the output converted back). Orthogonalization: classical
 * Gram-Schmidt with one re-orthogonalization pass in every step (with a good
 * preconditioner A M^-1 is close to the identity, so the first projection
 * cancels most of w and the second pass is always needed). Stops when the
 * Arnoldi residual norm drops below rtol * ||b - A x0||. */
typedef struct tp_solver_s* tp_solver;

typedef struct {
  int iterations;          /* preconditioned Arnoldi steps taken */
  int restarts;
  int converged;           /* 1 if the tolerance was met */
  double rel_residual;     /* final Arnoldi estimate ||r|| / ||r0|| */
  double true_rel_residual;/* ||b - A x|| / ||b - A x0|| recomputed in FP64 at the end */
  const double* history;   /* host array of relative residual estimates, one per iteration + 1;
                              owned by the solver, valid until the next solve or destroy */
  int history_len;
  int reorthogonalizations;/* Arnoldi steps with the second Gram-Schmidt pass (every step) */
  int vcycle_graph;        /* 1 if every preconditioner application of this solve was one launch of
                              the V-cycle's captured CUDA graph; 0 if the V-cycle ran as direct
                              launches (capture unavailable) or there is no preconditioner */
} tp_solve_info;

/* A: the FP64 operator (must be TP_FP64). mg: preconditioner built on A's
 * mesh (NULL: no preconditioner). With a double-word operator (tp_op_opts.dword)
 * the Arnoldi products A z_j use double-word arithmetic, while the initial
 * residual and the true residual at the end are evaluated in FP64 arithmetic.
 * Double-word products carry ~2^-48 relative to the operator's summed terms
 * (FP64: 2^-53), which for smooth Krylov vectors exceed A z by orders of
 * magnitude: the Arnoldi estimate then stops being trustworthy near 1e-10
 * (measured true residuals 1.5e-10 at k = 3, 128^3 and 2.4e-10 at k = 7, 64^3
 * for rtol = 1e-10), so tight tolerances want the FP64 operator. Allocates (restart+1)+restart+1 FP64
 * vectors of A's size plus two vectors of mg's precision. Errors:
 * TP_ERR_INVALID_ARG, TP_ERR_OOM, TP_ERR_CUDA. */
tp_status tp_fgmres_create(tp_solver* out, tp_op A, tp_mg mg, int restart);
/* Solves A x = b. x (in: initial guess, out: solution) and b are DEVICE FP64
 * vectors, 16-byte aligned. Runs on `stream` and synchronizes it (the
 * Arnoldi scalars are read on the host every iteration). Returns TP_OK when
 * converged, TP_ERR_NOT_CONVERGED after maxit iterations (x holds the last
 * iterate), TP_ERR_NONFINITE if a NaN/Inf appears in the Arnoldi process.
 * `info` (may be NULL) is filled in every case. */
tp_status tp_fgmres_solve(tp_solver s, double* x, const double* b, double rtol, int maxit, tp_solve_info* info,
                          void* stream);
tp_status tp_solver_destroy(tp_solver s);

/* ------------------------------------------------------------------ batched solves
 * Many independent Poisson problems of Sec. 7.2 type (manufactured sine-mode
 * solutions, see below) with uneven sizes and degrees solved together on one GPU:
 * every problem gets its own FP64 operator, low-precision multigrid and FGMRES at
 * set-up; the solves then run concurrently, `streams` host worker threads with one
 * CUDA stream each taking problems largest-first from a shared queue, every
 * preconditioner application being one launch of the V-cycle's captured CUDA graph. */
typedef struct {
  int nx, ny, nz;      /* cells of the unit-cube mesh */
  int k;               /* degree 1..7 */
  int nmodes;          /* manufactured solution sum_m a[m] sin(p pi x) sin(q pi y) sin(r pi z) */
  const double* a;     /* HOST, nmodes coefficients */
  const int* pqr;      /* HOST, 3*nmodes wave numbers >= 1 */
  double* x;           /* DEVICE FP64 output vector (ndofs) or NULL (solution discarded) */
} tp_batch_problem;

typedef struct {
  int mg_precision;    /* TP_FP32 (default) or TP_FP64 */
  int kernel;          /* level-operator kernel, as tp_mg_opts.kernel */
  int ec;              /* as tp_mg_opts.ec */
  int restart;         /* FGMRES restart (default 30) */
  double rtol;         /* relative residual target (default 1e-10) */
  int maxit;           /* per problem (default 300) */
  int streams;         /* concurrent worker streams (default 8; 1 = one after another) */
  int autotune;        /* 1: autotune every problem's apply tile shapes (tp_op_opts.autotune) */
  int smoother;        /* as tp_mg_opts.smoother (default TP_SMOOTHER_CHEBYSHEV) */
} tp_batch_opts;

typedef struct {
  int iterations, converged, status;  /* status: tp_status of that problem's solve */
  double true_rel_residual;
  double l2_error;                    /* || u_h - u ||_L2 against the manufactured solution */
  double seconds;                     /* wall time of that problem's solve */
} tp_batch_result;

/* Solves all problems (set-up and error evaluation are not part of *total_seconds,
 * the wall time of the concurrent solve phase). results: `count` entries, filled in
 * order. Allocates and frees all per-problem objects; blocks until done. Errors:
 * TP_ERR_INVALID_ARG, TP_ERR_OOM, TP_ERR_CUDA, or the first failing solve's status;
 * problems that only miss the tolerance report TP_ERR_NOT_CONVERGED in their result. */
tp_status tp_batch_solve(const tp_batch_problem* probs, int count, const tp_batch_opts* opts,
                         tp_batch_result* results, double* total_seconds);

/* Batched solves over the caller's own problems: entry i solves A_i x[i] = b[i] with
 * solvers[i] (its FP64 operator A_i and, optionally, its V-cycle preconditioner, built
 * by tp_fgmres_create on meshes and degrees of any size), x[i] the initial guess and
 * result, b[i] the right-hand side (DEVICE FP64 vectors of A_i's size, owned by the
 * caller). The solves run concurrently as in tp_batch_solve (opts: rtol, maxit and
 * streams are used; NULL = defaults). The solvers run at the same time, so no solver
 * and no multigrid object may appear twice. infos and statuses (count entries each,
 * may be NULL) receive each solve's tp_solve_info (its history stays owned by that
 * solver) and tp_status; *total_seconds (may be NULL) the wall time of the concurrent
 * phase. Blocks until done. Errors: TP_ERR_INVALID_ARG (NULL entries, duplicates,
 * options), TP_ERR_CUDA, or the first solve's hard failure; solves that only miss the
 * tolerance report TP_ERR_NOT_CONVERGED in statuses. */
tp_status tp_batch_solve_solvers(const tp_solver* solvers, double* const* x, const double* const* b, int count,
                                 const tp_batch_opts* opts, tp_solve_info* infos, tp_status* statuses,
                                 double* total_seconds);

/* ------------------------------------------------------------------ Poisson problem data
 * Manufactured problems of Sec. 7.2: u = sum_m a[m] sin(p pi x/lx) sin(q pi y/ly) sin(r pi z/lz)
 * with (p, q, r) = pqr[3m..3m+2] >= 1, 1 <= nmodes <= 16; on the unit cube the
 * single mode a = 1, (1, 1, 1) is the paper's u = sin(pi x) sin(pi y) sin(pi z).
 * u vanishes on the boundary (g = 0 in Eq. (1)). a and pqr are HOST arrays. */

/* b = load vector of f = -Laplace u (b_a = int f phi_a), DEVICE FP64 vector in
 * the operator's layout, computed per mode as a tensor product of 1D load
 * vectors (30-point Gauss per cell). Allocates and frees small device
 * buffers; synchronizes `stream`. */
tp_status tp_rhs_sines(tp_op op, double* b, int nmodes, const double* a, const int* pqr, void* stream);

/* *err = || u_h - u ||_L2 for the DEVICE FP64 coefficient vector u_h, by
 * per-cell tensor Gauss quadrature with k+4 points per direction (FP64).
 * Allocates a scratch array of ncells doubles; synchronizes `stream`.
 * TP_ERR_UNSUPPORTED for degrees above 7. */
tp_status tp_l2_error_sines(tp_op op, const double* u_h, int nmodes, const double* a, const int* pqr, double* err,
                            void* stream);

/* Text of the last error on the calling thread ("" if none). */
const char* tp_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* TP_H */
