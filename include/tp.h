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
  TP_ERR_UNSUPPORTED = 7    /* valid request this build does not implement */
} tp_status;

typedef enum { TP_FP64 = 0, TP_FP32 = 1, TP_FP16 = 2, TP_BF16 = 3 } tp_precision;

/* Penalty of Eq. (2): (k+1)^2/h (default) or the paper's k(k+1)(1/h+ + 1/h-),
 * h the cell width normal to the face, on interior and boundary faces alike. */
typedef enum { TP_PENALTY_CONFIG = 0, TP_PENALTY_PAPER = 1 } tp_penalty;

/* Kernel family for tp_apply. AUTO picks the fastest measured family for the
 * precision; CUDA_CORE forces the FMA-pipe sum-factorization kernel (the
 * paper's CUDA-core comparator, App. A); TENSOR forces the tensor-core kernel. */
typedef enum { TP_KERNEL_AUTO = 0, TP_KERNEL_CUDA_CORE = 1, TP_KERNEL_TENSOR = 2 } tp_kernel;

typedef struct {
  int penalty;  /* tp_penalty */
  int kernel;   /* tp_kernel */
  int ec;       /* 1: error-corrected half-precision products (Algorithm 1) where supported */
} tp_op_opts;

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
} tp_op_info_t;

/* Uniform Cartesian mesh of [0,lx]x[0,ly]x[0,lz] with nx*ny*nz cells
 * (Sec. 2: cells mapped from the reference cube [0,1]^3). Host-only object.
 * Errors: TP_ERR_INVALID_ARG if out is NULL, a count < 1, a length <= 0 or
 * the DoF count would overflow 2^62. */
tp_status tp_mesh_create(tp_mesh* out, int nx, int ny, int nz, double lx, double ly, double lz);
tp_status tp_mesh_destroy(tp_mesh m);

/* SIPG Laplace operator of degree k on mesh m, for vectors of precision p,
 * on the current CUDA device (Sec. 2, Eq. (2) and Sec. 2.1, Eq. (9)).
 * 1 <= k <= 7. opts may be NULL (config penalty, AUTO kernel, no EC).
 * The 1D matrices are computed on the host in FP64 and uploaded once; the
 * library owns that device memory until tp_op_destroy. The mesh may be
 * destroyed after this call. Errors: TP_ERR_INVALID_ARG (k, p, opts),
 * TP_ERR_OOM, TP_ERR_CUDA, TP_ERR_UNSUPPORTED (kernel family not built for p). */
tp_status tp_dg_laplace_create(tp_op* out, tp_mesh m, int k, tp_precision p, const tp_op_opts* opts);
tp_status tp_op_get_info(tp_op op, tp_op_info_t* info);
tp_status tp_op_destroy(tp_op op);

/* y = A x: the matrix-free cell loop of Sec. 2.1 (gather, cell operation,
 * face operations, scatter) as one kernel launch, asynchronous on `stream`.
 * x and y are DEVICE pointers owned by the caller, ndofs entries of the
 * operator's precision in the layout above, 16-byte aligned, not
 * overlapping. Errors: TP_ERR_INVALID_ARG (NULL/unaligned/overlapping
 * pointers), TP_ERR_CUDA (launch failure). Ownership: nothing is retained. */
tp_status tp_apply(tp_op op, void* y, const void* x, void* stream);

/* y = A x with HOST vectors: copies x to a library-owned device buffer,
 * applies, copies y back, and synchronizes `stream` before returning.
 * Pinned host memory gives the fastest copies; pageable memory works.
 * The staging buffers (2*ndofs entries) are allocated on first use and kept
 * until tp_op_destroy. Errors as tp_apply, plus TP_ERR_OOM. */
tp_status tp_apply_host(tp_op op, void* y_host, const void* x_host, void* stream);

/* Text of the last error on the calling thread ("" if none). */
const char* tp_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* TP_H */
