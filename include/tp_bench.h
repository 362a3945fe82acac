/*
 * libtp_bench -- measurement support (not part of the method).
 *
 * A separate shared library (paper_2407_09621_gb300/libtp_bench.so), built
 * beside libtp.so by the same build step; the method's library does not
 * contain these functions.
 *
 * The paper reports arithmetic rates against the hardware peak of the pipe a
 * kernel runs on (Sec. 4.2, Sec. 6). The FP64 and FP32 FMA-pipe peaks of the
 * GPU are not published per part and clocks, so the library measures them
 * with a register-only kernel: every thread runs a fixed number of
 * independent fused multiply-add chains, no memory traffic except one store
 * per thread at the end.
 *
 * The tensor-core apply (apply_umma.cu) is shaped by how fast one thread can
 * issue tcgen05.mma products; tp_bench_umma_issue measures that rate.
 */
#ifndef TP_BENCH_H
#define TP_BENCH_H

#include "tp.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Measures the FMA-pipe throughput for precision p (TP_FP64: DFMA,
 * TP_FP32: FFMA) on the current device, on `stream` (NULL = default),
 * best of 5 timed launches after 2 warm-ups, CUDA-event timed.
 * *tflops receives flops/s / 1e12 (FMA = 2 flops). Allocates and frees a
 * small device buffer. Blocks until done. Errors: TP_ERR_INVALID_ARG (NULL
 * out, other precisions), TP_ERR_CUDA, TP_ERR_OOM; the message is in
 * tp_bench_last_error(). */
tp_status tp_bench_fma_peak(int precision, double* tflops, void* stream);

/* Measures the tcgen05.mma rate on the current device, on `stream`: one CTA
 * per SM in which `issuers` warps (1, 2 or 4; one thread each) issue 2048
 * products in all of M = 128, N = n (64, 128, 192 or 256), K = 16, FP16
 * operands of zeros, FP32 accumulation, each warp into its own TMEM columns
 * (n x issuers <= 512). A comes from shared memory (a_in_tmem = 0) or from
 * TMEM (a_in_tmem = 1, then n x issuers <= 448); B from shared memory.
 * *clk_per_mma receives the SM cycles per product of a CTA (issue of the
 * first product to completion of the last, over all its products), *tflops
 * the tensor rate over the whole GPU (best of 3 timed launches after 2
 * warm-ups, CUDA-event timed). Needs sm_103a. Allocates and frees small
 * device buffers; blocks until done. Every wait in the kernel is bounded
 * (1 s). Errors: TP_ERR_INVALID_ARG (NULL out, other n / issuers),
 * TP_ERR_TIMEOUT (a wait gave up), TP_ERR_CUDA, TP_ERR_OOM; the message is in
 * tp_bench_last_error(). */
tp_status tp_bench_umma_issue(int n, int issuers, int a_in_tmem, double* clk_per_mma, double* tflops,
                              void* stream);

/* Text of the last error of this library on the calling thread ("" if none). */
const char* tp_bench_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* TP_BENCH_H */
