/*
 * submat_debug.h -- test hooks of the submatrix library.
 *
 * These entry points exercise one kernel in isolation so that tests can
 * compare it with a plain reference of the same operation.  They are not
 * steps of the density-matrix path.  Conventions (status codes, streams,
 * submat_last_error) are those of submat.h.
 */
#ifndef SUBMAT_DEBUG_H
#define SUBMAT_DEBUG_H

#include "submat.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Grouped BF16 tensor-core GEMM (the Newton-Schulz product engine):
 *   C_s = A_s B_s^T,  s = 0..count-1,
 * for square matrices stored back to back as [count][ld][ld] on the device.
 *   ld     leading dimension, a multiple of 64 (<= 8192)
 *   n      logical dimension (n <= ld); only used for the residual
 *   A_hi, A_lo, B_hi, B_lo   device BF16 arrays [count][ld][ld]; the *_lo may be
 *          NULL when split == 0
 *   split  0: C = A_hi B_hi^T;  1: C = A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T
 *   sym    1: only tiles with ti <= tj are computed and each is mirrored
 *          (B must then be symmetric and A B^T symmetric)
 *   C      device FP32 [count][ld][ld] (output)
 *   res2   device double[count] or NULL: accumulates ||C_s - I_n||_F^2
 *   skip_arrive  test hook: nonzero makes the epilogue withhold its release
 *          of the accumulator, so a bounded wait must expire
 *   timeout_s    limit of each device wait (seconds; <= 0 selects 2 s)
 *   tile_n       output tile width: 128 or 256 (0 selects 128)
 * Returns OK, INVALID_ARG, TIMEOUT (a bounded wait expired; the kernel freed
 * its resources and returned), CUDA.
 */
submat_status submat_debug_tc_gemm(int count, int ld, int n, const void* A_hi, const void* A_lo,
                                   const void* B_hi, const void* B_lo, int split, int sym,
                                   float* C, double* res2, int skip_arrive, double timeout_s,
                                   int tile_n, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SUBMAT_DEBUG_H */
