/*
 * fno.h -- C ABI of the kernels of the learned warm start: a Fourier neural operator
 * (FNO) that maps problem parameters and the porosity field to an initial
 * (u_r, u_z, T) for the lattice Boltzmann solver of lbm.h.
 *
 * The paper has no counterpart for any of this: the warm start is an addition around
 * the paper's method, whose iteration always runs to convergence from the guess and
 * decides the result (Sec. 4 defines the problems it is trained on).
 *
 * All arrays are FP32 in device memory, row-major; the GEMM rounds its operands to
 * BF16 when it stages them and accumulates in FP32 on the tensor cores.  Every call
 * is asynchronous on `stream` (NULL = legacy default stream) and returns 0, or
 * FNO_ERR_INVALID for a bad argument, FNO_ERR_CUDA for a failed launch;
 * fno_last_error() gives the message.  No call allocates device memory.
 */
#ifndef FNO_H
#define FNO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FNO_OK 0
#define FNO_ERR_INVALID 1
#define FNO_ERR_CUDA 2

/* Batched GEMM: for b in [0, batch):
 *   C_b = alpha * op(A_b) op(B_b) + beta * C_b (+ bias[n] broadcast over rows, if bias != NULL)
 * op(A) is M x K: A stored M x K with row stride lda (transA = 0) or K x M (transA = 1);
 * op(B) is K x N: B stored K x N with row stride ldb (transB = 0) or N x K (transB = 1);
 * C is M x N with row stride ldc.  X_b = X + b * strideX (stride 0 shares one matrix).
 * beta = 0 ignores the old contents of C (which may be uninitialised). */
int fno_gemm(int transA, int transB, int M, int N, int K, float alpha, const float *A, int64_t lda,
             int64_t strideA, const float *B, int64_t ldb, int64_t strideB, float beta, float *C, int64_t ldc,
             int64_t strideC, int batch, const float *bias, void *stream);

/* y = GELU(x) (exact form 0.5 x (1 + erf(x / sqrt 2))), n elements; y may alias x. */
int fno_gelu_fwd(const float *x, float *y, int64_t n, void *stream);
/* dx (+)= GELU'(x) * dy; accumulate = 1 adds to dx. */
int fno_gelu_bwd(const float *x, const float *dy, float *dx, int64_t n, int accumulate, void *stream);

/* Per-mode complex channel mixing.  X, Y hold for each batch b and retained mode
 * (kr, kz) the real parts at [b][kr][kz][c] and the imaginary parts at
 * [b][kr][nkz + kz][c] (nkz kz-modes, nkr kr-modes, C channels in X, O in Y);
 * R[kr][kz][c][o][2] holds complex weights (re, im).
 *   Y[b, kr, kz, o] = sum_c X[b, kr, kz, c] * R[kr, kz, c, o]        (complex) */
int fno_mix_fwd(const float *X, const float *R, float *Y, int batch, int nkr, int nkz, int C, int O, void *stream);
/* Gradients of fno_mix_fwd: dX = (dL/dX) (overwritten), dR (+)= dL/dR (accumulate = 1 adds). */
int fno_mix_bwd(const float *X, const float *R, const float *dY, float *dX, float *dR, int batch, int nkr, int nkz,
                int C, int O, int accumulate, void *stream);

/* out[n] (+)= sum over rows of X[rows x N] (row stride ldx). */
int fno_colsum(const float *X, int64_t rows, int N, int64_t ldx, float *out, int accumulate, void *stream);

/* Mean squared error over n elements: *loss (device double) += sum (y - t)^2 / n;
 * dy = 2 (y - t) / n. */
int fno_mse(const float *y, const float *t, float *dy, double *loss, int64_t n, void *stream);

/* Adam step t >= 1 (bias-corrected) on n parameters: m, v updated in place. */
int fno_adam(float *w, const float *g, float *m, float *v, int64_t n, float lr, float beta1, float beta2, float eps,
             int t, void *stream);

/* Tensor-core path of fno_gemm: 0 = mma.sync m16n8k16 (default), 1 = tcgen05.mma with
 * the accumulator in tensor memory (persistent CTAs, 128 x N tiles with N <= 256 chosen
 * so that there are four tiles per SM, two stage buffers).  Process-wide. */
int fno_set_tensor_path(int path);
/* Status of the tcgen05 path, synchronous:
 *   0  no bounded wait ran out since the last clear;
 *   1  a tcgen05 GEMM gave up a wait (its output is invalid), then saw every MMA it had
 *      issued complete before freeing its tensor memory: later GEMMs are unaffected;
 *   2  a recovery wait ran out as well, so tensor memory may have been freed under an
 *      MMA still in flight and a later GEMM could compute a wrong result unnoticed.
 *      From the first call that reads 2, the tcgen05 path is off for the rest of the
 *      process: fno_gemm runs on mma.sync, fno_set_tensor_path(1) fails, and this call
 *      keeps returning 2;
 *  -1  CUDA error.  clear = 1 resets the device flag (not the process-wide state of 2). */
int fno_tensor_path_status(int clear);

/* Test hooks for the failure path (no counterpart in the paper).
 * fno_test_wait_timeout(1): the next tcgen05 GEMM CTAs replace their first wait for an
 * MMA commit by a short bounded wait on a barrier that nothing arrives at, so the timeout
 * path runs (each CTA then waits for its real commits before freeing tensor memory);
 * 0 restores normal waits.  fno_test_set_tc_error(v) writes v in {0, 1, 2} into the
 * device flag read by fno_tensor_path_status, to exercise the host's handling of it. */
int fno_test_wait_timeout(int enable);
int fno_test_set_tc_error(int value);

const char *fno_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FNO_H */
