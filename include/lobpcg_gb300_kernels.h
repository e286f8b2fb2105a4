/*
 * lobpcg_gb300_kernels.h -- C ABI of the solver's dense building blocks.
 *
 * These are the contractions and small dense eigen-solves that one block
 * iteration of LOBPCG (Algorithm 1 of Bottin, Leroux, Knyazev, Zerah 2007)
 * is made of, exposed one by one so that each can be checked against a CPU
 * reference and timed on its own.  lobpcg_solve uses the same kernels.
 *
 * Common rules
 *   - Matrices are column-major with a leading dimension (elements).
 *   - Complex numbers are interleaved (re, im); prec = LOBPCG_C128 selects
 *     complex128 with FP64 arithmetic, LOBPCG_C64 complex64 with FP32, and
 *     (GEMMs) LOBPCG_C128_DF32 complex128 with double-FP32 arithmetic:
 *     every operand split into two FP32 parts, exact FP32 products by FMA
 *     (Dekker's TwoProd) and pair accumulators (Knuth's TwoSum), about 2^-47
 *     relative per product, run on the FP32 units (FP64 class, several
 *     times the FP64 rate of this GPU), or LOBPCG_C128_TC complex128 on the
 *     tensor cores: each real value split exactly into six 8-bit BF16
 *     digits with a power-of-two scale per 64 terms of the reduction, the
 *     digit products of equal weight summed exactly in FP32 per 64 terms,
 *     those sums added in double-FP32 (error about 2^-44 of sum |a||b|,
 *     FP64 class; error-free slicing after Ozaki, Ogita, Oishi and Rump,
 *     Numer. Algorithms 2012).
 *   - Pointers are device pointers; work is enqueued on `stream`
 *     (cudaStream_t, NULL = legacy default stream) and the call returns
 *     without synchronising, except where noted.
 *   - Return LOBPCG_OK or a negative LOBPCG_ERR_* code (header lobpcg_gb300.h);
 *     lobpcg_k_last_error() gives the message of the last failure.  The
 *     precision, the sizes, NULL pointers and leading dimensions are checked
 *     before any device work (ERR_ARG); a GEMM with an empty output (m, n or
 *     M = 0) is a no-op that returns LOBPCG_OK.
 *   - Scratch memory the kernels need is allocated by the library and kept
 *     for later calls (one pool per device).
 */
#ifndef LOBPCG_GB300_KERNELS_H
#define LOBPCG_GB300_KERNELS_H

#include "lobpcg_gb300.h"


#ifdef __cplusplus
extern "C" {
#endif

/*
 * C = alpha * A^H B + beta * C: the Gram and projection contractions of
 * Algorithm 1, step 4 (blocks of [Psi W P]^H [Psi W P] and of
 * [Psi W P]^H H[Psi W P]; Sec. 4.1 computes them with zgemm) and of the
 * KB projection beta^H X (Sec. 4.3).
 *   A is K x m (lda >= K), B is K x n (ldb >= K), C is m x n (ldc >= m).
 *   alpha, beta are real.  K may be large (the plane-wave count); the
 *   reduction over K is split across the GPU and summed in a fixed order, so
 *   results are bitwise reproducible for a given shape.
 */
int lobpcg_k_gemm_cn(int prec, int m, int n, int K, double alpha, const void *A, int lda,
                     const void *B, int ldb, double beta, void *C, int ldc, void *stream);

/*
 * Lower triangle of C = A^H B, complex128 (prec = LOBPCG_C128,
 * LOBPCG_C128_DF32 or LOBPCG_C128_TC): the FP64-class Gram matrices of
 * Algorithm 1, step 4 and of the all-band Rayleigh-Ritz closing a sweep
 * (Sec. 3.2).  Both Grams of the Rayleigh-Ritz pencil are Hermitian and the
 * pencil solver reads only their lower triangles, so 64 x 64 output tiles
 * strictly above the diagonal are skipped: about half the work for n >> 64.
 *   A and B are K x n (lda, ldb >= K), C is n x n (ldc >= n).  Every element
 *   C(i, j) with i >= j is written; tiles strictly above the diagonal are
 *   left untouched, and the rest of the upper triangle holds A^H B values
 *   (LOBPCG_C128_TC writes the entries with i >= j only).
 *   Same split and fixed summation order as lobpcg_k_gemm_cn.
 */
int lobpcg_k_gram_lower(int prec, int n, int K, const void *A, int lda, const void *B, int ldb, void *C,
                        int ldc, void *stream);

/*
 * D = alpha * A B + beta * C: the Ritz updates of Algorithm 1, steps 4-5
 * (Psi Delta + W Lambda + P Gamma and W Lambda + P Gamma), the KB
 * back-projection beta (E B) and the block-constraint update Y (Y^H W).
 *   A is M x k (lda >= M), B is k x n (ldb >= k), C and D are M x n
 *   (ldc, ldd >= M).  C may equal D (in-place accumulate) or be NULL when
 *   beta = 0.  alpha, beta are real.
 */
int lobpcg_k_gemm_nn(int prec, int M, int n, int k, double alpha, const void *A, int lda,
                     const void *B, int ldb, double beta, const void *C, int ldc,
                     void *D, int ldd, void *stream);

/*
 * Rayleigh-Ritz step of Algorithm 1, step 4, in FP64: the lowest m
 * eigenpairs of the Hermitian pencil A c = theta S c, where S is the Gram
 * matrix of a basis Z and A = Z^H H Z (n x n complex128, column-major,
 * lower triangles used).
 *   S is scaled to unit diagonal and factored by Cholesky; a basis vector
 *   whose pivot falls below drop_tol (relative to its own norm) is taken as
 *   dependent on the earlier ones and removed from the subspace.
 *   theta  (device, m doubles)          Ritz values, ascending.
 *   C      (device, n x m complex128, ld n) coefficients: Z C are the Ritz vectors,
 *          C^H S C = I.
 *   ndropped (device int, may be NULL)  number of basis vectors removed.
 * S and A are not modified.  Errors: ERR_ARG (m > n, n > 4096), ERR_OOM, ERR_CUDA.
 */
int lobpcg_k_rayleigh_ritz(int n, int m, const void *S, const void *A, double drop_tol,
                           double *theta, void *C, int *ndropped, void *stream);

/*
 * The same Rayleigh-Ritz step with the parts that one SM's FP64 units limit on
 * this GPU in double-FP32 arithmetic (the LOBPCG_C128_DF32 scheme above): the
 * Cholesky diagonal blocks, the column work of the Householder
 * tridiagonalisation, the small dense products, the fine multisection rounds
 * and the back-transformation.  Inverse iteration's serial recurrences stay
 * FP64.  Same arguments, layout and errors as lobpcg_k_rayleigh_ritz; results
 * agree with it to about 1e-13 relative.
 */
int lobpcg_k_rayleigh_ritz_df32(int n, int m, const void *S, const void *A, double drop_tol,
                                double *theta, void *C, int *ndropped, void *stream);

/*
 * The same Rayleigh-Ritz step in FP32 arithmetic: S, A and C are complex64
 * (n x n and n x m, column-major), theta is float.  A building block only:
 * the mixed-precision schedule assembles its pencils from FP32 Gram blocks
 * but solves them in FP64 class.
 */
int lobpcg_k_rayleigh_ritz32(int n, int m, const void *S, const void *A, double drop_tol,
                             float *theta, void *C, int *ndropped, void *stream);

/*
 * Hermitian eigen-decomposition in FP64: A = V diag(w) V^H, eigenvalues ascending.
 *   A   (device, n x n complex128, ld n; lower triangle used, not modified),
 *   w   (device, n doubles), V (device, n x n complex128, ld n).
 * Householder tridiagonalisation (in one thread-block cluster's shared memory
 * up to n = 416, else one cooperative grid), multisection and inverse iteration
 * on the tridiagonal matrix, compact-WY back-transformation.
 */
int lobpcg_k_heev(int n, const void *A, double *w, void *V, void *stream);

/*
 * Engine of the complex64 (LOBPCG_C64) GEMMs issued by the calling host
 * thread (a per-thread setting); lobpcg_solve and lobpcg_apply_H set it from
 * their handle's lobpcg_options.gemm_split on entry, and every k-point lane
 * thread of a solve does likewise, so handles with different engines used
 * from different threads do not interfere.
 *   0 (auto) or 2: 5th-generation tensor cores (tcgen05, accumulators in TMEM)
 *      with 3xTF32 split operands and FP32 accumulation (relative error about
 *      1e-6 of sum |a||b|) for long reductions (A^H B with K >= 1024) and tall
 *      products (A B with M >= 1024); CUDA cores for the other shapes.
 *   3: CUDA cores only (FP32 products, FP64 accumulation every 256 terms).
 * Returns ERR_ARG for other values (1, BF16x3, is not built).
 */
int lobpcg_k_set_gemm_mode(int mode);

/*
 * Poll limit of the waits inside the tensor-core GEMMs on the current device:
 * before a CTA refills a shared-memory stage it waits, at most `polls` times,
 * for the MMAs that read it.  polls < 0 restores the default (2^26 polls,
 * seconds).  A wait that runs out makes the CTA stop issuing, wait (with the
 * default limit) for the MMAs it already issued, free its tensor memory and
 * return with a device flag set, which lobpcg_k_check_timeouts and every
 * solve sweep turn into LOBPCG_ERR_TIMEOUT.  This exists so that tests can
 * drive the timeout path (polls = 0) without hanging or faulting the GPU.
 * Errors: ERR_CUDA.
 */
int lobpcg_k_set_spin_limit(long long polls);

/*
 * Synchronises the device, then returns LOBPCG_ERR_TIMEOUT if a tensor-core
 * GEMM launched so far stopped because an mbarrier wait ran out (its output is
 * then not valid), else LOBPCG_OK.  Clears the condition.
 */
int lobpcg_k_check_timeouts(void);

/* Message of the last failure of a lobpcg_k_* call on this host thread. */
const char *lobpcg_k_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LOBPCG_GB300_KERNELS_H */
