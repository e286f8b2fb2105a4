/*
 * lobpcg_gb300.h -- C ABI of a GB300 (sm_103a) block LOBPCG plane-wave eigensolver.
 *
 * The library finds the lowest Kohn-Sham eigenpairs of a FIXED plane-wave
 * Hamiltonian (Bottin, Leroux, Knyazev, Zerah 2007, "Large scale ab initio
 * calculations based on three levels of parallelization"):
 *
 *   H = T + V_loc + V_KB   on the sphere  1/2 |k+G|^2 <= Ecut      (Sec. 2.1)
 *
 *   T      kinetic diagonal 1/2 |k+G|^2,
 *   V_loc  local potential applied through a zero-padded 3D FFT: inverse FFT
 *          of the sphere to the N^3 grid, pointwise V(r), forward FFT back
 *          to the sphere (Sec. 2.2 item iii, Sec. 4.1),
 *   V_KB   Kleinman-Bylander non-local part  sum_p E_p |beta_p><beta_p|
 *          (Sec. 2.2 item iv, Sec. 4.3),
 *
 * by block LOBPCG (Sec. 3.2, Algorithm 1) iterated block after block with
 * each block orthogonal to the previous ones, each sweep closed by a
 * Rayleigh-Ritz step over all bands (Sec. 3.2, last paragraph).  The overlap
 * operator O is the identity (norm-conserving case, Sec. 2.1).
 *
 * Conventions shared by every call
 *   - Cell: cubic, side a (bohr), volume Omega = a^3; G_n = (2 pi / a) n for
 *     integer triplets n; k-points in reduced coordinates, q = (2 pi/a)(n + k).
 *   - Grid: N^3 points r_j = a j / N; real-space arrays are C-order [x][y][z].
 *   - Sphere: n is in the basis of k-point k when
 *         |n + k|^2 <= 2 Ecut (a / 2 pi)^2 + 1e-9
 *     (index units; lattice points exactly on the sphere are kept).  Every
 *     basis index must lie in [-N/2, N/2-1] or lobpcg_create fails.
 *   - Plane-wave order ("G order") of k-point k: sorted by n_x, then n_y,
 *     then n_z (signed); lobpcg_gvectors returns it.  Every coefficient
 *     array below is in this order.
 *   - Complex numbers are interleaved (re, im): complex128 = 2 x double,
 *     complex64 = 2 x float.  Blocks of vectors are column-major
 *     npw_k x nb (each band's npw_k coefficients contiguous, ld = npw_k).
 *   - V_loc matrix elements: the grid potential's discrete Fourier
 *     coefficient Vt((n - n') mod N), Vt(n) = N^-3 sum_j V(r_j) e^{-2 pi i n.j/N}.
 *
 * Ownership and streams
 *   - The library copies the potential, projectors and energies at create
 *     and owns every device buffer it allocates; it never frees caller memory.
 *   - lobpcg_apply_H enqueues on the CUDA stream given at create
 *     (lobpcg_set_stream changes it) and returns after enqueueing.
 *     lobpcg_solve runs after the work already queued on that stream, on
 *     library streams (one per concurrent k-point, high priority, plus
 *     low-priority side streams), and returns synchronised.
 *   - A handle is not thread-safe: one host thread at a time per handle.
 *
 * Errors
 *   - Every call returns an int status: LOBPCG_OK (0) on success, a negative
 *     LOBPCG_ERR_* code on failure, LOBPCG_NOT_CONVERGED (positive) when a
 *     solve ran out of sweeps with its outputs filled.  The library never
 *     calls exit/abort.  lobpcg_last_error returns a message for the last
 *     failure on a handle.
 */
#ifndef LOBPCG_GB300_H
#define LOBPCG_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LOBPCG_OK               0
#define LOBPCG_NOT_CONVERGED    1   /* solve: outputs filled, max residual > tol */
#define LOBPCG_ERR_ARG         -1   /* invalid argument (sizes, pointers, k index, options) */
#define LOBPCG_ERR_OOM         -2   /* a device allocation failed or exceeded the handle's cap */
#define LOBPCG_ERR_CUDA        -3   /* a CUDA runtime call failed; message has the CUDA error */
#define LOBPCG_ERR_TIMEOUT     -4   /* a bounded device wait ran out (never a hang) */
#define LOBPCG_ERR_BREAKDOWN   -5   /* the Rayleigh-Ritz basis collapsed beyond recovery */
#define LOBPCG_ERR_UNSUPPORTED -6   /* grid size or option not supported by this build */

/* Arithmetic of lobpcg_apply_H (element type of X and Y, and compute precision). */
#define LOBPCG_C128 0               /* complex128 in/out, FP64 FFT and GEMMs */
#define LOBPCG_C64  1               /* complex64  in/out, FP32 FFT and GEMMs */
#define LOBPCG_C128_DF32 2          /* complex128 in/out, FFT and GEMMs in double-FP32 arithmetic:
                                       pairs of FP32 numbers, error-free TwoSum / TwoProd steps,
                                       about 2^-47 relative per operation (FP64 class) at several
                                       times this GPU's FP64 rate */
#define LOBPCG_C128_TC 3            /* complex128 in/out, FFT in double-FP32 arithmetic and GEMMs
                                       on the tensor cores: each real value split exactly into six
                                       8-bit BF16 digits with one power-of-two scale per 64 terms of
                                       the reduction, digit products summed exactly in FP32 per
                                       64 terms, partial sums in double-FP32 (error about 2^-44 of
                                       sum |a||b|, FP64 class) */

/* Precision schedule of lobpcg_solve (lobpcg_options.precision). */
#define LOBPCG_FP64  0              /* every step in FP64 */
#define LOBPCG_MIXED 1              /* FP32 FFTs / 3xTF32 tensor-core GEMMs for W and P;
                                       X, HX and the residuals stored in FP64; the X block
                                       start, Cholesky, Rayleigh-Ritz and X updates in FP64
                                       class (arithmetic chosen by lobpcg_options.fp64_gemm);
                                       residual norms and convergence in FP64 */

typedef struct lobpcg_ctx lobpcg_ctx;   /* opaque handle */

/* Cubic cell: side a (bohr), FFT grid edge N, plane-wave cutoff ecut (Ha). */
typedef struct {
    double a;
    int    N;
    double ecut;
} lobpcg_cell;

typedef struct {
    int    block_size;   /* m: bands per LOBPCG block (Sec. 3.2); M must be a multiple */
    int    nline;        /* Algorithm 1 iterations per block visit (paper: 4) */
    int    max_sweeps;   /* sweeps over all blocks before giving up */
    int    precision;    /* LOBPCG_FP64 or LOBPCG_MIXED */
    int    gemm_split;   /* complex64 GEMM engine: 0 = auto (= 2), 2 = tensor cores with 3xTF32 split
                            operands for long reductions and tall products, 3 = CUDA cores only;
                            1 (BF16x3) is not built: ERR_UNSUPPORTED */
    int    use_graph;    /* 1: the FP32 H application of each block iteration (FFT passes + KB GEMMs,
                            about ten kernels) is recorded once per buffer pair as a CUDA graph and
                            replayed as one launch.  Ignored while options.timing is on and on the
                            legacy default stream (which cannot be captured). */
    int    autotune;     /* 1: the first lobpcg_solve of the handle times, per k-point, the FFT
                            band-batch budget (32 .. 256 MB) of the FP32 and of the FP64-class H
                            application and keeps the fastest; lobpcg_stats.ms_autotune reports
                            the time it took (not included in ms_total). */
    double tol;          /* convergence: max_i ||H x_i - theta_i x_i||_2 <= tol (Ha), ||x_i|| = 1 */
    long long mem_cap;   /* 0: no cap; else maximum bytes the handle may allocate (ERR_OOM above it) */
    int    timing;       /* 1: time each phase of lobpcg_solve with CUDA events on its lane streams */
    int    nbuf;         /* extra buffer bands iterated above the M requested ones but not required to
                            converge (rounded up to whole blocks; 0 = none).  They give the top wanted
                            bands a gap to the unresolved spectrum. */
    double mixed_switch; /* MIXED only: a block whose smallest residual after the previous sweep is
                            below this (Ha) runs its iterations in FP64 (default 0 = never) */
    double mixed_early;  /* MIXED only: a block all of whose bands had residuals above this (Ha) in the
                            previous sweep visits "early": its start and its X updates use the FP32
                            copies, and its H X is not refreshed in FP64.  The sweep-end Rayleigh-Ritz
                            does likewise when every block was early.  (default 1e-3; 0 = never) */
    int    fp64_gemm;    /* arithmetic of the FP64-class work limited by this GPU's FP64 units: the tall
                            GEMMs (Grams, constraint, Ritz updates, KB projections of FP64 H X) and, in
                            the Rayleigh-Ritz step, the Cholesky diagonal blocks, the tridiagonalisation's
                            column work and the small products.  0 = auto (MIXED: tall GEMMs on the
                            tensor cores as in 3, the rest double-FP32; FP64: native FP64), 1 = native
                            FP64, 2 = double-FP32 on the FP32 units (about 2^-47 relative per operation)
                            on both schedules, 3 = like 2 but the tall GEMMs on the tensor cores with
                            exact BF16 digit slices (the LOBPCG_C128_TC arithmetic).  With 2 and 3
                            the fine multisection rounds and the back-transformation run in
                            double-FP32 as well; inverse iteration's serial recurrences stay FP64. */
    int    gamma_real;   /* 1: k-points at Gamma (k = 0) are solved in the real-orbital form (the
                            Gamma-point trick of plane-wave codes; the paper expands complex orbitals,
                            Sec. 2.1): eigenvectors with c(-G) = conj(c(G)), stored packed on the half
                            sphere (G = 0 and one of each +-G pair), coefficient matrices real, and H
                            applied to two real bands at once as one complex band.  Valid when H
                            commutes with c(G) -> conj(c(-G)): a real local potential and projectors
                            real in r space up to one phase each (true of the synthetic cells).  The
                            start vectors are projected onto the real form; the returned vectors are
                            full-sphere complex128 with the symmetry.  Ignored by lobpcg_solve_pcg and
                            at other k-points.  0 (default): complex orbitals everywhere. */
} lobpcg_options;

/* Phases of a solve, for the per-phase timers of lobpcg_stats. */
#define LOBPCG_PH_FFT        0   /* V_loc + kinetic through the FFT passes */
#define LOBPCG_PH_NONLOCAL   1   /* KB projection and back-projection GEMMs */
#define LOBPCG_PH_GRAM       2   /* Gram matrices of the Rayleigh-Ritz basis */
#define LOBPCG_PH_CONSTRAINT 3   /* orthogonality constraint against earlier blocks */
#define LOBPCG_PH_RR         4   /* FP64 Cholesky + Rayleigh-Ritz eigensolves */
#define LOBPCG_PH_UPDATE     5   /* Ritz updates, residual, preconditioner, casts, copies */
#define LOBPCG_PH_COUNT      6

typedef struct {
    int    sweeps;            /* sweeps done */
    int    iterations;        /* Algorithm 1 iterations done (all blocks, all k) */
    int    converged;         /* 1 if every band of every k met tol */
    int    restarts;          /* Rayleigh-Ritz basis vectors dropped as dependent */
    double max_resid;         /* final max residual over all k and bands (Ha) */
    double ms_total;          /* wall time of the solve, ms */
    long long band_applies_fp64;  /* single-band H applications done in FP64 */
    long long band_applies_fp32;  /* single-band H applications done in FP32 */
    long long kernel_launches;    /* kernels launched by the solve */
    /* per phase (index LOBPCG_PH_*), filled when options.timing = 1: */
    double    ph_ms[LOBPCG_PH_COUNT];      /* device time, CUDA events on the lane streams (summed) */
    double    ph_flops[LOBPCG_PH_COUNT];   /* algorithmic floating-point operations */
    double    ph_bytes[LOBPCG_PH_COUNT];   /* algorithmic DRAM bytes */
    long long ph_calls[LOBPCG_PH_COUNT];   /* timed calls */
    double    ph_fp64_flops[LOBPCG_PH_COUNT];  /* part of ph_flops done in FP64 arithmetic */
    long long block_visits_fp32;  /* block visits run with the mixed FP32/FP64 schedule */
    long long block_visits_fp64;  /* block visits run entirely in FP64 */
    double    ph_ms_fp64[LOBPCG_PH_COUNT];     /* part of ph_ms spent in calls doing FP64 arithmetic */
    double    ph_bytes_fp64[LOBPCG_PH_COUNT];  /* part of ph_bytes moved by those calls */
    long long block_visits_settled;  /* MIXED: block visits without inner iterations, the block's
                                        residuals being all below tol / 100 after the previous sweep */
    double    ms_autotune;            /* wall time of the autotuner in this call (options.autotune) */
} lobpcg_stats;

/* Fill *opt with defaults: m = 64, nline = 4, max_sweeps = 100, FP64, tol = 1e-8. */
int lobpcg_default_options(lobpcg_options *opt);

/*
 * Create a solver for nk k-points of one cell (Sec. 2.1 basis; Sec. 5.2 k-points).
 *   cell      a, N, ecut as above.  Supported N: products of 2, 3 and 5, 4 <= N <= 256.
 *   kpts      host, nk x 3 doubles, reduced coordinates.
 *   vloc_r    host, N^3 doubles, the real local potential V(r_j), C-order [x][y][z].
 *   nproj     number of KB projectors (>= 0), the same set for every k.
 *   proj_E    host, nproj doubles: KB energies E_p (Ha); may be NULL when nproj = 0.
 *   beta      host, nk pointers; beta[k] is npw_k x nproj complex128, column-major,
 *             rows in G order.  Because npw_k and the G order are only known
 *             after the basis is built, pass beta = NULL here and give the
 *             projectors afterwards with lobpcg_set_projectors, or precompute
 *             the order with the same rule.  May be NULL when nproj = 0.
 *   opt       options (NULL = defaults).
 *   stream    cudaStream_t to enqueue on (NULL = legacy default stream).
 * On success *out receives a handle.  Errors: ERR_ARG, ERR_UNSUPPORTED,
 * ERR_OOM, ERR_CUDA (then *out is NULL).  The options, the cell, N and every
 * host value (potential, k-points, energies: all finite) are checked before
 * the first device call, so ERR_ARG and ERR_UNSUPPORTED need no GPU.
 */
int lobpcg_create(lobpcg_ctx **out, const lobpcg_cell *cell, int nk, const double *kpts,
                  const double *vloc_r, int nproj, const double *proj_E,
                  const void *const *beta, const lobpcg_options *opt, void *stream);

/* Upload (or replace) the Kleinman-Bylander projectors of k-point k (the v_nl
 * term of Sec. 2.2 item iv and Sec. 4.3): beta_k is host npw_k x nproj
 * complex128, column-major, rows in G order.  The library copies it; the call
 * returns once the host buffer may be reused.  nproj = 0: a no-op.
 * Errors: ERR_ARG (ctx or beta_k NULL, k out of range), ERR_OOM, ERR_CUDA. */
int lobpcg_set_projectors(lobpcg_ctx *ctx, int k, const void *beta_k);

/* Change the CUDA stream (cudaStream_t; NULL = legacy default stream) that
 * later calls enqueue on and that lobpcg_solve orders its work after.
 * Errors: ERR_ARG (ctx NULL). */
int lobpcg_set_stream(lobpcg_ctx *ctx, void *stream);

/* Replace the options of an existing handle (block size, tolerance,
 * precision ...); they apply from the next call.  The options are checked as
 * at create: ERR_ARG or ERR_UNSUPPORTED leaves the old ones in place. */
int lobpcg_set_options(lobpcg_ctx *ctx, const lobpcg_options *opt);

/* Number of plane waves npw_k of k-point k (the sphere of Sec. 2.1, >= 1), or
 * ERR_ARG (ctx NULL, k out of range). */
int lobpcg_npw(const lobpcg_ctx *ctx, int k);

/* Write the G order of k-point k: miller is host int32 npw_k x 3, caller-owned
 * (row g = (n_x, n_y, n_z), sorted by n_x, then n_y, then n_z).
 * Errors: ERR_ARG (ctx or miller NULL, k out of range). */
int lobpcg_gvectors(const lobpcg_ctx *ctx, int k, int32_t *miller);

/*
 * Y = H X for nb bands of k-point k (Sec. 2.2 items iii and iv).
 *   X, Y       npw_k x nb, column-major (ld = npw_k), complex128 when
 *              precision = LOBPCG_C128, LOBPCG_C128_DF32 or LOBPCG_C128_TC, complex64 when
 *              LOBPCG_C64.  Device
 *              pointers run fully asynchronously on the handle's stream; host
 *              pointers are staged through device buffers and the call returns
 *              after Y has been written back (synchronous).  X and Y must not
 *              overlap.
 *   nb         >= 0 (0 is a no-op).
 * Errors: ERR_ARG (k, nb, NULL pointers, overlapping X/Y), ERR_OOM, ERR_CUDA.
 */
int lobpcg_apply_H(lobpcg_ctx *ctx, int k, const void *X, void *Y, int nb, int precision);

/*
 * Electron density of nb bands of k-point k on the real-space grid, the first
 * step of the self-consistent loop (Sec. 2.1; computed by the same FFT as the
 * local potential, Sec. 2.2 item iii, per-band contributions summed over
 * bands as in Sec. 4.1):
 *     rho(r_j) += sum_b f_b |psi_b(r_j)|^2,
 *     psi_b(r) = Omega^-1/2 sum_G X[G, b] e^{i(k+G).r}   (Omega = a^3),
 * so that (Omega / N^3) sum_j rho(r_j) = sum_b f_b for orthonormal bands.
 *   X          device, npw_k x nb column-major, complex128 (precision =
 *              LOBPCG_C128: FP64 transforms, or LOBPCG_C128_DF32:
 *              double-FP32 transforms) or complex64 (LOBPCG_C64: FP32
 *              transforms, FP32 sums over each band batch).
 *   f          host, nb doubles: occupations (k-point weight included).
 *   rho        device, N^3 doubles, C-order [x][y][z] (the layout of vloc_r),
 *              accumulated into (zero it for a fresh density; call once per
 *              k-point to sum over k).  The bands are summed in band order
 *              within each grid point and nothing is summed atomically, so
 *              the result is bitwise reproducible.
 * Enqueued on the handle's stream; returns after the work is queued and the
 * occupations are copied.  Errors: ERR_ARG (k, nb, NULL or host X / rho,
 * non-finite f), ERR_OOM, ERR_CUDA, ERR_UNSUPPORTED.
 */
int lobpcg_density(lobpcg_ctx *ctx, int k, const void *X, int nb, const double *f, double *rho, int precision);

/*
 * Allocation-free Y = (T + V_loc) X for nb bands of k-point k.  The paper has
 * no counterpart: this entry point exists for callers that cannot allocate
 * device memory while they run (code inside another framework's memory pool
 * or under a fixed device-memory budget, loops that must not touch the
 * allocator because allocation can synchronise the device).  It runs the same
 * FFT passes as lobpcg_apply_H, without the KB projector part, and allocates
 * nothing: the FFT half-box lives in a 32 MiB file-scope device array that
 * every GPU loading the library holds until the process exits.
 *   X, Y       device pointers only, npw_k x nb column-major, complex128
 *              (precision = LOBPCG_C128) or complex64 (LOBPCG_C64); must not overlap.
 *   limit      one band's half-box, Px * N^2 complex numbers (Px = x-planes the
 *              sphere occupies, about N/2 + 1), must fit in 32 MiB, else
 *              LOBPCG_ERR_ARG; bands are processed in batches that fit.
 * lobpcg_create looks up the array's device address on the handle's device
 * (host code cannot use the array's name as an address; the lookup also loads
 * the device module that holds the array, which is when CUDA reserves its
 * 32 MiB), so the call itself does no set-up; the handle's device must be the
 * current device (else ERR_ARG).  All calls share the array: calls that
 * overlap on the GPU race on it.  Errors: ERR_ARG, ERR_CUDA; the message is
 * lobpcg_last_error(NULL).
 */
int lobpcg_apply_local_noalloc(lobpcg_ctx *ctx, int k, const void *X, void *Y, int nb, int precision);

/*
 * Lowest nbands eigenpairs of every k-point by block LOBPCG (Algorithm 1),
 * block by block with the orthogonality constraint, each sweep closed by an
 * all-band Rayleigh-Ritz step (Sec. 3.2).
 *   nbands     M, a multiple of the block size, 1 <= M <= npw_k for every k.
 *   X          nk pointers; X[k] is npw_k x M complex128 (column-major).
 *              In: start vectors (any full-rank block).  Out: orthonormal
 *              eigenvectors, ascending eigenvalues.  Device pointers are used
 *              in place; host pointers (pinned or pageable) are copied to a
 *              library device buffer and the result copied back.
 *   eig        host nk x M doubles (out): eigenvalues, ascending per k.
 *   resid      host nk x M doubles (out): ||H x_i - eps_i x_i||_2 in FP64.
 *   stats      optional (NULL allowed) statistics.
 * Synchronous: returns once eig/resid are on the host.
 * Returns OK, NOT_CONVERGED (outputs filled) or an error code.
 */
int lobpcg_solve(lobpcg_ctx *ctx, int nbands, void *const *X, double *eig, double *resid,
                 lobpcg_stats *stats);

/*
 * The same eigenpairs by band-by-band preconditioned conjugate gradient, the
 * method Sec. 3.3 compares LOBPCG with (Teter, Payne and Allan 1989; the
 * iterative-diagonalisation form of Bylander et al. 1990): every band in
 * order, kept orthogonal to the bands before it, takes options.nline
 * iterations of steepest descent preconditioned by the Teter ratio (the
 * preconditioner of lobpcg_solve), Fletcher-Reeves conjugation and an exact
 * line minimisation of the Rayleigh quotient on span[x, d]; each sweep is
 * closed by the all-band Rayleigh-Ritz step and residual test of
 * lobpcg_solve.  Same arguments, ownership, buffer bands and results as
 * lobpcg_solve; options.precision = LOBPCG_FP64 runs FP64 throughout,
 * LOBPCG_MIXED runs the H applications and GEMMs in the FP64-class engines
 * (options.fp64_gemm).  block_size only sets the buffer-band rounding.
 */
int lobpcg_solve_pcg(lobpcg_ctx *ctx, int nbands, void *const *X, double *eig, double *resid,
                     lobpcg_stats *stats);

/* Sizes in bytes of lobpcg_cell, lobpcg_options and lobpcg_stats as this library
 * was compiled, so that a binding can check its own layouts against them (any
 * pointer may be NULL).  Always LOBPCG_OK; needs no device. */
int lobpcg_struct_sizes(int64_t *cell, int64_t *options, int64_t *stats);

/* Number of kernels the library has launched in this process so far (all handles). */
long long lobpcg_launch_count(void);

/* Message describing the last error on ctx ("" if none); ctx may be NULL for create errors. */
const char *lobpcg_last_error(const lobpcg_ctx *ctx);

/* Free every resource of the handle.  NULL is ignored. */
void lobpcg_destroy(lobpcg_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* LOBPCG_GB300_H */
