// Internal declarations shared by the library's translation units.
// Complex numbers are interleaved (re, im) pairs, layout-compatible with
// float2 / double2 and with numpy complex64 / complex128.
#pragma once

#include <atomic>
#include <mutex>

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/lobpcg_gb300.h"

namespace lg {

template <typename R>
struct alignas(2 * sizeof(R)) cx {
    R x, y;
};

template <typename R>
__host__ __device__ __forceinline__ cx<R> mkc(R a, R b) { cx<R> r; r.x = a; r.y = b; return r; }
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return mkc<R>(a.x + b.x, a.y + b.y); }
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return mkc<R>(a.x - b.x, a.y - b.y); }
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator*(cx<R> a, cx<R> b) {
    return mkc<R>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator*(R s, cx<R> a) { return mkc<R>(s * a.x, s * a.y); }
template <typename R>
__host__ __device__ __forceinline__ cx<R> conjc(cx<R> a) { return mkc<R>(a.x, -a.y); }
// a * conj(b)
template <typename R>
__host__ __device__ __forceinline__ cx<R> mul_conj(cx<R> a, cx<R> b) {
    return mkc<R>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
// acc += conj(a) * b
template <typename R>
__host__ __device__ __forceinline__ void fma_cn(cx<R> &acc, cx<R> a, cx<R> b) {
    acc.x = fma(a.x, b.x, acc.x); acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y); acc.y = fma(-a.y, b.x, acc.y);
}
// acc += a * b
template <typename R>
__host__ __device__ __forceinline__ void fma_nn(cx<R> &acc, cx<R> a, cx<R> b) {
    acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
}
template <typename R>
__host__ __device__ __forceinline__ R abs2(cx<R> a) { return a.x * a.x + a.y * a.y; }

template <typename To, typename From>
__host__ __device__ __forceinline__ cx<To> cvt(cx<From> a) { return mkc<To>((To)a.x, (To)a.y); }

typedef cx<double> z64;   // complex128
typedef cx<float> c32;    // complex64

// ------------------------------------------------------------------ status
struct Status {
    int code = LOBPCG_OK;
    std::string msg;
};

// Thread-local message for calls that have no handle (create, lobpcg_k_*).
void set_global_error(const std::string &m);
const char *global_error();

#define LG_CUDA_TRY(...)                                                                    \
    do {                                                                                    \
        cudaError_t _e = (__VA_ARGS__);                                                     \
        if (_e != cudaSuccess) {                                                            \
            return ::lg::fail(LOBPCG_ERR_CUDA, std::string(#__VA_ARGS__ " failed: ") +       \
                                                   cudaGetErrorString(_e));                 \
        }                                                                                   \
    } while (0)

#define LG_TRY(...)                                  \
    do {                                             \
        int _s = (__VA_ARGS__);                      \
        if (_s < 0) return _s;                       \
    } while (0)

// Records a message for the current call and returns `code`.
int fail(int code, const std::string &m);
// Message recorded by the last fail() on this host thread.
const std::string &last_fail();

// Checks a kernel launch (configuration errors are reported at launch time) and
// counts it in the process-wide launch counter.
int check_launch(const char *what);
long long launch_count();

// ------------------------------------------------------------------ phase timers
// CUDA-event timing of solver phases on one stream (no-op when disabled).
struct Prof {
    bool on = false;
    cudaStream_t s = nullptr;
    struct Rec { int ph; bool f64; cudaEvent_t a, b; };
    std::vector<cudaEvent_t> pool;
    std::vector<Rec> recs;
    double ms[LOBPCG_PH_COUNT] = {0};
    double ms64[LOBPCG_PH_COUNT] = {0};   // part of ms[] spent in scopes doing FP64 arithmetic
    double flops[LOBPCG_PH_COUNT] = {0};
    double fp64_flops[LOBPCG_PH_COUNT] = {0};
    double bytes[LOBPCG_PH_COUNT] = {0};
    double bytes64[LOBPCG_PH_COUNT] = {0};
    long long calls[LOBPCG_PH_COUNT] = {0};
    cudaEvent_t get();
    // Start timing phase `ph`; returns the start event (nullptr when off).
    cudaEvent_t begin(int ph);
    void end(int ph, cudaEvent_t a, double fl, double by, bool fp64);
    // Wait for the recorded events and add their durations to ms[].
    void collect();
    ~Prof();
};

// RAII scope of one timed phase.
struct PhaseScope {
    Prof *p;
    int ph;
    double fl, by;
    bool f64;
    cudaEvent_t a;
    PhaseScope(Prof *p_, int ph_, double fl_, double by_, bool f64_)
        : p(p_), ph(ph_), fl(fl_), by(by_), f64(f64_), a(p_ ? p_->begin(ph_) : nullptr) {}
    ~PhaseScope() { if (p) p->end(ph, a, fl, by, f64); }
};

// ------------------------------------------------------------------ device memory
// A grow-only device buffer owned by the library.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

// Allocation accounting with an optional cap (lobpcg_options.mem_cap).
struct Allocator {
    long long cap = 0;
    std::atomic<long long> used{0};  // concurrent k-point lanes allocate from one allocator
    int alloc(void **p, size_t bytes);
    void free(void *p, size_t bytes);
    // Make `b` at least `bytes` large (contents are not preserved).
    int ensure(DevBuf &b, size_t bytes);
    void release(DevBuf &b);
};

// ------------------------------------------------------------------ FFT geometry (one k-point)
struct FFTGeom {
    int N = 0;
    int Px = 0, Py = 0;           // active x planes and y rows of the sphere
    int nx0 = 0, ny0 = 0;         // signed index of plane 0 / row 0
    int npw = 0;
    long long zlines = 0;         // occupied z-lines summed over planes (FFTs in passes A and C)
    // device tables
    int *plane_begin = nullptr;   // Px+1: sphere range of each x plane
    int2 *plane_yrange = nullptr; // Px: [py_lo, py_hi] rows holding coefficients
    int *gmap = nullptr;          // npw: py * N + (n_z mod N)
};

// Radix plan of a length-N 1D FFT (Stockham, radices 8, 4, 2, 5, 3).
struct FFTPlan {
    int N = 0;
    int nstage = 0;
    int radix[12];
};
// Mixed-radix plan of a length-N line (radices 8, 4, 2, 5, 3; allow8 = false leaves out 8).
bool make_fft_plan(int N, FFTPlan &plan, bool allow8 = true);

// Local-potential application Y = V_loc X (+ T X) for a block of bands on one k-point.
//   X, Y: npw x nb column-major (ld = ldx / ldy) of cx<R>; T: npw kinetic (nullable)
//   vt:   device potential pre-scaled by 1/N^3, layout [z][x][y] ([y][x][z] for the
//         FP32 register variant)
//   tw:   device twiddles e^{-2 pi i t / N}, t < N
//   T2:   scratch of at least nbatch * Px * N * N cx<R>
//   df:   complex128 only: transform in double-FP32 arithmetic (FP32 pairs, ~2^-48 per
//         operation) instead of FP64
//   vt_pair: optional, with df: vt as (hi, lo) FP32 pairs in vt's layout (read instead of
//         converting vt on the fly)
template <typename R>
int fft_vloc_apply(const FFTGeom &g, const FFTPlan &plan, const cx<R> *X, int ldx, cx<R> *Y, int ldy,
                   int nb, const R *kin, const R *vt, const cx<R> *tw, cx<R> *T2, int nbatch,
                   cudaStream_t s, bool df = false, const float2 *vt_pair = nullptr);
// FP32 register-resident variant of the three passes for the grid edges it is
// compiled for (8, 12, 16, 20, 24, 36, 48, 64, 72, 96, 120, 128, 160).  Its scratch is laid out T2[b][px][y][z]
// and its potential table vt as [y][x][z] (pre-scaled by 1/N^3);
// fft_vloc_apply<float> routes to it whenever fft_reg_supported(N).
bool fft_reg_supported(int N);
int fft_reg_prepare();                        // twiddle constants on the current device (once)
size_t fft_reg_smem_need(const FFTGeom &g);
int fft_reg_apply(const FFTGeom &g, const c32 *X, int ldx, c32 *Y, int ldy, int nb, const float *kin,
                  const float *vt, c32 *T2, int nbatch, cudaStream_t s);
// Density rho[x][y][z] += scale sum_b f_b |psi_b(r)|^2 of nb bands (Sec. 2.1, first step of the SC
// loop) by pass A and an inverse x-transform: FP64 (df = false) or double-FP32 (df) passes for
// complex128, the FP32 register passes (f32: the occupations in FP32) for complex64.  T2: scratch
// as for fft_vloc_apply; rho (device, N^3 FP64) is accumulated into.
template <typename R>
int fft_density(const FFTGeom &g, const FFTPlan &plan, const cx<R> *X, int ldx, int nb, const cx<R> *tw,
                const double *f, const float *f32, double scale, double *rho, cx<R> *T2, int nbatch, cudaStream_t s,
                bool df);
int fft_reg_density(const FFTGeom &g, const c32 *X, int ldx, int nb, const float *f, double scale, double *rho,
                    c32 *T2, int nbatch, cudaStream_t s);
// Algorithmic floating-point operations of the three passes for one band
// (5 n log2 n per length-n complex line FFT, plus the V and T multiplies).
double fft_flops_per_band(const FFTGeom &g);
// Shared memory the passes need; 0 when the grid does not fit on one SM.
template <typename R>
size_t fft_smem_need(const FFTGeom &g);

// Read-only view of one k-point's FFT tables inside a handle (for entry points
// that run the FFT passes on scratch they own).
struct LocalView {
    const FFTGeom *geom = nullptr;
    const FFTPlan *plan = nullptr;
    int npw = 0;
    const double *kin64 = nullptr, *vt64 = nullptr;
    const float *kin32 = nullptr, *vt32 = nullptr;
    const z64 *tw64 = nullptr;
    const c32 *tw32 = nullptr;
    cudaStream_t stream = nullptr;
    int device = 0;
};
// Looks up the allocation-free entry point's scratch address on the current device
// (loading the module that holds it); lobpcg_create calls it on the handle's device.
int noalloc_prepare();
}  // namespace lg
struct lobpcg_ctx;
namespace lg {
int ctx_local_view(const lobpcg_ctx *c, int k, LocalView *v);
bool is_device_pointer(const void *p);

// ------------------------------------------------------------------ BLAS-like kernels
// Scratch for split-K partial sums (grown on demand).
struct GemmWork {
    Allocator *alloc = nullptr;
    DevBuf part;
    bool df = false;  // complex128 gemm_small in double-FP32 arithmetic
    // The FP64-class tall products (zgemm_cn_df, zgemm_nn_df, zgemm_cn_lower with df) run on the
    // tensor cores with exact 8-bit BF16 slices (oz_gemm.cu) instead of double-FP32 CUDA cores.
    bool oz = false;
    DevBuf oz_a, oz_e, oz_p;  // digit tiles, chunk exponents, FP64 partial tiles
};
template <typename R>
int gemm_cn(GemmWork &w, int m, int n, int K, R alpha, const cx<R> *A, int lda, const cx<R> *B, int ldb,
            R beta, cx<R> *C, int ldc, cudaStream_t s);
// Lower triangle of C = A^H B (n x n, complex128): 64 x 64 tiles strictly above the
// diagonal are skipped (Hermitian Grams whose consumers read the lower triangle only).
// df = true: double-FP32 arithmetic (FP64 class, ~2^-47 per product) instead of FP64.
int zgemm_cn_lower(GemmWork &w, int n, int K, const z64 *A, int lda, const z64 *B, int ldb, z64 *C, int ldc,
                   cudaStream_t s, bool df = false);
// Complex128 C = alpha A^H B + beta C and D = alpha A B + beta C in double-FP32
// arithmetic on the FP32 units (tall products; K split as for gemm_cn).
int zgemm_cn_df(GemmWork &w, int m, int n, int K, double alpha, const z64 *A, int lda, const z64 *B, int ldb,
                double beta, z64 *C, int ldc, cudaStream_t s);
// w (nullable) carries the engine choice (w->oz) and its scratch.
int zgemm_nn_df(GemmWork *w, int M, int n, int k, double alpha, const z64 *A, int lda, const z64 *B, int ldb,
                double beta, const z64 *C, int ldc, z64 *D, int ldd, cudaStream_t s);
// FP64-class complex128 products on the tensor cores: digits of 8 bits (six BF16 slices per real
// value, per-64-term chunk power-of-two scales), exact FP32 accumulation per chunk, double-FP32
// sums across chunks (error about 2^-44 of sum |a||b|).  C = alpha A^H B + beta C (lower: only
// i >= j written) and D = alpha A B + beta C.
int oz_gemm_cn(GemmWork &w, int m, int n, int K, double alpha, const z64 *A, int lda, const z64 *B, int ldb,
               double beta, z64 *C, int ldc, cudaStream_t s, bool lower);
int oz_gemm_nn(GemmWork &w, int M, int n, int k, double alpha, const z64 *A, int lda, const z64 *B, int ldb,
               double beta, const z64 *C, int ldc, z64 *D, int ldd, cudaStream_t s);
int oz_check_error();   // LOBPCG_ERR_TIMEOUT if a wait inside oz_gemm ran out (clears the flag)
// Complex64 products on the tensor cores (3xTF32 split operands, FP32 accumulation):
// C = alpha A^H B + beta C (K split over the GPU, FP64 partial sums) and
// D = alpha A B + beta C.  gemm_cn<float> / gemm_nn<float> route here for long
// reductions / tall products unless the GEMM mode says otherwise.
int tc_gemm_cn(GemmWork &w, int m, int n, int K, float alpha, const c32 *A, int lda, const c32 *B, int ldb,
               float beta, c32 *C, int ldc, cudaStream_t s);
// Poll limit of the tensor-core GEMMs' ring waits on the current device (< 0: the default).
int tc_set_spin_limit(long long polls);
int tc_gemm_nn(int M, int n, int k, float alpha, const c32 *A, int lda, const c32 *B, int ldb, float beta,
               const c32 *C, int ldc, c32 *D, int ldd, cudaStream_t s);
int tc_check_error();   // LOBPCG_ERR_TIMEOUT if a bounded device wait ran out (clears the flag)
int *device_wait_flag(); // device address of that flag (kernels with bounded waits set it)
// FP32 GEMM engine, process-wide: 0 = auto / 2 = tensor cores (TF32x3) where the shape suits them,
// 3 = CUDA cores only.
void set_gemm_mode(int mode);
int gemm_mode();
template <typename R>
int gemm_nn(int M, int n, int k, R alpha, const cx<R> *A, int lda, const cx<R> *B, int ldb, R beta,
            const cx<R> *C, int ldc, cx<R> *D, int ldd, cudaStream_t s);
// Small general complex128 product: C = alpha op(A) op(B) + beta C, op in {'N','C'}.
// Small general complex product in precision R; w (nullable) enables a split of the reduction dimension.
template <typename R>
int gemm_small(GemmWork *w, char opA, char opB, int m, int n, int k, double alpha, const cx<R> *A, int lda,
               const cx<R> *B, int ldb, double beta, cx<R> *C, int ldc, cudaStream_t s);
// w (nullable) enables a split of the reduction dimension.
int zgemm_small(GemmWork *w, char opA, char opB, int m, int n, int k, double alpha, const z64 *A, int lda,
                const z64 *B, int ldb, double beta, z64 *C, int ldc, cudaStream_t s);

// ------------------------------------------------------------------ Gamma-point real form (vec.cu)
// Packed half-sphere storage of real-form vectors (c(-G) = conj(c(G))): z[0] = c(0), z[g] =
// sqrt(2) c(G_g) for G_g in the half set; half[g] / mirror[g]: sphere positions of G_g / -G_g.
template <typename R>
int gamma_pack_full(int nz, int nb, const cx<R> *C, int ldc, const int *half, const int *mirror, cx<R> *Z, int ldz,
                    cudaStream_t s);
template <typename R>
int gamma_unpack_full(int nz, int nb, const cx<R> *Z, int ldz, const int *half, const int *mirror, cx<R> *C, int ldc,
                      cudaStream_t s);
// bands 2i, 2i+1 of Z -> sphere column i of C as c_a + i c_b, and back from Y = H C
template <typename R>
int gamma_unpack_pairs(int nz, int nb, const cx<R> *Z, int ldz, const int *half, const int *mirror, cx<R> *C, int ldc,
                       cudaStream_t s);
template <typename R>
int gamma_pack_pairs(int nz, int nb, const cx<R> *Y, int ldy, const int *half, const int *mirror, cx<R> *Z, int ldz,
                     cudaStream_t s);
template <typename R>
int zero_imag(int rows, int cols, cx<R> *A, int lda, cudaStream_t s);

// ------------------------------------------------------------------ band-by-band PCG (pcg.cu)
// Device-side steps of one band of the PCG comparison method: every scalar lives in sc (device),
// so a band iteration never waits for the host.  Vectors are npw long, FP64; Y (npw x j, ld ldy)
// holds the orthonormal bands before this one.
struct PcgBand {
    int npw = 0, j = 0, ldy = 0;
    cudaStream_t s = nullptr;
    const double *kin = nullptr;
    const z64 *Y = nullptr;
    z64 *x = nullptr, *hx = nullptr, *xi = nullptr, *eta = nullptr, *d = nullptr, *dh = nullptr, *hd = nullptr;
    double *part = nullptr, *sc = nullptr;   // reduction partials, scalar block (16 doubles)
    z64 *gpart = nullptr, *G = nullptr;      // projection partials and coefficients
    int prepare_start();                     // x off span(Y), normalised
    int after_hx();                          // eps = <x|Hx>, Ekin(x)
    int direction(bool first);               // steps 1-5: dh (normalised search direction)
    int step();                              // step 6 with hd = H dh: line minimum, x and Hx updated
    int project(z64 *v, const z64 *x);       // v off span(Y) twice, then off x (x may be NULL)
    int sums(int nq, const z64 *a0, const z64 *b0, const z64 *a1, const z64 *b1, const z64 *a2, const z64 *b2,
             int mode, int act);
    int vec(int op, z64 *v, const z64 *a, const z64 *b, z64 *w);
};
// Doubles of scratch a PcgBand needs for npw plane waves and up to M earlier bands (part, sc,
// gpart, G carved from one buffer).
size_t pcg_scratch_doubles(int npw, int M);
void pcg_carve(PcgBand &pb, double *base, int npw, int M);   // sets sc, part, gpart, G

// ------------------------------------------------------------------ dense FP64 eigen-solvers
// Orders the cooperative launches (grid-barrier kernels) of concurrent streams one after
// another, so that two such grids never compete for residency.
struct CoopGate {
    std::mutex mu;
    cudaEvent_t ev = nullptr;
    bool used = false;
};
struct EigWork {
    Allocator *alloc = nullptr;
    DevBuf buf;      // generic workspace
    DevBuf ibuf;     // integer workspace
    GemmWork gw;
    CoopGate *gate = nullptr;  // set when several streams may run Rayleigh-Ritz steps at once
    int coop_share = 1;        // >1: cooperative grids use at most 1/coop_share of the resident blocks
    // FP64 Rayleigh-Ritz: run the parts limited by one SM's FP64 units (Cholesky diagonal
    // blocks, the tridiagonalisation's column work, the small products) in double-FP32
    bool df = false;
};
// Rayleigh-Ritz: lowest m pairs of A c = theta S c (n x n, ld n). See lobpcg_k_rayleigh_ritz.
// lead (a multiple of 32): the first lead columns of S are known to be the identity's (an
// orthonormal block orthogonal to the rest), so their factorisation is skipped.
int rayleigh_ritz(EigWork &w, int n, int m, const z64 *S, int lds, const z64 *A, int lda, double drop_tol,
                  double *theta, z64 *C, int ldc, int *ndropped, cudaStream_t s, int lead = 0);
// The same Rayleigh-Ritz in FP32 arithmetic (complex64 pencil, float Ritz values).
int rayleigh_ritz32(EigWork &w, int n, int m, const c32 *S, int lds, const c32 *A, int lda, double drop_tol,
                    float *theta, c32 *C, int ldc, int *ndropped, cudaStream_t s);
// Copy the lower triangle of A (n x n, ld n) onto the upper one (imaginary diagonal cleared).
int hermitize_lower(EigWork &w, int n, z64 *A, cudaStream_t s);
// Lowest m eigenpairs of a Hermitian matrix (n x n, ld lda, lower triangle; overwritten).
int heev_lowest(EigWork &w, int n, int m, z64 *A, int lda, double *theta, z64 *V, int ldv, cudaStream_t s);

// ------------------------------------------------------------------ vector kernels
template <typename R>
int residual_precond(int npw, int m, const z64 *X, int ldx, const z64 *HX, int ldhx, const double *theta,
                     const double *kin, cx<R> *W, int ldw, double *work, double *part, cudaStream_t s);
// Mixed schedule: R = HX - X theta (FP64) stored in FP32, and W = K(R) in FP32.
int residual_precond_mixed(int npw, int m, const z64 *X, int ldx, const z64 *HX, int ldhx, const double *theta,
                           const double *kin, c32 *R, c32 *W, int ld, double *work, double *part, cudaStream_t s);
// V += alpha D (FP64 columns).
int axpy_cols(int rows, int cols, double alpha, const z64 *D, int ldd, z64 *V, int ldv, cudaStream_t s);
// Assemble the FP64 Rayleigh-Ritz pencil of the mixed schedule (see api.cu).
int assemble_gram_mixed(int nz, int mx, const c32 *S32, int lds32, const c32 *A32, int lda32, const double *theta,
                        z64 *S, z64 *A, cudaStream_t s);
// Overwrite diag(S) = diag(X^H X), diag(A) = diag(X^H HX) in FP64 (m x m, ld m).
int diag_pencil(int npw, int m, const z64 *X, int ldx, const z64 *HX, int ldhx, z64 *S, z64 *A, double *part,
                cudaStream_t s);
// Deterministic pseudo-random complex entries in [-1, 1) (buffer-band start vectors).
int fill_random(int rows, int cols, z64 *X, int ldx, unsigned seed, cudaStream_t s);
int column_resid_norms(int npw, int m, const z64 *X, int ldx, const z64 *HX, int ldhx, const double *theta,
                       double *out, double *part, cudaStream_t s);
// FP32-output pencil assembly, FP64 Rayleigh quotients, FP32 residual and preconditioner (mixed schedule).
int assemble_gram_mixed32(int nz, int mx, const c32 *S32, int lds32, const c32 *A32, int lda32, const double *theta,
                          c32 *S, c32 *A, cudaStream_t s);
int rayleigh_quotients(int npw, int m, const z64 *X, int ldx, const z64 *HX, int ldhx, double *theta, double *part,
                       cudaStream_t s);
// E = C - I (leading rows x cols, FP32) and its largest component magnitude on the host (synchronises).
int near_identity32(int rows, int cols, const z64 *C, int ldc, c32 *E, int lde, unsigned int *dmax, float *hmax,
                    cudaStream_t s);
// Scale column j of C by conj(C_jj)/|C_jj| (leading rows x cols, j < min(rows, cols)).
int fix_phases(int rows, int cols, z64 *C, int ldc, cudaStream_t s);
// out = A + fp64(T).
int add_cast(int rows, int cols, const z64 *A, int lda, const c32 *T, int ldt, z64 *out, int ldo, cudaStream_t s);
int residual32(int npw, int m, const z64 *X, int ldx, const z64 *HX, int ldhx, const double *theta, c32 *R, int ldr,
               cudaStream_t s);
int precond32(int npw, int m, const z64 *X, int ldx, const double *kin, const c32 *R, int ldr, c32 *W, int ldw,
              double *work, double *part, cudaStream_t s);
// Per-column sums (kinetic energies, Rayleigh quotients, pencil diagonals, residual norms) take a
// scratch `part` of colsum_part_elems(m) doubles: their rows are split over many blocks and the
// partials added in a fixed order.  part = NULL: one block per column.
size_t colsum_part_elems(int m);
template <typename Ro, typename Ri>
int copy_cast(int rows, int cols, const cx<Ri> *A, int lda, cx<Ro> *B, int ldb, cudaStream_t s);
int scale_rows_real(int rows, int cols, const double *d, z64 *A, int lda, cudaStream_t s);
template <typename R>
int scale_rows(int rows, int cols, const R *d, cx<R> *A, int lda, cudaStream_t s);

}  // namespace lg
