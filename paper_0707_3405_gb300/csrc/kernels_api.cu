// C ABI of the dense building blocks (include/lobpcg_gb300_kernels.h): the
// GEMMs and FP64 eigen-solvers of one LOBPCG block iteration, callable on
// their own.  Scratch memory comes from one library-owned pool.
#include "common.cuh"
#include "lobpcg_gb300_kernels.h"

#include <mutex>

using namespace lg;

namespace {

struct Pool {
    Allocator alloc;
    GemmWork gw;
    EigWork ew;
    Pool() {
        gw.alloc = &alloc;
        ew.alloc = &alloc;
        ew.gw.alloc = &alloc;
    }
};

Pool &pool() {
    static Pool p;
    return p;
}
std::mutex &pool_mutex() {
    static std::mutex mu;
    return mu;
}

}  // namespace

extern "C" {

namespace {
// Engine flag of the pool's GEMM scratch for one call (FP64-class on the tensor cores or not).
struct OzScope {
    GemmWork &w;
    OzScope(GemmWork &w_, bool on) : w(w_) { w.oz = on; }
    ~OzScope() { w.oz = false; }
};
}  // namespace

int lobpcg_k_gemm_cn(int prec, int m, int n, int K, double alpha, const void *A, int lda, const void *B, int ldb,
                     double beta, void *C, int ldc, void *stream) {
    if (prec != LOBPCG_C128 && prec != LOBPCG_C128_DF32 && prec != LOBPCG_C128_TC && prec != LOBPCG_C64)
        return fail(LOBPCG_ERR_ARG, "unknown precision");
    if (m < 0 || n < 0 || K < 0) return fail(LOBPCG_ERR_ARG, "negative size");
    if (m == 0 || n == 0) return LOBPCG_OK;
    if (!A || !B || !C || lda < K || ldb < K || ldc < m) return fail(LOBPCG_ERR_ARG, "bad pointer or leading dimension");
    std::lock_guard<std::mutex> lk(pool_mutex());
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (prec == LOBPCG_C128)
        return gemm_cn<double>(pool().gw, m, n, K, alpha, static_cast<const z64 *>(A), lda, static_cast<const z64 *>(B),
                               ldb, beta, static_cast<z64 *>(C), ldc, s);
    if (prec == LOBPCG_C128_DF32 || prec == LOBPCG_C128_TC) {
        OzScope oz(pool().gw, prec == LOBPCG_C128_TC);
        return zgemm_cn_df(pool().gw, m, n, K, alpha, static_cast<const z64 *>(A), lda, static_cast<const z64 *>(B),
                           ldb, beta, static_cast<z64 *>(C), ldc, s);
    }
    if (prec == LOBPCG_C64)
        return gemm_cn<float>(pool().gw, m, n, K, (float)alpha, static_cast<const c32 *>(A), lda,
                              static_cast<const c32 *>(B), ldb, (float)beta, static_cast<c32 *>(C), ldc, s);
    return fail(LOBPCG_ERR_ARG, "unknown precision");
}

int lobpcg_k_gram_lower(int prec, int n, int K, const void *A, int lda, const void *B, int ldb, void *C,
                        int ldc, void *stream) {
    if (prec != LOBPCG_C128 && prec != LOBPCG_C128_DF32 && prec != LOBPCG_C128_TC)
        return fail(LOBPCG_ERR_ARG, "unknown precision");
    if (n < 0 || K < 0) return fail(LOBPCG_ERR_ARG, "negative size");
    if (n == 0) return LOBPCG_OK;
    if (!A || !B || !C || lda < K || ldb < K || ldc < n) return fail(LOBPCG_ERR_ARG, "bad pointer or leading dimension");
    std::lock_guard<std::mutex> lk(pool_mutex());
    OzScope oz(pool().gw, prec == LOBPCG_C128_TC);
    return zgemm_cn_lower(pool().gw, n, K, static_cast<const z64 *>(A), lda, static_cast<const z64 *>(B), ldb,
                          static_cast<z64 *>(C), ldc, reinterpret_cast<cudaStream_t>(stream),
                          prec != LOBPCG_C128);
}

int lobpcg_k_gemm_nn(int prec, int M, int n, int k, double alpha, const void *A, int lda, const void *B, int ldb,
                     double beta, const void *C, int ldc, void *D, int ldd, void *stream) {
    if (prec != LOBPCG_C128 && prec != LOBPCG_C128_DF32 && prec != LOBPCG_C128_TC && prec != LOBPCG_C64)
        return fail(LOBPCG_ERR_ARG, "unknown precision");
    if (M < 0 || n < 0 || k < 0) return fail(LOBPCG_ERR_ARG, "negative size");
    if (M == 0 || n == 0) return LOBPCG_OK;
    if (!A || !B || !D || lda < M || ldb < k || ldd < M || (beta != 0.0 && (!C || ldc < M)))
        return fail(LOBPCG_ERR_ARG, "bad pointer or leading dimension");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (prec == LOBPCG_C128)
        return gemm_nn<double>(M, n, k, alpha, static_cast<const z64 *>(A), lda, static_cast<const z64 *>(B), ldb, beta,
                               static_cast<const z64 *>(C), ldc, static_cast<z64 *>(D), ldd, s);
    if (prec == LOBPCG_C128_DF32)
        return zgemm_nn_df(nullptr, M, n, k, alpha, static_cast<const z64 *>(A), lda, static_cast<const z64 *>(B), ldb,
                           beta, static_cast<const z64 *>(C), ldc, static_cast<z64 *>(D), ldd, s);
    if (prec == LOBPCG_C128_TC) {
        std::lock_guard<std::mutex> lk(pool_mutex());
        OzScope oz(pool().gw, true);
        return zgemm_nn_df(&pool().gw, M, n, k, alpha, static_cast<const z64 *>(A), lda, static_cast<const z64 *>(B),
                           ldb, beta, static_cast<const z64 *>(C), ldc, static_cast<z64 *>(D), ldd, s);
    }
    if (prec == LOBPCG_C64)
        return gemm_nn<float>(M, n, k, (float)alpha, static_cast<const c32 *>(A), lda, static_cast<const c32 *>(B), ldb,
                              (float)beta, static_cast<const c32 *>(C), ldc, static_cast<c32 *>(D), ldd, s);
    return fail(LOBPCG_ERR_ARG, "unknown precision");
}

int lobpcg_k_rayleigh_ritz(int n, int m, const void *S, const void *A, double drop_tol, double *theta, void *C,
                           int *ndropped, void *stream) {
    if (n < 1 || m < 1 || m > n || n > 4096) return fail(LOBPCG_ERR_ARG, "need 1 <= m <= n <= 4096");
    if (!S || !A || !theta || !C) return fail(LOBPCG_ERR_ARG, "NULL pointer");
    std::lock_guard<std::mutex> lk(pool_mutex());
    return rayleigh_ritz(pool().ew, n, m, static_cast<const z64 *>(S), n, static_cast<const z64 *>(A), n, drop_tol,
                         theta, static_cast<z64 *>(C), n, ndropped, reinterpret_cast<cudaStream_t>(stream));
}

int lobpcg_k_rayleigh_ritz_df32(int n, int m, const void *S, const void *A, double drop_tol, double *theta, void *C,
                                int *ndropped, void *stream) {
    if (n < 1 || m < 1 || m > n || n > 4096) return fail(LOBPCG_ERR_ARG, "need 1 <= m <= n <= 4096");
    if (!S || !A || !theta || !C) return fail(LOBPCG_ERR_ARG, "NULL pointer");
    std::lock_guard<std::mutex> lk(pool_mutex());
    EigWork &ew = pool().ew;
    ew.df = true;
    const int rc = rayleigh_ritz(ew, n, m, static_cast<const z64 *>(S), n, static_cast<const z64 *>(A), n, drop_tol,
                                 theta, static_cast<z64 *>(C), n, ndropped, reinterpret_cast<cudaStream_t>(stream));
    ew.df = false;
    return rc;
}

int lobpcg_k_rayleigh_ritz32(int n, int m, const void *S, const void *A, double drop_tol, float *theta, void *C,
                             int *ndropped, void *stream) {
    if (n < 1 || m < 1 || m > n || n > 4096) return fail(LOBPCG_ERR_ARG, "need 1 <= m <= n <= 4096");
    if (!S || !A || !theta || !C) return fail(LOBPCG_ERR_ARG, "NULL pointer");
    std::lock_guard<std::mutex> lk(pool_mutex());
    return rayleigh_ritz32(pool().ew, n, m, static_cast<const c32 *>(S), n, static_cast<const c32 *>(A), n, drop_tol,
                           theta, static_cast<c32 *>(C), n, ndropped, reinterpret_cast<cudaStream_t>(stream));
}

int lobpcg_k_heev(int n, const void *A, double *w, void *V, void *stream) {
    if (n < 1 || n > 4096) return fail(LOBPCG_ERR_ARG, "need 1 <= n <= 4096");
    if (!A || !w || !V) return fail(LOBPCG_ERR_ARG, "NULL pointer");
    std::lock_guard<std::mutex> lk(pool_mutex());
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // work on a copy (the tridiagonalisation overwrites its input)
    DevBuf cp;
    int rc = pool().alloc.ensure(cp, sizeof(z64) * (size_t)n * n);
    if (rc < 0) return rc;
    cudaError_t e = cudaMemcpyAsync(cp.p, A, sizeof(z64) * (size_t)n * n, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) {
        pool().alloc.release(cp);
        return fail(LOBPCG_ERR_CUDA, cudaGetErrorString(e));
    }
    rc = hermitize_lower(pool().ew, n, static_cast<z64 *>(cp.p), s);
    if (rc == 0) rc = heev_lowest(pool().ew, n, n, static_cast<z64 *>(cp.p), n, w, static_cast<z64 *>(V), n, s);
    cudaStreamSynchronize(s);
    pool().alloc.release(cp);
    return rc;
}

int lobpcg_k_set_gemm_mode(int mode) {
    if (mode != 0 && mode != 2 && mode != 3) return fail(LOBPCG_ERR_ARG, "gemm mode must be 0, 2 or 3");
    set_gemm_mode(mode);
    return LOBPCG_OK;
}

int lobpcg_k_set_spin_limit(long long polls) { return tc_set_spin_limit(polls); }

int lobpcg_k_check_timeouts(void) {
    LG_CUDA_TRY(cudaDeviceSynchronize());
    return tc_check_error();
}

const char *lobpcg_k_last_error(void) { return global_error(); }

}  // extern "C"
