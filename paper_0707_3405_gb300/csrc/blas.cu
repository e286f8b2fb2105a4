// Complex GEMMs on the CUDA cores (FP64 and FP32): the Gram, projection,
// constraint and update contractions of Algorithm 1 (Sec. 3.2; the paper
// runs them as zgemm, Sec. 4.1 and 5.1) and the small dense products of the
// Rayleigh-Ritz step.
//
// One tiled kernel serves every operand form: op(A) and op(B) are either the
// matrix or its conjugate transpose, chosen at compile time so that tile
// loads stay coalesced.  64 x 64 output tile, K step 16, 256 threads, each
// thread owning a 4 x 4 register tile (rows tx + 16 i, columns ty + 16 j, so
// stores to column-major C are coalesced).  A long reduction dimension is
// split over grid.z; the partial tiles are summed afterwards in a fixed
// order, so results are bitwise reproducible.
#include "common.cuh"

#include <algorithm>

namespace lg {

namespace {

constexpr int BM = 64, BN = 64, BK = 16, TH = 256;

template <typename R, bool CA, bool CB>
__global__ void __launch_bounds__(TH)
k_gemm(int m, int n, int K, int kchunk, R alpha, const cx<R> *__restrict__ A, int lda,
       const cx<R> *__restrict__ B, int ldb, R beta, const cx<R> *C, int ldc, cx<R> *D, int ldd,
       cx<R> *__restrict__ part) {
    __shared__ cx<R> As[BK][BM + 1];
    __shared__ cx<R> Bs[BK][BN + 1];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int i0 = blockIdx.x * BM, j0 = blockIdx.y * BN;
    const int kbeg = blockIdx.z * kchunk;
    const int kend = min(K, kbeg + kchunk);
    const cx<R> zero = mkc<R>(0, 0);
    cx<R> acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = zero;

    for (int k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
        for (int r = 0; r < (BK * BM) / TH; ++r) {
            const int e = tid + r * TH;
            int i, kk;
            if (!CA) { i = e % BM; kk = e / BM; } else { kk = e % BK; i = e / BK; }
            const int gi = i0 + i, gk = k0 + kk;
            cx<R> v = zero;
            if (gi < m && gk < kend) v = CA ? conjc(A[(size_t)gi * lda + gk]) : A[(size_t)gk * lda + gi];
            As[kk][i] = v;
        }
#pragma unroll
        for (int r = 0; r < (BK * BN) / TH; ++r) {
            const int e = tid + r * TH;
            int j, kk;
            if (!CB) { kk = e % BK; j = e / BK; } else { j = e % BN; kk = e / BN; }
            const int gj = j0 + j, gk = k0 + kk;
            cx<R> v = zero;
            if (gj < n && gk < kend) v = CB ? conjc(B[(size_t)gk * ldb + gj]) : B[(size_t)gj * ldb + gk];
            Bs[kk][j] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            cx<R> a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][tx + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][ty + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) fma_nn(acc[i][j], a[i], b[j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int gj = j0 + ty + 16 * j;
        if (gj >= n) continue;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int gi = i0 + tx + 16 * i;
            if (gi >= m) continue;
            if (part) {
                part[((size_t)blockIdx.z * n + gj) * m + gi] = acc[i][j];
            } else {
                cx<R> v = alpha * acc[i][j];
                if (beta != (R)0) v = v + beta * C[(size_t)gj * ldc + gi];
                D[(size_t)gj * ldd + gi] = v;
            }
        }
    }
}

template <typename R>
__global__ void k_reduce_parts(int m, int n, int nsplit, R alpha, const cx<R> *__restrict__ part, R beta,
                               const cx<R> *C, int ldc, cx<R> *D, int ldd) {
    const size_t tot = (size_t)m * n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        const int gi = (int)(e % m), gj = (int)(e / m);
        cx<R> s = part[e];
        for (int z = 1; z < nsplit; ++z) s = s + part[(size_t)z * tot + e];
        cx<R> v = alpha * s;
        if (beta != (R)0) v = v + beta * C[(size_t)gj * ldc + gi];
        D[(size_t)gj * ldd + gi] = v;
    }
}

int num_sms() {
    static int v = 0;
    if (!v) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 132;
    }
    return v;
}

// Launch op(A) op(B) with an optional split of the reduction dimension.
template <typename R, bool CA, bool CB>
int launch_gemm(GemmWork *w, int m, int n, int K, R alpha, const cx<R> *A, int lda, const cx<R> *B, int ldb,
                R beta, const cx<R> *C, int ldc, cx<R> *D, int ldd, cudaStream_t s, bool allow_split) {
    if (m <= 0 || n <= 0) return LOBPCG_OK;
    const int tm = (m + BM - 1) / BM, tn = (n + BN - 1) / BN;
    const int tiles = tm * tn;
    int nsplit = 1;
    if (allow_split && w && K > 4 * BK) {
        const int want = (2 * num_sms() + tiles - 1) / tiles;
        const int maxs = (K + 4 * BK - 1) / (4 * BK);
        nsplit = std::max(1, std::min(want, maxs));
    }
    if (K <= 0) nsplit = 1;
    int kchunk = (K + nsplit - 1) / nsplit;
    kchunk = ((kchunk + BK - 1) / BK) * BK;
    if (kchunk <= 0) kchunk = BK;
    nsplit = K > 0 ? (K + kchunk - 1) / kchunk : 1;
    if (nsplit == 1) {
        k_gemm<R, CA, CB><<<dim3(tm, tn, 1), TH, 0, s>>>(m, n, K, kchunk, alpha, A, lda, B, ldb, beta, C, ldc, D,
                                                         ldd, nullptr);
        return check_launch("gemm");
    }
    const size_t need = sizeof(cx<R>) * (size_t)nsplit * m * n;
    LG_TRY(w->alloc->ensure(w->part, need));
    cx<R> *part = reinterpret_cast<cx<R> *>(w->part.p);
    k_gemm<R, CA, CB><<<dim3(tm, tn, nsplit), TH, 0, s>>>(m, n, K, kchunk, alpha, A, lda, B, ldb, beta, C, ldc, D,
                                                          ldd, part);
    LG_TRY(check_launch("gemm split"));
    const size_t tot = (size_t)m * n;
    const int blocks = (int)std::min<size_t>((tot + 255) / 256, 4096);
    k_reduce_parts<R><<<blocks, 256, 0, s>>>(m, n, nsplit, alpha, part, beta, C, ldc, D, ldd);
    return check_launch("gemm reduce");
}

}  // namespace

template <typename R>
int gemm_cn(GemmWork &w, int m, int n, int K, R alpha, const cx<R> *A, int lda, const cx<R> *B, int ldb, R beta,
            cx<R> *C, int ldc, cudaStream_t s) {
    return launch_gemm<R, true, false>(&w, m, n, K, alpha, A, lda, B, ldb, beta, C, ldc, C, ldc, s, true);
}

template <typename R>
int gemm_nn(int M, int n, int k, R alpha, const cx<R> *A, int lda, const cx<R> *B, int ldb, R beta,
            const cx<R> *C, int ldc, cx<R> *D, int ldd, cudaStream_t s) {
    return launch_gemm<R, false, false>(nullptr, M, n, k, alpha, A, lda, B, ldb, beta, C, ldc, D, ldd, s, false);
}

int zgemm_small(char opA, char opB, int m, int n, int k, double alpha, const z64 *A, int lda, const z64 *B,
                int ldb, double beta, z64 *C, int ldc, cudaStream_t s) {
    const bool ca = (opA == 'C'), cb = (opB == 'C');
    if (!ca && !cb) return launch_gemm<double, false, false>(nullptr, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, C, ldc, s, false);
    if (ca && !cb) return launch_gemm<double, true, false>(nullptr, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, C, ldc, s, false);
    if (!ca && cb) return launch_gemm<double, false, true>(nullptr, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, C, ldc, s, false);
    return launch_gemm<double, true, true>(nullptr, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, C, ldc, s, false);
}

template int gemm_cn<double>(GemmWork &, int, int, int, double, const z64 *, int, const z64 *, int, double, z64 *,
                             int, cudaStream_t);
template int gemm_cn<float>(GemmWork &, int, int, int, float, const c32 *, int, const c32 *, int, float, c32 *, int,
                            cudaStream_t);
template int gemm_nn<double>(int, int, int, double, const z64 *, int, const z64 *, int, double, const z64 *, int,
                             z64 *, int, cudaStream_t);
template int gemm_nn<float>(int, int, int, float, const c32 *, int, const c32 *, int, float, const c32 *, int, c32 *,
                            int, cudaStream_t);

}  // namespace lg
