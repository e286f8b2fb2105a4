// Complex GEMMs on the CUDA cores (FP64 and FP32): the Gram, projection,
// constraint and update contractions of Algorithm 1 (Sec. 3.2; the paper
// runs them as zgemm, Sec. 4.1 and 5.1) and the small dense products of the
// Rayleigh-Ritz step.
//
// One tiled kernel serves every operand form: op(A) and op(B) are either the
// matrix or its conjugate transpose, chosen at compile time so that tile
// loads stay coalesced.  K step 16, 256 threads, each thread owning a T x T
// register tile (rows tx + 16 i, columns ty + 16 j, so stores to column-major
// C are coalesced): 64 x 64 output tiles for tall-skinny and large products,
// 32 x 32 for the small dense ones.  A long reduction dimension is
// split over grid.z; the partial tiles are summed afterwards in a fixed
// order, so results are bitwise reproducible.
#include "common.cuh"

#include <algorithm>
#include <type_traits>

namespace lg {

namespace {

constexpr int BK = 16, TH = 256;

// T x T register tile per thread, 16 x 16 threads: (16 T) x (16 T) output tile.
// FP32 products are accumulated in FP32 for at most KFLUSH terms and then added
// into FP64 accumulators, so that long reductions (the plane-wave count) keep
// about 1e-6 relative accuracy; split partial sums are FP64.
constexpr int KFLUSH = 256;

template <typename R, bool CA, bool CB, int T>
__global__ void __launch_bounds__(TH)
k_gemm(int m, int n, int K, int kchunk, R alpha, const cx<R> *__restrict__ A, int lda,
       const cx<R> *__restrict__ B, int ldb, R beta, const cx<R> *C, int ldc, cx<R> *D, int ldd,
       z64 *__restrict__ part, int lower) {
    constexpr int BM = 16 * T, BN = 16 * T;
    __shared__ cx<R> As[BK][BM + 1];
    __shared__ cx<R> Bs[BK][BN + 1];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int i0 = blockIdx.x * BM, j0 = blockIdx.y * BN;
    // lower-triangle output: a tile strictly above the diagonal is neither computed nor written
    if (lower && blockIdx.x < blockIdx.y) return;
    const int kbeg = blockIdx.z * kchunk;
    const int kend = min(K, kbeg + kchunk);
    const cx<R> zero = mkc<R>(0, 0);
    constexpr bool F32 = sizeof(R) == 4;
    cx<R> acc[T][T];
    z64 acc64[F32 ? T : 1][F32 ? T : 1];
#pragma unroll
    for (int i = 0; i < T; ++i)
#pragma unroll
        for (int j = 0; j < T; ++j) acc[i][j] = zero;
    if (F32) {
#pragma unroll
        for (int i = 0; i < (F32 ? T : 1); ++i)
#pragma unroll
            for (int j = 0; j < (F32 ? T : 1); ++j) acc64[i][j] = mkc(0.0, 0.0);
    }
    int since_flush = 0;

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
            cx<R> a[T], b[T];
#pragma unroll
            for (int i = 0; i < T; ++i) a[i] = As[kk][tx + 16 * i];
#pragma unroll
            for (int j = 0; j < T; ++j) b[j] = Bs[kk][ty + 16 * j];
#pragma unroll
            for (int i = 0; i < T; ++i)
#pragma unroll
                for (int j = 0; j < T; ++j) fma_nn(acc[i][j], a[i], b[j]);
        }
        __syncthreads();
        if (F32) {
            since_flush += BK;
            if (since_flush >= KFLUSH) {
                since_flush = 0;
#pragma unroll
                for (int i = 0; i < (F32 ? T : 1); ++i)
#pragma unroll
                    for (int j = 0; j < (F32 ? T : 1); ++j) {
                        acc64[i][j] = acc64[i][j] + cvt<double, R>(acc[i][j]);
                        acc[i][j] = zero;
                    }
            }
        }
    }
#pragma unroll
    for (int j = 0; j < T; ++j) {
        const int gj = j0 + ty + 16 * j;
        if (gj >= n) continue;
#pragma unroll
        for (int i = 0; i < T; ++i) {
            const int gi = i0 + tx + 16 * i;
            if (gi >= m) continue;
            z64 t = cvt<double, R>(acc[i][j]);
            if (F32) t = t + acc64[F32 ? i : 0][F32 ? j : 0];
            if (part) {
                part[((size_t)blockIdx.z * n + gj) * m + gi] = t;
            } else {
                z64 v = (double)alpha * t;
                if (beta != (R)0) v = v + (double)beta * cvt<double, R>(C[(size_t)gj * ldc + gi]);
                D[(size_t)gj * ldd + gi] = cvt<R, double>(v);
            }
        }
    }
}

// ------------------------------------------------------------------ double-FP32 engine
// FP64-class complex products without FP64 arithmetic in the inner loop (this
// GPU runs FP64 at a small fraction of its FP32 rate).  Each operand is split
// into an unevaluated pair of FP32 numbers x = hi + lo (|lo| <= 2^-24 |hi|).
// A real product is formed as hi*hi exactly (Dekker's TwoProd through one FMA)
// plus the two cross terms hi*lo and lo*hi; the accumulator is a pair too, and
// each product enters it through Knuth's TwoSum, so nothing of the high part is
// ever rounded away.  The neglected lo*lo term and the FP32 rounding of the
// low-order parts leave about 2^-47 relative per product (FP64 class).  Tiles,
// split and summation order are those of k_gemm; partial tiles are FP64.
struct dfc {
    float rh, rl, ih, il;  // Re = rh + rl, Im = ih + il
};

__device__ __forceinline__ dfc to_dfc(z64 v, bool conj) {
    const float rh = __double2float_rn(v.x), ih = __double2float_rn(v.y);
    const float rl = __double2float_rn(v.x - (double)rh), il = __double2float_rn(v.y - (double)ih);
    return conj ? dfc{rh, rl, -ih, -il} : dfc{rh, rl, ih, il};
}

// (sh, sl) += (xh + xl)(yh + yl); the intrinsics keep the compiler from contracting the steps.
__device__ __forceinline__ void df_mac(float &sh, float &sl, float xh, float xl, float yh, float yl) {
    const float p = __fmul_rn(xh, yh);
    float e = __fmaf_rn(xh, yh, -p);
    e = __fmaf_rn(xh, yl, e);
    e = __fmaf_rn(xl, yh, e);
    const float t = __fadd_rn(sh, p);
    const float z = __fsub_rn(t, sh);
    const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, z)), __fsub_rn(p, z));
    sh = t;
    sl = __fadd_rn(sl, __fadd_rn(err, e));
}

__device__ __forceinline__ void df_norm(float &h, float &l) {
    const float t = __fadd_rn(h, l);
    l = __fsub_rn(l, __fsub_rn(t, h));
    h = t;
}

template <bool CA, bool CB, int T>
__global__ void __launch_bounds__(TH, 2)
k_gemm_df(int m, int n, int K, int kchunk, double alpha, const z64 *__restrict__ A, int lda,
          const z64 *__restrict__ B, int ldb, double beta, const z64 *C, int ldc, z64 *D, int ldd,
          z64 *__restrict__ part, int lower) {
    constexpr int BM = 16 * T, BN = 16 * T;
    __shared__ dfc As[BK][BM + 1];
    __shared__ dfc Bs[BK][BN + 1];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int i0 = blockIdx.x * BM, j0 = blockIdx.y * BN;
    if (lower && blockIdx.x < blockIdx.y) return;
    const int kbeg = blockIdx.z * kchunk;
    const int kend = min(K, kbeg + kchunk);
    dfc acc[T][T];
#pragma unroll
    for (int i = 0; i < T; ++i)
#pragma unroll
        for (int j = 0; j < T; ++j) acc[i][j] = dfc{0.f, 0.f, 0.f, 0.f};
    const z64 zero = mkc(0.0, 0.0);
    for (int k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
        for (int r = 0; r < (BK * BM) / TH; ++r) {
            const int e = tid + r * TH;
            int i, kk;
            if (!CA) { i = e % BM; kk = e / BM; } else { kk = e % BK; i = e / BK; }
            const int gi = i0 + i, gk = k0 + kk;
            z64 v = zero;
            if (gi < m && gk < kend) v = CA ? A[(size_t)gi * lda + gk] : A[(size_t)gk * lda + gi];
            As[kk][i] = to_dfc(v, CA);
        }
#pragma unroll
        for (int r = 0; r < (BK * BN) / TH; ++r) {
            const int e = tid + r * TH;
            int j, kk;
            if (!CB) { kk = e % BK; j = e / BK; } else { j = e % BN; kk = e / BN; }
            const int gj = j0 + j, gk = k0 + kk;
            z64 v = zero;
            if (gj < n && gk < kend) v = CB ? B[(size_t)gk * ldb + gj] : B[(size_t)gj * ldb + gk];
            Bs[kk][j] = to_dfc(v, CB);
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < BK; ++kk) {
            dfc a[T], b[T];
#pragma unroll
            for (int i = 0; i < T; ++i) a[i] = As[kk][tx + 16 * i];
#pragma unroll
            for (int j = 0; j < T; ++j) b[j] = Bs[kk][ty + 16 * j];
#pragma unroll
            for (int i = 0; i < T; ++i)
#pragma unroll
                for (int j = 0; j < T; ++j) {
                    dfc &c = acc[i][j];
                    df_mac(c.rh, c.rl, a[i].rh, a[i].rl, b[j].rh, b[j].rl);
                    df_mac(c.rh, c.rl, -a[i].ih, -a[i].il, b[j].ih, b[j].il);
                    df_mac(c.ih, c.il, a[i].rh, a[i].rl, b[j].ih, b[j].il);
                    df_mac(c.ih, c.il, a[i].ih, a[i].il, b[j].rh, b[j].rl);
                }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < T; ++i)
#pragma unroll
            for (int j = 0; j < T; ++j) {
                df_norm(acc[i][j].rh, acc[i][j].rl);
                df_norm(acc[i][j].ih, acc[i][j].il);
            }
    }
#pragma unroll
    for (int j = 0; j < T; ++j) {
        const int gj = j0 + ty + 16 * j;
        if (gj >= n) continue;
#pragma unroll
        for (int i = 0; i < T; ++i) {
            const int gi = i0 + tx + 16 * i;
            if (gi >= m) continue;
            const dfc &c = acc[i][j];
            const z64 t = mkc((double)c.rh + (double)c.rl, (double)c.ih + (double)c.il);
            if (part) {
                part[((size_t)blockIdx.z * n + gj) * m + gi] = t;
            } else {
                z64 v = alpha * t;
                if (beta != 0.0) v = v + beta * C[(size_t)gj * ldc + gi];
                D[(size_t)gj * ldd + gi] = v;
            }
        }
    }
}

template <typename R>
__global__ void k_reduce_parts(int m, int n, int nsplit, R alpha, const z64 *__restrict__ part, R beta,
                               const cx<R> *C, int ldc, cx<R> *D, int ldd, int lower_tile) {
    const size_t tot = (size_t)m * n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        const int gi = (int)(e % m), gj = (int)(e / m);
        if (lower_tile && gi / lower_tile < gj / lower_tile) continue;  // tile not computed
        z64 s = part[e];
        for (int z = 1; z < nsplit; ++z) s = s + part[(size_t)z * tot + e];
        z64 v = (double)alpha * s;
        if (beta != (R)0) v = v + (double)beta * cvt<double, R>(C[(size_t)gj * ldc + gi]);
        D[(size_t)gj * ldd + gi] = cvt<R, double>(v);
    }
}

int num_sms() {
    static std::atomic<int> cached{0};
    int v = cached.load();
    if (!v) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 132;
        cached.store(v);
    }
    return v;
}

// Launch op(A) op(B) with an optional split of the reduction dimension.
// Small products use 32 x 32 tiles so that they still spread over the GPU.
template <typename R, bool CA, bool CB, int T, bool DF = false>
int launch_gemm_t(GemmWork *w, int m, int n, int K, R alpha, const cx<R> *A, int lda, const cx<R> *B, int ldb,
                  R beta, const cx<R> *C, int ldc, cx<R> *D, int ldd, cudaStream_t s, bool allow_split,
                  int min_chunk, bool lower) {
    constexpr int BM = 16 * T, BN = 16 * T;
    if (m <= 0 || n <= 0) return LOBPCG_OK;
    const int tm = (m + BM - 1) / BM, tn = (n + BN - 1) / BN;
    int tiles = tm * tn;
    if (lower) {  // tiles on or below the diagonal
        tiles = 0;
        for (int tj = 0; tj < tn; ++tj) tiles += std::max(0, tm - tj);
    }
    int nsplit = 1;
    if (allow_split && w && K > min_chunk) {
        const int want = (2 * num_sms() + tiles - 1) / tiles;
        const int maxs = (K + min_chunk - 1) / min_chunk;
        nsplit = std::max(1, std::min(want, maxs));
    }
    if (K <= 0) nsplit = 1;
    int kchunk = (K + nsplit - 1) / nsplit;
    kchunk = ((kchunk + BK - 1) / BK) * BK;
    if (kchunk <= 0) kchunk = BK;
    nsplit = K > 0 ? (K + kchunk - 1) / kchunk : 1;
    auto kern = [&](dim3 grid, z64 *part) {
        if constexpr (DF)
            k_gemm_df<CA, CB, T><<<grid, TH, 0, s>>>(m, n, K, kchunk, alpha, A, lda, B, ldb, beta, C, ldc, D, ldd,
                                                     part, lower ? 1 : 0);
        else
            k_gemm<R, CA, CB, T><<<grid, TH, 0, s>>>(m, n, K, kchunk, alpha, A, lda, B, ldb, beta, C, ldc, D, ldd,
                                                     part, lower ? 1 : 0);
    };
    if (nsplit == 1) {
        kern(dim3(tm, tn, 1), nullptr);
        return check_launch("gemm");
    }
    const size_t need = sizeof(z64) * (size_t)nsplit * m * n;
    LG_TRY(w->alloc->ensure(w->part, need));
    z64 *part = reinterpret_cast<z64 *>(w->part.p);
    kern(dim3(tm, tn, nsplit), part);
    LG_TRY(check_launch("gemm split"));
    const size_t tot = (size_t)m * n;
    const int blocks = (int)std::min<size_t>((tot + 255) / 256, 4096);
    k_reduce_parts<R><<<blocks, 256, 0, s>>>(m, n, nsplit, alpha, part, beta, C, ldc, D, ldd, lower ? BM : 0);
    return check_launch("gemm reduce");
}

template <typename R, bool CA, bool CB>
int launch_gemm(GemmWork *w, int m, int n, int K, R alpha, const cx<R> *A, int lda, const cx<R> *B, int ldb,
                R beta, const cx<R> *C, int ldc, cx<R> *D, int ldd, cudaStream_t s, bool allow_split,
                bool lower = false) {
    if constexpr (std::is_same<R, double>::value) {
        if (w && w->df) {  // double-FP32 arithmetic, same tiles and split
            if ((long long)m * n <= 512LL * 512LL && K <= 8192)
                return launch_gemm_t<R, CA, CB, 2, true>(w, m, n, K, alpha, A, lda, B, ldb, beta, C, ldc, D, ldd, s,
                                                         allow_split, 2 * BK, lower);
            return launch_gemm_t<R, CA, CB, 4, true>(w, m, n, K, alpha, A, lda, B, ldb, beta, C, ldc, D, ldd, s,
                                                     allow_split, 4 * BK, lower);
        }
    }
    // tall-skinny and large products: 64 x 64 tiles; small dense ones: 32 x 32 tiles + fine split
    if ((long long)m * n <= 512LL * 512LL && K <= 8192)
        return launch_gemm_t<R, CA, CB, 2>(w, m, n, K, alpha, A, lda, B, ldb, beta, C, ldc, D, ldd, s, allow_split,
                                           2 * BK, lower);
    return launch_gemm_t<R, CA, CB, 4>(w, m, n, K, alpha, A, lda, B, ldb, beta, C, ldc, D, ldd, s, allow_split,
                                       4 * BK, lower);
}

}  // namespace

namespace {
// per host thread: each handle call (and each k-point lane thread of a solve) sets it from its
// own options, so handles with different engines on different threads do not interfere
thread_local int g_gemm_mode = 0;
// tensor-core thresholds: a long reduction (A^H B) or a tall product (A B)
constexpr int kTcMinK = 1024, kTcMinM = 1024;
}  // namespace

void set_gemm_mode(int mode) { g_gemm_mode = mode; }
int gemm_mode() { return g_gemm_mode; }

template <typename R>
int gemm_cn(GemmWork &w, int m, int n, int K, R alpha, const cx<R> *A, int lda, const cx<R> *B, int ldb, R beta,
            cx<R> *C, int ldc, cudaStream_t s) {
    if constexpr (std::is_same<R, float>::value) {
        if (g_gemm_mode != 3 && K >= kTcMinK) return tc_gemm_cn(w, m, n, K, alpha, A, lda, B, ldb, beta, C, ldc, s);
    }
    return launch_gemm<R, true, false>(&w, m, n, K, alpha, A, lda, B, ldb, beta, C, ldc, C, ldc, s, true);
}

int zgemm_cn_lower(GemmWork &w, int n, int K, const z64 *A, int lda, const z64 *B, int ldb, z64 *C, int ldc,
                   cudaStream_t s, bool df) {
    if (df && w.oz) return oz_gemm_cn(w, n, n, K, 1.0, A, lda, B, ldb, 0.0, C, ldc, s, true);
    if (df)
        return launch_gemm_t<double, true, false, 4, true>(&w, n, n, K, 1.0, A, lda, B, ldb, 0.0, C, ldc, C, ldc, s,
                                                          true, 4 * BK, true);
    return launch_gemm<double, true, false>(&w, n, n, K, 1.0, A, lda, B, ldb, 0.0, C, ldc, C, ldc, s, true, true);
}

int zgemm_cn_df(GemmWork &w, int m, int n, int K, double alpha, const z64 *A, int lda, const z64 *B, int ldb,
                double beta, z64 *C, int ldc, cudaStream_t s) {
    if (m <= 0 || n <= 0) return LOBPCG_OK;
    if (w.oz) return oz_gemm_cn(w, m, n, K, alpha, A, lda, B, ldb, beta, C, ldc, s, false);
    return launch_gemm_t<double, true, false, 4, true>(&w, m, n, K, alpha, A, lda, B, ldb, beta, C, ldc, C, ldc, s,
                                                      true, 4 * BK, false);
}

int zgemm_nn_df(GemmWork *w, int M, int n, int k, double alpha, const z64 *A, int lda, const z64 *B, int ldb,
                double beta, const z64 *C, int ldc, z64 *D, int ldd, cudaStream_t s) {
    if (M <= 0 || n <= 0) return LOBPCG_OK;
    if (w && w->oz && k > 0) return oz_gemm_nn(*w, M, n, k, alpha, A, lda, B, ldb, beta, C, ldc, D, ldd, s);
    return launch_gemm_t<double, false, false, 4, true>(nullptr, M, n, k, alpha, A, lda, B, ldb, beta, C, ldc, D,
                                                       ldd, s, false, 4 * BK, false);
}

template <typename R>
int gemm_nn(int M, int n, int k, R alpha, const cx<R> *A, int lda, const cx<R> *B, int ldb, R beta,
            const cx<R> *C, int ldc, cx<R> *D, int ldd, cudaStream_t s) {
    if constexpr (std::is_same<R, float>::value) {
        if (g_gemm_mode != 3 && M >= kTcMinM && k > 0)
            return tc_gemm_nn(M, n, k, alpha, A, lda, B, ldb, beta, C, ldc, D, ldd, s);
    }
    return launch_gemm<R, false, false>(nullptr, M, n, k, alpha, A, lda, B, ldb, beta, C, ldc, D, ldd, s, false);
}

template <typename R>
int gemm_small(GemmWork *w, char opA, char opB, int m, int n, int k, double alpha, const cx<R> *A, int lda,
               const cx<R> *B, int ldb, double beta, cx<R> *C, int ldc, cudaStream_t s) {
    const bool ca = (opA == 'C'), cb = (opB == 'C');
    const bool sp = w != nullptr;
    const R al = (R)alpha, be = (R)beta;
    if (!ca && !cb) return launch_gemm<R, false, false>(w, m, n, k, al, A, lda, B, ldb, be, C, ldc, C, ldc, s, sp);
    if (ca && !cb) return launch_gemm<R, true, false>(w, m, n, k, al, A, lda, B, ldb, be, C, ldc, C, ldc, s, sp);
    if (!ca && cb) return launch_gemm<R, false, true>(w, m, n, k, al, A, lda, B, ldb, be, C, ldc, C, ldc, s, sp);
    return launch_gemm<R, true, true>(w, m, n, k, al, A, lda, B, ldb, be, C, ldc, C, ldc, s, sp);
}
template int gemm_small<double>(GemmWork *, char, char, int, int, int, double, const z64 *, int, const z64 *, int,
                                double, z64 *, int, cudaStream_t);
template int gemm_small<float>(GemmWork *, char, char, int, int, int, double, const c32 *, int, const c32 *, int,
                               double, c32 *, int, cudaStream_t);

int zgemm_small(GemmWork *w, char opA, char opB, int m, int n, int k, double alpha, const z64 *A, int lda,
                const z64 *B, int ldb, double beta, z64 *C, int ldc, cudaStream_t s) {
    return gemm_small<double>(w, opA, opB, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, s);
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
