// FP64 Rayleigh-Ritz for block LOBPCG (Algorithm 1, step 4 of Bottin et al.
// 2007: "apply the Rayleigh-Ritz method within the subspace spanned by the
// columns of Psi, W and P"; the paper calls LAPACK for it, Sec. 4.2) and the
// all-band subspace diagonalisation that closes each sweep (Sec. 3.2).
//
// Given the Gram matrix S = Z^H Z and A = Z^H H Z of a basis Z (n x n):
//   1. scale to unit diagonal, S' = D S D, A' = D A D, D = diag(S)^-1/2;
//   2. blocked Cholesky S' = L L^H; a column whose pivot^2 is below drop_tol
//      is dependent on the earlier ones and is removed (its L column becomes
//      e_j, its L row is cleared), which turns the problem into plain RR on
//      the remaining columns;
//   3. Ahat = L^-1 A' L^-H (explicit blocked triangular inverse);
//   4. lowest m eigenpairs of Ahat: complex Householder tridiagonalisation
//      (reflectors in the LAPACK larfg convention, real sub-diagonal),
//      eigenvalues by multisection on Sturm counts (a warp per eigenvalue),
//      eigenvectors by inverse iteration with partial-pivoting tridiagonal
//      LU and modified Gram-Schmidt inside clusters of close eigenvalues,
//      back-transformation by the reflectors in blocks of 32 (compact WY form);
//   5. C = D L^-H Q.
// Every step runs on the GPU in FP64; no host synchronisation.
#include "common.cuh"
#include "df64.cuh"

#include <cooperative_groups.h>

#include <algorithm>
#include <cfloat>
#include <climits>
#include <type_traits>

namespace lg {

namespace {

constexpr int NBK = 32;  // Cholesky / inverse block size

template <typename RT> struct Lim;
template <> struct Lim<double> {
    static __device__ __forceinline__ double eps() { return DBL_EPSILON; }
    static __device__ __forceinline__ double tiny() { return DBL_MIN; }
    static __device__ __forceinline__ double big() { return DBL_MAX; }
};
template <> struct Lim<float> {
    static __device__ __forceinline__ float eps() { return FLT_EPSILON; }
    static __device__ __forceinline__ float tiny() { return FLT_MIN; }
    static __device__ __forceinline__ float big() { return FLT_MAX; }
};
__device__ __forceinline__ z64 ldcg_cx(const z64 *p) {
    const double2 t = __ldcg(reinterpret_cast<const double2 *>(p));
    return mkc(t.x, t.y);
}
__device__ __forceinline__ c32 ldcg_cx(const c32 *p) {
    const float2 t = __ldcg(reinterpret_cast<const float2 *>(p));
    return mkc(t.x, t.y);
}
__device__ __forceinline__ cx<df64> ldcg_cx(const cx<df64> *p) {
    const float4 t = __ldcg(reinterpret_cast<const float4 *>(p));
    return mkc(df64(t.x, t.y), df64(t.z, t.w));
}
// Load a complex stored as cx<PT> into the compute type CT.
template <typename CT, typename PT>
__device__ __forceinline__ cx<CT> ld_as(const cx<PT> *p) {
    if constexpr (std::is_same<CT, PT>::value) return *p;
    else return mkc<CT>((CT)p->x, (CT)p->y);
}
template <typename CT, typename PT>
__device__ __forceinline__ cx<CT> ldcg_as(const cx<PT> *p) {
    const cx<PT> v = ldcg_cx(p);
    if constexpr (std::is_same<CT, PT>::value) return v;
    else return mkc<CT>((CT)v.x, (CT)v.y);
}
template <typename PT, typename CT>
__device__ __forceinline__ cx<PT> as_store(cx<CT> v) {
    if constexpr (std::is_same<CT, PT>::value) return v;
    else return mkc<PT>((PT)v.x, (PT)v.y);
}


template <typename RT>
__device__ __forceinline__ RT warp_sum(RT v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Deterministic block sum (blockDim.x multiple of 32, <= 1024). Result on all threads.
template <typename RT>
__device__ RT block_sum(RT v, RT *sh) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    RT t = 0.0;
    for (int i = 0; i < nw; ++i) t += sh[i];
    return t;
}

// ------------------------------------------------------------------ scaling
template <typename RT>
__global__ void k_scale_gram(int n, const cx<RT> *__restrict__ S, int lds, const cx<RT> *__restrict__ A, int lda,
                             cx<RT> *__restrict__ Ss, cx<RT> *__restrict__ As, RT *__restrict__ d) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= n) return;
    const RT si = S[(size_t)i * lds + i].x, sj = S[(size_t)j * lds + j].x;
    const RT di = si > 0.0 ? 1.0 / sqrt(si) : 0.0;
    const RT dj = sj > 0.0 ? 1.0 / sqrt(sj) : 0.0;
    if (j == 0) d[i] = di;
    cx<RT> s, a;
    if (i >= j) {
        s = S[(size_t)j * lds + i];
        a = A[(size_t)j * lda + i];
    } else {
        s = conjc(S[(size_t)i * lds + j]);
        a = conjc(A[(size_t)i * lda + j]);
    }
    if (i == j) { s.y = 0.0; a.y = 0.0; }
    Ss[(size_t)j * n + i] = (di * dj) * s;
    As[(size_t)j * n + i] = (di * dj) * a;
}

// ------------------------------------------------------------------ Cholesky with dropping
// Factor the kb x kb diagonal block at k0 (already updated by earlier panels),
// write L_kk over it and its inverse into Linv.
// CT: compute type (double-FP32 where one SM's FP64 units would be the limit).
template <typename RT, typename CT = RT>
__global__ void __launch_bounds__(256)
k_chol_diag(int n, int k0, int kb, cx<RT> *__restrict__ L, cx<RT> *__restrict__ Linv, RT drop_tol_in,
            int *__restrict__ dropped, int *__restrict__ ndrop) {
    __shared__ cx<CT> T[NBK][NBK + 1];
    __shared__ cx<CT> I[NBK][NBK + 1];
    __shared__ int dflag[NBK];
    const CT drop_tol = (CT)drop_tol_in;
    const int tid = threadIdx.x;
    for (int e = tid; e < NBK * NBK; e += blockDim.x) {
        const int r = e % NBK, c = e / NBK;
        cx<CT> v = mkc<CT>(0.0, 0.0);
        if (r < kb && c < kb && r >= c) v = ld_as<CT>(L + (size_t)(k0 + c) * n + k0 + r);
        T[r][c] = v;
        I[r][c] = mkc<CT>(0.0, 0.0);
    }
    __syncthreads();
    for (int j = 0; j < kb; ++j) {
        const CT p = T[j][j].x;
        const bool drop = !(p > drop_tol);
        __syncthreads();
        if (drop) {
            for (int r = j + 1 + tid; r < kb; r += blockDim.x) T[r][j] = mkc<CT>(0.0, 0.0);
            if (tid == 0) { T[j][j] = mkc<CT>(1.0, 0.0); dflag[j] = 1; }
        } else {
            const CT rt = sqrt(p), inv = (CT)1.0 / rt;
            for (int r = j + 1 + tid; r < kb; r += blockDim.x) T[r][j] = inv * T[r][j];
            if (tid == 0) { T[j][j] = mkc<CT>(rt, 0.0); dflag[j] = 0; }
        }
        __syncthreads();
        if (!drop) {
            const int rem = kb - j - 1;
            for (int e = tid; e < rem * rem; e += blockDim.x) {
                const int r = j + 1 + e % rem, c = j + 1 + e / rem;
                if (r >= c) T[r][c] = T[r][c] - mul_conj(T[r][j], T[c][j]);
            }
        }
        __syncthreads();
    }
    // clear the rows of dropped columns inside the block
    for (int e = tid; e < kb * kb; e += blockDim.x) {
        const int r = e % kb, c = e / kb;
        if (c < r && dflag[r]) T[r][c] = mkc<CT>(0.0, 0.0);
    }
    __syncthreads();
    // inverse of the lower-triangular block (real positive diagonal) by forward substitution,
    // column c on the 8 lanes of one warp segment: I[r][c] = -(1 / T[r][r]) sum_{l=c}^{r-1} T[r][l] I[l][c],
    // each lane taking every 8th l, the segment adding its partial sums by shuffles (fixed order)
    __shared__ CT rdiag[NBK];
    if (tid < kb) rdiag[tid] = (CT)1.0 / T[tid][tid].x;
    __syncthreads();
    {
        const int c = tid >> 3, sub = tid & 7;
        const bool on = c < kb;
        for (int r = 0; r < kb; ++r) {
            cx<CT> sacc = mkc<CT>(0.0, 0.0);
            if (on && c < r)
                for (int l = c + sub; l < r; l += 8) sacc = sacc + T[r][l] * I[l][c];
#pragma unroll
            for (int o = 1; o < 8; o <<= 1) {
                sacc.x += __shfl_xor_sync(0xffffffffu, sacc.x, o);
                sacc.y += __shfl_xor_sync(0xffffffffu, sacc.y, o);
            }
            if (on && sub == 0) {
                if (c < r) I[r][c] = (-rdiag[r]) * sacc;
                else if (c == r) I[r][r] = mkc<CT>(rdiag[r], 0.0);
            }
            __syncwarp();
        }
    }
    __syncthreads();
    for (int e = tid; e < kb * kb; e += blockDim.x) {
        const int r = e % kb, c = e / kb;
        L[(size_t)(k0 + c) * n + k0 + r] = (r >= c) ? as_store<RT>(T[r][c]) : mkc<RT>(0.0, 0.0);
        Linv[(size_t)(k0 + c) * n + k0 + r] = (r >= c) ? as_store<RT>(I[r][c]) : mkc<RT>(0.0, 0.0);
    }
    if (tid < kb) {
        dropped[k0 + tid] = dflag[tid];
        if (dflag[tid]) atomicAdd(ndrop, 1);
    }
}

// Panel: L21 = S21 Linv_kk^H for rows k0+kb..n-1 (8 rows per block, 32 columns).
template <typename RT>
__global__ void __launch_bounds__(256)
k_chol_panel(int n, int k0, int kb, cx<RT> *__restrict__ L, const cx<RT> *__restrict__ Linv,
             const int *__restrict__ dropped) {
    __shared__ cx<RT> Di[NBK][NBK + 1];
    __shared__ cx<RT> Srow[8][NBK + 1];
    const int tid = threadIdx.x;
    for (int e = tid; e < NBK * NBK; e += blockDim.x) {
        const int r = e % NBK, c = e / NBK;
        Di[r][c] = (r < kb && c < kb) ? Linv[(size_t)(k0 + c) * n + k0 + r] : mkc<RT>(0.0, 0.0);
    }
    const int rl = tid / NBK, c = tid % NBK;
    const int row = k0 + kb + blockIdx.x * 8 + rl;
    if (row < n && c < kb) Srow[rl][c] = L[(size_t)(k0 + c) * n + row];
    __syncthreads();
    if (row < n && c < kb) {
        cx<RT> s = mkc<RT>(0.0, 0.0);
        for (int l = 0; l <= c; ++l) s = s + mul_conj(Srow[rl][l], Di[c][l]);
        if (dropped[k0 + c]) s = mkc<RT>(0.0, 0.0);
        L[(size_t)(k0 + c) * n + row] = s;
    }
}

// Leading identity block (a basis whose first `lead` vectors are orthonormal and orthogonal to the
// rest, as [X W P] of a mixed block iteration): its Cholesky factor and inverse are the identity.
template <typename RT>
__global__ void k_lead_identity(int n, int lead, cx<RT> *__restrict__ L, cx<RT> *__restrict__ Linv,
                                int *__restrict__ dropped) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (i >= n) return;
    const cx<RT> v = mkc<RT>(i == j ? 1.0 : 0.0, 0.0);
    L[(size_t)j * n + i] = v;
    if (i < lead) Linv[(size_t)j * n + i] = v;
    if (i == 0) dropped[j] = 0;
}

template <typename RT>
__global__ void k_zero_dropped_rows(int n, cx<RT> *__restrict__ L, const int *__restrict__ dropped) {
    const int j = blockIdx.x;
    if (!dropped[j]) return;
    for (int c = threadIdx.x; c < j; c += blockDim.x) L[(size_t)c * n + j] = mkc<RT>(0.0, 0.0);
}

// ------------------------------------------------------------------ hermitize / dropped rows
template <typename RT>
__global__ void k_hermitize_rowsum(int n, cx<RT> *__restrict__ A, const int *__restrict__ dropped,
                                   RT *__restrict__ rowsum) {
    const int i = blockIdx.x;
    __shared__ RT sh[32];
    RT s = 0.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        cx<RT> v = (i >= j) ? A[(size_t)j * n + i] : conjc(A[(size_t)i * n + j]);
        if (i == j) v.y = 0.0;
        if (dropped && (dropped[i] || dropped[j])) v = mkc<RT>(0.0, 0.0);
        s += sqrt(abs2(v));
        if (i >= j) {
            A[(size_t)j * n + i] = v;
            A[(size_t)i * n + j] = conjc(v);
        }
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) rowsum[i] = s;
}

template <typename RT>
__global__ void k_set_dropped_diag(int n, cx<RT> *__restrict__ A, const int *__restrict__ dropped,
                                   const int *__restrict__ ndrop, const RT *__restrict__ rowsum) {
    if (*ndrop == 0) return;
    __shared__ RT sh[32];
    RT mx = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) mx = fmax(mx, rowsum[i]);
    // deterministic max via shuffles
#pragma unroll
    for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = mx;
    __syncthreads();
    RT m2 = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m2 = fmax(m2, sh[w]);
    const RT sigma = 2.0 * m2 + 1.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        if (dropped[i]) A[(size_t)i * n + i] = mkc<RT>(sigma, 0.0);
}

// ------------------------------------------------------------------ tridiagonalisation
// Reflector of x = A[i+1:n, i] in the LAPACK larfg convention:
//   H = I - tau v v^H, v[0] = 1, H^H x = beta e_1 with beta real.
template <typename RT>
struct Refl {
    cx<RT> tau;
    RT beta;
    cx<RT> scal;  // v[r] = x[r] * scal for r >= 1
};

// Reflector from alpha = x[0] and s = sum_{r>=1} |x[r]|^2 (LAPACK larfg convention).
template <typename RT>
__device__ __forceinline__ Refl<RT> reflector_from(cx<RT> alpha, RT s) {
    Refl<RT> R;
    if (s == 0.0 && alpha.y == 0.0) {
        R.tau = mkc<RT>(0.0, 0.0);
        R.beta = alpha.x;
        R.scal = mkc<RT>(0.0, 0.0);
        return R;
    }
    const RT beta = -copysign(sqrt(abs2(alpha) + s), alpha.x);
    R.beta = beta;
    R.tau = mkc<RT>((beta - alpha.x) / beta, -alpha.y / beta);
    const cx<RT> den = mkc<RT>(alpha.x - beta, alpha.y);
    const RT dd = abs2(den);
    R.scal = mkc<RT>(den.x / dd, -den.y / dd);
    return R;
}

template <typename RT, bool CG = false, typename PT = RT>
__device__ Refl<RT> make_reflector(const cx<PT> *__restrict__ col, int L, RT *sh) {
    RT s = 0.0;
    for (int r = 1 + threadIdx.x; r < L; r += blockDim.x) s += abs2(CG ? ldcg_as<RT>(col + r) : ld_as<RT>(col + r));
    s = block_sum(s, sh);
    return reflector_from<RT>(CG ? ldcg_as<RT>(col) : ld_as<RT>(col), s);
}

// Block sum whose cross-warp step is one warp's shuffle tree (a fixed order): for large
// blocks, where every thread summing all warp partials would cost more issue slots than
// the rest of the step.  sh holds 33 entries; every thread gets the result.
template <typename RT>
__device__ RT block_sum_tree(RT v, RT *sh) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    if (wid == 0) {
        RT t = lane < nw ? sh[lane] : RT(0.0);
        t = warp_sum(t);
        if (lane == 0) sh[32] = t;
    }
    __syncthreads();
    return sh[32];
}

// make_reflector with the tree sum and the scalar arithmetic in one thread, broadcast
// through shared memory (*rb).
template <typename RT, typename PT = RT>
__device__ Refl<RT> make_reflector_bc(const cx<PT> *__restrict__ col, int L, RT *sh, Refl<RT> *rb) {
    RT s = 0.0;
    for (int r = 1 + threadIdx.x; r < L; r += blockDim.x) s += abs2(ld_as<RT>(col + r));
    s = block_sum_tree(s, sh);
    if (threadIdx.x == 0) *rb = reflector_from<RT>(ld_as<RT>(col), s);
    __syncthreads();
    return *rb;
}

// Step i, part 1: reflector (every block, redundantly) and y = A22 v by 32x32 tiles;
// the last block to finish forms w = tau y - |tau|^2/2 (v^H y) v.
template <typename RT>
__global__ void __launch_bounds__(256)
k_tri_step1(int n, int i, cx<RT> *__restrict__ A, int lda, cx<RT> *__restrict__ Hv, cx<RT> *__restrict__ taus,
            RT *__restrict__ dg, RT *__restrict__ eg, cx<RT> *__restrict__ ypart, cx<RT> *__restrict__ wv,
            unsigned int *__restrict__ counter) {
    __shared__ RT sh[32];
    __shared__ cx<RT> vs[32];
    __shared__ cx<RT> acc[8][33];
    __shared__ bool last;
    const int L = n - i - 1;
    const cx<RT> *col = A + (size_t)i * lda + i + 1;
    const Refl<RT> R = make_reflector<RT>(col, L, sh);
    const int tr = blockIdx.x, tc = blockIdx.y;
    const int tid = threadIdx.x;
    if (tr == 0 && tc == 0) {
        for (int r = tid; r < L; r += blockDim.x) Hv[(size_t)i * n + i + 1 + r] = (r == 0) ? mkc<RT>(1.0, 0.0) : col[r] * R.scal;
        if (tid == 0) {
            taus[i] = R.tau;
            dg[i] = A[(size_t)i * lda + i].x;
            eg[i] = R.beta;
        }
    }
    // v entries of this column tile
    if (tid < 32) {
        const int c = tc * 32 + tid;
        vs[tid] = (c < L) ? ((c == 0) ? mkc<RT>(1.0, 0.0) : col[c] * R.scal) : mkc<RT>(0.0, 0.0);
    }
    __syncthreads();
    const int rl = tid & 31, cg = tid >> 5;  // 32 rows x 8 column groups of 4
    const int r = tr * 32 + rl;
    cx<RT> s = mkc<RT>(0.0, 0.0);
    if (r < L) {
        const cx<RT> *A22 = A + (size_t)(i + 1) * lda + i + 1;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int cl = cg * 4 + q, c = tc * 32 + cl;
            if (c < L) s = s + A22[(size_t)c * lda + r] * vs[cl];
        }
    }
    acc[cg][rl] = s;
    __syncthreads();
    if (tid < 32) {
        cx<RT> t = acc[0][tid];
        for (int g = 1; g < 8; ++g) t = t + acc[g][tid];
        const int rr = tr * 32 + tid;
        if (rr < L) ypart[(size_t)tc * n + rr] = t;
    }
    // last-block reduction (no waiting: only the block that arrives last continues)
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        const unsigned int total = gridDim.x * gridDim.y;
        const unsigned int prev = atomicAdd(counter + i, 1u);
        last = (prev == total - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    const int ncb = gridDim.y;
    // y = sum of partials (fixed order), dot = v^H y
    RT dre = 0.0, dim = 0.0;
    for (int rr = tid; rr < L; rr += blockDim.x) {
        cx<RT> y = mkc<RT>(0.0, 0.0);
        for (int c = 0; c < ncb; ++c) {
            y = y + ldcg_cx(ypart + (size_t)c * n + rr);
        }
        const cx<RT> v = (rr == 0) ? mkc<RT>(1.0, 0.0) : col[rr] * R.scal;
        // conj(v) * y
        dre += v.x * y.x + v.y * y.y;
        dim += v.x * y.y - v.y * y.x;
        wv[rr] = y;  // stash y, scaled below
    }
    dre = block_sum(dre, sh);
    (void)dim;  // v^H A v is real for Hermitian A
    const RT t2 = 0.5 * abs2(R.tau) * dre;
    __syncthreads();
    for (int rr = tid; rr < L; rr += blockDim.x) {
        const cx<RT> v = (rr == 0) ? mkc<RT>(1.0, 0.0) : col[rr] * R.scal;
        const cx<RT> y = wv[rr];
        wv[rr] = R.tau * y - t2 * v;
    }
}

// Step i, part 2: A22 -= w v^H + v w^H on 32x32 tiles.
template <typename RT>
__global__ void __launch_bounds__(256)
k_tri_step2(int n, int i, cx<RT> *__restrict__ A, int lda, const cx<RT> *__restrict__ Hv, const cx<RT> *__restrict__ wv) {
    __shared__ cx<RT> vr[32], wr[32], vc[32], wc[32];
    const int L = n - i - 1;
    const int tr = blockIdx.x, tc = blockIdx.y, tid = threadIdx.x;
    const cx<RT> *v = Hv + (size_t)i * n + i + 1;
    if (tid < 32) {
        const int r = tr * 32 + tid, c = tc * 32 + tid;
        vr[tid] = r < L ? v[r] : mkc<RT>(0.0, 0.0);
        wr[tid] = r < L ? wv[r] : mkc<RT>(0.0, 0.0);
        vc[tid] = c < L ? v[c] : mkc<RT>(0.0, 0.0);
        wc[tid] = c < L ? wv[c] : mkc<RT>(0.0, 0.0);
    }
    __syncthreads();
    cx<RT> *A22 = A + (size_t)(i + 1) * lda + i + 1;
    for (int e = tid; e < 32 * 32; e += blockDim.x) {
        const int rl = e & 31, cl = e >> 5;
        const int r = tr * 32 + rl, c = tc * 32 + cl;
        if (r < L && c < L) {
            cx<RT> a = A22[(size_t)c * lda + r];
            a = a - mul_conj(wr[rl], vc[cl]) - mul_conj(vr[rl], wc[cl]);
            A22[(size_t)c * lda + r] = a;
        }
    }
}

// Grid-wide barrier for co-resident blocks (cooperative launch): a monotone arrival
// counter; block 0 thread 0 of every block waits for `target` arrivals.  Bounded: a
// wait that runs out (or sees another block's failure) sets *err and the blocks leave.
__device__ __forceinline__ bool grid_barrier(unsigned int *count, unsigned int target, int *err) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(count, 1u);
        int ok = 0;
        for (long long it = 0; it < (1LL << 22); ++it) {
            if (*reinterpret_cast<volatile unsigned int *>(count) >= target) { ok = 1; break; }
            if (*reinterpret_cast<volatile int *>(err)) break;
        }
        if (!ok) atomicExch(err, 1);
        __threadfence();
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

// Whole Householder tridiagonalisation in one cooperative launch (same arithmetic as
// k_tri_step1 / k_tri_step2, same fixed summation order): per column, every block
// forms the reflector, multiplies its 32 x 32 tiles of A22 by v, [barrier], sums the
// partial products for all rows and forms w, updates its tiles, [barrier].  Data
// written by other blocks is read through L2 (__ldcg).  Dynamic shared memory: v and w
// (2 n complex).
template <typename RT>
__global__ void __launch_bounds__(256)
k_tri_coop(int n, cx<RT> *__restrict__ A, int lda, cx<RT> *__restrict__ Hv, cx<RT> *__restrict__ taus,
           RT *__restrict__ dg, RT *__restrict__ eg, cx<RT> *__restrict__ ypart, unsigned int *bar, int *err) {
    extern __shared__ __align__(16) unsigned char dsm[];
    cx<RT> *vsh = reinterpret_cast<cx<RT> *>(dsm);
    cx<RT> *wsh = vsh + n;
    __shared__ RT sh[32];
    __shared__ cx<RT> acc[8][33];
    const int tid = threadIdx.x, G = gridDim.x;
    unsigned int arrivals = 0;
    for (int i = 0; i + 1 < n; ++i) {
        const int L = n - i - 1;
        const int tl = (L + 31) / 32, ntiles = tl * tl;
        const cx<RT> *col = A + (size_t)i * lda + i + 1;
        const Refl<RT> R = make_reflector<RT, true>(col, L, sh);
        for (int r = tid; r < L; r += blockDim.x) vsh[r] = (r == 0) ? mkc<RT>(1.0, 0.0) : ldcg_cx(col + r) * R.scal;
        if (blockIdx.x == 0) {
            for (int r = tid; r < L; r += blockDim.x) Hv[(size_t)i * n + i + 1 + r] = vsh[r];
            if (tid == 0) {
                taus[i] = R.tau;
                dg[i] = ldcg_cx(A + (size_t)i * lda + i).x;
                eg[i] = R.beta;
            }
        }
        __syncthreads();
        const cx<RT> *A22 = A + (size_t)(i + 1) * lda + i + 1;
        const int rl = tid & 31, cg = tid >> 5;
        for (int t = blockIdx.x; t < ntiles; t += G) {
            const int tr = t % tl, tc = t / tl;
            const int r = tr * 32 + rl;
            cx<RT> sacc = mkc<RT>(0.0, 0.0);
            if (r < L) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int c = tc * 32 + cg * 4 + q;
                    if (c < L) sacc = sacc + ldcg_cx(A22 + (size_t)c * lda + r) * vsh[c];
                }
            }
            acc[cg][rl] = sacc;
            __syncthreads();
            if (tid < 32) {
                cx<RT> u = acc[0][tid];
                for (int g = 1; g < 8; ++g) u = u + acc[g][tid];
                const int rr = tr * 32 + tid;
                if (rr < L) ypart[(size_t)tc * n + rr] = u;
            }
            __syncthreads();
        }
        arrivals += G;
        if (!grid_barrier(bar, arrivals, err)) return;
        // y = sum of the tile-column partials (fixed order), dot = v^H y, w = tau y - |tau|^2/2 (v^H y) v
        RT dre = 0.0;
        for (int rr = tid; rr < L; rr += blockDim.x) {
            cx<RT> y = mkc<RT>(0.0, 0.0);
            for (int c = 0; c < tl; ++c) y = y + ldcg_cx(ypart + (size_t)c * n + rr);
            const cx<RT> v = vsh[rr];
            dre += v.x * y.x + v.y * y.y;
            wsh[rr] = y;
        }
        dre = block_sum(dre, sh);
        const RT t2 = 0.5 * abs2(R.tau) * dre;
        for (int rr = tid; rr < L; rr += blockDim.x) wsh[rr] = R.tau * wsh[rr] - t2 * vsh[rr];
        __syncthreads();
        // A22 -= w v^H + v w^H on this block's tiles
        cx<RT> *A22w = A + (size_t)(i + 1) * lda + i + 1;
        for (int t = blockIdx.x; t < ntiles; t += G) {
            const int tr = t % tl, tc = t / tl;
            for (int e = tid; e < 32 * 32; e += blockDim.x) {
                const int r = tr * 32 + (e & 31), c = tc * 32 + (e >> 5);
                if (r < L && c < L) {
                    cx<RT> a = ldcg_cx(A22w + (size_t)c * lda + r);
                    a = a - mul_conj(wsh[r], vsh[c]) - mul_conj(vsh[r], wsh[c]);
                    A22w[(size_t)c * lda + r] = a;
                }
            }
        }
        arrivals += G;
        if (!grid_barrier(bar, arrivals, err)) return;
    }
    if (blockIdx.x == 0 && tid == 0) dg[n - 1] = ldcg_cx(A + (size_t)(n - 1) * lda + n - 1).x;
}

// Fused single-launch tridiagonalisation: one grid barrier per column.
// Block g owns the TS x TS tiles t = g, g + G, ... of the matrix (row-major tile index) and keeps
// them in shared memory for the whole factorisation.  Invariant at the top of column i (after a
// barrier): ypart[i & 1] holds, per tile column, the partial products A^(i)[J,J] v_i
// (J = i+1..n-1, A^(i) = the matrix after reflectors 0..i-1), and colbuf[i & 1] holds column
// i+1 of A^(i) from row i+1 down.  Column i then runs:
//   (a) y_i = sum of the partials (fixed order), w_i = tau y_i - |tau|^2/2 (v_i^H y_i) v_i;
//   (b) column i+1 of A^(i+1) = colbuf - w_i v_i^H - v_i w_i^H restricted to it, its diagonal
//       (-> d[i+1]) and reflector i+1 (every block, redundantly, same arithmetic);
//   (c) each owned tile: A -= w_i v_i^H + v_i w_i^H on J x J and, in the same pass, the partial
//       product with v_{i+1} on J' x J' (J' = i+2..n-1) -> ypart[(i+1) & 1];
//   (d) owners of column i+2 publish it (rows i+2..) -> colbuf[(i+1) & 1];  barrier.
// Same formulas as k_tri_step1 / k_tri_step2.  Small tiles spread the FP64 work of a column
// over more SMs (this GPU has few FP64 units per SM).  256 threads: TS rows x (256 / TS)
// column groups of CPT = TS*TS/256 columns.  Dynamic shared memory: the owned tiles, then
// v_i, w_i, v_{i+1} and the working column (n complex each).
template <typename RT, int TS, typename CT = RT>
__global__ void __launch_bounds__(256)
k_tri_fused(int n, const cx<RT> *__restrict__ A, int lda, cx<RT> *__restrict__ Hv, cx<RT> *__restrict__ taus,
            RT *__restrict__ dg, RT *__restrict__ eg, cx<RT> *__restrict__ ypart_st, cx<RT> *__restrict__ colbuf_st,
            unsigned int *bar, int *err) {
    static_assert(sizeof(cx<CT>) == sizeof(cx<RT>), "the compute type keeps the storage size");
    cx<CT> *ypart = reinterpret_cast<cx<CT> *>(ypart_st);   // scratch kept in the compute type
    cx<CT> *colbuf = reinterpret_cast<cx<CT> *>(colbuf_st);
    constexpr int TT = TS * TS, NG = 256 / TS, CPT = TT / 256;
    extern __shared__ __align__(16) unsigned char dsm[];
    const int T = (n + TS - 1) / TS, G = gridDim.x, g = blockIdx.x, tid = threadIdx.x;
    const int nown = (T * T - g + G - 1) / G;  // tiles g, g+G, ... below T*T
    cx<CT> *tiles = reinterpret_cast<cx<CT> *>(dsm);  // nown x [TS cols][TS rows]
    cx<CT> *v = tiles + (size_t)nown * TT;             // v_i on [0, n)
    cx<CT> *w = v + n;                                  // w_i
    cx<CT> *vn = w + n;                                 // v_{i+1}
    cx<CT> *x = vn + n;                                 // working column
    __shared__ CT sh[32];
    __shared__ cx<CT> acc[NG][TS + 1];
    const int rl = tid % TS, cg = tid / TS;
    const cx<CT> zero = mkc<CT>(0.0, 0.0);
    unsigned int arrivals = 0;
    // load the owned tiles (entries outside the matrix are zero)
    for (int q = 0; q < nown; ++q) {
        const int t = g + q * G, TR = t / T, TC = t % T;
        for (int e = tid; e < TT; e += blockDim.x) {
            const int r = TR * TS + (e % TS), c = TC * TS + (e / TS);
            tiles[(size_t)q * TT + e] = (r < n && c < n) ? ld_as<CT>(A + (size_t)c * lda + r) : zero;
        }
    }
    // reflector 0 from column 0 (read from A, unmodified), d[0]
    Refl<CT> R = make_reflector<CT, false, RT>(A + 1, n - 1, sh);
    for (int r = tid; r < n; r += blockDim.x)
        v[r] = (r < 1) ? zero : (r == 1 ? mkc<CT>(1.0, 0.0) : ld_as<CT>(A + r) * R.scal);
    if (g == 0 && tid == 0) dg[0] = A[0].x;
    __syncthreads();
    // partial products A^(0)[J,J] v_0 and column 1 of A^(0)
    for (int q = 0; q < nown; ++q) {
        const int t = g + q * G, TR = t / T, TC = t % T;
        const cx<CT> *tl = tiles + (size_t)q * TT;
        const int r = TR * TS + rl;
        cx<CT> sacc = zero;
#pragma unroll
        for (int k = 0; k < CPT; ++k) {
            const int cl = cg * CPT + k, c = TC * TS + cl;
            if (r >= 1 && r < n && c >= 1 && c < n) sacc = sacc + tl[cl * TS + rl] * v[c];
        }
        acc[cg][rl] = sacc;
        __syncthreads();
        if (tid < TS) {
            cx<CT> u = acc[0][tid];
            for (int k = 1; k < NG; ++k) u = u + acc[k][tid];
            const int rr = TR * TS + tid;
            if (rr < n) ypart[(size_t)TC * n + rr] = u;
            if (n > 1 && TC == 1 / TS && rr >= 1 && rr < n) colbuf[rr] = tl[(1 % TS) * TS + tid];
        }
        __syncthreads();
    }
    arrivals += G;
    if (!grid_barrier(bar, arrivals, err)) return;

    for (int i = 0; i + 1 < n; ++i) {
        const int par = i & 1;
        const cx<CT> *yp = ypart + (size_t)par * T * n;
        const cx<CT> *cb = colbuf + (size_t)par * n;
        // (a) y_i and w_i on J = [i+1, n); loads issued in groups of 8 before they are summed
        CT dre = 0.0;
        for (int r = i + 1 + tid; r < n; r += blockDim.x) {
            cx<CT> y = zero;
            for (int c = 0; c < T; c += 8) {
                cx<CT> t8[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) t8[k] = (c + k < T) ? ldcg_cx(yp + (size_t)(c + k) * n + r) : zero;
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    if (c + k < T) y = y + t8[k];
            }
            dre += v[r].x * y.x + v[r].y * y.y;
            w[r] = y;
        }
        dre = block_sum(dre, sh);
        const CT t2 = (CT)0.5 * abs2(R.tau) * dre;
        for (int r = i + 1 + tid; r < n; r += blockDim.x) w[r] = R.tau * w[r] - t2 * v[r];
        __syncthreads();
        // (b) column i+1 of A^(i+1) from row i+1; d[i+1]; reflector i+1
        const cx<CT> vi1 = v[i + 1], wi1 = w[i + 1];
        for (int r = i + 1 + tid; r < n; r += blockDim.x)
            x[r] = ldcg_cx(cb + r) - mul_conj(w[r], vi1) - mul_conj(v[r], wi1);
        __syncthreads();
        if (g == 0) {  // reflectors kept in the compute type (read by the back-transformation)
            cx<CT> *HvC = reinterpret_cast<cx<CT> *>(Hv);
            for (int r = i + 1 + tid; r < n; r += blockDim.x) HvC[(size_t)i * n + r] = v[r];
            if (tid == 0) {
                reinterpret_cast<cx<CT> *>(taus)[i] = R.tau;
                eg[i] = (RT)R.beta;
                dg[i + 1] = (RT)x[i + 1].x;
            }
        }
        if (i + 2 >= n) break;  // last column: nothing left to transform
        const Refl<CT> Rn = make_reflector<CT>(x + i + 2, n - i - 2, sh);
        for (int r = tid; r < n; r += blockDim.x)
            vn[r] = (r < i + 2) ? zero : (r == i + 2 ? mkc<CT>(1.0, 0.0) : x[r] * Rn.scal);
        __syncthreads();
        // (c) update the owned tiles with (w_i, v_i) and multiply by v_{i+1}; (d) publish column i+2
        cx<CT> *ypn = ypart + (size_t)(1 - par) * T * n;
        cx<CT> *cbn = colbuf + (size_t)(1 - par) * n;
        const int c2 = i + 2;
        for (int q = 0; q < nown; ++q) {
            const int t = g + q * G, TR = t / T, TC = t % T;
            cx<CT> *tl = tiles + (size_t)q * TT;
            if (TR * TS + TS - 1 < i + 1 || TC * TS + TS - 1 < i + 1) {
                // tile outside J x J: its share of y_{i+1} is zero (uniform branch)
                if (tid < TS) {
                    const int rr = TR * TS + tid;
                    if (rr < n) ypn[(size_t)TC * n + rr] = zero;
                }
                continue;
            }
            const int r = TR * TS + rl;
            const bool rin = r >= i + 1 && r < n;
            const cx<CT> wr = rin ? w[r] : zero, vr = rin ? v[r] : zero;
            cx<CT> sacc = zero;
#pragma unroll
            for (int k = 0; k < CPT; ++k) {
                const int cl = cg * CPT + k, c = TC * TS + cl;
                if (rin && c >= i + 1 && c < n) {
                    cx<CT> a = tl[cl * TS + rl];
                    a = a - mul_conj(wr, v[c]) - mul_conj(vr, w[c]);
                    tl[cl * TS + rl] = a;
                    if (r >= c2 && c >= c2) sacc = sacc + a * vn[c];
                }
            }
            acc[cg][rl] = sacc;
            __syncthreads();
            if (tid < TS) {
                cx<CT> u = acc[0][tid];
                for (int k = 1; k < NG; ++k) u = u + acc[k][tid];
                const int rr = TR * TS + tid;
                if (rr < n) ypn[(size_t)TC * n + rr] = u;
                if (TC == c2 / TS && rr >= c2 && rr < n) cbn[rr] = tl[(c2 % TS) * TS + tid];
            }
            __syncthreads();
        }
        R = Rn;
        for (int r = tid; r < n; r += blockDim.x) v[r] = vn[r];
        arrivals += G;
        if (!grid_barrier(bar, arrivals, err)) return;
    }
}

// a - w_r conj(v_c) - v_r conj(w_c), each real part through fused multiply-adds
template <typename CT>
__device__ __forceinline__ cx<CT> rank2_entry(cx<CT> a, cx<CT> wr, cx<CT> vr, cx<CT> vc, cx<CT> wc) {
    CT re = fma(-wr.x, vc.x, a.x);
    re = fma(-wr.y, vc.y, re);
    re = fma(-vr.x, wc.x, re);
    re = fma(-vr.y, wc.y, re);
    CT im = fma(-wr.y, vc.x, a.y);
    im = fma(wr.x, vc.y, im);
    im = fma(-vr.y, wc.x, im);
    im = fma(vr.x, wc.y, im);
    return mkc<CT>(re, im);
}
// acc + a b
template <typename CT>
__device__ __forceinline__ cx<CT> cmac(cx<CT> acc, cx<CT> a, cx<CT> b) {
    CT re = fma(a.x, b.x, acc.x);
    re = fma(-a.y, b.y, re);
    CT im = fma(a.x, b.y, acc.y);
    im = fma(a.y, b.x, im);
    return mkc<CT>(re, im);
}

// The same reduction held in the shared memory of one thread-block cluster of CS CTAs, for
// matrices small enough to fit there (n up to about 416 with 16 CTAs).  CTA q keeps the rows
// r = q + CS j of the full Hermitian matrix, row-major, so that y = A v needs no reduction
// across CTAs.  Per column i, after one cluster barrier every CTA holds y_i = A^(i) v_i and
// column i+1 of A^(i), both gathered through distributed shared memory, and forms w_i, the
// next column, d, e and reflector i+1 on its own: the same operations on the same values in
// the same order, so the same bits in every CTA.  Then each CTA applies the rank-2 update to
// its rows of the trailing block and, in the same pass, multiplies them by v_{i+1} (one warp
// per row), and sends its entries of y_{i+1} and of column i+2 to every CTA.  The gathered
// vectors alternate between two buffers, so that one barrier per column orders every write
// after the reads of the buffer it overwrites.  Outputs as k_tri_fused (Hv, taus in the
// compute type; d, e).  Dynamic shared memory: nr x n matrix entries (nr = ceil(n / CS)) and
// 7 n vector entries.
template <typename RT, typename CT>
__global__ void __launch_bounds__(1024, 1)
k_tri_cluster(int n, const cx<RT> *__restrict__ A, int lda, cx<RT> *__restrict__ Hv, cx<RT> *__restrict__ taus,
              RT *__restrict__ dg, RT *__restrict__ eg) {
    static_assert(sizeof(cx<CT>) == sizeof(cx<RT>), "the compute type keeps the storage size");
    namespace cgn = cooperative_groups;
    cgn::cluster_group cl = cgn::this_cluster();
    const int CS = (int)cl.num_blocks(), q = (int)cl.block_rank();
    const int nr = (n + CS - 1) / CS;
    extern __shared__ __align__(16) unsigned char dsm[];
    cx<CT> *M = reinterpret_cast<cx<CT> *>(dsm);       // local row j = global row q + CS j
    cx<CT> *vb = M + (size_t)nr * n;                    // v_i and v_{i+1}, by parity of i
    cx<CT> *w = vb + 2 * n;                             // w_i
    cx<CT> *yg = w + n;                                 // gathered y, two parities
    cx<CT> *cg = yg + 2 * n;                            // gathered next column, two parities
    __shared__ CT sh[33];
    __shared__ Refl<CT> rb;
    const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5, nw = blockDim.x >> 5;
    const cx<CT> zero = mkc<CT>(0.0, 0.0);
    // every CTA of the cluster running before any of them writes another's shared memory
    cl.sync();
    for (size_t e = tid; e < (size_t)nr * n; e += blockDim.x) {
        const int j = (int)(e / n), c = (int)(e % n), r = q + CS * j;
        M[e] = r < n ? ld_as<CT>(A + (size_t)c * lda + r) : zero;
    }
    // reflector 0 from column 0 of A, d[0]
    Refl<CT> R = make_reflector_bc<CT, RT>(A + 1, n - 1, sh, &rb);
    for (int r = tid; r < n; r += blockDim.x)
        vb[r] = (r < 1) ? zero : (r == 1 ? mkc<CT>(1.0, 0.0) : ld_as<CT>(A + r) * R.scal);
    if (q == 0 && tid == 0) dg[0] = A[0].x;
    __syncthreads();
    // y_0 = A[J,J] v_0 and column 1 on the owned rows of J = [1, n), sent to every CTA
    for (int j = wp; j < nr; j += nw) {
        const int r = q + CS * j;
        if (r < 1 || r >= n) continue;
        const cx<CT> *Mr = M + (size_t)j * n;
        cx<CT> acc = zero;
        for (int c = 1 + lane; c < n; c += 32) acc = cmac(acc, Mr[c], vb[c]);
        acc.x = warp_sum(acc.x);
        acc.y = warp_sum(acc.y);
        if (lane < CS) {
            cl.map_shared_rank(yg, lane)[r] = acc;
            cl.map_shared_rank(cg, lane)[r] = Mr[1];
        }
    }
    cl.sync();
    for (int i = 0; i + 1 < n; ++i) {
        const int par = i & 1;
        cx<CT> *v = vb + (size_t)par * n, *vn = vb + (size_t)(1 - par) * n;
        const cx<CT> *yv = yg + (size_t)par * n;
        cx<CT> *x = cg + (size_t)par * n;
        // w_i = tau y - |tau|^2 / 2 (v^H y) v on J = [i+1, n)
        CT dre = 0.0;
        for (int r = i + 1 + tid; r < n; r += blockDim.x) dre += v[r].x * yv[r].x + v[r].y * yv[r].y;
        dre = block_sum_tree(dre, sh);
        const CT t2 = (CT)0.5 * abs2(R.tau) * dre;
        for (int r = i + 1 + tid; r < n; r += blockDim.x) w[r] = R.tau * yv[r] - t2 * v[r];
        __syncthreads();
        // column i+1 of A^(i+1) (in place of the gathered column of A^(i)), d[i+1]
        const cx<CT> vi1 = v[i + 1], wi1 = w[i + 1];
        for (int r = i + 1 + tid; r < n; r += blockDim.x) x[r] = x[r] - mul_conj(w[r], vi1) - mul_conj(v[r], wi1);
        __syncthreads();
        if (q == 0) {
            cx<CT> *HvC = reinterpret_cast<cx<CT> *>(Hv);
            for (int r = i + 1 + tid; r < n; r += blockDim.x) HvC[(size_t)i * n + r] = v[r];
            if (tid == 0) {
                reinterpret_cast<cx<CT> *>(taus)[i] = R.tau;
                eg[i] = (RT)R.beta;
                dg[i + 1] = (RT)x[i + 1].x;
            }
        }
        if (i + 2 >= n) break;  // last column: nothing left to transform
        const Refl<CT> Rn = make_reflector_bc<CT>(x + i + 2, n - i - 2, sh, &rb);
        for (int r = tid; r < n; r += blockDim.x)
            vn[r] = (r < i + 2) ? zero : (r == i + 2 ? mkc<CT>(1.0, 0.0) : x[r] * Rn.scal);
        __syncthreads();
        // rank-2 update of the owned rows of the trailing block [i+2, n)^2, times v_{i+1}
        const int c2 = i + 2, nxt = 1 - par;
        for (int j = wp; j < nr; j += nw) {
            const int r = q + CS * j;
            if (r < c2 || r >= n) continue;
            cx<CT> *Mr = M + (size_t)j * n;
            const cx<CT> wr = w[r], vr = v[r];
            cx<CT> acc = zero;
            for (int c = c2 + lane; c < n; c += 32) {
                const cx<CT> a = rank2_entry(Mr[c], wr, vr, v[c], w[c]);
                Mr[c] = a;
                acc = cmac(acc, a, vn[c]);
            }
            acc.x = warp_sum(acc.x);
            acc.y = warp_sum(acc.y);
            __syncwarp();
            if (lane < CS) {
                cl.map_shared_rank(yg, lane)[(size_t)nxt * n + r] = acc;
                cl.map_shared_rank(cg, lane)[(size_t)nxt * n + r] = Mr[c2];
            }
        }
        R = Rn;
        cl.sync();
    }
}

template <typename RT>
__global__ void k_tri_last(int n, const cx<RT> *__restrict__ A, int lda, RT *__restrict__ dg) {
    if (threadIdx.x == 0) dg[n - 1] = A[(size_t)(n - 1) * lda + n - 1].x;
}

// ------------------------------------------------------------------ eigenvalues (multisection)
template <typename RT>
__device__ __forceinline__ int sturm_count(const RT *__restrict__ d, const RT *__restrict__ e, int n,
                                           RT x, RT pivmin) {
    int c = 0;
    RT q = d[0] - x;
    if (fabs(q) < pivmin) q = -pivmin;
    c += (q < 0.0);
    for (int i = 1; i < n; ++i) {
        const RT ei = e[i - 1];
        q = d[i] - x - (ei * ei) / q;
        if (fabs(q) < pivmin) q = -pivmin;
        c += (q < 0.0);
    }
    return c;
}

template <typename RT>
__device__ void tri_bounds(const RT *__restrict__ d, const RT *__restrict__ e, int n, RT &lo,
                           RT &hi, RT &tnorm, RT &pivmin) {
    lo = Lim<RT>::big();
    hi = -Lim<RT>::big();
    RT emax2 = 0.0;
    for (int i = 0; i < n; ++i) {
        RT r = 0.0;
        if (i > 0) r += fabs(e[i - 1]);
        if (i < n - 1) { r += fabs(e[i]); emax2 = fmax(emax2, e[i] * e[i]); }
        lo = fmin(lo, d[i] - r);
        hi = fmax(hi, d[i] + r);
    }
    tnorm = fmax(fabs(lo), fabs(hi));
    pivmin = Lim<RT>::tiny() * fmax((RT)1.0, emax2);
    const RT pad = 2.0 * Lim<RT>::eps() * tnorm * n + 2.0 * pivmin;
    lo -= pad;
    hi += pad;
}

// Multisection: each round the 32 lanes of a warp evaluate Sturm counts at 32
// points inside the bracket and keep the 1/33 of it that holds eigenvalue k
// (about 5 bits per round).  The FP64 divisions of the Sturm counts are the cost
// (this GPU has few FP64 units per SM).
constexpr int kMsLanes = 32;
constexpr int kMsMaxN = 4096;  // FP32 pre-bracketing copies of d and e^2 (shared memory)
// FP32 Sturm count on FP32 copies of d and e^2 (shared memory).
__device__ __forceinline__ int sturm_count32(const float *__restrict__ d, const float *__restrict__ e2, int n, float x,
                                             float pivmin) {
    int c = 0;
    float q = d[0] - x;
    if (fabsf(q) < pivmin) q = -pivmin;
    c += (q < 0.f);
    for (int i = 1; i < n; ++i) {
        q = d[i] - x - e2[i - 1] / q;
        if (fabsf(q) < pivmin) q = -pivmin;
        c += (q < 0.f);
    }
    return c;
}

// One warp per eigenvalue index k < m, one warp per block so that the m warps spread over
// the SMs.  FP64 (RT = double): a few cheap FP32 rounds first narrow the bracket.  FP32
// Sturm counts are exact for a matrix whose entries are within a few FP32 roundings of T
// (Kahan; Demmel, Dhillon and Ren 1995), so the FP32 bracket widened by a margin well above
// that perturbation still holds the eigenvalue; the first FP64 round checks it (its end
// lanes evaluate the two bracket ends) and falls back to the Gershgorin bracket if not.
template <typename RT>
__global__ void __launch_bounds__(32)
k_multisect(int n, int m, const RT *__restrict__ d, const RT *__restrict__ e, RT *__restrict__ theta) {
    const int k = blockIdx.x;
    const int sub = threadIdx.x;
    if (k >= m) return;
    RT lo, hi, tnorm, pivmin;
    tri_bounds(d, e, n, lo, hi, tnorm, pivmin);
    bool check = false;
    const RT lo_g = lo, hi_g = hi;
    if constexpr (sizeof(RT) == 8) {
        __shared__ float ds[kMsMaxN], e2s[kMsMaxN];
        if (n <= kMsMaxN) {
            for (int i = sub; i < n; i += kMsLanes) {
                ds[i] = (float)d[i];
                e2s[i] = (i + 1 < n) ? (float)(e[i] * e[i]) : 0.f;
            }
            __syncwarp();
            const float tn = (float)tnorm;
            const float piv = FLT_MIN * fmaxf(1.f, tn * tn);
            const float margin = 32.f * FLT_EPSILON * tn + 4.f * piv;
            float l32 = (float)lo, h32 = (float)hi;
            for (int it = 0; it < 8 && h32 - l32 > 4.f * margin; ++it) {  // warp-uniform
                const float w = h32 - l32;
                const float x = l32 + w * (float)(sub + 1) / (float)(kMsLanes + 1);
                const int c = sturm_count32(ds, e2s, n, x, piv);
                const unsigned mask = __ballot_sync(0xffffffffu, c <= k);
                const int T = __popc(mask) - 1;
                const float xlo = __shfl_sync(0xffffffffu, x, T < 0 ? 0 : T);
                const float xhi = __shfl_sync(0xffffffffu, x, T < kMsLanes - 1 ? T + 1 : kMsLanes - 1);
                if (T >= 0) l32 = xlo;
                if (T < kMsLanes - 1) h32 = xhi;
            }
            lo = fmax(lo_g, (RT)l32 - (RT)margin);
            hi = fmin(hi_g, (RT)h32 + (RT)margin);
            check = true;
        }
    }
    for (int it = 0; it < 32; ++it) {
        const RT w = hi - lo;
        if (w <= 2.0 * Lim<RT>::eps() * fmax(fabs(lo), fabs(hi)) + 4.0 * pivmin) break;  // warp-uniform
        RT x;
        if (check)  // bracket ends on the end lanes, 30 points between
            x = (sub == 0) ? lo : (sub == kMsLanes - 1) ? hi : lo + w * (RT)sub / (RT)(kMsLanes - 1);
        else
            x = lo + w * (RT)(sub + 1) / (RT)(kMsLanes + 1);
        const int c = sturm_count(d, e, n, x, pivmin);
        if (check) {
            check = false;
            const bool ok = __shfl_sync(0xffffffffu, c, 0) <= k && __shfl_sync(0xffffffffu, c, kMsLanes - 1) > k;
            if (!ok) {  // the FP32 bracket missed (not expected): restart from Gershgorin
                lo = lo_g;
                hi = hi_g;
                continue;
            }
        }
        const unsigned mask = __ballot_sync(0xffffffffu, c <= k);
        const int T = __popc(mask) - 1;  // counts are monotone in sub: lanes 0..T have c <= k
        const RT xlo = __shfl_sync(0xffffffffu, x, T < 0 ? 0 : T);
        const RT xhi = __shfl_sync(0xffffffffu, x, T < kMsLanes - 1 ? T + 1 : kMsLanes - 1);
        if (T >= 0) lo = xlo;
        if (T < kMsLanes - 1) hi = xhi;
    }
    if (sub == 0) theta[k] = 0.5 * (lo + hi);
}

// Double-FP32 Sturm count on pair copies of d and e^2 (shared memory): the same recurrence,
// its divisions on the FP32 units (one SM sub-partition issues an FP64 instruction for a whole
// warp in 64 cycles on this GPU, an FP32 one in 1).  About 2^-47 relative per operation: the
// count is exact for a matrix within a few such roundings of T.
__device__ __forceinline__ int sturm_count_df(const df64 *__restrict__ d, const df64 *__restrict__ e2, int n, df64 x,
                                              float pivmin) {
    int c = 0;
    df64 q = d[0] - x;
    if (fabsf(q.hi) < pivmin) q = df64(-pivmin);
    c += (q.hi < 0.f);
    for (int i = 1; i < n; ++i) {
        q = (d[i] - x) - e2[i - 1] / q;
        if (fabsf(q.hi) < pivmin) q = df64(-pivmin);
        c += (q.hi < 0.f);
    }
    return c;
}

// Multisection of the FP64-class Rayleigh-Ritz step (same rounds as k_multisect): FP32 rounds
// narrow the bracket, double-FP32 rounds finish it; the bracket bounds come from FP32 copies of
// T with a generous pad.  Dynamic shared memory: d, e^2 as pairs, then as floats (24 n bytes).
__global__ void __launch_bounds__(32)
k_multisect_df(int n, int m, const double *__restrict__ d, const double *__restrict__ e, double *__restrict__ theta) {
    extern __shared__ __align__(16) unsigned char smraw[];
    df64 *dd = reinterpret_cast<df64 *>(smraw);
    df64 *de2 = dd + n;
    float *ds = reinterpret_cast<float *>(de2 + n);
    float *e2s = ds + n;
    const int k = blockIdx.x, sub = threadIdx.x;
    if (k >= m) return;
    for (int i = sub; i < n; i += kMsLanes) {
        dd[i] = df64(d[i]);
        const df64 ei = (i + 1 < n) ? df64(e[i]) : df64(0.f);
        de2[i] = ei * ei;
        ds[i] = dd[i].hi;
        e2s[i] = de2[i].hi;
    }
    __syncwarp();
    // Gershgorin bracket in FP32, padded well above its rounding
    float lo_f = FLT_MAX, hi_f = -FLT_MAX, emax2 = 0.f;
    for (int i = 0; i < n; ++i) {
        float r = 0.f;
        if (i > 0) r += sqrtf(e2s[i - 1]);
        if (i < n - 1) { r += sqrtf(e2s[i]); emax2 = fmaxf(emax2, e2s[i]); }
        lo_f = fminf(lo_f, ds[i] - r);
        hi_f = fmaxf(hi_f, ds[i] + r);
    }
    const float tn = fmaxf(fabsf(lo_f), fabsf(hi_f));
    const float piv = FLT_MIN * fmaxf(1.f, fmaxf(emax2, tn * tn));
    const float gpad = 64.f * FLT_EPSILON * tn * (float)n + 4.f * piv;
    lo_f -= gpad;
    hi_f += gpad;
    const float margin = 32.f * FLT_EPSILON * tn + 4.f * piv;
    float l32 = lo_f, h32 = hi_f;
    for (int it = 0; it < 8 && h32 - l32 > 4.f * margin; ++it) {  // warp-uniform
        const float w = h32 - l32;
        const float x = l32 + w * (float)(sub + 1) / (float)(kMsLanes + 1);
        const int c = sturm_count32(ds, e2s, n, x, piv);
        const unsigned mask = __ballot_sync(0xffffffffu, c <= k);
        const int T = __popc(mask) - 1;
        const float xlo = __shfl_sync(0xffffffffu, x, T < 0 ? 0 : T);
        const float xhi = __shfl_sync(0xffffffffu, x, T < kMsLanes - 1 ? T + 1 : kMsLanes - 1);
        if (T >= 0) l32 = xlo;
        if (T < kMsLanes - 1) h32 = xhi;
    }
    const df64 lo_g(lo_f), hi_g(hi_f);
    df64 lo = fmax(lo_g, df64(l32) - df64(margin)), hi = fmin(hi_g, df64(h32) + df64(margin));
    bool check = true;
    const float eps_df = 0x1p-45f;
    for (int it = 0; it < 40; ++it) {
        const df64 w = hi - lo;
        if (w.hi <= 2.f * eps_df * fmaxf(fabsf(lo.hi), fabsf(hi.hi)) + 4.f * piv) break;  // warp-uniform
        df64 x;
        if (check)  // bracket ends on the end lanes, 30 points between
            x = (sub == 0) ? lo : (sub == kMsLanes - 1) ? hi : lo + w * df64((float)sub / (float)(kMsLanes - 1));
        else
            x = lo + w * df64((float)(sub + 1) / (float)(kMsLanes + 1));
        const int c = sturm_count_df(dd, de2, n, x, piv);
        if (check) {
            check = false;
            const bool ok = __shfl_sync(0xffffffffu, c, 0) <= k && __shfl_sync(0xffffffffu, c, kMsLanes - 1) > k;
            if (!ok) {  // the FP32 bracket missed (not expected): restart from Gershgorin
                lo = lo_g;
                hi = hi_g;
                continue;
            }
        }
        const unsigned mask = __ballot_sync(0xffffffffu, c <= k);
        const int T = __popc(mask) - 1;
        const df64 xlo = __shfl_sync(0xffffffffu, x, T < 0 ? 0 : T);
        const df64 xhi = __shfl_sync(0xffffffffu, x, T < kMsLanes - 1 ? T + 1 : kMsLanes - 1);
        if (T >= 0) lo = xlo;
        if (T < kMsLanes - 1) hi = xhi;
    }
    if (sub == 0) theta[k] = (double)((lo + hi) * df64(0.5f));
}

// ------------------------------------------------------------------ eigenvectors (inverse iteration)
template <typename RT>
__device__ __forceinline__ RT hash_uniform(unsigned int a, unsigned int b) {
    unsigned int h = a * 0x9E3779B1u ^ (b + 0x7F4A7C15u) * 0x85EBCA77u;
    h ^= h >> 16; h *= 0x7FEB352Du; h ^= h >> 15; h *= 0x846CA68Bu; h ^= h >> 16;
    return (RT)h * (2.0 / 4294967296.0) - 1.0;
}

// One warp per eigenvalue index; the warp whose eigenvalue starts a cluster of
// close eigenvalues computes all vectors of that cluster, in order: lane 0 runs the
// LU of T - lambda I with partial pivoting and the solves (sequential recurrences,
// kept in shared memory), from a pseudo-random start, three times; after each solve
// the warp orthogonalises against the cluster's earlier vectors (modified
// Gram-Schmidt) and normalises.  Dynamic shared memory: 6 n reals + n pivots.
template <typename RT>
__global__ void __launch_bounds__(32)
k_inviter(int n, int m, const RT *__restrict__ d, const RT *__restrict__ e, const RT *__restrict__ theta,
          RT *Z) {
    extern __shared__ __align__(16) unsigned char smraw[];
    RT *dd = reinterpret_cast<RT *>(smraw);
    RT *du = dd + n, *du2 = du + n, *dl = du2 + n, *z = dl + n, *rdd = z + n;
    signed char *pv = reinterpret_cast<signed char *>(rdd + n);
    const int k = blockIdx.x, lane = threadIdx.x;
    if (k >= m) return;
    RT lo, hi, tnorm, pivmin;
    tri_bounds(d, e, n, lo, hi, tnorm, pivmin);
    // vectors of eigenvalues closer than gaptol are orthogonalised against each other;
    // elsewhere orthogonality is ~ eps |T| / gap (LAPACK uses 1e-3 |T| for single precision)
    const RT gaptol = (sizeof(RT) == 4 ? (RT)1e-3 : (RT)1e-5) * fmax(tnorm, Lim<RT>::tiny());
    const RT pert = 10.0 * Lim<RT>::eps() * fmax(tnorm, Lim<RT>::tiny());
    if (k > 0 && theta[k] - theta[k - 1] <= gaptol) return;  // not a cluster start
    RT lam_prev = -Lim<RT>::big();
    for (int j = k; j < m; ++j) {
        if (j > k && theta[j] - theta[j - 1] > gaptol) break;
        RT lam = theta[j];
        if (j > k && lam < lam_prev + pert) lam = lam_prev + pert;
        lam_prev = lam;
        RT *zj = Z + (size_t)j * n;
        if (lane == 0) {
            for (int i = 0; i < n; ++i) dd[i] = d[i] - lam;
            for (int i = 0; i + 1 < n; ++i) { du[i] = e[i]; dl[i] = e[i]; du2[i] = 0.0; }
            for (int i = 0; i + 1 < n; ++i) {
                if (fabs(dd[i]) >= fabs(dl[i])) {
                    pv[i] = 0;
                    if (dd[i] == 0.0) dd[i] = pert;
                    const RT f = dl[i] / dd[i];
                    dl[i] = f;
                    dd[i + 1] -= f * du[i];
                } else {
                    pv[i] = 1;
                    const RT f = dd[i] / dl[i];
                    dd[i] = dl[i];
                    dl[i] = f;
                    const RT t = du[i];
                    du[i] = dd[i + 1];
                    dd[i + 1] = t - f * dd[i + 1];
                    if (i + 2 < n) { du2[i] = du[i + 1]; du[i + 1] = -f * du[i + 1]; }
                }
            }
            if (dd[n - 1] == 0.0) dd[n - 1] = pert;
        }
        __syncwarp();
        // reciprocal pivots, all lanes: the three solves below then multiply instead of divide
        for (int i = lane; i < n; i += 32) rdd[i] = (RT)1.0 / dd[i];
        for (int i = lane; i < n; i += 32) z[i] = hash_uniform<RT>((unsigned)j, (unsigned)i);
        __syncwarp();
        for (int it = 0; it < 3; ++it) {
            if (lane == 0) {
                for (int i = 0; i + 1 < n; ++i) {
                    if (pv[i] == 0) {
                        z[i + 1] -= dl[i] * z[i];
                    } else {
                        const RT t = z[i];
                        z[i] = z[i + 1];
                        z[i + 1] = t - dl[i] * z[i];
                    }
                }
                z[n - 1] = z[n - 1] * rdd[n - 1];
                if (n > 1) z[n - 2] = (z[n - 2] - du[n - 2] * z[n - 1]) * rdd[n - 2];
                for (int i = n - 3; i >= 0; --i) z[i] = (z[i] - du[i] * z[i + 1] - du2[i] * z[i + 2]) * rdd[i];
            }
            __syncwarp();
            for (int p = k; p < j; ++p) {
                const RT *zp = Z + (size_t)p * n;
                RT sp = 0.0;
                for (int i = lane; i < n; i += 32) sp += z[i] * zp[i];
                sp = warp_sum(sp);
                for (int i = lane; i < n; i += 32) z[i] -= sp * zp[i];
                __syncwarp();
            }
            RT nr = 0.0;
            for (int i = lane; i < n; i += 32) nr += z[i] * z[i];
            nr = warp_sum(nr);
            const RT inv = nr > 0.0 ? 1.0 / sqrt(nr) : 0.0;
            for (int i = lane; i < n; i += 32) z[i] *= inv;
            __syncwarp();
        }
        for (int i = lane; i < n; i += 32) zj[i] = z[i];
        __syncwarp();
    }
}

// ------------------------------------------------------------------ back-transformation
// V = H_0 H_1 ... H_{n-2} Z with H_i = I - tau_i v_i v_i^H, applied kWy reflectors at a time in
// the compact WY form (Schreiber and Van Loan, 1989): H_{i0} ... H_{i0+k-1} = I - Y T Y^H with
// Y = [v_{i0} ... v_{i0+k-1}] and T upper triangular, T_jj = tau_j and
// T[0:j, j] = -tau_j T[0:j, 0:j] (Y[:, 0:j]^H v_j).  Each block then costs one reduction
// (t = Y^H z) instead of one per reflector.  v_i is read only on its support r >= i + 1.
constexpr int kWy = 32;

// Partial Gram matrices G = Y^H Y of each block of kWy reflectors (block b: reflectors
// 32 b ...), over row chunk ch of the block's rows [32 b + 1, n): grid (blocks, chunks).  The
// chunk of Y is staged in shared memory (zero where v_k has no support, r <= 32 b + k); thread
// (k, g) accumulates G[k][g + 8 u], u = 0..3.  Gp[b][ch] is a full kWy x kWy row-major matrix.
constexpr int kWyRows = 64;   // rows of a chunk
template <typename CT>
__global__ void __launch_bounds__(256)
k_wy_gram(int n, int nch, const cx<CT> *__restrict__ Hv, cx<CT> *__restrict__ Gp) {
    __shared__ cx<CT> Ys[kWyRows][kWy + 1];
    const int b = blockIdx.x, ch = blockIdx.y, i0 = b * kWy, kb = min(kWy, n - 1 - i0);
    const int rows = n - (i0 + 1), per = (rows + nch - 1) / nch;
    const int r0 = i0 + 1 + ch * per, r1 = min(n, r0 + per);
    const int tid = threadIdx.x, k = tid >> 3, g = tid & 7;
    const cx<CT> zero = mkc<CT>(0.0, 0.0);
    cx<CT> acc[4] = {zero, zero, zero, zero};
    for (int c0 = r0; c0 < r1; c0 += kWyRows) {
        __syncthreads();
        for (int e = tid; e < kWyRows * kWy; e += blockDim.x) {
            const int kk = e / kWyRows, rr = e % kWyRows, r = c0 + rr;
            Ys[rr][kk] = (kk < kb && r < r1 && r > i0 + kk) ? Hv[(size_t)(i0 + kk) * n + r] : zero;
        }
        __syncthreads();
        const int nr = min(kWyRows, r1 - c0);
        for (int rr = 0; rr < nr; ++rr) {
            const cx<CT> a = conjc(Ys[rr][k]);
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u] = cmac(acc[u], a, Ys[rr][g + 8 * u]);
        }
    }
    cx<CT> *out = Gp + ((size_t)b * nch + ch) * kWy * kWy;
#pragma unroll
    for (int u = 0; u < 4; ++u) out[k * kWy + g + 8 * u] = acc[u];
}

// T of each block from its Gram (chunk partials summed in chunk order): T_jj = tau_j, then
// pairs of adjacent diagonal blocks of width h = 1, 2, 4, 8, 16 merged by
// T12 = -T11 G12 T22 (the product of the two blocks' WY forms), each merge level in two
// parallel matrix products.  kWy x kWy row-major into Tf[b], zero outside the reflectors.
template <typename CT>
__global__ void __launch_bounds__(256)
k_wy_t(int n, int nch, const cx<CT> *__restrict__ Gp, const cx<CT> *__restrict__ taus, cx<CT> *__restrict__ Tf) {
    __shared__ cx<CT> G[kWy][kWy + 1];
    __shared__ cx<CT> T[kWy][kWy + 1];
    __shared__ cx<CT> X[kWy][kWy + 1];
    const int b = blockIdx.x, i0 = b * kWy, kb = min(kWy, n - 1 - i0), tid = threadIdx.x;
    const cx<CT> zero = mkc<CT>(0.0, 0.0);
    for (int e = tid; e < kWy * kWy; e += blockDim.x) {
        const int k = e / kWy, j = e % kWy;
        cx<CT> sum = zero;
        for (int ch = 0; ch < nch; ++ch) sum = sum + Gp[((size_t)b * nch + ch) * kWy * kWy + e];
        G[k][j] = sum;
        T[k][j] = (k == j && k < kb) ? taus[i0 + k] : zero;
    }
    __syncthreads();
    for (int h = 1; h < kWy; h *= 2) {
        // entries of the merges at this level: (kWy / 2h) merges x h x h
        const int nent = (kWy / (2 * h)) * h * h;
        // X = T11 G12
        for (int e = tid; e < nent; e += blockDim.x) {
            const int mg = e / (h * h), k = (e % (h * h)) / h, l = e % h;
            const int a = mg * 2 * h;
            cx<CT> u = zero;
            for (int p = k; p < h; ++p) u = cmac(u, T[a + k][a + p], G[a + p][a + h + l]);
            X[a + k][a + h + l] = u;
        }
        __syncthreads();
        // T12 = -X T22
        for (int e = tid; e < nent; e += blockDim.x) {
            const int mg = e / (h * h), k = (e % (h * h)) / h, l = e % h;
            const int a = mg * 2 * h;
            cx<CT> u = zero;
            for (int p = 0; p <= l; ++p) u = cmac(u, X[a + k][a + h + p], T[a + h + p][a + h + l]);
            T[a + k][a + h + l] = zero - u;
        }
        __syncthreads();
    }
    for (int e = tid; e < kWy * kWy; e += blockDim.x) Tf[(size_t)b * kWy * kWy + e] = T[e / kWy][e % kWy];
}

// NV eigenvectors per CTA (z in shared memory in the compute type CT), blocks from the last
// to the first: t = Y^H z (a warp per reflector, KU reflectors at once for independent
// accumulation chains, fixed-order warp sums), s = T t (eight lanes per entry, combined by a
// shuffle tree), z -= Y s (a thread per row, KU partial sums).  Dynamic shared memory:
// NV n entries.
template <typename RT, typename CT, int NV>
__global__ void __launch_bounds__(256)
k_backtransform_wy(int n, int m, const cx<CT> *__restrict__ Hv, const cx<CT> *__restrict__ Tf,
                   const RT *__restrict__ Z, cx<RT> *__restrict__ V, int ldv) {
    constexpr int KU = NV >= 4 ? 1 : 4;
    extern __shared__ __align__(16) unsigned char smraw[];
    cx<CT> *z = reinterpret_cast<cx<CT> *>(smraw);   // [NV][n]
    __shared__ cx<CT> t[NV][kWy], sv[NV][kWy];
    const int j0 = blockIdx.x * NV, tid = threadIdx.x, lane = tid & 31, wp = tid >> 5, nw = blockDim.x >> 5;
    const cx<CT> zero = mkc<CT>(0.0, 0.0);
    for (int e = tid; e < NV * n; e += blockDim.x) {
        const int vv = e / n, r = e % n;
        z[e] = (j0 + vv < m) ? mkc<CT>((CT)Z[(size_t)(j0 + vv) * n + r], CT(0.0)) : zero;
    }
    __syncthreads();
    const int nblk = (n - 1 + kWy - 1) / kWy;
    for (int b = nblk - 1; b >= 0; --b) {
        const int i0 = b * kWy, kb = min(kWy, n - 1 - i0);
        // t_k = v_{i0+k}^H z, reflectors k = k0 + nw u (u < KU) together
        for (int k0 = wp; k0 < kWy; k0 += nw * KU) {
            cx<CT> acc[KU][NV];
#pragma unroll
            for (int u = 0; u < KU; ++u)
#pragma unroll
                for (int vv = 0; vv < NV; ++vv) acc[u][vv] = zero;
            for (int r = i0 + 1 + lane; r < n; r += 32) {
                cx<CT> zr[NV];
#pragma unroll
                for (int vv = 0; vv < NV; ++vv) zr[vv] = z[vv * n + r];
#pragma unroll
                for (int u = 0; u < KU; ++u) {
                    const int k = k0 + nw * u;
                    if (k < kb && r > i0 + k) {   // v_{i0+k} lives on r >= i0 + k + 1
                        const cx<CT> a = conjc(Hv[(size_t)(i0 + k) * n + r]);
#pragma unroll
                        for (int vv = 0; vv < NV; ++vv) acc[u][vv] = cmac(acc[u][vv], a, zr[vv]);
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < KU; ++u) {
                const int k = k0 + nw * u;
#pragma unroll
                for (int vv = 0; vv < NV; ++vv) {
                    const CT re = warp_sum(acc[u][vv].x), im = warp_sum(acc[u][vv].y);
                    if (lane == 0 && k < kWy) t[vv][k] = mkc<CT>(re, im);
                }
            }
        }
        __syncthreads();
        // s = T t: entry (vv, k) from eight lanes, lane part p taking l = k + p, k + p + 8, ...
        const cx<CT> *Tb = Tf + (size_t)b * kWy * kWy;
        for (int e = tid; e < NV * kWy * 8; e += blockDim.x) {
            const int p = e & 7, k = (e >> 3) % kWy, vv = (e >> 3) / kWy;
            cx<CT> u = zero;
            for (int l = k + p; l < kb; l += 8) u = cmac(u, Tb[k * kWy + l], t[vv][l]);
#pragma unroll
            for (int o = 1; o < 8; o <<= 1) {
                u.x += __shfl_xor_sync(0xffffffffu, u.x, o);
                u.y += __shfl_xor_sync(0xffffffffu, u.y, o);
            }
            if (p == 0) sv[vv][k] = u;
        }
        __syncthreads();
        // z -= Y s on the rows the block touches
        for (int r = i0 + 1 + tid; r < n; r += blockDim.x) {
            const int kmax = min(kb, r - i0);   // v_{i0+k}[r] is zero for r <= i0 + k
            cx<CT> d[NV][KU];                   // KU partial sums per vector
#pragma unroll
            for (int vv = 0; vv < NV; ++vv)
#pragma unroll
                for (int q = 0; q < KU; ++q) d[vv][q] = zero;
            for (int k = 0; k < kmax; k += KU) {
#pragma unroll
                for (int q = 0; q < KU; ++q) {
                    if (k + q < kmax) {
                        const cx<CT> a = Hv[(size_t)(i0 + k + q) * n + r];
#pragma unroll
                        for (int vv = 0; vv < NV; ++vv) d[vv][q] = cmac(d[vv][q], a, sv[vv][k + q]);
                    }
                }
            }
#pragma unroll
            for (int vv = 0; vv < NV; ++vv) {
                cx<CT> tot = d[vv][0];
#pragma unroll
                for (int q = 1; q < KU; ++q) tot = tot + d[vv][q];
                z[vv * n + r] = z[vv * n + r] - tot;
            }
        }
        __syncthreads();
    }
    for (int e = tid; e < NV * n; e += blockDim.x) {
        const int vv = e / n, r = e % n;
        if (j0 + vv < m) V[(size_t)(j0 + vv) * ldv + r] = mkc<RT>((RT)z[e].x, (RT)z[e].y);
    }
}

template <typename RT>
__global__ void k_scale_rows_copy(int n, int m, const RT *__restrict__ d, const cx<RT> *__restrict__ T, int ldt,
                                  cx<RT> *__restrict__ C, int ldc) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (i < n) C[(size_t)j * ldc + i] = d[i] * T[(size_t)j * ldt + i];
}

__global__ void k_copy_int(const int *__restrict__ a, int *__restrict__ b) { *b = *a; }

size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

// Raise a kernel's dynamic shared-memory ceiling to the device maximum.  The attribute is
// process-wide, so it is never lowered: launches of different sizes on concurrent streams
// then never see a ceiling below their own request.
int allow_max_dyn_smem(const void *fn) {
    int dev = 0, smem_max = 0;
    LG_CUDA_TRY(cudaGetDevice(&dev));
    LG_CUDA_TRY(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa;
    LG_CUDA_TRY(cudaFuncGetAttributes(&fa, fn));
    LG_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     smem_max - (int)fa.sharedSizeBytes));
    return LOBPCG_OK;
}

// The cluster-resident tridiagonalisation when the matrix fits one cluster's shared memory
// (16 CTAs above n = 192, else 8) and the device can place such a cluster; done = false
// leaves the reduction to the grid-wide kernels.
template <typename RT, typename CT>
int launch_tri_cluster(int n, const cx<RT> *A, int lda, cx<RT> *Hv, cx<RT> *taus, RT *dg, RT *eg, cudaStream_t s,
                       bool &done) {
    done = false;
    const int CS = n > 192 ? 16 : 8;
    const int nr = (n + CS - 1) / CS;
    const size_t dsm = sizeof(cx<CT>) * ((size_t)nr * n + 7 * (size_t)n);
    int dev = 0, smem_max = 0, cl_ok = 0;
    LG_CUDA_TRY(cudaGetDevice(&dev));
    LG_CUDA_TRY(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    LG_CUDA_TRY(cudaDeviceGetAttribute(&cl_ok, cudaDevAttrClusterLaunch, dev));
    const void *fn = (const void *)k_tri_cluster<RT, CT>;
    cudaFuncAttributes fa;
    LG_CUDA_TRY(cudaFuncGetAttributes(&fa, fn));
    if (!cl_ok || dsm + fa.sharedSizeBytes > (size_t)smem_max) return LOBPCG_OK;
    // the same (largest) limit from every caller: concurrent lanes launch this kernel with
    // different sizes, and a per-call limit set by one would invalidate another's launch
    LG_TRY(allow_max_dyn_smem(fn));
    if (CS > 8) LG_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CS);
    cfg.blockDim = dim3(std::min(1024, 32 * nr));  // one warp per owned row
    cfg.dynamicSmemBytes = dsm;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CS;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, fn, &cfg) != cudaSuccess || ncl < 1) {
        (void)cudaGetLastError();  // this cluster shape cannot be placed: not an error
        return LOBPCG_OK;
    }
    LG_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_tri_cluster<RT, CT>, n, A, lda, Hv, taus, dg, eg));
    LG_TRY(check_launch("tridiagonalisation (cluster)"));
    done = true;
    return LOBPCG_OK;
}
constexpr int kTriClusterMaxN = 416;
constexpr int kWyChunks = 8;   // row chunks of the back-transformation's Gram partials

// T factors, then the blocked application; NV eigenvectors per CTA, as many as keep about
// 128 CTAs or more (each CTA reads every reflector once).
template <typename RT, typename CT>
int backtransform_wy(int n, int m, const cx<CT> *Hv, const cx<CT> *taus, cx<CT> *Tf, cx<CT> *Gp, const RT *Z,
                     cx<RT> *V, int ldv, cudaStream_t s) {
    const int nblk = (n - 1 + kWy - 1) / kWy;
    const int nch = kWyChunks;
    k_wy_gram<CT><<<dim3(nblk, nch), 256, 0, s>>>(n, nch, Hv, Gp);
    LG_TRY(check_launch("back-transform Gram partials"));
    k_wy_t<CT><<<nblk, 256, 0, s>>>(n, nch, Gp, taus, Tf);
    LG_TRY(check_launch("back-transform T factors"));
    const int NV = m >= 8 * 128 ? 8 : m >= 4 * 128 ? 4 : m >= 2 * 128 ? 2 : 1;
    const size_t smem = sizeof(cx<CT>) * (size_t)NV * n;
    const int grid = (m + NV - 1) / NV;
    auto run = [&](auto kern) -> int {
        if (smem > 48 * 1024) LG_TRY(allow_max_dyn_smem((const void *)kern));
        kern<<<grid, 256, smem, s>>>(n, m, Hv, Tf, Z, V, ldv);
        return check_launch("back-transform (compact WY)");
    };
    if (NV == 8) return run(k_backtransform_wy<RT, CT, 8>);
    if (NV == 4) return run(k_backtransform_wy<RT, CT, 4>);
    if (NV == 2) return run(k_backtransform_wy<RT, CT, 2>);
    return run(k_backtransform_wy<RT, CT, 1>);
}

template <typename RT>
int heev_lowest_t(EigWork &w, int n, int m, cx<RT> *A, int lda, RT *theta, cx<RT> *V, int ldv, cudaStream_t s) {
    if (n <= 0 || m <= 0) return LOBPCG_OK;
    if (m > n) return fail(LOBPCG_ERR_ARG, "heev: m > n");
    // workspace carve-up
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes); return o; };
    const size_t o_hv = take(sizeof(cx<RT>) * (size_t)n * n);
    const size_t o_tau = take(sizeof(cx<RT>) * n);
    const size_t o_d = take(sizeof(RT) * n);
    const size_t o_e = take(sizeof(RT) * n);
    const size_t o_yp = take(sizeof(cx<RT>) * 2 * (size_t)((n + 15) / 16) * n);
    const size_t o_wv = take(sizeof(cx<RT>) * 2 * (size_t)n);
    const size_t o_z = take(sizeof(RT) * (size_t)n * m);
    const size_t o_cnt = take(sizeof(unsigned int) * n);
    const size_t o_tf = take(sizeof(cx<RT>) * (size_t)kWy * kWy * ((n + kWy - 1) / kWy));
    const size_t o_gp = take(sizeof(cx<RT>) * (size_t)kWy * kWy * kWyChunks * ((n + kWy - 1) / kWy));
    LG_TRY(w.alloc->ensure(w.buf, off));
    char *base = reinterpret_cast<char *>(w.buf.p);
    cx<RT> *Hv = reinterpret_cast<cx<RT> *>(base + o_hv);
    cx<RT> *taus = reinterpret_cast<cx<RT> *>(base + o_tau);
    RT *dg = reinterpret_cast<RT *>(base + o_d);
    RT *eg = reinterpret_cast<RT *>(base + o_e);
    cx<RT> *yp = reinterpret_cast<cx<RT> *>(base + o_yp);
    cx<RT> *wv = reinterpret_cast<cx<RT> *>(base + o_wv);
    RT *Z = reinterpret_cast<RT *>(base + o_z);
    unsigned int *cnt = reinterpret_cast<unsigned int *>(base + o_cnt);
    cx<RT> *Tf = reinterpret_cast<cx<RT> *>(base + o_tf);
    cx<RT> *Gp = reinterpret_cast<cx<RT> *>(base + o_gp);
    LG_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(unsigned int) * n, s));
    LG_CUDA_TRY(cudaMemsetAsync(taus, 0, sizeof(cx<RT>) * n, s));
    bool coop_done = false, hv_df = false;
    if (n >= 2 && n <= kTriClusterMaxN) {
        bool done = false, df = false;
        if constexpr (std::is_same<RT, double>::value) {
            df = w.df;  // the double-FP32 compute type, as in the grid-wide kernel below
            if (df) LG_TRY((launch_tri_cluster<RT, df64>(n, A, lda, Hv, taus, dg, eg, s, done)));
        }
        if (!df) LG_TRY((launch_tri_cluster<RT, RT>(n, A, lda, Hv, taus, dg, eg, s, done)));
        coop_done = done;
        hv_df = done && df;
    }
    if (!coop_done && n >= 2) {
        // fused version: tiles resident in shared memory, one grid barrier per column; 16 x 16
        // tiles for small matrices (more SMs share a column's FP64 work), else 32 x 32
        int dev = 0, sms = 0, coop = 0, smem_max = 0;
        LG_CUDA_TRY(cudaGetDevice(&dev));
        LG_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        LG_CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
        LG_CUDA_TRY(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        const bool small_tiles = n <= 256;
        const int TS = small_tiles ? 16 : 32;
        const int T = (n + TS - 1) / TS;
        // with concurrent streams each cooperative grid gets its share of the SMs, so that all of
        // them fit at once (no gate needed then)
        const int share = std::max(1, w.coop_share);
        const int G = std::max(1, std::min(T * T, sms / share));
        const int nown = (T * T + G - 1) / G;
        const size_t dsm = sizeof(cx<RT>) * ((size_t)nown * TS * TS + 4 * (size_t)n);
        const size_t static_sm = sizeof(RT) * 32 + sizeof(cx<RT>) * 16 * 33 + 64;
        int *err = device_wait_flag();
        const void *fn = small_tiles ? (const void *)k_tri_fused<RT, 16> : (const void *)k_tri_fused<RT, 32>;
        bool fn_df = false;
        if constexpr (std::is_same<RT, double>::value) {
            if (w.df) {  // the column's vector work in double-FP32 (this GPU has few FP64 units per SM)
                fn = small_tiles ? (const void *)k_tri_fused<RT, 16, df64> : (const void *)k_tri_fused<RT, 32, df64>;
                fn_df = true;
            }
        }
        if (coop && err && dsm + static_sm <= (size_t)smem_max) {
            LG_TRY(allow_max_dyn_smem(fn));
            int per_sm = 0;
            LG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, dsm));
            if (per_sm >= 1 && (size_t)G * share <= (size_t)sms * per_sm) {
                unsigned int *bar = cnt;
                const cx<RT> *Ac = A;
                void *args[] = {(void *)&n, (void *)&Ac, (void *)&lda, (void *)&Hv, (void *)&taus, (void *)&dg,
                                (void *)&eg, (void *)&yp, (void *)&wv, (void *)&bar, (void *)&err};
                if (w.gate && share == 1) {
                    // one cooperative grid at a time across concurrent streams
                    std::lock_guard<std::mutex> lk(w.gate->mu);
                    if (w.gate->used) LG_CUDA_TRY(cudaStreamWaitEvent(s, w.gate->ev, 0));
                    LG_CUDA_TRY(cudaLaunchCooperativeKernel(fn, dim3(G), dim3(256), args, dsm, s));
                    LG_CUDA_TRY(cudaEventRecord(w.gate->ev, s));
                    w.gate->used = true;
                } else {
                    LG_CUDA_TRY(cudaLaunchCooperativeKernel(fn, dim3(G), dim3(256), args, dsm, s));
                }
                LG_TRY(check_launch("tridiagonalisation (fused cooperative)"));
                coop_done = true;
                hv_df = fn_df;  // reflectors stored as pairs
            }
        }
    }
    if (!coop_done && n >= 2 && n <= 1024) {
        // one cooperative launch; falls back to two launches per column if it cannot run
        const int tl0 = (n - 1 + 31) / 32;
        const size_t dsm = 2 * sizeof(cx<RT>) * (size_t)n;
        int per_sm = 0, dev = 0, sms = 0, coop = 0;
        LG_CUDA_TRY(cudaGetDevice(&dev));
        LG_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        LG_CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
        if (dsm > 48 * 1024)
            LG_TRY(allow_max_dyn_smem((const void *)k_tri_coop<RT>));
        LG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tri_coop<RT>, 256, dsm));
        const int G = std::min(tl0 * tl0, sms * std::max(per_sm, 0));
        int *err = device_wait_flag();
        if (coop && G >= 1 && err) {
            unsigned int *bar = cnt;            // arrival counter (zeroed above)
            void *args[] = {(void *)&n, (void *)&A, (void *)&lda, (void *)&Hv, (void *)&taus, (void *)&dg, (void *)&eg,
                            (void *)&yp, (void *)&bar, (void *)&err};
            if (w.gate) {
                std::lock_guard<std::mutex> lk(w.gate->mu);
                if (w.gate->used) LG_CUDA_TRY(cudaStreamWaitEvent(s, w.gate->ev, 0));
                LG_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)k_tri_coop<RT>, dim3(G), dim3(256), args, dsm, s));
                LG_CUDA_TRY(cudaEventRecord(w.gate->ev, s));
                w.gate->used = true;
            } else {
                LG_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)k_tri_coop<RT>, dim3(G), dim3(256), args, dsm, s));
            }
            LG_TRY(check_launch("tridiagonalisation (cooperative)"));
            coop_done = true;
        }
    }
    if (!coop_done) {
        for (int i = 0; i + 1 < n; ++i) {
            const int L = n - i - 1;
            const int tl = (L + 31) / 32;
            k_tri_step1<RT><<<dim3(tl, tl), 256, 0, s>>>(n, i, A, lda, Hv, taus, dg, eg, yp, wv, cnt);
            LG_TRY(check_launch("tridiag step 1"));
            k_tri_step2<RT><<<dim3(tl, tl), 256, 0, s>>>(n, i, A, lda, Hv, wv);
            LG_TRY(check_launch("tridiag step 2"));
        }
        k_tri_last<RT><<<1, 32, 0, s>>>(n, A, lda, dg);
        LG_TRY(check_launch("tridiag last"));
    }
    bool ms_done = false;
    if constexpr (std::is_same<RT, double>::value) {
        if (w.df) {  // FP64-class path: the fine rounds in double-FP32
            const size_t smem_ms = 24 * (size_t)n;
            if (smem_ms > 48 * 1024) LG_TRY(allow_max_dyn_smem((const void *)k_multisect_df));
            k_multisect_df<<<m, kMsLanes, smem_ms, s>>>(n, m, dg, eg, theta);
            LG_TRY(check_launch("multisection (double-FP32)"));
            ms_done = true;
        }
    }
    if (!ms_done) {
        k_multisect<RT><<<m, kMsLanes, 0, s>>>(n, m, dg, eg, theta);
        LG_TRY(check_launch("multisection"));
    }
    const size_t smem_ii = 6 * sizeof(RT) * (size_t)n + (size_t)n;
    if (smem_ii > 48 * 1024)
        LG_TRY(allow_max_dyn_smem((const void *)k_inviter<RT>));
    k_inviter<RT><<<m, 32, smem_ii, s>>>(n, m, dg, eg, theta, Z);
    LG_TRY(check_launch("inverse iteration"));
    if (n == 1) {
        LG_CUDA_TRY(cudaMemcpy2DAsync(V, sizeof(cx<RT>) * ldv, Z, sizeof(RT), sizeof(RT), m, cudaMemcpyDeviceToDevice, s));
        LG_CUDA_TRY(cudaMemset2DAsync(reinterpret_cast<char *>(V) + sizeof(RT), sizeof(cx<RT>) * ldv, 0, sizeof(RT), m, s));
        return check_launch("back-transform (n = 1)");
    }
    if constexpr (sizeof(cx<RT>) == sizeof(cx<df64>)) {
        if (hv_df)
            return backtransform_wy<RT, df64>(n, m, reinterpret_cast<const cx<df64> *>(Hv),
                                              reinterpret_cast<const cx<df64> *>(taus),
                                              reinterpret_cast<cx<df64> *>(Tf), reinterpret_cast<cx<df64> *>(Gp), Z,
                                              V, ldv, s);
    }
    return backtransform_wy<RT, RT>(n, m, Hv, taus, Tf, Gp, Z, V, ldv, s);
}

template <typename RT>
int hermitize_lower_t(EigWork &w, int n, cx<RT> *A, cudaStream_t s) {
    LG_TRY(w.alloc->ensure(w.ibuf, sizeof(RT) * (size_t)n + 256));
    k_hermitize_rowsum<RT><<<n, 128, 0, s>>>(n, A, nullptr, reinterpret_cast<RT *>(w.ibuf.p));
    return check_launch("hermitize");
}

template <typename RT>
int rayleigh_ritz_t(EigWork &w, int n, int m, const cx<RT> *S, int lds, const cx<RT> *A, int lda, double drop_tol,
                    RT *theta, cx<RT> *C, int ldc, int *ndropped, cudaStream_t s, int lead = 0) {
    if (n <= 0 || m <= 0) return LOBPCG_OK;
    if (m > n) return fail(LOBPCG_ERR_ARG, "rayleigh_ritz: m > n");
    if (n > 4096) return fail(LOBPCG_ERR_ARG, "rayleigh_ritz: n > 4096");
    // own workspace (separate from heev's)
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes); return o; };
    const size_t o_ss = take(sizeof(cx<RT>) * (size_t)n * n);
    const size_t o_as = take(sizeof(cx<RT>) * (size_t)n * n);
    const size_t o_li = take(sizeof(cx<RT>) * (size_t)n * n);
    const size_t o_tm = take(sizeof(cx<RT>) * (size_t)n * n);
    const size_t o_q = take(sizeof(cx<RT>) * (size_t)n * m);
    const size_t o_d = take(sizeof(RT) * n);
    const size_t o_rs = take(sizeof(RT) * n);
    const size_t o_dr = take(sizeof(int) * n);
    const size_t o_nd = take(sizeof(int));
    LG_TRY(w.alloc->ensure(w.ibuf, off));
    char *base = reinterpret_cast<char *>(w.ibuf.p);
    cx<RT> *Ss = reinterpret_cast<cx<RT> *>(base + o_ss);
    cx<RT> *As = reinterpret_cast<cx<RT> *>(base + o_as);
    cx<RT> *Li = reinterpret_cast<cx<RT> *>(base + o_li);
    cx<RT> *Tm = reinterpret_cast<cx<RT> *>(base + o_tm);
    cx<RT> *Q = reinterpret_cast<cx<RT> *>(base + o_q);
    RT *d = reinterpret_cast<RT *>(base + o_d);
    RT *rs = reinterpret_cast<RT *>(base + o_rs);
    int *dr = reinterpret_cast<int *>(base + o_dr);
    int *nd = reinterpret_cast<int *>(base + o_nd);

    w.gw.df = std::is_same<RT, double>::value && w.df;  // the small products below
    LG_CUDA_TRY(cudaMemsetAsync(nd, 0, sizeof(int), s));
    LG_CUDA_TRY(cudaMemsetAsync(Li, 0, sizeof(cx<RT>) * (size_t)n * n, s));
    k_scale_gram<RT><<<dim3((n + 127) / 128, n), 128, 0, s>>>(n, S, lds, A, lda, Ss, As, d);
    LG_TRY(check_launch("scale gram"));
    if (lead % NBK != 0 || lead > n || lead < 0) lead = 0;
    if (lead > 0) {
        k_lead_identity<RT><<<dim3((n + 127) / 128, lead), 128, 0, s>>>(n, lead, Ss, Li, dr);
        LG_TRY(check_launch("leading identity"));
    }
    // blocked Cholesky with dropping (L overwrites Ss), after the leading identity columns
    for (int k0 = lead; k0 < n; k0 += NBK) {
        const int kb = std::min(NBK, n - k0);
        bool chol_done = false;
        if constexpr (std::is_same<RT, double>::value) {
            if (w.df) {  // one block: double-FP32 instead of that SM's FP64 units
                k_chol_diag<RT, df64><<<1, 256, 0, s>>>(n, k0, kb, Ss, Li, (RT)drop_tol, dr, nd);
                chol_done = true;
            }
        }
        if (!chol_done) k_chol_diag<RT><<<1, 256, 0, s>>>(n, k0, kb, Ss, Li, (RT)drop_tol, dr, nd);
        LG_TRY(check_launch("cholesky diag"));
        const int rem = n - k0 - kb;
        if (rem > 0) {
            k_chol_panel<RT><<<(rem + 7) / 8, 256, 0, s>>>(n, k0, kb, Ss, Li, dr);
            LG_TRY(check_launch("cholesky panel"));
            const cx<RT> *L21 = Ss + (size_t)k0 * n + k0 + kb;
            cx<RT> *S22 = Ss + (size_t)(k0 + kb) * n + k0 + kb;
            LG_TRY(gemm_small<RT>(&w.gw, 'N', 'C', rem, rem, kb, -1.0, L21, n, L21, n, 1.0, S22, n, s));
        }
    }
    k_zero_dropped_rows<RT><<<n, 128, 0, s>>>(n, Ss, dr);
    LG_TRY(check_launch("zero dropped rows"));
    // off-diagonal blocks of L^-1, block row by block row
    for (int r0 = NBK; r0 < n; r0 += NBK) {
        const int kb = std::min(NBK, n - r0);
        // Tm(kb x r0) = L[r0:r0+kb, 0:r0] * Li[0:r0, 0:r0]
        LG_TRY(gemm_small<RT>(&w.gw, 'N', 'N', kb, r0, r0, 1.0, Ss + r0, n, Li, n, 0.0, Tm, n, s));
        // Li[r0:r0+kb, 0:r0] = -Li_rr * Tm
        LG_TRY(gemm_small<RT>(&w.gw, 'N', 'N', kb, r0, kb, -1.0, Li + (size_t)r0 * n + r0, n, Tm, n, 0.0, Li + r0, n, s));
    }
    // Ahat = Li As Li^H
    LG_TRY(gemm_small<RT>(&w.gw, 'N', 'N', n, n, n, 1.0, Li, n, As, n, 0.0, Tm, n, s));
    LG_TRY(gemm_small<RT>(&w.gw, 'N', 'C', n, n, n, 1.0, Tm, n, Li, n, 0.0, As, n, s));
    k_hermitize_rowsum<RT><<<n, 128, 0, s>>>(n, As, dr, rs);
    LG_TRY(check_launch("hermitize"));
    k_set_dropped_diag<RT><<<1, 1024, 0, s>>>(n, As, dr, nd, rs);
    LG_TRY(check_launch("dropped diag"));
    LG_TRY(heev_lowest_t<RT>(w, n, m, As, n, theta, Q, n, s));
    // C = D Li^H Q
    LG_TRY(gemm_small<RT>(&w.gw, 'C', 'N', n, m, n, 1.0, Li, n, Q, n, 0.0, Tm, n, s));
    k_scale_rows_copy<RT><<<dim3((n + 127) / 128, m), 128, 0, s>>>(n, m, d, Tm, n, C, ldc);
    LG_TRY(check_launch("scale C"));
    if (ndropped) {
        k_copy_int<<<1, 1, 0, s>>>(nd, ndropped);
        LG_TRY(check_launch("copy ndropped"));
    }
    return LOBPCG_OK;
}

int heev_lowest(EigWork &w, int n, int m, z64 *A, int lda, double *theta, z64 *V, int ldv, cudaStream_t s) {
    return heev_lowest_t<double>(w, n, m, A, lda, theta, V, ldv, s);
}
int hermitize_lower(EigWork &w, int n, z64 *A, cudaStream_t s) { return hermitize_lower_t<double>(w, n, A, s); }
int rayleigh_ritz(EigWork &w, int n, int m, const z64 *S, int lds, const z64 *A, int lda, double drop_tol,
                  double *theta, z64 *C, int ldc, int *ndropped, cudaStream_t s, int lead) {
    return rayleigh_ritz_t<double>(w, n, m, S, lds, A, lda, drop_tol, theta, C, ldc, ndropped, s, lead);
}
int rayleigh_ritz32(EigWork &w, int n, int m, const c32 *S, int lds, const c32 *A, int lda, double drop_tol,
                    float *theta, c32 *C, int ldc, int *ndropped, cudaStream_t s) {
    return rayleigh_ritz_t<float>(w, n, m, S, lds, A, lda, drop_tol, theta, C, ldc, ndropped, s);
}

}  // namespace lg
