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
//      back-transformation by the reflectors;
//   5. C = D L^-H Q.
// Every step runs on the GPU in FP64; no host synchronisation.
#include "common.cuh"

#include <algorithm>
#include <cfloat>

namespace lg {

namespace {

constexpr int NBK = 32;  // Cholesky / inverse block size

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Deterministic block sum (blockDim.x multiple of 32, <= 1024). Result on all threads.
__device__ double block_sum(double v, double *sh) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double t = 0.0;
    for (int i = 0; i < nw; ++i) t += sh[i];
    return t;
}

// ------------------------------------------------------------------ scaling
__global__ void k_scale_gram(int n, const z64 *__restrict__ S, int lds, const z64 *__restrict__ A, int lda,
                             z64 *__restrict__ Ss, z64 *__restrict__ As, double *__restrict__ d) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= n) return;
    const double si = S[(size_t)i * lds + i].x, sj = S[(size_t)j * lds + j].x;
    const double di = si > 0.0 ? 1.0 / sqrt(si) : 0.0;
    const double dj = sj > 0.0 ? 1.0 / sqrt(sj) : 0.0;
    if (j == 0) d[i] = di;
    z64 s, a;
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
__global__ void __launch_bounds__(256)
k_chol_diag(int n, int k0, int kb, z64 *__restrict__ L, z64 *__restrict__ Linv, double drop_tol,
            int *__restrict__ dropped, int *__restrict__ ndrop) {
    __shared__ z64 T[NBK][NBK + 1];
    __shared__ z64 I[NBK][NBK + 1];
    __shared__ int dflag[NBK];
    const int tid = threadIdx.x;
    for (int e = tid; e < NBK * NBK; e += blockDim.x) {
        const int r = e % NBK, c = e / NBK;
        z64 v = mkc(0.0, 0.0);
        if (r < kb && c < kb && r >= c) v = L[(size_t)(k0 + c) * n + k0 + r];
        T[r][c] = v;
        I[r][c] = mkc(0.0, 0.0);
    }
    __syncthreads();
    for (int j = 0; j < kb; ++j) {
        const double p = T[j][j].x;
        const bool drop = !(p > drop_tol);
        __syncthreads();
        if (drop) {
            for (int r = j + 1 + tid; r < kb; r += blockDim.x) T[r][j] = mkc(0.0, 0.0);
            if (tid == 0) { T[j][j] = mkc(1.0, 0.0); dflag[j] = 1; }
        } else {
            const double rt = sqrt(p), inv = 1.0 / rt;
            for (int r = j + 1 + tid; r < kb; r += blockDim.x) T[r][j] = inv * T[r][j];
            if (tid == 0) { T[j][j] = mkc(rt, 0.0); dflag[j] = 0; }
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
        if (c < r && dflag[r]) T[r][c] = mkc(0.0, 0.0);
    }
    __syncthreads();
    // inverse of the lower-triangular block, one column per thread
    if (tid < kb) {
        const int c = tid;
        I[c][c] = mkc(1.0 / T[c][c].x, 0.0);  // real positive diagonal
        for (int r = c + 1; r < kb; ++r) {
            z64 s = mkc(0.0, 0.0);
            for (int l = c; l < r; ++l) s = s + T[r][l] * I[l][c];
            I[r][c] = (-1.0 / T[r][r].x) * s;
        }
    }
    __syncthreads();
    for (int e = tid; e < kb * kb; e += blockDim.x) {
        const int r = e % kb, c = e / kb;
        L[(size_t)(k0 + c) * n + k0 + r] = (r >= c) ? T[r][c] : mkc(0.0, 0.0);
        Linv[(size_t)(k0 + c) * n + k0 + r] = (r >= c) ? I[r][c] : mkc(0.0, 0.0);
    }
    if (tid < kb) {
        dropped[k0 + tid] = dflag[tid];
        if (dflag[tid]) atomicAdd(ndrop, 1);
    }
}

// Panel: L21 = S21 Linv_kk^H for rows k0+kb..n-1 (8 rows per block, 32 columns).
__global__ void __launch_bounds__(256)
k_chol_panel(int n, int k0, int kb, z64 *__restrict__ L, const z64 *__restrict__ Linv,
             const int *__restrict__ dropped) {
    __shared__ z64 Di[NBK][NBK + 1];
    __shared__ z64 Srow[8][NBK + 1];
    const int tid = threadIdx.x;
    for (int e = tid; e < NBK * NBK; e += blockDim.x) {
        const int r = e % NBK, c = e / NBK;
        Di[r][c] = (r < kb && c < kb) ? Linv[(size_t)(k0 + c) * n + k0 + r] : mkc(0.0, 0.0);
    }
    const int rl = tid / NBK, c = tid % NBK;
    const int row = k0 + kb + blockIdx.x * 8 + rl;
    if (row < n && c < kb) Srow[rl][c] = L[(size_t)(k0 + c) * n + row];
    __syncthreads();
    if (row < n && c < kb) {
        z64 s = mkc(0.0, 0.0);
        for (int l = 0; l <= c; ++l) s = s + mul_conj(Srow[rl][l], Di[c][l]);
        if (dropped[k0 + c]) s = mkc(0.0, 0.0);
        L[(size_t)(k0 + c) * n + row] = s;
    }
}

__global__ void k_zero_dropped_rows(int n, z64 *__restrict__ L, const int *__restrict__ dropped) {
    const int j = blockIdx.x;
    if (!dropped[j]) return;
    for (int c = threadIdx.x; c < j; c += blockDim.x) L[(size_t)c * n + j] = mkc(0.0, 0.0);
}

// ------------------------------------------------------------------ hermitize / dropped rows
__global__ void k_hermitize_rowsum(int n, z64 *__restrict__ A, const int *__restrict__ dropped,
                                   double *__restrict__ rowsum) {
    const int i = blockIdx.x;
    __shared__ double sh[32];
    double s = 0.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        z64 v = (i >= j) ? A[(size_t)j * n + i] : conjc(A[(size_t)i * n + j]);
        if (i == j) v.y = 0.0;
        if (dropped && (dropped[i] || dropped[j])) v = mkc(0.0, 0.0);
        s += sqrt(abs2(v));
        if (i >= j) {
            A[(size_t)j * n + i] = v;
            A[(size_t)i * n + j] = conjc(v);
        }
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) rowsum[i] = s;
}

__global__ void k_set_dropped_diag(int n, z64 *__restrict__ A, const int *__restrict__ dropped,
                                   const int *__restrict__ ndrop, const double *__restrict__ rowsum) {
    if (*ndrop == 0) return;
    __shared__ double sh[32];
    double mx = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) mx = fmax(mx, rowsum[i]);
    // deterministic max via shuffles
#pragma unroll
    for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = mx;
    __syncthreads();
    double m2 = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m2 = fmax(m2, sh[w]);
    const double sigma = 2.0 * m2 + 1.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        if (dropped[i]) A[(size_t)i * n + i] = mkc(sigma, 0.0);
}

// ------------------------------------------------------------------ tridiagonalisation
// Reflector of x = A[i+1:n, i] in the LAPACK larfg convention:
//   H = I - tau v v^H, v[0] = 1, H^H x = beta e_1 with beta real.
struct Refl {
    z64 tau;
    double beta;
    z64 scal;  // v[r] = x[r] * scal for r >= 1
};

__device__ Refl make_reflector(const z64 *__restrict__ col, int L, double *sh) {
    double s = 0.0;
    for (int r = 1 + threadIdx.x; r < L; r += blockDim.x) s += abs2(col[r]);
    s = block_sum(s, sh);
    const z64 alpha = col[0];
    Refl R;
    if (s == 0.0 && alpha.y == 0.0) {
        R.tau = mkc(0.0, 0.0);
        R.beta = alpha.x;
        R.scal = mkc(0.0, 0.0);
        return R;
    }
    const double beta = -copysign(sqrt(abs2(alpha) + s), alpha.x);
    R.beta = beta;
    R.tau = mkc((beta - alpha.x) / beta, -alpha.y / beta);
    const z64 den = mkc(alpha.x - beta, alpha.y);
    const double dd = abs2(den);
    R.scal = mkc(den.x / dd, -den.y / dd);
    return R;
}

// Step i, part 1: reflector (every block, redundantly) and y = A22 v by 32x32 tiles;
// the last block to finish forms w = tau y - |tau|^2/2 (v^H y) v.
__global__ void __launch_bounds__(256)
k_tri_step1(int n, int i, z64 *__restrict__ A, int lda, z64 *__restrict__ Hv, z64 *__restrict__ taus,
            double *__restrict__ dg, double *__restrict__ eg, z64 *__restrict__ ypart, z64 *__restrict__ wv,
            unsigned int *__restrict__ counter) {
    __shared__ double sh[32];
    __shared__ z64 vs[32];
    __shared__ z64 acc[8][33];
    __shared__ bool last;
    const int L = n - i - 1;
    const z64 *col = A + (size_t)i * lda + i + 1;
    const Refl R = make_reflector(col, L, sh);
    const int tr = blockIdx.x, tc = blockIdx.y;
    const int tid = threadIdx.x;
    if (tr == 0 && tc == 0) {
        for (int r = tid; r < L; r += blockDim.x) Hv[(size_t)i * n + i + 1 + r] = (r == 0) ? mkc(1.0, 0.0) : col[r] * R.scal;
        if (tid == 0) {
            taus[i] = R.tau;
            dg[i] = A[(size_t)i * lda + i].x;
            eg[i] = R.beta;
        }
    }
    // v entries of this column tile
    if (tid < 32) {
        const int c = tc * 32 + tid;
        vs[tid] = (c < L) ? ((c == 0) ? mkc(1.0, 0.0) : col[c] * R.scal) : mkc(0.0, 0.0);
    }
    __syncthreads();
    const int rl = tid & 31, cg = tid >> 5;  // 32 rows x 8 column groups of 4
    const int r = tr * 32 + rl;
    z64 s = mkc(0.0, 0.0);
    if (r < L) {
        const z64 *A22 = A + (size_t)(i + 1) * lda + i + 1;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int cl = cg * 4 + q, c = tc * 32 + cl;
            if (c < L) s = s + A22[(size_t)c * lda + r] * vs[cl];
        }
    }
    acc[cg][rl] = s;
    __syncthreads();
    if (tid < 32) {
        z64 t = acc[0][tid];
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
    double dre = 0.0, dim = 0.0;
    for (int rr = tid; rr < L; rr += blockDim.x) {
        z64 y = mkc(0.0, 0.0);
        for (int c = 0; c < ncb; ++c) {
            const double2 t = __ldcg(reinterpret_cast<const double2 *>(ypart + (size_t)c * n + rr));
            y = y + mkc(t.x, t.y);
        }
        const z64 v = (rr == 0) ? mkc(1.0, 0.0) : col[rr] * R.scal;
        // conj(v) * y
        dre += v.x * y.x + v.y * y.y;
        dim += v.x * y.y - v.y * y.x;
        wv[rr] = y;  // stash y, scaled below
    }
    dre = block_sum(dre, sh);
    (void)dim;  // v^H A v is real for Hermitian A
    const double t2 = 0.5 * abs2(R.tau) * dre;
    __syncthreads();
    for (int rr = tid; rr < L; rr += blockDim.x) {
        const z64 v = (rr == 0) ? mkc(1.0, 0.0) : col[rr] * R.scal;
        const z64 y = wv[rr];
        wv[rr] = R.tau * y - t2 * v;
    }
}

// Step i, part 2: A22 -= w v^H + v w^H on 32x32 tiles.
__global__ void __launch_bounds__(256)
k_tri_step2(int n, int i, z64 *__restrict__ A, int lda, const z64 *__restrict__ Hv, const z64 *__restrict__ wv) {
    __shared__ z64 vr[32], wr[32], vc[32], wc[32];
    const int L = n - i - 1;
    const int tr = blockIdx.x, tc = blockIdx.y, tid = threadIdx.x;
    const z64 *v = Hv + (size_t)i * n + i + 1;
    if (tid < 32) {
        const int r = tr * 32 + tid, c = tc * 32 + tid;
        vr[tid] = r < L ? v[r] : mkc(0.0, 0.0);
        wr[tid] = r < L ? wv[r] : mkc(0.0, 0.0);
        vc[tid] = c < L ? v[c] : mkc(0.0, 0.0);
        wc[tid] = c < L ? wv[c] : mkc(0.0, 0.0);
    }
    __syncthreads();
    z64 *A22 = A + (size_t)(i + 1) * lda + i + 1;
    for (int e = tid; e < 32 * 32; e += blockDim.x) {
        const int rl = e & 31, cl = e >> 5;
        const int r = tr * 32 + rl, c = tc * 32 + cl;
        if (r < L && c < L) {
            z64 a = A22[(size_t)c * lda + r];
            a = a - mul_conj(wr[rl], vc[cl]) - mul_conj(vr[rl], wc[cl]);
            A22[(size_t)c * lda + r] = a;
        }
    }
}

__global__ void k_tri_last(int n, const z64 *__restrict__ A, int lda, double *__restrict__ dg) {
    if (threadIdx.x == 0) dg[n - 1] = A[(size_t)(n - 1) * lda + n - 1].x;
}

// ------------------------------------------------------------------ eigenvalues (multisection)
__device__ __forceinline__ int sturm_count(const double *__restrict__ d, const double *__restrict__ e, int n,
                                           double x, double pivmin) {
    int c = 0;
    double q = d[0] - x;
    if (fabs(q) < pivmin) q = -pivmin;
    c += (q < 0.0);
    for (int i = 1; i < n; ++i) {
        const double ei = e[i - 1];
        q = d[i] - x - (ei * ei) / q;
        if (fabs(q) < pivmin) q = -pivmin;
        c += (q < 0.0);
    }
    return c;
}

__device__ void tri_bounds(const double *__restrict__ d, const double *__restrict__ e, int n, double &lo,
                           double &hi, double &tnorm, double &pivmin) {
    lo = DBL_MAX;
    hi = -DBL_MAX;
    double emax2 = 0.0;
    for (int i = 0; i < n; ++i) {
        double r = 0.0;
        if (i > 0) r += fabs(e[i - 1]);
        if (i < n - 1) { r += fabs(e[i]); emax2 = fmax(emax2, e[i] * e[i]); }
        lo = fmin(lo, d[i] - r);
        hi = fmax(hi, d[i] + r);
    }
    tnorm = fmax(fabs(lo), fabs(hi));
    pivmin = DBL_MIN * fmax(1.0, emax2);
    const double pad = 2.0 * DBL_EPSILON * tnorm * n + 2.0 * pivmin;
    lo -= pad;
    hi += pad;
}

// Four lanes per eigenvalue index k < m (eight eigenvalues per warp): each round
// the group evaluates 4 Sturm counts inside the bracket and keeps the fifth of it
// that holds eigenvalue k.  FP64 divisions are scarce on this GPU, so few lanes per
// eigenvalue (less total work) beat wide multisection (fewer rounds).
constexpr int kMsG = 4;
__global__ void k_multisect(int n, int m, const double *__restrict__ d, const double *__restrict__ e,
                            double *__restrict__ theta) {
    const int gid = (int)((blockIdx.x * blockDim.x + threadIdx.x) / kMsG);
    const int sub = threadIdx.x & (kMsG - 1);
    const int lane = threadIdx.x & 31;
    const int base = lane & ~(kMsG - 1);
    const bool active = gid < m;
    const int k = active ? gid : m - 1;
    double lo, hi, tnorm, pivmin;
    tri_bounds(d, e, n, lo, hi, tnorm, pivmin);
    for (int it = 0; it < 48; ++it) {
        const double w = hi - lo;
        const bool done = w <= 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)) + 4.0 * pivmin;
        if (__all_sync(0xffffffffu, done)) break;
        const double x = lo + w * (double)(sub + 1) / (double)(kMsG + 1);
        const int c = done ? 0 : sturm_count(d, e, n, x, pivmin);
        const unsigned mask = __ballot_sync(0xffffffffu, c <= k);
        const int T = __popc((mask >> base) & ((1u << kMsG) - 1u)) - 1;  // counts are monotone in sub
        const double xlo = __shfl_sync(0xffffffffu, x, base + (T < 0 ? 0 : T));
        const double xhi = __shfl_sync(0xffffffffu, x, base + (T < kMsG - 1 ? T + 1 : kMsG - 1));
        if (!done) {
            if (T >= 0) lo = xlo;
            if (T < kMsG - 1) hi = xhi;
        }
    }
    if (active && sub == 0) theta[k] = 0.5 * (lo + hi);
}

// ------------------------------------------------------------------ eigenvectors (inverse iteration)
__device__ __forceinline__ double hash_uniform(unsigned int a, unsigned int b) {
    unsigned int h = a * 0x9E3779B1u ^ (b + 0x7F4A7C15u) * 0x85EBCA77u;
    h ^= h >> 16; h *= 0x7FEB352Du; h ^= h >> 15; h *= 0x846CA68Bu; h ^= h >> 16;
    return (double)h * (2.0 / 4294967296.0) - 1.0;
}

// One thread per eigenvalue index; the thread whose eigenvalue starts a cluster
// of close eigenvalues computes all vectors of that cluster, in order, on its own
// (LU of T - lambda I with partial pivoting, three solves from a pseudo-random
// start, each followed by modified Gram-Schmidt against the cluster's earlier
// vectors and a normalisation).
__global__ void k_inviter(int n, int m, const double *__restrict__ d, const double *__restrict__ e,
                          const double *__restrict__ theta, double *Z, double *scratch, signed char *pivs) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= m) return;
    double lo, hi, tnorm, pivmin;
    tri_bounds(d, e, n, lo, hi, tnorm, pivmin);
    const double gaptol = 1e-5 * fmax(tnorm, DBL_MIN);
    const double pert = 10.0 * DBL_EPSILON * fmax(tnorm, DBL_MIN);
    if (k > 0 && theta[k] - theta[k - 1] <= gaptol) return;  // not a cluster start
    double lam_prev = -DBL_MAX;
    for (int j = k; j < m; ++j) {
        if (j > k && theta[j] - theta[j - 1] > gaptol) break;
        double lam = theta[j];
        if (j > k && lam < lam_prev + pert) lam = lam_prev + pert;
        lam_prev = lam;
        double *dd = scratch + (size_t)j * 5 * n;
        double *du = dd + n, *du2 = du + n, *dl = du2 + n;
        double *z = Z + (size_t)j * n;
        signed char *pv = pivs + (size_t)j * n;
        for (int i = 0; i < n; ++i) dd[i] = d[i] - lam;
        for (int i = 0; i + 1 < n; ++i) { du[i] = e[i]; dl[i] = e[i]; du2[i] = 0.0; }
        for (int i = 0; i + 1 < n; ++i) {
            if (fabs(dd[i]) >= fabs(dl[i])) {
                pv[i] = 0;
                if (dd[i] == 0.0) dd[i] = pert;
                const double f = dl[i] / dd[i];
                dl[i] = f;
                dd[i + 1] -= f * du[i];
            } else {
                pv[i] = 1;
                const double f = dd[i] / dl[i];
                dd[i] = dl[i];
                dl[i] = f;
                const double t = du[i];
                du[i] = dd[i + 1];
                dd[i + 1] = t - f * dd[i + 1];
                if (i + 2 < n) { du2[i] = du[i + 1]; du[i + 1] = -f * du[i + 1]; }
            }
        }
        if (dd[n - 1] == 0.0) dd[n - 1] = pert;
        for (int i = 0; i < n; ++i) z[i] = hash_uniform((unsigned)j, (unsigned)i);
        for (int it = 0; it < 3; ++it) {
            for (int i = 0; i + 1 < n; ++i) {
                if (pv[i] == 0) {
                    z[i + 1] -= dl[i] * z[i];
                } else {
                    const double t = z[i];
                    z[i] = z[i + 1];
                    z[i + 1] = t - dl[i] * z[i];
                }
            }
            z[n - 1] = z[n - 1] / dd[n - 1];
            if (n > 1) z[n - 2] = (z[n - 2] - du[n - 2] * z[n - 1]) / dd[n - 2];
            for (int i = n - 3; i >= 0; --i) z[i] = (z[i] - du[i] * z[i + 1] - du2[i] * z[i + 2]) / dd[i];
            for (int p = k; p < j; ++p) {
                const double *zp = Z + (size_t)p * n;
                double s = 0.0;
                for (int i = 0; i < n; ++i) s += z[i] * zp[i];
                for (int i = 0; i < n; ++i) z[i] -= s * zp[i];
            }
            double nr = 0.0;
            for (int i = 0; i < n; ++i) nr += z[i] * z[i];
            const double inv = nr > 0.0 ? 1.0 / sqrt(nr) : 0.0;
            for (int i = 0; i < n; ++i) z[i] *= inv;
        }
    }
}

// ------------------------------------------------------------------ back-transformation
// V[:, j] = H_0 H_1 ... H_{n-2} z_j (complex), one block per eigenvector.
__global__ void __launch_bounds__(256)
k_backtransform(int n, int m, const z64 *__restrict__ Hv, const z64 *__restrict__ taus, const double *__restrict__ Z,
                z64 *__restrict__ V, int ldv) {
    extern __shared__ __align__(16) unsigned char smraw[];
    z64 *z = reinterpret_cast<z64 *>(smraw);
    __shared__ double sh[32], sh2[32];
    const int j = blockIdx.x;
    for (int r = threadIdx.x; r < n; r += blockDim.x) z[r] = mkc(Z[(size_t)j * n + r], 0.0);
    __syncthreads();
    for (int i = n - 2; i >= 0; --i) {
        const z64 tau = taus[i];
        if (tau.x == 0.0 && tau.y == 0.0) continue;
        const int L = n - i - 1;
        const z64 *v = Hv + (size_t)i * n + i + 1;
        double sre = 0.0, sim = 0.0;
        for (int r = threadIdx.x; r < L; r += blockDim.x) {
            const z64 a = v[r], b = z[i + 1 + r];
            sre += a.x * b.x + a.y * b.y;
            sim += a.x * b.y - a.y * b.x;
        }
        sre = block_sum(sre, sh);
        sim = block_sum(sim, sh2);
        const z64 ts = tau * mkc(sre, sim);
        for (int r = threadIdx.x; r < L; r += blockDim.x) z[i + 1 + r] = z[i + 1 + r] - ts * v[r];
        __syncthreads();
    }
    for (int r = threadIdx.x; r < n; r += blockDim.x) V[(size_t)j * ldv + r] = z[r];
}

__global__ void k_scale_rows_copy(int n, int m, const double *__restrict__ d, const z64 *__restrict__ T, int ldt,
                                  z64 *__restrict__ C, int ldc) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (i < n) C[(size_t)j * ldc + i] = d[i] * T[(size_t)j * ldt + i];
}

__global__ void k_copy_int(const int *__restrict__ a, int *__restrict__ b) { *b = *a; }

size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

int heev_lowest(EigWork &w, int n, int m, z64 *A, int lda, double *theta, z64 *V, int ldv, cudaStream_t s) {
    if (n <= 0 || m <= 0) return LOBPCG_OK;
    if (m > n) return fail(LOBPCG_ERR_ARG, "heev: m > n");
    const int nt = (n + 31) / 32;
    // workspace carve-up
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes); return o; };
    const size_t o_hv = take(sizeof(z64) * (size_t)n * n);
    const size_t o_tau = take(sizeof(z64) * n);
    const size_t o_d = take(sizeof(double) * n);
    const size_t o_e = take(sizeof(double) * n);
    const size_t o_yp = take(sizeof(z64) * (size_t)nt * n);
    const size_t o_wv = take(sizeof(z64) * n);
    const size_t o_z = take(sizeof(double) * (size_t)n * m);
    const size_t o_sc = take(sizeof(double) * 5 * (size_t)n * m);
    const size_t o_pv = take((size_t)n * m);
    const size_t o_cnt = take(sizeof(unsigned int) * n);
    LG_TRY(w.alloc->ensure(w.buf, off));
    char *base = reinterpret_cast<char *>(w.buf.p);
    z64 *Hv = reinterpret_cast<z64 *>(base + o_hv);
    z64 *taus = reinterpret_cast<z64 *>(base + o_tau);
    double *dg = reinterpret_cast<double *>(base + o_d);
    double *eg = reinterpret_cast<double *>(base + o_e);
    z64 *yp = reinterpret_cast<z64 *>(base + o_yp);
    z64 *wv = reinterpret_cast<z64 *>(base + o_wv);
    double *Z = reinterpret_cast<double *>(base + o_z);
    double *sc = reinterpret_cast<double *>(base + o_sc);
    signed char *pv = reinterpret_cast<signed char *>(base + o_pv);
    unsigned int *cnt = reinterpret_cast<unsigned int *>(base + o_cnt);
    LG_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(unsigned int) * n, s));
    LG_CUDA_TRY(cudaMemsetAsync(taus, 0, sizeof(z64) * n, s));
    for (int i = 0; i + 1 < n; ++i) {
        const int L = n - i - 1;
        const int tl = (L + 31) / 32;
        k_tri_step1<<<dim3(tl, tl), 256, 0, s>>>(n, i, A, lda, Hv, taus, dg, eg, yp, wv, cnt);
        LG_TRY(check_launch("tridiag step 1"));
        k_tri_step2<<<dim3(tl, tl), 256, 0, s>>>(n, i, A, lda, Hv, wv);
        LG_TRY(check_launch("tridiag step 2"));
    }
    k_tri_last<<<1, 32, 0, s>>>(n, A, lda, dg);
    LG_TRY(check_launch("tridiag last"));
    k_multisect<<<(m * kMsG + 255) / 256, 256, 0, s>>>(n, m, dg, eg, theta);
    LG_TRY(check_launch("multisection"));
    k_inviter<<<(m + 63) / 64, 64, 0, s>>>(n, m, dg, eg, theta, Z, sc, pv);
    LG_TRY(check_launch("inverse iteration"));
    const size_t smem = sizeof(z64) * (size_t)n;
    if (smem > 48 * 1024) {
        LG_CUDA_TRY(cudaFuncSetAttribute(k_backtransform, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    }
    k_backtransform<<<m, 256, smem, s>>>(n, m, Hv, taus, Z, V, ldv);
    return check_launch("back-transform");
}

int hermitize_lower(EigWork &w, int n, z64 *A, cudaStream_t s) {
    LG_TRY(w.alloc->ensure(w.ibuf, sizeof(double) * (size_t)n + 256));
    k_hermitize_rowsum<<<n, 128, 0, s>>>(n, A, nullptr, reinterpret_cast<double *>(w.ibuf.p));
    return check_launch("hermitize");
}

int rayleigh_ritz(EigWork &w, int n, int m, const z64 *S, int lds, const z64 *A, int lda, double drop_tol,
                  double *theta, z64 *C, int ldc, int *ndropped, cudaStream_t s) {
    if (n <= 0 || m <= 0) return LOBPCG_OK;
    if (m > n) return fail(LOBPCG_ERR_ARG, "rayleigh_ritz: m > n");
    if (n > 4096) return fail(LOBPCG_ERR_ARG, "rayleigh_ritz: n > 4096");
    // own workspace (separate from heev's)
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes); return o; };
    const size_t o_ss = take(sizeof(z64) * (size_t)n * n);
    const size_t o_as = take(sizeof(z64) * (size_t)n * n);
    const size_t o_li = take(sizeof(z64) * (size_t)n * n);
    const size_t o_tm = take(sizeof(z64) * (size_t)n * n);
    const size_t o_q = take(sizeof(z64) * (size_t)n * m);
    const size_t o_d = take(sizeof(double) * n);
    const size_t o_rs = take(sizeof(double) * n);
    const size_t o_dr = take(sizeof(int) * n);
    const size_t o_nd = take(sizeof(int));
    LG_TRY(w.alloc->ensure(w.ibuf, off));
    char *base = reinterpret_cast<char *>(w.ibuf.p);
    z64 *Ss = reinterpret_cast<z64 *>(base + o_ss);
    z64 *As = reinterpret_cast<z64 *>(base + o_as);
    z64 *Li = reinterpret_cast<z64 *>(base + o_li);
    z64 *Tm = reinterpret_cast<z64 *>(base + o_tm);
    z64 *Q = reinterpret_cast<z64 *>(base + o_q);
    double *d = reinterpret_cast<double *>(base + o_d);
    double *rs = reinterpret_cast<double *>(base + o_rs);
    int *dr = reinterpret_cast<int *>(base + o_dr);
    int *nd = reinterpret_cast<int *>(base + o_nd);

    LG_CUDA_TRY(cudaMemsetAsync(nd, 0, sizeof(int), s));
    LG_CUDA_TRY(cudaMemsetAsync(Li, 0, sizeof(z64) * (size_t)n * n, s));
    k_scale_gram<<<dim3((n + 127) / 128, n), 128, 0, s>>>(n, S, lds, A, lda, Ss, As, d);
    LG_TRY(check_launch("scale gram"));
    // blocked Cholesky with dropping (L overwrites Ss)
    for (int k0 = 0; k0 < n; k0 += NBK) {
        const int kb = std::min(NBK, n - k0);
        k_chol_diag<<<1, 256, 0, s>>>(n, k0, kb, Ss, Li, drop_tol, dr, nd);
        LG_TRY(check_launch("cholesky diag"));
        const int rem = n - k0 - kb;
        if (rem > 0) {
            k_chol_panel<<<(rem + 7) / 8, 256, 0, s>>>(n, k0, kb, Ss, Li, dr);
            LG_TRY(check_launch("cholesky panel"));
            const z64 *L21 = Ss + (size_t)k0 * n + k0 + kb;
            z64 *S22 = Ss + (size_t)(k0 + kb) * n + k0 + kb;
            LG_TRY(zgemm_small(&w.gw, 'N', 'C', rem, rem, kb, -1.0, L21, n, L21, n, 1.0, S22, n, s));
        }
    }
    k_zero_dropped_rows<<<n, 128, 0, s>>>(n, Ss, dr);
    LG_TRY(check_launch("zero dropped rows"));
    // off-diagonal blocks of L^-1, block row by block row
    for (int r0 = NBK; r0 < n; r0 += NBK) {
        const int kb = std::min(NBK, n - r0);
        // Tm(kb x r0) = L[r0:r0+kb, 0:r0] * Li[0:r0, 0:r0]
        LG_TRY(zgemm_small(&w.gw, 'N', 'N', kb, r0, r0, 1.0, Ss + r0, n, Li, n, 0.0, Tm, n, s));
        // Li[r0:r0+kb, 0:r0] = -Li_rr * Tm
        LG_TRY(zgemm_small(&w.gw, 'N', 'N', kb, r0, kb, -1.0, Li + (size_t)r0 * n + r0, n, Tm, n, 0.0, Li + r0, n, s));
    }
    // Ahat = Li As Li^H
    LG_TRY(zgemm_small(&w.gw, 'N', 'N', n, n, n, 1.0, Li, n, As, n, 0.0, Tm, n, s));
    LG_TRY(zgemm_small(&w.gw, 'N', 'C', n, n, n, 1.0, Tm, n, Li, n, 0.0, As, n, s));
    k_hermitize_rowsum<<<n, 128, 0, s>>>(n, As, dr, rs);
    LG_TRY(check_launch("hermitize"));
    k_set_dropped_diag<<<1, 1024, 0, s>>>(n, As, dr, nd, rs);
    LG_TRY(check_launch("dropped diag"));
    LG_TRY(heev_lowest(w, n, m, As, n, theta, Q, n, s));
    // C = D Li^H Q
    LG_TRY(zgemm_small(&w.gw, 'C', 'N', n, m, n, 1.0, Li, n, Q, n, 0.0, Tm, n, s));
    k_scale_rows_copy<<<dim3((n + 127) / 128, m), 128, 0, s>>>(n, m, d, Tm, n, C, ldc);
    LG_TRY(check_launch("scale C"));
    if (ndropped) {
        k_copy_int<<<1, 1, 0, s>>>(nd, ndropped);
        LG_TRY(check_launch("copy ndropped"));
    }
    return LOBPCG_OK;
}

}  // namespace lg
