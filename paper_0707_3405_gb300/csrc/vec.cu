// Per-column and elementwise kernels of Algorithm 1 (Bottin et al. 2007, Sec. 3.2):
//   step 2  R = H Psi - Psi Upsilon (O = I),
//   step 3  W = K(R) with the Teter-Payne-Allan plane-wave preconditioner,
// the FP64 residual norms of the convergence test, precision casts and
// row scalings.
#include "common.cuh"

#include <cstring>

#include <algorithm>

namespace lg {

namespace {

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Two deterministic block sums at once (256 threads).
__device__ void block_sum2(double &a, double &b) {
    __shared__ double sa[8], sb[8];
    a = warp_sum_d(a);
    b = warp_sum_d(b);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) { sa[w] = a; sb[w] = b; }
    __syncthreads();
    double ta = 0.0, tb = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { ta += sa[i]; tb += sb[i]; }
    a = ta;
    b = tb;
}

// ------------------------------------------------------------------ per-column sums
// Two sums per column over the plane waves, split over chunks of rows so that the FP64 work of
// a few columns spreads over the whole GPU (one block per column would leave it to that block's
// SM, whose FP64 units are few); the chunk partials are added in a fixed order (reproducible).
enum ColOp { kEkin = 0, kRayleigh = 1, kDiag = 2, kResid = 3 };
constexpr int kMaxChunks = 32;

template <int OP>
__global__ void __launch_bounds__(256)
k_colsum2(int npw, int chunk, const z64 *__restrict__ X, int ldx, const z64 *__restrict__ HX, int ldhx,
          const double *__restrict__ kin, const double *__restrict__ theta, double *__restrict__ part) {
    const int c = blockIdx.x, j = blockIdx.y, nch = gridDim.x;
    const int g0 = c * chunk, g1 = min(npw, g0 + chunk);
    const z64 *x = X + (size_t)j * ldx;
    const z64 *h = (OP == kEkin) ? nullptr : HX + (size_t)j * ldhx;
    const double th = (OP == kResid) ? theta[j] : 0.0;
    double a = 0.0, b = 0.0;
    for (int g = g0 + threadIdx.x; g < g1; g += blockDim.x) {
        const z64 xv = x[g];
        const double xx = abs2(xv);
        if (OP == kEkin) {
            a += kin[g] * xx;
            b += xx;
        } else if (OP == kResid) {
            const z64 hv = h[g];
            const double p = hv.x - th * xv.x, q = hv.y - th * xv.y;
            a += p * p + q * q;
            b += xx;
        } else {
            const z64 hv = h[g];
            a += xx;
            b += xv.x * hv.x + xv.y * hv.y;
        }
    }
    block_sum2(a, b);
    if (threadIdx.x == 0) {
        part[((size_t)j * nch + c) * 2] = a;
        part[((size_t)j * nch + c) * 2 + 1] = b;
    }
}

template <int OP>
__global__ void k_colsum2_finish(int m, int nch, const double *__restrict__ part, double *__restrict__ out,
                                 z64 *__restrict__ S, z64 *__restrict__ A, int n) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    double a = 0.0, b = 0.0;
    for (int c = 0; c < nch; ++c) {
        a += part[((size_t)j * nch + c) * 2];
        b += part[((size_t)j * nch + c) * 2 + 1];
    }
    if (OP == kEkin) out[j] = b > 0.0 ? a / b : 1.0;
    else if (OP == kRayleigh) out[j] = a > 0.0 ? b / a : 0.0;
    else if (OP == kDiag) {
        S[(size_t)j * n + j] = mkc(a, 0.0);
        A[(size_t)j * n + j] = mkc(b, 0.0);
    } else out[j] = b > 0.0 ? sqrt(a / b) : 0.0;
}

// Chunks per column for m columns of npw rows: about four blocks per SM in all, at least 2048 rows
// per chunk.
int col_chunks(int npw, int m) {
    int nch = (4 * 152 + m - 1) / std::max(1, m);
    nch = std::min(nch, (npw + 2047) / 2048);
    return std::max(1, std::min(nch, kMaxChunks));
}

template <int OP>
int colsum2(int npw, int m, const z64 *X, int ldx, const z64 *HX, int ldhx, const double *kin, const double *theta,
            double *part, double *out, z64 *S, z64 *A, int n, cudaStream_t s) {
    const int nch = col_chunks(npw, m);
    const int chunk = (npw + nch - 1) / nch;
    k_colsum2<OP><<<dim3(nch, m), 256, 0, s>>>(npw, chunk, X, ldx, HX, ldhx, kin, theta, part);
    LG_TRY(check_launch("column sums"));
    k_colsum2_finish<OP><<<(m + 127) / 128, 128, 0, s>>>(m, nch, part, out, S, A, n);
    return check_launch("column sums (finish)");
}

// Kinetic energy of each band, Ekin_i = sum T |x|^2 / sum |x|^2 (one block per column).
__global__ void __launch_bounds__(256)
k_ekin(int npw, const z64 *__restrict__ X, int ldx, const double *__restrict__ kin, double *__restrict__ ekin) {
    const int j = blockIdx.x;
    const z64 *x = X + (size_t)j * ldx;
    double num = 0.0, den = 0.0;
    for (int g = threadIdx.x; g < npw; g += blockDim.x) {
        const double a = abs2(x[g]);
        num += kin[g] * a;
        den += a;
    }
    block_sum2(num, den);
    if (threadIdx.x == 0) ekin[j] = den > 0.0 ? num / den : 1.0;
}

// W = K(x) (HX - theta X),  x = T(q) / Ekin_i,
// K(x) = (27 + 18x + 12x^2 + 8x^3) / (27 + 18x + 12x^2 + 8x^3 + 16x^4)  (Teter, Payne, Allan 1989).
template <typename R>
__global__ void k_resid_precond(int npw, int m, const z64 *__restrict__ X, int ldx, const z64 *__restrict__ HX,
                                int ldhx, const double *__restrict__ theta, const double *__restrict__ kin,
                                const double *__restrict__ ekin, cx<R> *__restrict__ W, int ldw) {
    const int j = blockIdx.y;
    const double th = theta[j];
    const double ie = 1.0 / ekin[j];
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < npw; g += gridDim.x * blockDim.x) {
        const z64 x = X[(size_t)j * ldx + g], hx = HX[(size_t)j * ldhx + g];
        const double t = kin[g] * ie;
        const double p = 27.0 + t * (18.0 + t * (12.0 + 8.0 * t));
        const double t2 = t * t;
        const double k = p / (p + 16.0 * t2 * t2);
        const z64 r = mkc(hx.x - th * x.x, hx.y - th * x.y);
        W[(size_t)j * ldw + g] = mkc<R>((R)(k * r.x), (R)(k * r.y));
    }
}

// Mixed schedule: R = HX - theta X in FP64, stored in FP32 together with W = K(R).
__global__ void k_resid_precond_mixed(int npw, int m, const z64 *__restrict__ X, int ldx, const z64 *__restrict__ HX,
                                      int ldhx, const double *__restrict__ theta, const double *__restrict__ kin,
                                      const double *__restrict__ ekin, c32 *__restrict__ R, c32 *__restrict__ W,
                                      int ld) {
    const int j = blockIdx.y;
    const double th = theta[j];
    const double ie = 1.0 / ekin[j];
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < npw; g += gridDim.x * blockDim.x) {
        const z64 x = X[(size_t)j * ldx + g], hx = HX[(size_t)j * ldhx + g];
        const double t = kin[g] * ie;
        const double p = 27.0 + t * (18.0 + t * (12.0 + 8.0 * t));
        const double t2 = t * t;
        const double k = p / (p + 16.0 * t2 * t2);
        const double rx = hx.x - th * x.x, ry = hx.y - th * x.y;
        R[(size_t)j * ld + g] = mkc<float>((float)rx, (float)ry);
        W[(size_t)j * ld + g] = mkc<float>((float)(k * rx), (float)(k * ry));
    }
}

__global__ void k_axpy_cols(int rows, int cols, double alpha, const z64 *__restrict__ D, int ldd, z64 *__restrict__ V,
                            int ldv) {
    const size_t tot = (size_t)rows * cols;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % rows), j = (int)(e / rows);
        const z64 d = D[(size_t)j * ldd + i];
        z64 &v = V[(size_t)j * ldv + i];
        v = mkc(v.x + alpha * d.x, v.y + alpha * d.y);
    }
}

// Rayleigh quotients theta_j = Re(x_j^H (Hx)_j) / x_j^H x_j in FP64 (one block per column).
__global__ void __launch_bounds__(256)
k_rayleigh_quotients(int npw, const z64 *__restrict__ X, int ldx, const z64 *__restrict__ HX, int ldhx,
                     double *__restrict__ theta) {
    const int j = blockIdx.x;
    double xx = 0.0, xh = 0.0;
    for (int g = threadIdx.x; g < npw; g += blockDim.x) {
        const z64 x = X[(size_t)j * ldx + g], h = HX[(size_t)j * ldhx + g];
        xx += abs2(x);
        xh += x.x * h.x + x.y * h.y;
    }
    block_sum2(xx, xh);
    if (threadIdx.x == 0) theta[j] = xx > 0.0 ? xh / xx : 0.0;
}

// R = HX - X theta in FP64, stored in FP32.
__global__ void k_residual32(int npw, const z64 *__restrict__ X, int ldx, const z64 *__restrict__ HX, int ldhx,
                             const double *__restrict__ theta, c32 *__restrict__ R, int ldr) {
    const int j = blockIdx.y;
    const double th = theta[j];
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < npw; g += gridDim.x * blockDim.x) {
        const z64 x = X[(size_t)j * ldx + g], hx = HX[(size_t)j * ldhx + g];
        R[(size_t)j * ldr + g] = mkc<float>((float)(hx.x - th * x.x), (float)(hx.y - th * x.y));
    }
}

// W = K(R) (Teter-Payne-Allan, x = T(q)/Ekin_j) on FP32 columns.
__global__ void k_precond32(int npw, const c32 *__restrict__ R, int ldr, const double *__restrict__ kin,
                            const double *__restrict__ ekin, c32 *__restrict__ W, int ldw) {
    const int j = blockIdx.y;
    const double ie = 1.0 / ekin[j];
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < npw; g += gridDim.x * blockDim.x) {
        const double t = kin[g] * ie;
        const double p = 27.0 + t * (18.0 + t * (12.0 + 8.0 * t));
        const double t2 = t * t;
        const float k = (float)(p / (p + 16.0 * t2 * t2));
        const c32 r = R[(size_t)j * ldr + g];
        W[(size_t)j * ldw + g] = mkc<float>(k * r.x, k * r.y);
    }
}

// nz x nz pencil of the mixed schedule.
//   mx = 0: S = S32 (ld lds32), A = A32 (ld lda32), both full FP32 Grams.
//   mx > 0: the basis is [X W P] with X the orthonormal Ritz block (mx columns)
//     and [W P] projected out of span(X).  T1 = S32 = [R W P]^H [W P] (nz x nw,
//     ld lds32) and T2 = A32 = [W P]^H [HW HP] (nw x nw, ld lda32), nw = nz - mx:
//     S = [[I, 0], [0, T1[mx:, :]]],  A = [[diag(theta), T1[:mx, :]], [T1[:mx, :]^H, T2]].
template <typename Ro>
__global__ void k_assemble(int nz, int mx, const c32 *__restrict__ S32, int lds32, const c32 *__restrict__ A32,
                           int lda32, const double *__restrict__ theta, cx<Ro> *__restrict__ S,
                           cx<Ro> *__restrict__ A) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (i >= nz) return;
    z64 s, a;
    if (mx == 0) {
        s = cvt<double, float>(S32[(size_t)j * lds32 + i]);
        a = cvt<double, float>(A32[(size_t)j * lda32 + i]);
    } else if (i < mx && j < mx) {
        s = mkc(i == j ? 1.0 : 0.0, 0.0);
        a = mkc(i == j ? theta[i] : 0.0, 0.0);
    } else if (i >= mx && j >= mx) {
        if (i >= j) {
            s = cvt<double, float>(S32[(size_t)(j - mx) * lds32 + i]);
            a = cvt<double, float>(A32[(size_t)(j - mx) * lda32 + (i - mx)]);
        } else {
            s = conjc(cvt<double, float>(S32[(size_t)(i - mx) * lds32 + j]));
            a = conjc(cvt<double, float>(A32[(size_t)(i - mx) * lda32 + (j - mx)]));
        }
    } else if (j < mx) {  // i >= mx > j: conj(R_j^H Q_i)
        s = mkc(0.0, 0.0);
        a = conjc(cvt<double, float>(S32[(size_t)(i - mx) * lds32 + j]));
    } else {              // i < mx <= j: R_i^H Q_j
        s = mkc(0.0, 0.0);
        a = cvt<double, float>(S32[(size_t)(j - mx) * lds32 + i]);
    }
    S[(size_t)j * nz + i] = cvt<Ro, double>(s);
    A[(size_t)j * nz + i] = cvt<Ro, double>(a);
}

// FP64 diagonals of X^H X and X^H HX (one block per column) written onto the
// diagonals of the FP64 pencil S, A (ld n): exact Rayleigh quotients for the
// block-start Rayleigh-Ritz of the mixed schedule.
__global__ void __launch_bounds__(256)
k_diag_pencil(int npw, const z64 *__restrict__ X, int ldx, const z64 *__restrict__ HX, int ldhx, z64 *__restrict__ S,
              z64 *__restrict__ A, int n) {
    const int j = blockIdx.x;
    double xx = 0.0, xh = 0.0;
    for (int g = threadIdx.x; g < npw; g += blockDim.x) {
        const z64 x = X[(size_t)j * ldx + g], h = HX[(size_t)j * ldhx + g];
        xx += abs2(x);
        xh += x.x * h.x + x.y * h.y;
    }
    block_sum2(xx, xh);
    if (threadIdx.x == 0) {
        S[(size_t)j * n + j] = mkc(xx, 0.0);
        A[(size_t)j * n + j] = mkc(xh, 0.0);
    }
}

// ||HX_j - theta_j X_j|| / ||X_j|| (one block per column, FP64).
__global__ void __launch_bounds__(256)
k_resid_norm(int npw, const z64 *__restrict__ X, int ldx, const z64 *__restrict__ HX, int ldhx,
             const double *__restrict__ theta, double *__restrict__ out) {
    const int j = blockIdx.x;
    const double th = theta[j];
    double rr = 0.0, xx = 0.0;
    for (int g = threadIdx.x; g < npw; g += blockDim.x) {
        const z64 x = X[(size_t)j * ldx + g], hx = HX[(size_t)j * ldhx + g];
        const double a = hx.x - th * x.x, b = hx.y - th * x.y;
        rr += a * a + b * b;
        xx += abs2(x);
    }
    block_sum2(rr, xx);
    if (threadIdx.x == 0) out[j] = xx > 0.0 ? sqrt(rr / xx) : 0.0;
}

template <typename Ro, typename Ri>
__global__ void k_copy_cast(int rows, int cols, const cx<Ri> *__restrict__ A, int lda, cx<Ro> *__restrict__ B,
                            int ldb) {
    const size_t tot = (size_t)rows * cols;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % rows), j = (int)(e / rows);
        B[(size_t)j * ldb + i] = cvt<Ro, Ri>(A[(size_t)j * lda + i]);
    }
}

template <typename R>
__global__ void k_scale_rows(int rows, int cols, const R *__restrict__ d, cx<R> *__restrict__ A, int lda) {
    const size_t tot = (size_t)rows * cols;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % rows), j = (int)(e / rows);
        A[(size_t)j * lda + i] = d[i] * A[(size_t)j * lda + i];
    }
}

int grid_for(size_t n, int threads) {
    return (int)std::max<size_t>(1, std::min<size_t>((n + threads - 1) / threads, 152 * 16));
}

}  // namespace

size_t colsum_part_elems(int m) { return 2 * (size_t)std::max(m, 1) * kMaxChunks; }

// Ekin of each column into ekin[0..m)
static int ekin_cols(int npw, int m, const z64 *X, int ldx, const double *kin, double *ekin, double *part,
                     cudaStream_t s) {
    if (part) return colsum2<kEkin>(npw, m, X, ldx, nullptr, 0, kin, nullptr, part, ekin, nullptr, nullptr, 0, s);
    k_ekin<<<m, 256, 0, s>>>(npw, X, ldx, kin, ekin);
    return check_launch("ekin");
}

template <typename R>
int residual_precond(int npw, int m, const z64 *X, int ldx, const z64 *HX, int ldhx, const double *theta,
                     const double *kin, cx<R> *W, int ldw, double *work, double *part, cudaStream_t s) {
    if (m <= 0) return LOBPCG_OK;
    LG_TRY(ekin_cols(npw, m, X, ldx, kin, work, part, s));
    const int gx = std::max(1, std::min((npw + 255) / 256, 64));
    k_resid_precond<R><<<dim3(gx, m), 256, 0, s>>>(npw, m, X, ldx, HX, ldhx, theta, kin, work, W, ldw);
    return check_launch("residual/preconditioner");
}

int residual_precond_mixed(int npw, int m, const z64 *X, int ldx, const z64 *HX, int ldhx, const double *theta,
                           const double *kin, c32 *R, c32 *W, int ld, double *work, double *part, cudaStream_t s) {
    if (m <= 0) return LOBPCG_OK;
    LG_TRY(ekin_cols(npw, m, X, ldx, kin, work, part, s));
    const int gx = std::max(1, std::min((npw + 255) / 256, 64));
    k_resid_precond_mixed<<<dim3(gx, m), 256, 0, s>>>(npw, m, X, ldx, HX, ldhx, theta, kin, work, R, W, ld);
    return check_launch("residual/preconditioner (mixed)");
}

int axpy_cols(int rows, int cols, double alpha, const z64 *D, int ldd, z64 *V, int ldv, cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return LOBPCG_OK;
    k_axpy_cols<<<grid_for((size_t)rows * cols, 256), 256, 0, s>>>(rows, cols, alpha, D, ldd, V, ldv);
    return check_launch("axpy");
}

int assemble_gram_mixed(int nz, int mx, const c32 *S32, int lds32, const c32 *A32, int lda32, const double *theta,
                        z64 *S, z64 *A, cudaStream_t s) {
    k_assemble<double><<<dim3((nz + 127) / 128, nz), 128, 0, s>>>(nz, mx, S32, lds32, A32, lda32, theta, S, A);
    return check_launch("assemble gram");
}

int assemble_gram_mixed32(int nz, int mx, const c32 *S32, int lds32, const c32 *A32, int lda32, const double *theta,
                          c32 *S, c32 *A, cudaStream_t s) {
    k_assemble<float><<<dim3((nz + 127) / 128, nz), 128, 0, s>>>(nz, mx, S32, lds32, A32, lda32, theta, S, A);
    return check_launch("assemble gram (fp32)");
}

int rayleigh_quotients(int npw, int m, const z64 *X, int ldx, const z64 *HX, int ldhx, double *theta, double *part,
                       cudaStream_t s) {
    if (m <= 0) return LOBPCG_OK;
    if (part) return colsum2<kRayleigh>(npw, m, X, ldx, HX, ldhx, nullptr, nullptr, part, theta, nullptr, nullptr, 0, s);
    k_rayleigh_quotients<<<m, 256, 0, s>>>(npw, X, ldx, HX, ldhx, theta);
    return check_launch("rayleigh quotients");
}

int residual32(int npw, int m, const z64 *X, int ldx, const z64 *HX, int ldhx, const double *theta, c32 *R, int ldr,
               cudaStream_t s) {
    if (m <= 0) return LOBPCG_OK;
    const int gx = std::max(1, std::min((npw + 255) / 256, 64));
    k_residual32<<<dim3(gx, m), 256, 0, s>>>(npw, X, ldx, HX, ldhx, theta, R, ldr);
    return check_launch("residual (fp32 out)");
}

int precond32(int npw, int m, const z64 *X, int ldx, const double *kin, const c32 *R, int ldr, c32 *W, int ldw,
              double *work, double *part, cudaStream_t s) {
    if (m <= 0) return LOBPCG_OK;
    LG_TRY(ekin_cols(npw, m, X, ldx, kin, work, part, s));
    const int gx = std::max(1, std::min((npw + 255) / 256, 64));
    k_precond32<<<dim3(gx, m), 256, 0, s>>>(npw, R, ldr, kin, work, W, ldw);
    return check_launch("preconditioner (fp32)");
}

int diag_pencil(int npw, int m, const z64 *X, int ldx, const z64 *HX, int ldhx, z64 *S, z64 *A, double *part,
                cudaStream_t s) {
    if (m <= 0) return LOBPCG_OK;
    if (part) return colsum2<kDiag>(npw, m, X, ldx, HX, ldhx, nullptr, nullptr, part, nullptr, S, A, m, s);
    k_diag_pencil<<<m, 256, 0, s>>>(npw, X, ldx, HX, ldhx, S, A, m);
    return check_launch("diagonal of the pencil");
}

__global__ void k_fill_random(int rows, int cols, z64 *__restrict__ X, int ldx, unsigned seed) {
    const size_t tot = (size_t)rows * cols;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % rows), j = (int)(e / rows);
        unsigned h = (unsigned)i * 0x9E3779B1u ^ ((unsigned)j + seed) * 0x85EBCA77u;
        h ^= h >> 16; h *= 0x7FEB352Du; h ^= h >> 15; h *= 0x846CA68Bu; h ^= h >> 16;
        unsigned g = h * 0x27D4EB2Fu + 0x165667B1u;
        g ^= g >> 15; g *= 0x2C1B3C6Du; g ^= g >> 12;
        X[(size_t)j * ldx + i] = mkc((double)h * (2.0 / 4294967296.0) - 1.0, (double)g * (2.0 / 4294967296.0) - 1.0);
    }
}

int fill_random(int rows, int cols, z64 *X, int ldx, unsigned seed, cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return LOBPCG_OK;
    k_fill_random<<<grid_for((size_t)rows * cols, 256), 256, 0, s>>>(rows, cols, X, ldx, seed);
    return check_launch("fill random");
}

int column_resid_norms(int npw, int m, const z64 *X, int ldx, const z64 *HX, int ldhx, const double *theta,
                       double *out, double *part, cudaStream_t s) {
    if (m <= 0) return LOBPCG_OK;
    if (part) return colsum2<kResid>(npw, m, X, ldx, HX, ldhx, nullptr, theta, part, out, nullptr, nullptr, 0, s);
    k_resid_norm<<<m, 256, 0, s>>>(npw, X, ldx, HX, ldhx, theta, out);
    return check_launch("residual norms");
}

template <typename Ro, typename Ri>
int copy_cast(int rows, int cols, const cx<Ri> *A, int lda, cx<Ro> *B, int ldb, cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return LOBPCG_OK;
    k_copy_cast<Ro, Ri><<<grid_for((size_t)rows * cols, 256), 256, 0, s>>>(rows, cols, A, lda, B, ldb);
    return check_launch("copy/cast");
}

int scale_rows_real(int rows, int cols, const double *d, z64 *A, int lda, cudaStream_t s) {
    return scale_rows<double>(rows, cols, d, A, lda, s);
}

template <typename R>
int scale_rows(int rows, int cols, const R *d, cx<R> *A, int lda, cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return LOBPCG_OK;
    k_scale_rows<R><<<grid_for((size_t)rows * cols, 256), 256, 0, s>>>(rows, cols, d, A, lda);
    return check_launch("scale rows");
}

// E = C - I on the leading rows x cols block of C (FP64 in, FP32 out) and max |E| (as float bits,
// an atomic max on non-negative floats).
__global__ void k_near_identity32(int rows, int cols, const z64 *__restrict__ C, int ldc, c32 *__restrict__ E,
                                  int lde, unsigned int *__restrict__ maxbits) {
    const size_t tot = (size_t)rows * cols;
    float mx = 0.f;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % rows), j = (int)(e / rows);
        z64 v = C[(size_t)j * ldc + i];
        if (i == j) v.x -= 1.0;
        const c32 f = mkc<float>((float)v.x, (float)v.y);
        E[(size_t)j * lde + i] = f;
        mx = fmaxf(mx, fmaxf(fabsf(f.x), fabsf(f.y)));
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(maxbits, __float_as_uint(mx));
}

// out = A + fp64(T) column by column (out may be A).
__global__ void k_add_cast(int rows, int cols, const z64 *A, int lda, const c32 *__restrict__ T, int ldt, z64 *out,
                           int ldo) {
    const size_t tot = (size_t)rows * cols;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % rows), j = (int)(e / rows);
        const c32 t = T[(size_t)j * ldt + i];
        const z64 a = A[(size_t)j * lda + i];
        out[(size_t)j * ldo + i] = mkc(a.x + (double)t.x, a.y + (double)t.y);
    }
}

// Column j of C times conj(C_jj)/|C_jj| (a Ritz vector's phase is free): the diagonal becomes
// real and non-negative, so a rotation that only re-phases is the identity.
__global__ void k_fix_phases(int rows, int cols, z64 *__restrict__ C, int ldc) {
    const int j = blockIdx.x;
    if (j >= cols || j >= rows) return;
    const z64 p = C[(size_t)j * ldc + j];
    const double a = sqrt(p.x * p.x + p.y * p.y);
    if (!(a > 0.0)) return;
    const z64 ph = mkc(p.x / a, -p.y / a);
    __syncthreads();
    for (int i = threadIdx.x; i < rows; i += blockDim.x) C[(size_t)j * ldc + i] = C[(size_t)j * ldc + i] * ph;
}

int fix_phases(int rows, int cols, z64 *C, int ldc, cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return LOBPCG_OK;
    k_fix_phases<<<cols, 128, 0, s>>>(rows, cols, C, ldc);
    return check_launch("fix phases");
}

int near_identity32(int rows, int cols, const z64 *C, int ldc, c32 *E, int lde, unsigned int *dmax, float *hmax,
                    cudaStream_t s) {
    if (rows <= 0 || cols <= 0) {
        *hmax = 0.f;
        return LOBPCG_OK;
    }
    LG_CUDA_TRY(cudaMemsetAsync(dmax, 0, sizeof(unsigned int), s));
    k_near_identity32<<<grid_for((size_t)rows * cols, 256), 256, 0, s>>>(rows, cols, C, ldc, E, lde, dmax);
    LG_TRY(check_launch("near-identity part"));
    unsigned int h = 0;
    LG_CUDA_TRY(cudaMemcpyAsync(&h, dmax, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
    LG_CUDA_TRY(cudaStreamSynchronize(s));
    std::memcpy(hmax, &h, sizeof(float));
    return LOBPCG_OK;
}

int add_cast(int rows, int cols, const z64 *A, int lda, const c32 *T, int ldt, z64 *out, int ldo, cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return LOBPCG_OK;
    k_add_cast<<<grid_for((size_t)rows * cols, 256), 256, 0, s>>>(rows, cols, A, lda, T, ldt, out, ldo);
    return check_launch("add cast");
}

template int residual_precond<double>(int, int, const z64 *, int, const z64 *, int, const double *, const double *,
                                      z64 *, int, double *, double *, cudaStream_t);
template int residual_precond<float>(int, int, const z64 *, int, const z64 *, int, const double *, const double *,
                                     c32 *, int, double *, double *, cudaStream_t);
template int copy_cast<double, double>(int, int, const z64 *, int, z64 *, int, cudaStream_t);
template int copy_cast<float, double>(int, int, const z64 *, int, c32 *, int, cudaStream_t);
template int copy_cast<double, float>(int, int, const c32 *, int, z64 *, int, cudaStream_t);
template int copy_cast<float, float>(int, int, const c32 *, int, c32 *, int, cudaStream_t);
template int scale_rows<double>(int, int, const double *, z64 *, int, cudaStream_t);
template int scale_rows<float>(int, int, const float *, c32 *, int, cudaStream_t);


// ------------------------------------------------------------------ Gamma-point real form
// At k = 0, with H commuting with c(G) -> conj(c(-G)), the eigenvectors can be taken real in
// r space: c(-G) = conj(c(G)).  Such a vector is stored packed on the half sphere
// {G = 0} u S+ (S+: n_x > 0, or n_x = 0 and n_y > 0, or n_x = n_y = 0 and n_z > 0), G = 0 first:
//     z[0] = c(0) (real),  z[g] = sqrt(2) c(G_g)  (G_g in S+),
// so that Re(z_a^H z_b) = c_a^H c_b (the real inner product of the real form).  half[g] is the
// position of G_g in the sphere's order and mirror[g] the position of -G_g (mirror[0] = half[0]).
namespace {

constexpr double kRsqrt2 = 0.70710678118654752440;

// Sphere vectors (npw x nb) -> packed (nz x nb): z[g] = (c(G) + conj(c(-G))) / sqrt(2), z[0] = Re c(0)
// (the projection of an arbitrary vector onto the real form).
template <typename R>
__global__ void k_gamma_pack_full(int nz, int nb, const cx<R> *__restrict__ C, int ldc, const int *__restrict__ half,
                                  const int *__restrict__ mirror, cx<R> *__restrict__ Z, int ldz) {
    const size_t tot = (size_t)nz * nb;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        const int g = (int)(e % nz), b = (int)(e / nz);
        const cx<R> cp = C[(size_t)b * ldc + half[g]];
        if (g == 0) {
            Z[(size_t)b * ldz] = mkc<R>(cp.x, (R)0);
        } else {
            const cx<R> cq = C[(size_t)b * ldc + mirror[g]];
            Z[(size_t)b * ldz + g] = mkc<R>((R)kRsqrt2 * (cp.x + cq.x), (R)kRsqrt2 * (cp.y - cq.y));
        }
    }
}

// Packed (nz x nb) -> sphere vectors (npw x nb): c(G) = z / sqrt(2), c(-G) = conj(z) / sqrt(2).
template <typename R>
__global__ void k_gamma_unpack_full(int nz, int nb, const cx<R> *__restrict__ Z, int ldz, const int *__restrict__ half,
                                    const int *__restrict__ mirror, cx<R> *__restrict__ C, int ldc) {
    const size_t tot = (size_t)nz * nb;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        const int g = (int)(e % nz), b = (int)(e / nz);
        const cx<R> z = Z[(size_t)b * ldz + g];
        if (g == 0) {
            C[(size_t)b * ldc + half[0]] = mkc<R>(z.x, (R)0);
        } else {
            C[(size_t)b * ldc + half[g]] = mkc<R>((R)kRsqrt2 * z.x, (R)kRsqrt2 * z.y);
            C[(size_t)b * ldc + mirror[g]] = mkc<R>((R)kRsqrt2 * z.x, -(R)kRsqrt2 * z.y);
        }
    }
}

// Two packed real-form bands a = band 2i, b = band 2i+1 -> one sphere vector c_a + i c_b
// (column i of C; b = 0 past the last band).  H is complex-linear, so one application gives
// H c_a + i H c_b.
template <typename R>
__global__ void k_gamma_unpack_pairs(int nz, int nb, const cx<R> *__restrict__ Z, int ldz, const int *__restrict__ half,
                                     const int *__restrict__ mirror, cx<R> *__restrict__ C, int ldc) {
    const int np = (nb + 1) / 2;
    const size_t tot = (size_t)nz * np;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        const int g = (int)(e % nz), i = (int)(e / nz);
        const cx<R> a = Z[(size_t)(2 * i) * ldz + g];
        const cx<R> b = (2 * i + 1 < nb) ? Z[(size_t)(2 * i + 1) * ldz + g] : mkc<R>((R)0, (R)0);
        cx<R> *Ci = C + (size_t)i * ldc;
        if (g == 0) {
            Ci[half[0]] = mkc<R>(a.x, b.x);
        } else {
            const R s = (R)kRsqrt2;
            Ci[half[g]] = mkc<R>(s * (a.x - b.y), s * (a.y + b.x));     // (a + i b) / sqrt(2)
            Ci[mirror[g]] = mkc<R>(s * (a.x + b.y), s * (b.x - a.y));   // (conj a + i conj b) / sqrt(2)
        }
    }
}

// Y = H c_a + i H c_b (sphere) -> packed H a, H b: with both images real-form,
// (H c_a)(G) = (Y(G) + conj(Y(-G))) / 2 and (H c_b)(G) = (Y(G) - conj(Y(-G))) / (2 i).
template <typename R>
__global__ void k_gamma_pack_pairs(int nz, int nb, const cx<R> *__restrict__ Y, int ldy, const int *__restrict__ half,
                                   const int *__restrict__ mirror, cx<R> *__restrict__ Z, int ldz) {
    const int np = (nb + 1) / 2;
    const size_t tot = (size_t)nz * np;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        const int g = (int)(e % nz), i = (int)(e / nz);
        const cx<R> *Yi = Y + (size_t)i * ldy;
        cx<R> a, b;
        if (g == 0) {
            const cx<R> y0 = Yi[half[0]];
            a = mkc<R>(y0.x, (R)0);
            b = mkc<R>(y0.y, (R)0);
        } else {
            const cx<R> yp = Yi[half[g]], yq = Yi[mirror[g]];
            const R s = (R)kRsqrt2;
            a = mkc<R>(s * (yp.x + yq.x), s * (yp.y - yq.y));   // (Y(G) + conj Y(-G)) / sqrt(2)
            const R u = yp.x - yq.x, v = yp.y + yq.y;          // Y(G) - conj Y(-G)
            b = mkc<R>(s * v, -s * u);                          // that / (i sqrt(2))
        }
        Z[(size_t)(2 * i) * ldz + g] = a;
        if (2 * i + 1 < nb) Z[(size_t)(2 * i + 1) * ldz + g] = b;
    }
}

template <typename R>
__global__ void k_zero_imag(int rows, int cols, cx<R> *__restrict__ A, int lda) {
    const size_t tot = (size_t)rows * cols;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % rows), j = (int)(e / rows);
        A[(size_t)j * lda + i].y = (R)0;
    }
}

int gamma_grid(size_t n) { return (int)std::max<size_t>(1, std::min<size_t>((n + 255) / 256, 152 * 16)); }

}  // namespace

template <typename R>
int gamma_pack_full(int nz, int nb, const cx<R> *C, int ldc, const int *half, const int *mirror, cx<R> *Z, int ldz,
                    cudaStream_t s) {
    if (nz <= 0 || nb <= 0) return LOBPCG_OK;
    k_gamma_pack_full<R><<<gamma_grid((size_t)nz * nb), 256, 0, s>>>(nz, nb, C, ldc, half, mirror, Z, ldz);
    return check_launch("gamma pack");
}
template <typename R>
int gamma_unpack_full(int nz, int nb, const cx<R> *Z, int ldz, const int *half, const int *mirror, cx<R> *C, int ldc,
                      cudaStream_t s) {
    if (nz <= 0 || nb <= 0) return LOBPCG_OK;
    k_gamma_unpack_full<R><<<gamma_grid((size_t)nz * nb), 256, 0, s>>>(nz, nb, Z, ldz, half, mirror, C, ldc);
    return check_launch("gamma unpack");
}
template <typename R>
int gamma_unpack_pairs(int nz, int nb, const cx<R> *Z, int ldz, const int *half, const int *mirror, cx<R> *C, int ldc,
                       cudaStream_t s) {
    if (nz <= 0 || nb <= 0) return LOBPCG_OK;
    k_gamma_unpack_pairs<R><<<gamma_grid((size_t)nz * ((nb + 1) / 2)), 256, 0, s>>>(nz, nb, Z, ldz, half, mirror, C,
                                                                                   ldc);
    return check_launch("gamma unpack pairs");
}
template <typename R>
int gamma_pack_pairs(int nz, int nb, const cx<R> *Y, int ldy, const int *half, const int *mirror, cx<R> *Z, int ldz,
                     cudaStream_t s) {
    if (nz <= 0 || nb <= 0) return LOBPCG_OK;
    k_gamma_pack_pairs<R><<<gamma_grid((size_t)nz * ((nb + 1) / 2)), 256, 0, s>>>(nz, nb, Y, ldy, half, mirror, Z,
                                                                                 ldz);
    return check_launch("gamma pack pairs");
}
template <typename R>
int zero_imag(int rows, int cols, cx<R> *A, int lda, cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return LOBPCG_OK;
    k_zero_imag<R><<<gamma_grid((size_t)rows * cols), 256, 0, s>>>(rows, cols, A, lda);
    return check_launch("real part");
}
#define LG_GAMMA_INST(R)                                                                                             \
    template int gamma_pack_full<R>(int, int, const cx<R> *, int, const int *, const int *, cx<R> *, int, cudaStream_t); \
    template int gamma_unpack_full<R>(int, int, const cx<R> *, int, const int *, const int *, cx<R> *, int,          \
                                      cudaStream_t);                                                               \
    template int gamma_unpack_pairs<R>(int, int, const cx<R> *, int, const int *, const int *, cx<R> *, int,         \
                                       cudaStream_t);                                                              \
    template int gamma_pack_pairs<R>(int, int, const cx<R> *, int, const int *, const int *, cx<R> *, int,           \
                                     cudaStream_t);                                                                \
    template int zero_imag<R>(int, int, cx<R> *, int, cudaStream_t);
LG_GAMMA_INST(double)
LG_GAMMA_INST(float)
#undef LG_GAMMA_INST

}  // namespace lg
