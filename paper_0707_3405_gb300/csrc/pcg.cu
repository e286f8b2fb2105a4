// Band-by-band preconditioned conjugate gradient for a fixed H (the method Sec. 3.3 of the
// paper compares LOBPCG with: Teter, Payne and Allan 1989, in the iterative-diagonalisation form
// of Bylander et al. 1990).  These are the per-band vector steps; the driver in api.cu runs them
// band after band and closes each sweep with the all-band Rayleigh-Ritz step of the LOBPCG
// solver.  For one band x (orthogonal to the bands Y before it), nline iterations of:
//   1. xi  = -(H x - eps x), eps = <x|H|x>;
//   2. xi  <- xi projected off span(Y) (classical Gram-Schmidt, twice) and off x;
//   3. eta = K(xi) (Teter ratio, x = T(q)/Ekin(x)), projected the same way;
//   4. d   = eta + gamma d_prev, gamma = <eta|xi> / <eta_prev|xi_prev> (0 on the first);
//   5. d^  = (d - x <x|d>) / ||.||;
//   6. exact line minimum of the Rayleigh quotient on cos(t) x + sin(t) d^ (the 2 x 2
//      Rayleigh-Ritz problem on span[x, d^]); x <- x(t*), H x likewise.
// Every scalar stays on the device (no host round trip inside a band); sums over the plane
// waves go through fixed-order two-stage reductions (reproducible).  FP64 arithmetic.
#include "common.cuh"

#include <algorithm>

namespace lg {

namespace {

constexpr int kThr = 256;
constexpr int kChunk = 4096;   // plane waves per reduction block

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Up to three sums per block over its chunk of plane waves (fixed order):
//   mode 0: Re/Im of conj(a) b      (dots)
//   mode 1: sum T |a|^2, sum |a|^2  (kinetic energy of a band)
// part[blk * 6 + 2 q + {0, 1}] for q < nq.
__global__ void __launch_bounds__(kThr)
k_pcg_sums(int npw, int nq, const z64 *__restrict__ a0, const z64 *__restrict__ b0, const z64 *__restrict__ a1,
           const z64 *__restrict__ b1, const z64 *__restrict__ a2, const z64 *__restrict__ b2, int mode,
           const double *__restrict__ kin, double *__restrict__ part) {
    __shared__ double sh[8][6];
    const int g0 = blockIdx.x * kChunk, g1 = min(npw, g0 + kChunk);
    double acc[6] = {0, 0, 0, 0, 0, 0};
    const z64 *A[3] = {a0, a1, a2}, *B[3] = {b0, b1, b2};
    for (int g = g0 + threadIdx.x; g < g1; g += kThr) {
        if (mode == 1) {
            const double xx = abs2(a0[g]);
            acc[0] += kin[g] * xx;
            acc[1] += xx;
        } else {
#pragma unroll
            for (int q = 0; q < 3; ++q)
                if (q < nq) {
                    const z64 u = A[q][g], v = B[q][g];
                    acc[2 * q] += u.x * v.x + u.y * v.y;
                    acc[2 * q + 1] += u.x * v.y - u.y * v.x;
                }
        }
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        const double v = wsum(acc[q]);
        if (lane == 0) sh[w][q] = v;
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        double t = 0.0;
        for (int i = 0; i < kThr / 32; ++i) t += sh[i][threadIdx.x];
        part[(size_t)blockIdx.x * 6 + threadIdx.x] = t;
    }
}

// Scalar block of one band (device):
enum {
    S_EPS = 0,     // Rayleigh quotient of x
    S_EKIN,        // kinetic energy of x (preconditioner scale)
    S_DOTP,        // <eta_prev|xi_prev> (0: no previous direction)
    S_GAMMA,       // conjugacy coefficient of this iteration
    S_C, S_S,      // cos, sin of the line minimum
    S_ND,          // 1 / ||d^|| (0 when d^ vanished)
    S_NX,          // 1 / ||x||
    S_CO0, S_CO1,  // coefficient <x|v> (re, im) of a projection off x
    S_NSCAL
};

// Sum the block partials in a fixed order into r[0..2 nq) and act on them:
//   act 0: r -> S_CO0/1 (the <x|v> of a projection)
//   act 1: ||x||^2 -> S_NX
//   act 2: <x|Hx> -> S_EPS
//   act 3: Ekin -> S_EKIN (r = sum T|x|^2, sum |x|^2)
//   act 4: <eta|xi> -> S_GAMMA (from S_DOTP), S_DOTP <- <eta|xi>
//   act 5: <x|d> -> S_CO0/1
//   act 6: ||d^||^2 -> S_ND
//   act 7: (<dh|H dh>, <x|H dh>) -> line minimum: S_C, S_S
__global__ void k_pcg_finish(int nblk, int nq, const double *__restrict__ part, int act, double *__restrict__ sc) {
    if (threadIdx.x != 0) return;
    double r[6] = {0, 0, 0, 0, 0, 0};
    for (int b = 0; b < nblk; ++b)
        for (int q = 0; q < 2 * nq; ++q) r[q] += part[(size_t)b * 6 + q];
    switch (act) {
        case 0: case 5: sc[S_CO0] = r[0]; sc[S_CO1] = r[1]; break;
        case 1: sc[S_NX] = r[0] > 0.0 ? 1.0 / sqrt(r[0]) : 0.0; break;
        case 2: sc[S_EPS] = r[0]; break;
        case 3: sc[S_EKIN] = r[1] > 0.0 ? r[0] / r[1] : 1.0; break;
        case 4: {
            const double dot = r[0], prev = sc[S_DOTP];
            sc[S_GAMMA] = prev != 0.0 ? dot / prev : 0.0;
            sc[S_DOTP] = dot;
            break;
        }
        case 6: sc[S_ND] = r[0] > 0.0 ? 1.0 / sqrt(r[0]) : 0.0; break;
        case 7: {
            // E(t) = A cos^2 + B sin^2 + 2 C sin cos is smallest where (cos 2t, sin 2t) points
            // against ((A - B)/2, C)
            const double A = sc[S_EPS], B = r[0], C = r[2];
            double c = 1.0, s = 0.0;
            if (sc[S_ND] != 0.0) {
                const double t = 0.5 * atan2(-2.0 * C, B - A);
                c = cos(t);
                s = sin(t);
            }
            sc[S_C] = c;
            sc[S_S] = s;
            break;
        }
        default: break;
    }
}

// Elementwise steps with device scalars.
//   op 0: v <- v - x * co                  (projection off x)
//   op 1: v <- v * nx                      (normalise)
//   op 2: xi <- -(hx - eps x)              (v = xi, a = x, b = hx)
//   op 3: eta <- K(xi), x = T/Ekin          (v = eta, a = xi)
//   op 4: d <- eta + gamma d               (v = d, a = eta)
//   op 5: dh <- d - x co                   (v = dh, a = d, b = x)
//   op 6: x <- c x + s dh, hx <- c hx + s hd (v = x, a = dh, w = hx, b = hd)
//   op 7: x <- x nx, hx <- hx nx           (v = x, w = hx)
//   op 8: dh <- dh nd
__global__ void k_pcg_vec(int npw, int op, z64 *__restrict__ v, const z64 *__restrict__ a,
                          const z64 *__restrict__ b, z64 *__restrict__ w, const double *__restrict__ kin,
                          const double *__restrict__ sc) {
    const double eps = sc[S_EPS], ekin = sc[S_EKIN], gam = sc[S_GAMMA], c = sc[S_C], s = sc[S_S];
    const double nd = sc[S_ND], nx = sc[S_NX];
    const z64 co = mkc(sc[S_CO0], sc[S_CO1]);
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < npw; g += gridDim.x * blockDim.x) {
        switch (op) {
            case 0: v[g] = v[g] - co * a[g]; break;
            case 1: v[g] = nx * v[g]; break;
            case 2: v[g] = eps * a[g] - b[g]; break;
            case 3: {
                const double x = kin[g] / ekin;
                const double p = 27.0 + x * (18.0 + x * (12.0 + 8.0 * x));
                v[g] = (p / (p + 16.0 * x * x * x * x)) * a[g];
                break;
            }
            case 4: v[g] = gam != 0.0 ? a[g] + gam * v[g] : a[g]; break;   // no previous d on the first
            case 5: v[g] = a[g] - co * b[g]; break;
            case 6: {
                v[g] = c * v[g] + s * a[g];
                w[g] = c * w[g] + s * b[g];
                break;
            }
            case 7: v[g] = nx * v[g]; w[g] = nx * w[g]; break;
            case 8: v[g] = nd * v[g]; break;
            default: break;
        }
    }
}

// G = Y^H v (j entries) by chunks: part[chunk * j + i], then summed in chunk order.
__global__ void __launch_bounds__(kThr)
k_gemv_cn_part(int npw, int j, const z64 *__restrict__ Y, int ldy, const z64 *__restrict__ v,
               z64 *__restrict__ part) {
    __shared__ z64 vs[kChunk / 4];
    constexpr int CH = kChunk / 4;
    const int g0 = blockIdx.x * CH, g1 = min(npw, g0 + CH), len = g1 - g0;
    for (int g = threadIdx.x; g < len; g += kThr) vs[g] = v[g0 + g];
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = blockIdx.y * 8 + w; i < j; i += gridDim.y * 8) {
        const z64 *y = Y + (size_t)i * ldy + g0;
        double re = 0.0, im = 0.0;
        for (int g = lane; g < len; g += 32) {
            const z64 a = y[g], b = vs[g];
            re += a.x * b.x + a.y * b.y;
            im += a.x * b.y - a.y * b.x;
        }
        re = wsum(re);
        im = wsum(im);
        if (lane == 0) part[(size_t)blockIdx.x * j + i] = mkc(re, im);
    }
}

__global__ void k_gemv_cn_fin(int j, int nch, const z64 *__restrict__ part, z64 *__restrict__ G) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= j) return;
    z64 t = mkc(0.0, 0.0);
    for (int c = 0; c < nch; ++c) t = t + part[(size_t)c * j + i];
    G[i] = t;
}

// v <- v - Y G (j columns).
__global__ void __launch_bounds__(kThr)
k_gemv_nn_sub(int npw, int j, const z64 *__restrict__ Y, int ldy, const z64 *__restrict__ G, z64 *__restrict__ v) {
    extern __shared__ z64 gs[];
    for (int i = threadIdx.x; i < j; i += kThr) gs[i] = G[i];
    __syncthreads();
    for (int g = blockIdx.x * kThr + threadIdx.x; g < npw; g += gridDim.x * kThr) {
        z64 acc = mkc(0.0, 0.0);
        for (int i = 0; i < j; ++i) fma_nn(acc, Y[(size_t)i * ldy + g], gs[i]);
        v[g] = v[g] - acc;
    }
}

int nblk_of(int npw) { return (npw + kChunk - 1) / kChunk; }
int vec_grid(int npw) { return std::max(1, std::min((npw + kThr - 1) / kThr, 152 * 8)); }

}  // namespace

size_t pcg_scratch_doubles(int npw, int M) {
    const size_t part = ((size_t)nblk_of(npw) * 6 + 1) / 2 * 2;
    const size_t nch = ((size_t)npw + kChunk / 4 - 1) / (kChunk / 4);
    return 64 + part + 2 * nch * std::max(M, 1) + 2 * (size_t)std::max(M, 1);
}

void pcg_carve(PcgBand &pb, double *base, int npw, int M) {
    const size_t part = ((size_t)nblk_of(npw) * 6 + 1) / 2 * 2;
    const size_t nch = ((size_t)npw + kChunk / 4 - 1) / (kChunk / 4);
    pb.sc = base;
    pb.part = base + 64;
    pb.gpart = reinterpret_cast<z64 *>(base + 64 + part);
    pb.G = reinterpret_cast<z64 *>(base + 64 + part + 2 * nch * std::max(M, 1));
}

int PcgBand::sums(int nq, const z64 *a0, const z64 *b0, const z64 *a1, const z64 *b1, const z64 *a2,
                  const z64 *b2, int mode, int act) {
    const int nb = nblk_of(npw);
    k_pcg_sums<<<nb, kThr, 0, s>>>(npw, nq, a0, b0, a1, b1, a2, b2, mode, kin, part);
    LG_TRY(check_launch("pcg sums"));
    k_pcg_finish<<<1, 32, 0, s>>>(nb, mode == 1 ? 1 : nq, part, act, sc);
    return check_launch("pcg scalars");
}

int PcgBand::vec(int op, z64 *v, const z64 *a, const z64 *b, z64 *w) {
    k_pcg_vec<<<vec_grid(npw), kThr, 0, s>>>(npw, op, v, a, b, w, kin, sc);
    return check_launch("pcg vector step");
}

// v <- v - Y (Y^H v), twice, then v <- v - x <x|v>.
int PcgBand::project(z64 *v, const z64 *x) {
    if (j > 0) {
        const int CH = kChunk / 4;
        const int nch = (npw + CH - 1) / CH;
        const int gy = std::max(1, std::min(32, (j + 7) / 8));
        for (int rep = 0; rep < 2; ++rep) {
            k_gemv_cn_part<<<dim3(nch, gy), kThr, 0, s>>>(npw, j, Y, ldy, v, gpart);
            LG_TRY(check_launch("pcg projection Y^H v"));
            k_gemv_cn_fin<<<(j + 255) / 256, 256, 0, s>>>(j, nch, gpart, G);
            LG_TRY(check_launch("pcg projection sums"));
            k_gemv_nn_sub<<<vec_grid(npw), kThr, sizeof(z64) * (size_t)j, s>>>(npw, j, Y, ldy, G, v);
            LG_TRY(check_launch("pcg projection v - Y G"));
        }
    }
    if (!x) return LOBPCG_OK;
    LG_TRY(sums(1, x, v, nullptr, nullptr, nullptr, nullptr, 0, 0));
    return vec(0, v, x, nullptr, nullptr);
}

int PcgBand::prepare_start() {
    // x off span(Y), normalised; H x and eps follow in the driver (apply_H)
    LG_TRY(project(x, nullptr));
    LG_TRY(sums(1, x, x, nullptr, nullptr, nullptr, nullptr, 0, 1));
    return vec(1, x, nullptr, nullptr, nullptr);
}

int PcgBand::after_hx() {
    LG_TRY(sums(1, x, hx, nullptr, nullptr, nullptr, nullptr, 0, 2));          // eps
    LG_TRY(sums(1, x, nullptr, nullptr, nullptr, nullptr, nullptr, 1, 3));     // Ekin
    return LOBPCG_OK;
}

int PcgBand::direction(bool first) {
    if (first) LG_CUDA_TRY(cudaMemsetAsync(sc + S_DOTP, 0, sizeof(double), s));
    LG_TRY(vec(2, xi, x, hx, nullptr));                                          // 1: xi = -(Hx - eps x)
    LG_TRY(project(xi, x));                                                      // 2
    LG_TRY(vec(3, eta, xi, nullptr, nullptr));                                   // 3: eta = K(xi)
    LG_TRY(project(eta, x));
    LG_TRY(sums(1, eta, xi, nullptr, nullptr, nullptr, nullptr, 0, 4));          // 4: gamma
    LG_TRY(vec(4, d, eta, nullptr, nullptr));                                    //    d = eta + gamma d
    LG_TRY(sums(1, x, d, nullptr, nullptr, nullptr, nullptr, 0, 5));            // 5: <x|d>
    LG_TRY(vec(5, dh, d, x, nullptr));                                           //    d - x <x|d>
    LG_TRY(sums(1, dh, dh, nullptr, nullptr, nullptr, nullptr, 0, 6));
    return vec(8, dh, nullptr, nullptr, nullptr);                                //    normalised
}

int PcgBand::step() {
    LG_TRY(sums(2, dh, hd, x, hd, nullptr, nullptr, 0, 7));                     // 6: line minimum
    LG_TRY(vec(6, x, dh, hd, hx));                                               //    rotate x, H x
    LG_TRY(sums(1, x, x, nullptr, nullptr, nullptr, nullptr, 0, 1));
    LG_TRY(vec(7, x, nullptr, nullptr, hx));                                     //    normalise
    return after_hx();                                                           //    eps, Ekin
}

}  // namespace lg
