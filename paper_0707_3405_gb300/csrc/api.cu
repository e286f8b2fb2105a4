// C ABI of the GB300 LOBPCG plane-wave eigensolver: handle, plane-wave basis,
// H application and the block LOBPCG driver (Bottin, Leroux, Knyazev, Zerah
// 2007).  See include/lobpcg_gb300.h for the contract of every entry point.
#include "common.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

// ------------------------------------------------------------------ shared helpers
namespace lg {

static thread_local std::string g_last_fail;

int fail(int code, const std::string &m) {
    g_last_fail = m;
    return code;
}
const std::string &last_fail() { return g_last_fail; }
void set_global_error(const std::string &m) { g_last_fail = m; }
const char *global_error() { return g_last_fail.c_str(); }

int check_launch(const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(LOBPCG_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    return LOBPCG_OK;
}

int Allocator::alloc(void **p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) return LOBPCG_OK;
    if (cap > 0 && used + (long long)bytes > cap)
        return fail(LOBPCG_ERR_OOM, "allocation of " + std::to_string(bytes) + " bytes exceeds the memory cap");
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(LOBPCG_ERR_OOM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
    }
    used += (long long)bytes;
    return LOBPCG_OK;
}

void Allocator::free(void *p, size_t bytes) {
    if (p) {
        cudaFree(p);
        used -= (long long)bytes;
    }
}

int Allocator::ensure(DevBuf &b, size_t bytes) {
    if (b.bytes >= bytes && b.p) return LOBPCG_OK;
    release(b);
    size_t want = std::max(bytes, (size_t)256);
    LG_TRY(alloc(&b.p, want));
    b.bytes = want;
    return LOBPCG_OK;
}

void Allocator::release(DevBuf &b) {
    free(b.p, b.bytes);
    b.p = nullptr;
    b.bytes = 0;
}

}  // namespace lg

using namespace lg;

// ------------------------------------------------------------------ handle
namespace {

struct KPoint {
    double k[3];
    int npw = 0;
    std::vector<int32_t> miller;
    FFTGeom geom;
    double *kin64 = nullptr;
    float *kin32 = nullptr;
    z64 *beta64 = nullptr;  // npw x nproj
    c32 *beta32 = nullptr;
    bool has_beta = false;
};

}  // namespace

struct lobpcg_ctx {
    lobpcg_cell cell{};
    lobpcg_options opt{};
    cudaStream_t stream = nullptr;
    Allocator alloc;
    std::vector<DevBuf> owned;  // fixed tables
    int nk = 0;
    std::vector<KPoint> kp;
    FFTPlan plan;
    double *vt64 = nullptr;
    float *vt32 = nullptr;
    z64 *tw64 = nullptr;
    c32 *tw32 = nullptr;
    int nproj = 0;
    double *E64 = nullptr;
    float *E32 = nullptr;
    size_t fft_budget = (size_t)128 << 20;
    DevBuf T2, nlB, stageX, stageY;
    GemmWork gw;
    EigWork ew;
    // solver buffers
    DevBuf Zb[2], HZb[2], Z32, HZ32, HXall, Tmp, Gram, Gram2, Cbuf, dtheta, dres, dwork, Gc;
    std::string err;
};

namespace {

template <typename T>
int upload(lobpcg_ctx *c, T **dst, const T *src, size_t count) {
    DevBuf b;
    LG_TRY(c->alloc.ensure(b, sizeof(T) * std::max<size_t>(count, 1)));
    c->owned.push_back(b);
    *dst = reinterpret_cast<T *>(b.p);
    if (count) LG_CUDA_TRY(cudaMemcpy(*dst, src, sizeof(T) * count, cudaMemcpyHostToDevice));
    return LOBPCG_OK;
}

int ret(lobpcg_ctx *c, int rc) {
    if (rc < 0 && c) c->err = last_fail();
    return rc;
}

// Plane-wave sphere of one k-point, sorted by (n_x, n_y, n_z) (Sec. 2.1 basis).
int build_basis(lobpcg_ctx *c, KPoint &K) {
    const double a = c->cell.a;
    const int N = c->cell.N;
    const double two_pi = 2.0 * M_PI;
    const double r2 = 2.0 * c->cell.ecut * (a / two_pi) * (a / two_pi);
    const int lim = (int)std::ceil(std::sqrt(r2)) + 2;
    K.miller.clear();
    std::vector<double> kin;
    for (int i = -lim; i <= lim; ++i)
        for (int j = -lim; j <= lim; ++j)
            for (int l = -lim; l <= lim; ++l) {
                const double dx = i + K.k[0], dy = j + K.k[1], dz = l + K.k[2];
                if (dx * dx + dy * dy + dz * dz <= r2 + 1e-9) {
                    if (i < -N / 2 || i > N - N / 2 - 1 || j < -N / 2 || j > N - N / 2 - 1 || l < -N / 2 ||
                        l > N - N / 2 - 1)
                        return fail(LOBPCG_ERR_ARG, "plane-wave sphere does not fit in the FFT box (ecut too large for N)");
                    K.miller.push_back(i);
                    K.miller.push_back(j);
                    K.miller.push_back(l);
                    const double s = two_pi / a;
                    kin.push_back(0.5 * s * s * (dx * dx + dy * dy + dz * dz));
                }
            }
    K.npw = (int)kin.size();
    if (K.npw < 1) return fail(LOBPCG_ERR_ARG, "empty plane-wave sphere");
    // FFT geometry
    FFTGeom &g = K.geom;
    g.N = N;
    g.npw = K.npw;
    int nx_lo = 1 << 30, nx_hi = -(1 << 30), ny_lo = 1 << 30, ny_hi = -(1 << 30);
    for (int p = 0; p < K.npw; ++p) {
        nx_lo = std::min(nx_lo, K.miller[3 * p]);
        nx_hi = std::max(nx_hi, K.miller[3 * p]);
        ny_lo = std::min(ny_lo, K.miller[3 * p + 1]);
        ny_hi = std::max(ny_hi, K.miller[3 * p + 1]);
    }
    g.nx0 = nx_lo;
    g.ny0 = ny_lo;
    g.Px = nx_hi - nx_lo + 1;
    g.Py = ny_hi - ny_lo + 1;
    std::vector<int> pb(g.Px + 1, 0);
    std::vector<int2> yr(g.Px);
    for (int px = 0; px < g.Px; ++px) yr[px] = make_int2(g.Py, -1);
    std::vector<int> gm(K.npw);
    for (int p = 0; p < K.npw; ++p) {
        const int px = K.miller[3 * p] - nx_lo, py = K.miller[3 * p + 1] - ny_lo;
        const int iz = ((K.miller[3 * p + 2] % N) + N) % N;
        pb[px + 1]++;
        yr[px].x = std::min(yr[px].x, py);
        yr[px].y = std::max(yr[px].y, py);
        gm[p] = py * N + iz;
    }
    for (int px = 0; px < g.Px; ++px) {
        pb[px + 1] += pb[px];
        if (yr[px].y < 0) yr[px] = make_int2(0, -1);  // empty plane: no rows
    }
    LG_TRY(upload(c, &g.plane_begin, pb.data(), pb.size()));
    LG_TRY(upload(c, &g.plane_yrange, yr.data(), yr.size()));
    LG_TRY(upload(c, &g.gmap, gm.data(), gm.size()));
    LG_TRY(upload(c, &K.kin64, kin.data(), kin.size()));
    std::vector<float> k32(kin.begin(), kin.end());
    LG_TRY(upload(c, &K.kin32, k32.data(), k32.size()));
    if (fft_smem_need<double>(g) == 0 || fft_smem_need<float>(g) == 0)
        return fail(LOBPCG_ERR_UNSUPPORTED, "FFT grid too large for one SM's shared memory");
    return LOBPCG_OK;
}

int set_beta(lobpcg_ctx *c, int k, const void *beta) {
    KPoint &K = c->kp[k];
    if (c->nproj == 0) return LOBPCG_OK;
    const size_t cnt = (size_t)K.npw * c->nproj;
    if (!K.beta64) {
        DevBuf b64, b32;
        LG_TRY(c->alloc.ensure(b64, sizeof(z64) * cnt));
        LG_TRY(c->alloc.ensure(b32, sizeof(c32) * cnt));
        c->owned.push_back(b64);
        c->owned.push_back(b32);
        K.beta64 = reinterpret_cast<z64 *>(b64.p);
        K.beta32 = reinterpret_cast<c32 *>(b32.p);
    }
    LG_CUDA_TRY(cudaMemcpy(K.beta64, beta, sizeof(z64) * cnt, cudaMemcpyHostToDevice));
    LG_TRY(copy_cast<float, double>(K.npw, c->nproj, K.beta64, K.npw, K.beta32, K.npw, c->stream));
    LG_CUDA_TRY(cudaStreamSynchronize(c->stream));
    K.has_beta = true;
    return LOBPCG_OK;
}

template <typename R> struct Tables;
template <> struct Tables<double> {
    static const double *kin(const KPoint &K) { return K.kin64; }
    static const z64 *beta(const KPoint &K) { return K.beta64; }
    static const double *vt(const lobpcg_ctx *c) { return c->vt64; }
    static const z64 *tw(const lobpcg_ctx *c) { return c->tw64; }
    static const double *E(const lobpcg_ctx *c) { return c->E64; }
};
template <> struct Tables<float> {
    static const float *kin(const KPoint &K) { return K.kin32; }
    static const c32 *beta(const KPoint &K) { return K.beta32; }
    static const float *vt(const lobpcg_ctx *c) { return c->vt32; }
    static const c32 *tw(const lobpcg_ctx *c) { return c->tw32; }
    static const float *E(const lobpcg_ctx *c) { return c->E32; }
};

// Y = H X on device buffers (Sec. 2.2 items iii and iv): FFT route for
// T + V_loc, then the KB projection B = beta^H X, B <- E B, Y += beta B.
template <typename R>
int apply_H_dev(lobpcg_ctx *c, int k, const cx<R> *X, int ldx, cx<R> *Y, int ldy, int nb) {
    if (nb <= 0) return LOBPCG_OK;
    KPoint &K = c->kp[k];
    const FFTGeom &g = K.geom;
    const size_t per_band = sizeof(cx<R>) * (size_t)g.Px * g.N * g.N;
    int nbatch = (int)std::max<size_t>(1, c->fft_budget / per_band);
    nbatch = std::min(std::min(nbatch, nb), 65535);
    LG_TRY(c->alloc.ensure(c->T2, per_band * nbatch));
    LG_TRY(fft_vloc_apply<R>(g, c->plan, X, ldx, Y, ldy, nb, Tables<R>::kin(K), Tables<R>::vt(c),
                             Tables<R>::tw(c), reinterpret_cast<cx<R> *>(c->T2.p), nbatch, c->stream));
    if (c->nproj > 0) {
        if (!K.has_beta) return fail(LOBPCG_ERR_ARG, "projectors of this k-point were not given");
        LG_TRY(c->alloc.ensure(c->nlB, sizeof(cx<R>) * (size_t)c->nproj * nb));
        cx<R> *B = reinterpret_cast<cx<R> *>(c->nlB.p);
        const cx<R> *beta = Tables<R>::beta(K);
        LG_TRY(gemm_cn<R>(c->gw, c->nproj, nb, K.npw, (R)1, beta, K.npw, X, ldx, (R)0, B, c->nproj, c->stream));
        LG_TRY(scale_rows<R>(c->nproj, nb, Tables<R>::E(c), B, c->nproj, c->stream));
        LG_TRY(gemm_nn<R>(K.npw, nb, c->nproj, (R)1, beta, K.npw, B, c->nproj, (R)1, Y, ldy, Y, ldy, c->stream));
    }
    return LOBPCG_OK;
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// ------------------------------------------------------------------ LOBPCG driver
struct Solver {
    lobpcg_ctx *c;
    int k, npw, M, m, nblk;
    bool mixed;
    z64 *X;  // user block, npw x M
    z64 *Z[2], *HZ[2];
    c32 *Z32, *HZ32;
    z64 *HX, *Tmp, *S, *A, *C, *G;
    double *theta, *res, *work;
    int *ndrop;
    double drop_tol;
    long long applies64 = 0, applies32 = 0;
    int iterations = 0;
    cudaStream_t s;

    z64 *col(z64 *base, int j) const { return base + (size_t)j * npw; }

    int applyH64(const z64 *Xin, z64 *Yout, int nb) {
        applies64 += nb;
        return apply_H_dev<double>(c, k, Xin, npw, Yout, npw, nb);
    }
    // H W in FP32 for the mixed schedule: W is rounded to complex64 first and the
    // rounded W is kept in the basis so that W and HW stay consistent.
    int applyH32_inplace(z64 *W, z64 *HW, int nb) {
        applies32 += nb;
        LG_TRY(copy_cast<float, double>(npw, nb, W, npw, Z32, npw, s));
        LG_TRY(copy_cast<double, float>(npw, nb, Z32, npw, W, npw, s));
        LG_TRY(apply_H_dev<float>(c, k, Z32, npw, HZ32, npw, nb));
        return copy_cast<double, float>(npw, nb, HZ32, npw, HW, npw, s);
    }

    // V <- V - Y (Y^H V), twice (classical Gram-Schmidt repeated); Y = first j bands.
    int constrain(z64 *V, int nv, int j) {
        if (j <= 0) return LOBPCG_OK;
        for (int rep = 0; rep < 2; ++rep) {
            LG_TRY(gemm_cn<double>(c->gw, j, nv, npw, 1.0, X, npw, V, npw, 0.0, G, j, s));
            LG_TRY(gemm_nn<double>(npw, nv, j, -1.0, X, npw, G, j, 1.0, V, npw, V, npw, s));
        }
        return LOBPCG_OK;
    }

    int gram(const z64 *Zc, const z64 *HZc, int nz) {
        LG_TRY(gemm_cn<double>(c->gw, nz, nz, npw, 1.0, Zc, npw, Zc, npw, 0.0, S, nz, s));
        return gemm_cn<double>(c->gw, nz, nz, npw, 1.0, Zc, npw, HZc, npw, 0.0, A, nz, s);
    }

    int block(int b) {
        int cur = 0;
        z64 *Xu = col(X, b * m);
        LG_CUDA_TRY(cudaMemcpyAsync(Z[cur], Xu, sizeof(z64) * (size_t)npw * m, cudaMemcpyDeviceToDevice, s));
        LG_TRY(constrain(Z[cur], m, b * m));
        LG_TRY(applyH64(Z[cur], HZ[cur], m));
        // Rayleigh-Ritz on the block alone: orthonormal Ritz basis, Upsilon (step 1)
        LG_TRY(gram(Z[cur], HZ[cur], m));
        LG_TRY(rayleigh_ritz(c->ew, m, m, S, m, A, m, drop_tol, theta, C, m, ndrop, s));
        LG_TRY(gemm_nn<double>(npw, m, m, 1.0, Z[cur], npw, C, m, 0.0, nullptr, npw, Z[1 - cur], npw, s));
        LG_TRY(gemm_nn<double>(npw, m, m, 1.0, HZ[cur], npw, C, m, 0.0, nullptr, npw, HZ[1 - cur], npw, s));
        cur = 1 - cur;
        int nP = 0;
        for (int it = 0; it < c->opt.nline; ++it) {
            z64 *Zc = Z[cur], *HZc = HZ[cur];
            z64 *W = col(Zc, m), *HW = col(HZc, m);
            // steps 2-3: R = HX - X Upsilon, W = K(R); constraint against earlier blocks
            LG_TRY(residual_precond<double>(npw, m, Zc, npw, HZc, npw, theta, c->kp[k].kin64, W, npw, work, s));
            LG_TRY(constrain(W, m, b * m));
            if (mixed) {
                LG_TRY(applyH32_inplace(W, HW, m));
            } else {
                LG_TRY(applyH64(W, HW, m));
            }
            // step 4: Rayleigh-Ritz on span[X, W, P]
            const int nz = (2 + nP) * m;
            LG_TRY(gram(Zc, HZc, nz));
            LG_TRY(rayleigh_ritz(c->ew, nz, m, S, nz, A, nz, drop_tol, theta, C, nz, ndrop, s));
            // steps 4-5: P = W Lambda + P Gamma, X = X Delta + P (and H images)
            z64 *Zn = Z[1 - cur], *HZn = HZ[1 - cur];
            LG_TRY(gemm_nn<double>(npw, m, nz - m, 1.0, col(Zc, m), npw, C + m, nz, 0.0, nullptr, npw, col(Zn, 2 * m),
                                   npw, s));
            LG_TRY(gemm_nn<double>(npw, m, m, 1.0, Zc, npw, C, nz, 1.0, col(Zn, 2 * m), npw, Zn, npw, s));
            LG_TRY(gemm_nn<double>(npw, m, nz - m, 1.0, col(HZc, m), npw, C + m, nz, 0.0, nullptr, npw,
                                   col(HZn, 2 * m), npw, s));
            LG_TRY(gemm_nn<double>(npw, m, m, 1.0, HZc, npw, C, nz, 1.0, col(HZn, 2 * m), npw, HZn, npw, s));
            cur = 1 - cur;
            nP = 1;
            ++iterations;
        }
        LG_CUDA_TRY(cudaMemcpyAsync(Xu, Z[cur], sizeof(z64) * (size_t)npw * m, cudaMemcpyDeviceToDevice, s));
        LG_CUDA_TRY(cudaMemcpyAsync(col(HX, b * m), HZ[cur], sizeof(z64) * (size_t)npw * m, cudaMemcpyDeviceToDevice, s));
        return LOBPCG_OK;
    }

    // Rayleigh-Ritz over all M bands closing a sweep (Sec. 3.2), then FP64 residuals.
    int final_rr(double *eig_h, double *res_h) {
        if (mixed) LG_TRY(applyH64(X, HX, M));  // FP64 refresh of H X for the residual test
        LG_TRY(gemm_cn<double>(c->gw, M, M, npw, 1.0, X, npw, X, npw, 0.0, S, M, s));
        LG_TRY(gemm_cn<double>(c->gw, M, M, npw, 1.0, X, npw, HX, npw, 0.0, A, M, s));
        LG_TRY(rayleigh_ritz(c->ew, M, M, S, M, A, M, drop_tol, theta, C, M, ndrop, s));
        LG_TRY(gemm_nn<double>(npw, M, M, 1.0, X, npw, C, M, 0.0, nullptr, npw, Tmp, npw, s));
        LG_CUDA_TRY(cudaMemcpyAsync(X, Tmp, sizeof(z64) * (size_t)npw * M, cudaMemcpyDeviceToDevice, s));
        LG_TRY(gemm_nn<double>(npw, M, M, 1.0, HX, npw, C, M, 0.0, nullptr, npw, Tmp, npw, s));
        LG_CUDA_TRY(cudaMemcpyAsync(HX, Tmp, sizeof(z64) * (size_t)npw * M, cudaMemcpyDeviceToDevice, s));
        LG_TRY(column_resid_norms(npw, M, X, npw, HX, npw, theta, res, s));
        LG_CUDA_TRY(cudaMemcpyAsync(eig_h, theta, sizeof(double) * M, cudaMemcpyDeviceToHost, s));
        LG_CUDA_TRY(cudaMemcpyAsync(res_h, res, sizeof(double) * M, cudaMemcpyDeviceToHost, s));
        LG_CUDA_TRY(cudaStreamSynchronize(s));
        return LOBPCG_OK;
    }
};

template <typename T>
T *carve(lobpcg_ctx *c, DevBuf &b, size_t count, int &rc) {
    rc = c->alloc.ensure(b, sizeof(T) * std::max<size_t>(count, 1));
    return reinterpret_cast<T *>(b.p);
}

int solve_k(lobpcg_ctx *c, int k, int M, z64 *X, double *eig_h, double *res_h, int &sweeps_done, long long &a64,
            long long &a32, int &iters) {
    Solver sv;
    sv.c = c;
    sv.k = k;
    sv.npw = c->kp[k].npw;
    sv.M = M;
    sv.m = c->opt.block_size;
    sv.nblk = M / sv.m;
    sv.mixed = c->opt.precision == LOBPCG_MIXED;
    sv.X = X;
    sv.s = c->stream;
    sv.drop_tol = sv.mixed ? 1e-10 : 1e-12;
    const int npw = sv.npw, m = sv.m;
    const int nzmax = std::max(3 * m, M);
    int rc = 0;
    for (int i = 0; i < 2; ++i) {
        sv.Z[i] = carve<z64>(c, c->Zb[i], (size_t)npw * 3 * m, rc);
        LG_TRY(rc);
        sv.HZ[i] = carve<z64>(c, c->HZb[i], (size_t)npw * 3 * m, rc);
        LG_TRY(rc);
    }
    sv.Z32 = carve<c32>(c, c->Z32, (size_t)npw * m, rc); LG_TRY(rc);
    sv.HZ32 = carve<c32>(c, c->HZ32, (size_t)npw * m, rc); LG_TRY(rc);
    sv.HX = carve<z64>(c, c->HXall, (size_t)npw * M, rc); LG_TRY(rc);
    sv.Tmp = carve<z64>(c, c->Tmp, (size_t)npw * M, rc); LG_TRY(rc);
    sv.S = carve<z64>(c, c->Gram, (size_t)nzmax * nzmax, rc); LG_TRY(rc);
    sv.A = carve<z64>(c, c->Gram2, (size_t)nzmax * nzmax, rc); LG_TRY(rc);
    sv.C = carve<z64>(c, c->Cbuf, (size_t)nzmax * nzmax, rc); LG_TRY(rc);
    sv.G = carve<z64>(c, c->Gc, (size_t)M * m, rc); LG_TRY(rc);
    sv.theta = carve<double>(c, c->dtheta, nzmax, rc); LG_TRY(rc);
    sv.res = carve<double>(c, c->dres, nzmax, rc); LG_TRY(rc);
    double *w = carve<double>(c, c->dwork, 4 * (size_t)nzmax + 64, rc); LG_TRY(rc);
    sv.work = w;
    sv.ndrop = reinterpret_cast<int *>(w + 4 * (size_t)nzmax);
    sweeps_done = 0;
    double maxr = 0.0;
    for (int sw = 0; sw < c->opt.max_sweeps; ++sw) {
        for (int b = 0; b < sv.nblk; ++b) LG_TRY(sv.block(b));
        LG_TRY(sv.final_rr(eig_h, res_h));
        ++sweeps_done;
        maxr = 0.0;
        for (int i = 0; i < M; ++i) maxr = std::max(maxr, res_h[i]);
        if (!(maxr == maxr)) return fail(LOBPCG_ERR_BREAKDOWN, "non-finite residual");
        if (maxr <= c->opt.tol) break;
    }
    a64 += sv.applies64;
    a32 += sv.applies32;
    iters += sv.iterations;
    return maxr <= c->opt.tol ? LOBPCG_OK : LOBPCG_NOT_CONVERGED;
}

int validate_options(const lobpcg_options &o) {
    if (o.block_size < 1) return fail(LOBPCG_ERR_ARG, "block_size must be >= 1");
    if (o.nline < 1) return fail(LOBPCG_ERR_ARG, "nline must be >= 1");
    if (o.max_sweeps < 1) return fail(LOBPCG_ERR_ARG, "max_sweeps must be >= 1");
    if (o.precision != LOBPCG_FP64 && o.precision != LOBPCG_MIXED) return fail(LOBPCG_ERR_ARG, "unknown precision");
    if (!(o.tol > 0.0)) return fail(LOBPCG_ERR_ARG, "tol must be > 0");
    if (3 * o.block_size > 4096) return fail(LOBPCG_ERR_ARG, "block_size too large (3 m must be <= 4096)");
    return LOBPCG_OK;
}

}  // namespace

// ------------------------------------------------------------------ C ABI
extern "C" {

int lobpcg_default_options(lobpcg_options *opt) {
    if (!opt) return fail(LOBPCG_ERR_ARG, "opt is NULL");
    std::memset(opt, 0, sizeof(*opt));
    opt->block_size = 64;
    opt->nline = 4;
    opt->max_sweeps = 100;
    opt->precision = LOBPCG_FP64;
    opt->gemm_split = 0;
    opt->use_graph = 0;
    opt->autotune = 0;
    opt->tol = 1e-8;
    opt->mem_cap = 0;
    return LOBPCG_OK;
}

static int create_impl(lobpcg_ctx *c, const lobpcg_cell *cell, int nk, const double *kpts, const double *vloc_r,
                       int nproj, const double *proj_E, const void *const *beta) {
    if (!cell || !kpts || !vloc_r) return fail(LOBPCG_ERR_ARG, "cell, kpts and vloc_r must not be NULL");
    if (!(cell->a > 0.0) || !(cell->ecut > 0.0)) return fail(LOBPCG_ERR_ARG, "a and ecut must be > 0");
    if (nk < 1) return fail(LOBPCG_ERR_ARG, "nk must be >= 1");
    if (nproj < 0 || (nproj > 0 && !proj_E)) return fail(LOBPCG_ERR_ARG, "bad projector arguments");
    if (cell->N < 4 || cell->N > 256 || !make_fft_plan(cell->N, c->plan))
        return fail(LOBPCG_ERR_UNSUPPORTED, "N must be a product of 2, 3 and 5 in [4, 256]");
    c->cell = *cell;
    c->nk = nk;
    c->nproj = nproj;
    const int N = cell->N;
    // potential: [x][y][z] -> [z][x][y], scaled by 1/N^3 (the forward FFT's normalisation)
    const size_t N3 = (size_t)N * N * N;
    std::vector<double> vt(N3);
    std::vector<float> vt32(N3);
    const double inv = 1.0 / (double)N3;
    for (int x = 0; x < N; ++x)
        for (int y = 0; y < N; ++y)
            for (int z = 0; z < N; ++z) {
                const double v = vloc_r[((size_t)x * N + y) * N + z] * inv;
                if (!std::isfinite(v)) return fail(LOBPCG_ERR_ARG, "vloc_r has non-finite values");
                vt[((size_t)z * N + x) * N + y] = v;
                vt32[((size_t)z * N + x) * N + y] = (float)v;
            }
    LG_TRY(upload(c, &c->vt64, vt.data(), N3));
    LG_TRY(upload(c, &c->vt32, vt32.data(), N3));
    // twiddles e^{-2 pi i t/N}, FP64 on the host, rounded for FP32
    std::vector<z64> tw(N);
    std::vector<c32> tw32(N);
    for (int t = 0; t < N; ++t) {
        const long double ang = -2.0L * 3.141592653589793238462643383279502884L * (long double)t / (long double)N;
        tw[t] = mkc<double>((double)std::cos(ang), (double)std::sin(ang));
        tw32[t] = mkc<float>((float)tw[t].x, (float)tw[t].y);
    }
    LG_TRY(upload(c, &c->tw64, tw.data(), N));
    LG_TRY(upload(c, &c->tw32, tw32.data(), N));
    if (nproj > 0) {
        std::vector<float> e32(proj_E, proj_E + nproj);
        LG_TRY(upload(c, &c->E64, proj_E, nproj));
        LG_TRY(upload(c, &c->E32, e32.data(), nproj));
    }
    c->kp.resize(nk);
    for (int k = 0; k < nk; ++k) {
        for (int d = 0; d < 3; ++d) {
            c->kp[k].k[d] = kpts[3 * k + d];
            if (!std::isfinite(kpts[3 * k + d])) return fail(LOBPCG_ERR_ARG, "non-finite k-point");
        }
        LG_TRY(build_basis(c, c->kp[k]));
    }
    c->gw.alloc = &c->alloc;
    c->ew.alloc = &c->alloc;
    c->ew.gw.alloc = &c->alloc;
    if (beta && nproj > 0) {
        for (int k = 0; k < nk; ++k)
            if (beta[k]) LG_TRY(set_beta(c, k, beta[k]));
    }
    return LOBPCG_OK;
}

int lobpcg_create(lobpcg_ctx **out, const lobpcg_cell *cell, int nk, const double *kpts, const double *vloc_r,
                  int nproj, const double *proj_E, const void *const *beta, const lobpcg_options *opt,
                  void *stream) {
    if (!out) return fail(LOBPCG_ERR_ARG, "out is NULL");
    *out = nullptr;
    std::unique_ptr<lobpcg_ctx> c(new lobpcg_ctx());
    lobpcg_default_options(&c->opt);
    if (opt) {
        LG_TRY(validate_options(*opt));
        c->opt = *opt;
    }
    c->alloc.cap = c->opt.mem_cap;
    c->stream = reinterpret_cast<cudaStream_t>(stream);
    int rc = create_impl(c.get(), cell, nk, kpts, vloc_r, nproj, proj_E, beta);
    if (rc < 0) {
        lobpcg_destroy(c.release());
        return rc;
    }
    *out = c.release();
    return LOBPCG_OK;
}

int lobpcg_set_projectors(lobpcg_ctx *ctx, int k, const void *beta_k) {
    if (!ctx) return fail(LOBPCG_ERR_ARG, "ctx is NULL");
    if (k < 0 || k >= ctx->nk) return ret(ctx, fail(LOBPCG_ERR_ARG, "k out of range"));
    if (ctx->nproj == 0) return LOBPCG_OK;
    if (!beta_k) return ret(ctx, fail(LOBPCG_ERR_ARG, "beta_k is NULL"));
    return ret(ctx, set_beta(ctx, k, beta_k));
}

int lobpcg_set_stream(lobpcg_ctx *ctx, void *stream) {
    if (!ctx) return fail(LOBPCG_ERR_ARG, "ctx is NULL");
    ctx->stream = reinterpret_cast<cudaStream_t>(stream);
    return LOBPCG_OK;
}

int lobpcg_set_options(lobpcg_ctx *ctx, const lobpcg_options *opt) {
    if (!ctx || !opt) return fail(LOBPCG_ERR_ARG, "ctx or opt is NULL");
    int rc = validate_options(*opt);
    if (rc < 0) return ret(ctx, rc);
    ctx->opt = *opt;
    ctx->alloc.cap = opt->mem_cap;
    return LOBPCG_OK;
}

int lobpcg_npw(const lobpcg_ctx *ctx, int k) {
    if (!ctx) return fail(LOBPCG_ERR_ARG, "ctx is NULL");
    if (k < 0 || k >= ctx->nk) return fail(LOBPCG_ERR_ARG, "k out of range");
    return ctx->kp[k].npw;
}

int lobpcg_gvectors(const lobpcg_ctx *ctx, int k, int32_t *miller) {
    if (!ctx || !miller) return fail(LOBPCG_ERR_ARG, "ctx or miller is NULL");
    if (k < 0 || k >= ctx->nk) return fail(LOBPCG_ERR_ARG, "k out of range");
    std::memcpy(miller, ctx->kp[k].miller.data(), sizeof(int32_t) * ctx->kp[k].miller.size());
    return LOBPCG_OK;
}

static int apply_impl(lobpcg_ctx *c, int k, const void *X, void *Y, int nb, int precision) {
    if (k < 0 || k >= c->nk) return fail(LOBPCG_ERR_ARG, "k out of range");
    if (nb < 0) return fail(LOBPCG_ERR_ARG, "nb must be >= 0");
    if (nb == 0) return LOBPCG_OK;
    if (!X || !Y) return fail(LOBPCG_ERR_ARG, "X and Y must not be NULL");
    if (precision != LOBPCG_C128 && precision != LOBPCG_C64) return fail(LOBPCG_ERR_ARG, "unknown precision");
    const int npw = c->kp[k].npw;
    const size_t esz = precision == LOBPCG_C128 ? sizeof(z64) : sizeof(c32);
    const size_t bytes = esz * (size_t)npw * nb;
    const char *xa = static_cast<const char *>(X), *ya = static_cast<const char *>(Y);
    if (xa < ya + bytes && ya < xa + bytes) return fail(LOBPCG_ERR_ARG, "X and Y overlap");
    const bool dx = is_device_ptr(X), dy = is_device_ptr(Y);
    const void *Xd = X;
    void *Yd = Y;
    if (!dx) {
        LG_TRY(c->alloc.ensure(c->stageX, bytes));
        LG_CUDA_TRY(cudaMemcpyAsync(c->stageX.p, X, bytes, cudaMemcpyHostToDevice, c->stream));
        Xd = c->stageX.p;
    }
    if (!dy) {
        LG_TRY(c->alloc.ensure(c->stageY, bytes));
        Yd = c->stageY.p;
    }
    if (precision == LOBPCG_C128)
        LG_TRY(apply_H_dev<double>(c, k, static_cast<const z64 *>(Xd), npw, static_cast<z64 *>(Yd), npw, nb));
    else
        LG_TRY(apply_H_dev<float>(c, k, static_cast<const c32 *>(Xd), npw, static_cast<c32 *>(Yd), npw, nb));
    if (!dy) {
        LG_CUDA_TRY(cudaMemcpyAsync(Y, Yd, bytes, cudaMemcpyDeviceToHost, c->stream));
    }
    if (!dx || !dy) LG_CUDA_TRY(cudaStreamSynchronize(c->stream));
    return LOBPCG_OK;
}

int lobpcg_apply_H(lobpcg_ctx *ctx, int k, const void *X, void *Y, int nb, int precision) {
    if (!ctx) return fail(LOBPCG_ERR_ARG, "ctx is NULL");
    return ret(ctx, apply_impl(ctx, k, X, Y, nb, precision));
}

static int solve_impl(lobpcg_ctx *c, int M, void *const *X, double *eig, double *resid, lobpcg_stats *st) {
    if (!X || !eig || !resid) return fail(LOBPCG_ERR_ARG, "X, eig and resid must not be NULL");
    const int m = c->opt.block_size;
    if (M < 1 || M % m) return fail(LOBPCG_ERR_ARG, "nbands must be a positive multiple of block_size");
    for (int k = 0; k < c->nk; ++k) {
        if (!X[k]) return fail(LOBPCG_ERR_ARG, "X[k] is NULL");
        if (M > c->kp[k].npw) return fail(LOBPCG_ERR_ARG, "nbands exceeds the plane-wave count");
        if (c->nproj > 0 && !c->kp[k].has_beta) return fail(LOBPCG_ERR_ARG, "projectors missing for a k-point");
        if (!is_device_ptr(X[k])) return fail(LOBPCG_ERR_ARG, "X[k] must be a device pointer");
    }
    const auto t0 = std::chrono::steady_clock::now();
    int worst = LOBPCG_OK, sweeps = 0, iters = 0;
    long long a64 = 0, a32 = 0;
    double maxr = 0.0;
    for (int k = 0; k < c->nk; ++k) {
        int sw = 0;
        int rc = solve_k(c, k, M, static_cast<z64 *>(X[k]), eig + (size_t)k * M, resid + (size_t)k * M, sw, a64, a32,
                         iters);
        if (rc < 0) return rc;
        if (rc == LOBPCG_NOT_CONVERGED) worst = rc;
        sweeps = std::max(sweeps, sw);
        for (int i = 0; i < M; ++i) maxr = std::max(maxr, resid[(size_t)k * M + i]);
    }
    if (st) {
        std::memset(st, 0, sizeof(*st));
        st->sweeps = sweeps;
        st->iterations = iters;
        st->converged = worst == LOBPCG_OK;
        st->max_resid = maxr;
        st->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        st->band_applies_fp64 = a64;
        st->band_applies_fp32 = a32;
    }
    return worst;
}

int lobpcg_solve(lobpcg_ctx *ctx, int nbands, void *const *X, double *eig, double *resid, lobpcg_stats *stats) {
    if (!ctx) return fail(LOBPCG_ERR_ARG, "ctx is NULL");
    return ret(ctx, solve_impl(ctx, nbands, X, eig, resid, stats));
}

const char *lobpcg_last_error(const lobpcg_ctx *ctx) {
    if (!ctx) return global_error();
    return ctx->err.c_str();
}

void lobpcg_destroy(lobpcg_ctx *ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    for (auto &b : ctx->owned) ctx->alloc.release(b);
    DevBuf *bufs[] = {&ctx->T2, &ctx->nlB, &ctx->stageX, &ctx->stageY, &ctx->Zb[0], &ctx->Zb[1], &ctx->HZb[0],
                      &ctx->HZb[1], &ctx->Z32, &ctx->HZ32, &ctx->HXall, &ctx->Tmp, &ctx->Gram, &ctx->Gram2,
                      &ctx->Cbuf, &ctx->dtheta, &ctx->dres, &ctx->dwork, &ctx->Gc, &ctx->gw.part, &ctx->ew.buf,
                      &ctx->ew.ibuf, &ctx->ew.gw.part};
    for (DevBuf *b : bufs) ctx->alloc.release(*b);
    delete ctx;
}

}  // extern "C"
