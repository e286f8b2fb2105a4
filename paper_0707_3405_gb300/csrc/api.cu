// C ABI of the GB300 LOBPCG plane-wave eigensolver: handle, plane-wave basis,
// H application and the block LOBPCG driver (Bottin, Leroux, Knyazev, Zerah
// 2007).  See include/lobpcg_gb300.h for the contract of every entry point.
#include "common.cuh"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <thread>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <tuple>
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

static std::atomic<long long> g_launches{0};
long long launch_count() { return g_launches.load(); }
// Correct the count for kernels recorded into a CUDA graph (not run) or run from one.
static void add_launches(long long d) { g_launches.fetch_add(d, std::memory_order_relaxed); }

int check_launch(const char *what) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(LOBPCG_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    return LOBPCG_OK;
}

cudaEvent_t Prof::get() {
    if (!pool.empty()) {
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

cudaEvent_t Prof::begin(int) {
    if (!on) return nullptr;
    cudaEvent_t a = get();
    if (a) cudaEventRecord(a, s);
    return a;
}

void Prof::end(int ph, cudaEvent_t a, double fl, double by, bool fp64) {
    if (!on) return;
    flops[ph] += fl;
    bytes[ph] += by;
    if (fp64) {
        fp64_flops[ph] += fl;
        bytes64[ph] += by;
    }
    calls[ph] += 1;
    cudaEvent_t b = get();
    if (!a || !b) return;
    cudaEventRecord(b, s);
    recs.push_back({ph, fp64, a, b});
    if (recs.size() > 4096) collect();
}

void Prof::collect() {
    if (recs.empty()) return;
    cudaEventSynchronize(recs.back().b);
    for (auto &r : recs) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
            ms[r.ph] += t;
            if (r.f64) ms64[r.ph] += t;
        } else {
            cudaGetLastError();
        }
        pool.push_back(r.a);
        pool.push_back(r.b);
    }
    recs.clear();
}

Prof::~Prof() {
    collect();
    for (auto e : pool) cudaEventDestroy(e);
}

int Allocator::alloc(void **p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) return LOBPCG_OK;
    // reserve first, so that concurrent lanes cannot pass the cap check together
    const long long before = used.fetch_add((long long)bytes);
    if (cap > 0 && before + (long long)bytes > cap) {
        used -= (long long)bytes;
        return fail(LOBPCG_ERR_OOM, "allocation of " + std::to_string(bytes) + " bytes exceeds the memory cap");
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        used -= (long long)bytes;
        cudaGetLastError();
        *p = nullptr;
        return fail(LOBPCG_ERR_OOM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
    }
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
    // FFT scratch budget per band batch (bytes; 0 = the handle default), chosen by the autotuner
    size_t fft_budget32 = 0, fft_budget64 = 0;
    bool tuned = false;
    // Gamma point: packed half-sphere tables of the real form (see gamma_pack_full)
    bool gamma = false;
    int n_half = 0;
    int *half = nullptr, *mirror = nullptr;
    double *kin_half64 = nullptr;
};

// Everything one k-point solve (or one apply_H call) writes: scratch, solver buffers and the
// stream it runs on.  Lane 0 serves apply_H on the handle's stream and runs a solve on its own
// high-priority stream; a multi-k solve adds lanes with their own streams so that k-points
// proceed concurrently.
struct Lane {
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    DevBuf T2, nlB, stageX, stageY;
    GemmWork gw;
    EigWork ew;
    DevBuf Zb[2], HZb[2], Z32, HZ32, HXall, Tmp, Gram, Gram2, Cbuf, dtheta, dres, dwork, Gc;
    DevBuf occ;  // occupations of a density call (FP64, then FP32)
    DevBuf pcgv, pcgs;  // PCG: seven band vectors, reduction and scalar scratch
    DevBuf rfi, rfo, Xpk;  // Gamma real form: sphere pairs in / out of an H application, packed X
    DevBuf X32all, HX32all, Q32[2], HQ32[2], D32, Small32, Xext, T32, E32;
    // CUDA graphs of the FP32 H application on fixed buffers (options.use_graph), keyed by
    // (k, X, Y, nb); a graph is only replayed while the scratch it recorded is still in place
    struct Graph {
        cudaGraphExec_t exec = nullptr;
        long long kernels = 0;
        const void *t2 = nullptr, *nlb = nullptr, *part = nullptr;
    };
    std::map<std::tuple<int, const void *, void *, int>, Graph> graphs;
    // Beside a full mixed sweep, each block's FP64-class H X is recomputed on a side stream with its
    // own scratch (side) into HXr, overlapping the latency-bound Rayleigh-Ritz steps of the later
    // blocks; the sweep end swaps it in.
    DevBuf HXr;
    std::unique_ptr<Lane> side;
    cudaStream_t solve_stream = nullptr;  // lane 0's own high-priority stream during a solve
    cudaEvent_t ev_main = nullptr, ev_side = nullptr;
    int make_side(Allocator *a) {
        if (!side) {
            // lowest priority: its blocks fill the gaps the solve's own kernels leave
            int least = 0, greatest = 0;
            LG_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&least, &greatest));
            side.reset(new Lane());
            LG_CUDA_TRY(cudaStreamCreateWithPriority(&side->stream, cudaStreamNonBlocking, least));
            side->own_stream = true;
        }
        side->bind(a, nullptr, 1);
        if (!ev_main) LG_CUDA_TRY(cudaEventCreateWithFlags(&ev_main, cudaEventDisableTiming));
        if (!ev_side) LG_CUDA_TRY(cudaEventCreateWithFlags(&ev_side, cudaEventDisableTiming));
        return LOBPCG_OK;
    }
    void clear_graphs() {
        for (auto &g : graphs)
            if (g.second.exec) cudaGraphExecDestroy(g.second.exec);
        graphs.clear();
    }
    void bind(Allocator *a, CoopGate *g, int share) {
        gw.alloc = a;
        ew.alloc = a;
        ew.gw.alloc = a;
        ew.gate = g;
        ew.coop_share = share;
    }
    void release(Allocator &a) {
        DevBuf *bufs[] = {&T2, &nlB, &stageX, &stageY, &Zb[0], &Zb[1], &HZb[0], &HZb[1], &Z32, &HZ32, &HXall,
                          &Tmp, &Gram, &Gram2, &Cbuf, &dtheta, &dres, &dwork, &Gc, &gw.part, &ew.buf, &ew.ibuf,
                          &ew.gw.part, &X32all, &HX32all, &Q32[0], &Q32[1], &HQ32[0], &HQ32[1], &D32, &Small32,
                          &Xext, &T32, &E32, &occ, &gw.oz_a, &gw.oz_e, &gw.oz_p, &pcgv, &pcgs, &rfi, &rfo,
                          &Xpk};
        clear_graphs();
        for (DevBuf *b : bufs) a.release(*b);
        a.release(HXr);
        if (side) {
            if (side->stream) cudaStreamSynchronize(side->stream);
            side->release(a);
            side.reset();
        }
        if (ev_main) cudaEventDestroy(ev_main);
        if (ev_side) cudaEventDestroy(ev_side);
        ev_main = ev_side = nullptr;
        if (solve_stream) cudaStreamDestroy(solve_stream);
        solve_stream = nullptr;
        if (own_stream && stream) cudaStreamDestroy(stream);
        stream = nullptr;
    }
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
    float2 *vtdf = nullptr;   // vt64 as (hi, lo) FP32 pairs, for the double-FP32 FFT passes
    float *vt32 = nullptr;
    z64 *tw64 = nullptr;
    c32 *tw32 = nullptr;
    int nproj = 0;
    double *E64 = nullptr;
    float *E32 = nullptr;
    size_t fft_budget = (size_t)128 << 20;
    int device = 0;
    std::vector<std::unique_ptr<Lane>> lanes;  // lanes[0]: apply_H on the handle's stream
    CoopGate gate;
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
    K.gamma = K.k[0] == 0.0 && K.k[1] == 0.0 && K.k[2] == 0.0;
    if (K.gamma) {
        // half set {0} u S+ (S+: n_x > 0, or n_x = 0 and n_y > 0, or n_x = n_y = 0 and n_z > 0),
        // G = 0 first, then S+ in sphere order; the sphere holds -G with every G
        std::map<std::tuple<int, int, int>, int> pos;
        for (int p = 0; p < K.npw; ++p) pos[std::make_tuple(K.miller[3 * p], K.miller[3 * p + 1], K.miller[3 * p + 2])] = p;
        std::vector<int> hv, mv;
        std::vector<double> kh;
        const auto z = pos.find(std::make_tuple(0, 0, 0));
        if (z == pos.end()) return fail(LOBPCG_ERR_ARG, "Gamma sphere without G = 0");
        hv.push_back(z->second);
        mv.push_back(z->second);
        kh.push_back(kin[z->second]);
        for (int p = 0; p < K.npw; ++p) {
            const int a = K.miller[3 * p], b = K.miller[3 * p + 1], d = K.miller[3 * p + 2];
            if (!(a > 0 || (a == 0 && b > 0) || (a == 0 && b == 0 && d > 0))) continue;
            const auto q = pos.find(std::make_tuple(-a, -b, -d));
            if (q == pos.end()) return fail(LOBPCG_ERR_ARG, "Gamma sphere not symmetric under G -> -G");
            hv.push_back(p);
            mv.push_back(q->second);
            kh.push_back(kin[p]);
        }
        K.n_half = (int)hv.size();
        LG_TRY(upload(c, &K.half, hv.data(), hv.size()));
        LG_TRY(upload(c, &K.mirror, mv.data(), mv.size()));
        LG_TRY(upload(c, &K.kin_half64, kh.data(), kh.size()));
    }
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
int apply_H_dev(lobpcg_ctx *c, Lane &L, int k, const cx<R> *X, int ldx, cx<R> *Y, int ldy, int nb,
                Prof *prof = nullptr, bool df = false) {
    if (nb <= 0) return LOBPCG_OK;
    KPoint &K = c->kp[k];
    const FFTGeom &g = K.geom;
    const bool f64 = sizeof(R) == 8;
    const size_t cb = sizeof(cx<R>);
    const size_t per_band = cb * (size_t)g.Px * g.N * g.N;
    const size_t kb = f64 ? K.fft_budget64 : K.fft_budget32;
    int nbatch = (int)std::max<size_t>(1, (kb ? kb : c->fft_budget) / per_band);
    nbatch = std::min(std::min(nbatch, nb), 65535);
    LG_TRY(c->alloc.ensure(L.T2, per_band * nbatch));
    {
        // algorithmic DRAM bytes: sphere X read twice (scatter, kinetic), Y written,
        // kinetic table, half-box written / read-written / read (4 Px N^2), V once per batch
        const double by = nb * (3.0 * cb * K.npw + sizeof(R) * (double)K.npw + 4.0 * per_band) +
                          std::ceil((double)nb / nbatch) * sizeof(R) * (double)g.N * g.N * g.N;
        PhaseScope ps(prof, LOBPCG_PH_FFT, nb * fft_flops_per_band(g), by, f64 && !df);
        LG_TRY(fft_vloc_apply<R>(g, c->plan, X, ldx, Y, ldy, nb, Tables<R>::kin(K), Tables<R>::vt(c),
                                 Tables<R>::tw(c), reinterpret_cast<cx<R> *>(L.T2.p), nbatch, L.stream, df,
                                 df ? c->vtdf : nullptr));
    }
    if (c->nproj > 0) {
        if (!K.has_beta) return fail(LOBPCG_ERR_ARG, "projectors of this k-point were not given");
        LG_TRY(c->alloc.ensure(L.nlB, cb * (size_t)c->nproj * nb));
        cx<R> *B = reinterpret_cast<cx<R> *>(L.nlB.p);
        const cx<R> *beta = Tables<R>::beta(K);
        const double fl = 16.0 * K.npw * (double)c->nproj * nb;
        const double by = cb * (2.0 * K.npw * c->nproj + 3.0 * K.npw * nb);
        PhaseScope ps(prof, LOBPCG_PH_NONLOCAL, fl, by, f64 && !df);
        if constexpr (sizeof(R) == 8) {
            if (df) {  // double-FP32 projections (FP64 class)
                LG_TRY(zgemm_cn_df(L.gw, c->nproj, nb, K.npw, 1.0, beta, K.npw, X, ldx, 0.0, B, c->nproj, L.stream));
                LG_TRY(scale_rows<R>(c->nproj, nb, Tables<R>::E(c), B, c->nproj, L.stream));
                return zgemm_nn_df(&L.gw, K.npw, nb, c->nproj, 1.0, beta, K.npw, B, c->nproj, 1.0, Y, ldy, Y, ldy,
                                   L.stream);
            }
        }
        LG_TRY(gemm_cn<R>(L.gw, c->nproj, nb, K.npw, (R)1, beta, K.npw, X, ldx, (R)0, B, c->nproj, L.stream));
        LG_TRY(scale_rows<R>(c->nproj, nb, Tables<R>::E(c), B, c->nproj, L.stream));
        LG_TRY(gemm_nn<R>(K.npw, nb, c->nproj, (R)1, beta, K.npw, B, c->nproj, (R)1, Y, ldy, Y, ldy, L.stream));
    }
    return LOBPCG_OK;
}

// H on packed real-form bands (Gamma point): bands 2i and 2i+1 go through one complex H
// application as c_a + i c_b and are separated afterwards (see gamma_pack_pairs), so the FFT and
// KB work is halved.  Zin, Zout: n_half x nb, ld n_half.
template <typename R>
int apply_real(lobpcg_ctx *c, Lane &L, int k, const cx<R> *Zin, cx<R> *Zout, int nb, Prof *prof, bool df) {
    if (nb <= 0) return LOBPCG_OK;
    KPoint &K = c->kp[k];
    const int np = (nb + 1) / 2;
    const size_t bytes = sizeof(cx<R>) * (size_t)K.npw * np;
    LG_TRY(c->alloc.ensure(L.rfi, bytes));
    LG_TRY(c->alloc.ensure(L.rfo, bytes));
    cx<R> *Ci = reinterpret_cast<cx<R> *>(L.rfi.p), *Co = reinterpret_cast<cx<R> *>(L.rfo.p);
    {
        PhaseScope ps(prof, LOBPCG_PH_UPDATE, 0.0, 2.0 * (double)bytes, false);
        LG_TRY(gamma_unpack_pairs<R>(K.n_half, nb, Zin, K.n_half, K.half, K.mirror, Ci, K.npw, L.stream));
    }
    LG_TRY(apply_H_dev<R>(c, L, k, Ci, K.npw, Co, K.npw, np, prof, df));
    PhaseScope ps(prof, LOBPCG_PH_UPDATE, 0.0, 2.0 * (double)bytes, false);
    return gamma_pack_pairs<R>(K.n_half, nb, Co, K.npw, K.half, K.mirror, Zout, K.n_half, L.stream);
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
// Algorithm 1 of the paper (Sec. 3.2) on one k-point, block after block with the
// orthogonality constraint, each sweep closed by an all-band Rayleigh-Ritz step.
//
// FP64 schedule: every vector, product and Gram matrix in FP64.
//
// Mixed schedule (the block iteration in FP32 around FP64 X and H X):
//   * block start in FP64: X_b is projected off the earlier blocks (H X_b along),
//     then rotated by the Rayleigh-Ritz step of the block alone, so that X_b is
//     orthonormal with X_b^H H X_b diagonal to FP64 accuracy;
//   * X_b and H X_b are kept in FP64; R = H X_b - X_b Theta is formed in FP64 with
//     exact FP64 Rayleigh quotients Theta;
//   * W = K(R), the constraint, H W (FP32 FFT, tensor-core KB GEMMs), P and H P
//     are FP32;
//   * R, W and P are projected out of span(X_b) in FP32, so the Rayleigh-Ritz basis
//     [X_b, W, P] has X-rows S = [I 0 0], A = [Theta, R^H W, R^H P]: the X-W and
//     X-P couplings come from the FP64 residual (relatively accurate however small
//     the residual is), never from X^H H W;
//   * the Gram blocks of W and P are FP32 tensor-core GEMMs, the Rayleigh-Ritz
//     solve is FP64;
//   * X_b <- X_b C_X + P and H X_b <- H X_b C_X + H P are FP64;
//   * every sweep ends with an FP64-class H X refresh (computed block by block on a
//     low-priority side stream while the later blocks run), the FP64-class all-band
//     Rayleigh-Ritz step and FP64 residual norms, which decide convergence;
//   * early visits (every band of the block above opt.mixed_early in the previous
//     sweep): the block start and the block's X updates run on the FP32 copies
//     (tensor cores, FP64 diagonals and eigensolve) and H X_b is not refreshed; X_b
//     and H X_b then carry FP32 accuracy, far below the residuals of such a block.
//     The first full visit of a block after early ones recomputes H X_b first;
//   * settled blocks (every band below tol/100 after the previous sweep) keep their
//     block start but take no inner iterations;
//   * the sweep-end Rayleigh-Ritz runs on the FP32 copies only when every block was
//     early, and convergence is only ever declared after a sweep that was not.
struct Solver {
    lobpcg_ctx *c;
    Lane *L = nullptr;
    Prof *prof;
    int k, npw, M, m, nblk;
    bool mixed;
    bool df = false;  // FP64-class tall GEMMs in double-FP32 arithmetic
    bool real = false;  // Gamma real form: packed half-sphere bands, real coefficient matrices
    const double *kin = nullptr;  // kinetic table of the stored rows (packed in the real form)
    double *part = nullptr;  // scratch of the per-column reductions (colsum_part_elems(nzmax))
    cudaStream_t s;
    z64 *X, *HX;             // all bands, FP64 (X is the caller's buffer)
    z64 *HXr = nullptr;      // side-stream H X of the current full sweep (see Lane::side)
    bool hxr_ready = false;  // every block's side refresh of this sweep is queued
    z64 *Z[2], *HZ[2];       // FP64 block bases [X W P] (mixed: only the X part)
    z64 *Tmp;                // npw x max(M, m) FP64 scratch
    z64 *S, *A, *C;          // Gram / projected / coefficient matrices, FP64
    z64 *G;                  // constraint coefficients, FP64
    double *theta, *res, *work;
    int *ndrop;
    double drop_tol;          // dependence threshold for FP64 Grams
    double drop_tol32;        // dependence threshold for FP32 Grams (mixed schedule)
    // mixed-only FP32 buffers
    c32 *X32all, *HX32all;   // FP32 copies of X and H X (all bands)
    c32 *Q32[2], *HQ32[2];   // [R W P] and [. HW HP], npw x 3m
    c32 *X32, *HX32;         // FP32 copies of X_b, H X_b
    c32 *S32, *A32, *C32, *G32, *D32;
    c32 *T32;                // npw x M FP32 scratch (early-sweep rotations)
    c32 *E32;                // C - I of a near-identity rotation (FP32)
    unsigned int *dmax;      // device scratch for max |C - I|
    bool early = false;      // current sweep is an early one of the mixed schedule
    long long applies64 = 0, applies32 = 0;
    int iterations = 0;
    int verbose = 0;          // LOBPCG_VERBOSE: 1 per sweep, 2 per iteration (synchronising diagnostics)
    std::vector<double> dbg;

    // Diagnostic print of the estimated residual max of a block (FP64 from X, HX).
    void trace(const char *tag, int b, int it, const z64 *Xb, const z64 *HXb, int nb) {
        if (verbose < 2) return;
        dbg.assign(2 * nb + 1, 0.0);
        double *dres = res;
        column_resid_norms(npw, nb, Xb, npw, HXb, npw, theta, dres, part, s);
        cudaMemcpyAsync(dbg.data(), dres, sizeof(double) * nb, cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(dbg.data() + nb, theta, sizeof(double) * nb, cudaMemcpyDeviceToHost, s);
        int nd = 0;
        cudaMemcpyAsync(&nd, ndrop, sizeof(int), cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
        double mx = 0.0;
        for (int i = 0; i < nb; ++i) mx = std::max(mx, dbg[i]);
        fprintf(stderr, "[lobpcg] k=%d %s block=%d it=%d max_resid_est=%.3e theta0=%.12f dropped=%d\n", k, tag, b,
                it, mx, dbg[nb], nd);
    }

    z64 *col(z64 *base, int j) const { return base + (size_t)j * npw; }
    c32 *col(c32 *base, int j) const { return base + (size_t)j * npw; }
    double cbytes64(double cols) const { return 16.0 * npw * cols; }
    double cbytes32(double cols) const { return 8.0 * npw * cols; }

    int applyH64(const z64 *Xin, z64 *Yout, int nb) {
        if (real) {
            applies64 += (nb + 1) / 2;
            return apply_real<double>(c, *L, k, Xin, Yout, nb, prof, df);
        }
        applies64 += nb;
        return apply_H_dev<double>(c, *L, k, Xin, npw, Yout, npw, nb, prof, df);
    }
    int applyH32(const c32 *Xin, c32 *Yout, int nb) {
        if (real) {
            applies32 += (nb + 1) / 2;
            return apply_real<float>(c, *L, k, Xin, Yout, nb, prof, false);
        }
        applies32 += nb;
        // (the legacy default stream cannot be captured)
        if (c->opt.use_graph && !prof && s != nullptr && s != cudaStreamLegacy) return graph_apply32(Xin, Yout, nb);
        return apply_H_dev<float>(c, *L, k, Xin, npw, Yout, npw, nb, prof);
    }
    // H W through a CUDA graph: the FFT passes and KB GEMMs of one block application (about ten
    // kernels) replay as one launch.  The first call on a buffer pair runs directly (allocating
    // its scratch) and records the graph for the next ones.
    int graph_apply32(const c32 *Xin, c32 *Yout, int nb) {
        const auto key = std::make_tuple(k, (const void *)Xin, (void *)Yout, nb);
        auto it = L->graphs.find(key);
        if (it != L->graphs.end() && it->second.t2 == L->T2.p && it->second.nlb == L->nlB.p &&
            it->second.part == L->gw.part.p) {
            LG_CUDA_TRY(cudaGraphLaunch(it->second.exec, s));
            add_launches(it->second.kernels);
            return LOBPCG_OK;
        }
        if (it != L->graphs.end()) {  // scratch moved since it was recorded
            cudaGraphExecDestroy(it->second.exec);
            L->graphs.erase(it);
        }
        LG_TRY(apply_H_dev<float>(c, *L, k, Xin, npw, Yout, npw, nb, nullptr));
        const long long l0 = launch_count();
        cudaGraph_t g = nullptr;
        LG_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        const int rc = apply_H_dev<float>(c, *L, k, Xin, npw, Yout, npw, nb, nullptr);
        const cudaError_t ec = cudaStreamEndCapture(s, &g);
        add_launches(l0 - launch_count());  // recorded, not run
        if (rc != LOBPCG_OK || ec != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            if (rc != LOBPCG_OK) return rc;
            LG_CUDA_TRY(ec);
        }
        Lane::Graph gr;
        size_t nn = 0;
        cudaGraphGetNodes(g, nullptr, &nn);
        std::vector<cudaGraphNode_t> nodes(nn);
        if (nn) cudaGraphGetNodes(g, nodes.data(), &nn);
        for (cudaGraphNode_t nd : nodes) {
            cudaGraphNodeType t;
            if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++gr.kernels;
        }
        const cudaError_t ei = cudaGraphInstantiate(&gr.exec, g, 0ULL);
        cudaGraphDestroy(g);
        LG_CUDA_TRY(ei);
        gr.t2 = L->T2.p;
        gr.nlb = L->nlB.p;
        gr.part = L->gw.part.p;
        L->graphs[key] = gr;
        return LOBPCG_OK;
    }

    // ---------------------------------------------------------- FP64 helpers
    // In the real form every coefficient matrix is the real part of the packed product
    // (Re(z_a^H z_b) is the real inner product of the real-form vectors).
    template <typename R>
    int realpart(int rows, int cols, cx<R> *Cc, int ldc) {
        return real ? zero_imag<R>(rows, cols, Cc, ldc, s) : LOBPCG_OK;
    }
    int gemm_cn64(int ph, int mm, int nn, const z64 *Aa, const z64 *Bb, z64 *Cc, int ldc) {
        {
            PhaseScope ps(prof, ph, 8.0 * mm * nn * (double)npw, cbytes64(mm + nn), !df);
            if (df) LG_TRY(zgemm_cn_df(L->gw, mm, nn, npw, 1.0, Aa, npw, Bb, npw, 0.0, Cc, ldc, s));
            else LG_TRY(gemm_cn<double>(L->gw, mm, nn, npw, 1.0, Aa, npw, Bb, npw, 0.0, Cc, ldc, s));
        }
        return realpart<double>(mm, nn, Cc, ldc);
    }
    // Hermitian Gram (lower triangle only; the Rayleigh-Ritz reads no more)
    int gram64(int nn, const z64 *Aa, const z64 *Bb, z64 *Cc) {
        {
            PhaseScope ps(prof, LOBPCG_PH_GRAM, 4.0 * nn * (nn + 1) * (double)npw, cbytes64(2 * nn), !df);
            LG_TRY(zgemm_cn_lower(L->gw, nn, npw, Aa, npw, Bb, npw, Cc, nn, s, df));
        }
        return realpart<double>(nn, nn, Cc, nn);
    }
    int gemm_nn64(int ph, int nn, int kk, double alpha, const z64 *Aa, const z64 *Bb, int ldb, double beta,
                  const z64 *Cc, z64 *Dd) {
        PhaseScope ps(prof, ph, 8.0 * nn * kk * (double)npw, cbytes64(kk + nn * (beta != 0.0 ? 2 : 1)), !df);
        if (df) return zgemm_nn_df(&L->gw, npw, nn, kk, alpha, Aa, npw, Bb, ldb, beta, Cc, npw, Dd, npw, s);
        return gemm_nn<double>(npw, nn, kk, alpha, Aa, npw, Bb, ldb, beta, Cc, npw, Dd, npw, s);
    }
    int gemm_cn32(int ph, int mm, int nn, const c32 *Aa, const c32 *Bb, c32 *Cc, int ldc) {
        {
            PhaseScope ps(prof, ph, 8.0 * mm * nn * (double)npw, cbytes32(mm + nn), false);
            LG_TRY(gemm_cn<float>(L->gw, mm, nn, npw, 1.0f, Aa, npw, Bb, npw, 0.0f, Cc, ldc, s));
        }
        return realpart<float>(mm, nn, Cc, ldc);
    }
    int gemm_nn32(int ph, int nn, int kk, float alpha, const c32 *Aa, const c32 *Bb, int ldb, float beta,
                  const c32 *Cc, c32 *Dd) {
        PhaseScope ps(prof, ph, 8.0 * nn * kk * (double)npw, cbytes32(kk + nn * (beta != 0.f ? 2 : 1)), false);
        return gemm_nn<float>(npw, nn, kk, alpha, Aa, npw, Bb, ldb, beta, Cc, npw, Dd, npw, s);
    }
    // Rayleigh-Ritz on the pencil in S, A.  `tol` is the dependence threshold on the squared
    // Cholesky pivot of the unit-diagonal Gram: a kept direction amplifies the Gram's rounding
    // by 1/pivot^2, so tol is ~1e3 x the Gram's unit roundoff (FP64 Grams 1e-12, FP32 Grams 1e-3).
    int rr(int nz, int mm, double tol, int lead = 0) {
        {
            const double n3 = (double)nz * nz * nz;
            PhaseScope ps(prof, LOBPCG_PH_RR, 8.0 * (3.0 * n3 + 2.0 * nz * (double)nz * mm), 0.0, true);
            LG_TRY(rayleigh_ritz(L->ew, nz, mm, S, nz, A, nz, tol, theta, C, nz, ndrop, s, lead));
        }
        return realpart<double>(nz, mm, C, nz);   // a real symmetric pencil has real Ritz vectors
    }
    template <typename Ro, typename Ri>
    int cast(int cols, const cx<Ri> *a, cx<Ro> *b) {
        PhaseScope ps(prof, LOBPCG_PH_UPDATE, 0.0, (double)npw * cols * (sizeof(cx<Ri>) + sizeof(cx<Ro>)), false);
        return copy_cast<Ro, Ri>(npw, cols, a, npw, b, npw, s);
    }
    int copy32(c32 *dst, const c32 *src, int cols) {
        PhaseScope ps(prof, LOBPCG_PH_UPDATE, 0.0, 2.0 * cbytes32(cols), false);
        LG_CUDA_TRY(cudaMemcpyAsync(dst, src, sizeof(c32) * (size_t)npw * cols, cudaMemcpyDeviceToDevice, s));
        return LOBPCG_OK;
    }
    int copy64(z64 *dst, const z64 *src, int cols) {
        PhaseScope ps(prof, LOBPCG_PH_UPDATE, 0.0, 2.0 * cbytes64(cols), false);
        LG_CUDA_TRY(cudaMemcpyAsync(dst, src, sizeof(z64) * (size_t)npw * cols, cudaMemcpyDeviceToDevice, s));
        return LOBPCG_OK;
    }

    // V <- V - Y (Y^H V), twice (classical Gram-Schmidt repeated); Y = first j bands.
    int constrain64(z64 *V, int nv, int j) {
        if (j <= 0) return LOBPCG_OK;
        for (int rep = 0; rep < 2; ++rep) {
            LG_TRY(gemm_cn64(LOBPCG_PH_CONSTRAINT, j, nv, X, V, G, j));
            LG_TRY(gemm_nn64(LOBPCG_PH_CONSTRAINT, nv, j, -1.0, X, G, j, 1.0, V, V));
        }
        return LOBPCG_OK;
    }
    // V <- V - Xb (Xb^H V) for the m columns of V, and HV <- HV - HXb (Xb^H V) when given
    int project_block64(const z64 *Xb, const z64 *HXb, z64 *V, z64 *HV) {
        LG_TRY(gemm_cn64(LOBPCG_PH_UPDATE, m, m, Xb, V, G, m));
        LG_TRY(gemm_nn64(LOBPCG_PH_UPDATE, m, m, -1.0, Xb, G, m, 1.0, V, V));
        if (HV) LG_TRY(gemm_nn64(LOBPCG_PH_UPDATE, m, m, -1.0, HXb, G, m, 1.0, HV, HV));
        return LOBPCG_OK;
    }
    int constrain32(c32 *V, int nv, const c32 *Y, int j, int ph) {
        if (j <= 0) return LOBPCG_OK;
        for (int rep = 0; rep < 2; ++rep) {
            LG_TRY(gemm_cn32(ph, j, nv, Y, V, G32, j));
            LG_TRY(gemm_nn32(ph, nv, j, -1.0f, Y, G32, j, 1.0f, V, V));
        }
        return LOBPCG_OK;
    }

    // ---------------------------------------------------------- FP64 block visit
    int block64(int b) {
        int cur = 0;
        z64 *Xu = col(X, b * m);
        LG_TRY(copy64(Z[cur], Xu, m));
        LG_TRY(constrain64(Z[cur], m, b * m));
        LG_TRY(applyH64(Z[cur], HZ[cur], m));
        // Rayleigh-Ritz on the block alone: orthonormal Ritz basis, Upsilon (step 1)
        LG_TRY(gram64(m, Z[cur], Z[cur], S));
        LG_TRY(gram64(m, Z[cur], HZ[cur], A));
        LG_TRY(rr(m, m, drop_tol));
        LG_TRY(gemm_nn64(LOBPCG_PH_UPDATE, m, m, 1.0, Z[cur], C, m, 0.0, nullptr, Z[1 - cur]));
        LG_TRY(gemm_nn64(LOBPCG_PH_UPDATE, m, m, 1.0, HZ[cur], C, m, 0.0, nullptr, HZ[1 - cur]));
        cur = 1 - cur;
        int nP = 0;
        for (int it = 0; it < c->opt.nline; ++it) {
            z64 *Zc = Z[cur], *HZc = HZ[cur];
            z64 *W = col(Zc, m), *HW = col(HZc, m);
            {   // steps 2-3: R = HX - X Upsilon, W = K(R)
                PhaseScope ps(prof, LOBPCG_PH_UPDATE, 20.0 * npw * m, cbytes64(3.0 * m), true);
                LG_TRY(residual_precond<double>(npw, m, Zc, npw, HZc, npw, theta, kin, W, npw, work, part, s));
            }
            LG_TRY(constrain64(W, m, b * m));
            // W and P off span(X_b) (P's H image likewise): span[X, W, P], hence the step in exact
            // arithmetic, is unchanged, but the Gram matrix stays away from singular when bands of
            // a degenerate shell converge and leave W and P as rounding noise close to span(X_b)
            LG_TRY(project_block64(Zc, nullptr, W, nullptr));
            LG_TRY(applyH64(W, HW, m));
            if (nP) LG_TRY(project_block64(Zc, HZc, col(Zc, 2 * m), col(HZc, 2 * m)));
            // step 4: Rayleigh-Ritz on span[X, W, P]
            const int nz = (2 + nP) * m;
            LG_TRY(gram64(nz, Zc, Zc, S));
            LG_TRY(gram64(nz, Zc, HZc, A));
            LG_TRY(rr(nz, m, drop_tol));
            // steps 4-5: P = W Lambda + P Gamma, X = X Delta + P (and their H images)
            z64 *Zn = Z[1 - cur], *HZn = HZ[1 - cur];
            LG_TRY(gemm_nn64(LOBPCG_PH_UPDATE, m, nz - m, 1.0, col(Zc, m), C + m, nz, 0.0, nullptr, col(Zn, 2 * m)));
            LG_TRY(gemm_nn64(LOBPCG_PH_UPDATE, m, m, 1.0, Zc, C, nz, 1.0, col(Zn, 2 * m), Zn));
            LG_TRY(gemm_nn64(LOBPCG_PH_UPDATE, m, nz - m, 1.0, col(HZc, m), C + m, nz, 0.0, nullptr, col(HZn, 2 * m)));
            LG_TRY(gemm_nn64(LOBPCG_PH_UPDATE, m, m, 1.0, HZc, C, nz, 1.0, col(HZn, 2 * m), HZn));
            cur = 1 - cur;
            nP = 1;
            ++iterations;
        }
        LG_TRY(copy64(Xu, Z[cur], m));
        LG_TRY(copy64(col(HX, b * m), HZ[cur], m));
        return LOBPCG_OK;
    }

    // ---------------------------------------------------------- mixed block visit
    // Rayleigh-Ritz of the mixed schedule: FP32 Gram blocks assembled into an FP64 pencil,
    // solved in FP64; the coefficients also come back in FP32 for the FP32 updates.
    int rr_mixed(int nz, int mm) {
        // the assembled pencil has S = I on the X block and no X-W / X-P overlap (see
        // assemble_gram_mixed): its Cholesky starts after that block
        LG_TRY(rr(nz, mm, drop_tol32, m));
        // a Ritz vector's phase is free: make C's X-diagonal real positive, so that a step which
        // barely moves X_b has C_X close to I (see near_identity)
        LG_TRY(fix_phases(nz, mm, C, nz, s));
        PhaseScope ps(prof, LOBPCG_PH_UPDATE, 0.0, 24.0 * nz * mm, false);
        return copy_cast<float, double>(nz, mm, C, nz, C32, nz, s);
    }
    int ritz_values(const z64 *Xb, const z64 *HXb) {
        PhaseScope ps(prof, LOBPCG_PH_UPDATE, 8.0 * npw * m, cbytes64(2.0 * m), true);
        return rayleigh_quotients(npw, m, Xb, npw, HXb, npw, theta, part, s);
    }

    // nline: Algorithm 1 iterations after the block start (0 for a block already converged far
    // below the tolerance, see solve_k)
    int block_mixed(int b, int nline) {
        const int j0 = b * m;
        int cur = 0;
        z64 *Xb = Z[cur], *HXb = HZ[cur];
        LG_TRY(copy64(Xb, col(X, j0), m));
        LG_TRY(copy64(HXb, col(HX, j0), m));
        // Block start in FP64: the inner iterations take X_b as orthonormal, X_b^H H X_b as
        // diagonal and X_b as orthogonal to the earlier blocks, and cannot repair an error there
        // (the residual is projected off span(X_b)); FP32 products here would leave ~1e-7
        // couplings and set a residual floor.  In early sweeps, far above that floor, the FP32
        // copies and the tensor cores do it.
        if (early) {
            LG_TRY(block_start_early(b, Xb, HXb));
        } else {
        if (b > 0) {
            // X_b <- X_b - Y (Y^H X_b), H X_b <- H X_b - (H Y)(Y^H X_b).  One pass: outside the
            // early sweeps X_b already leaves the earlier blocks only at the FP32 level of the
            // inner corrections (about 1e-7 of them), which a single FP64 projection removes.
            for (int rep = 0; rep < 1; ++rep) {
                LG_TRY(gemm_cn64(LOBPCG_PH_CONSTRAINT, j0, m, X, Xb, G, j0));
                LG_TRY(gemm_nn64(LOBPCG_PH_CONSTRAINT, m, j0, -1.0, X, G, j0, 1.0, Xb, Xb));
                LG_TRY(gemm_nn64(LOBPCG_PH_CONSTRAINT, m, j0, -1.0, HX, G, j0, 1.0, HXb, HXb));
            }
        }
        // Rayleigh-Ritz of the block alone (FP64 Grams), rotation in FP64
        LG_TRY(gram64(m, Xb, Xb, S));
        LG_TRY(gram64(m, Xb, HXb, A));
        LG_TRY(rr(m, m, drop_tol));
        LG_TRY(gemm_nn64(LOBPCG_PH_UPDATE, m, m, 1.0, Xb, C, m, 0.0, nullptr, Z[1 - cur]));
        LG_TRY(gemm_nn64(LOBPCG_PH_UPDATE, m, m, 1.0, HXb, C, m, 0.0, nullptr, HZ[1 - cur]));
        }
        cur = 1 - cur;
        trace("mixed-start", b, -1, Z[cur], HZ[cur], m);
        int nP = 0;
        for (int it = 0; it < nline; ++it) {
            Xb = Z[cur];
            HXb = HZ[cur];
            c32 *Q = Q32[cur], *HQ = HQ32[cur];
            c32 *R32 = Q, *W32 = col(Q, m), *P32 = col(Q, 2 * m);
            c32 *HW32 = col(HQ, m), *HP32 = col(HQ, 2 * m);
            LG_TRY(cast<float, double>(m, Xb, X32));
            LG_TRY(cast<float, double>(m, HXb, HX32));
            // step 1: exact FP64 Rayleigh quotients of the current block
            LG_TRY(ritz_values(Xb, HXb));
            {   // step 2: R = HX - X Upsilon in FP64, stored FP32, then projected out of span(X) in FP32
                PhaseScope ps(prof, LOBPCG_PH_UPDATE, 4.0 * npw * m, cbytes64(2.0 * m) + cbytes32(m), true);
                LG_TRY(residual32(npw, m, Xb, npw, HXb, npw, theta, R32, npw, s));
            }
            LG_TRY(constrain32(R32, m, X32, m, LOBPCG_PH_UPDATE));
            {   // step 3: W = K(R)
                PhaseScope ps(prof, LOBPCG_PH_UPDATE, 10.0 * npw * m, cbytes64(m) + 2.0 * cbytes32(m), false);
                LG_TRY(precond32(npw, m, Xb, npw, kin, R32, npw, W32, npw, work, part, s));
            }
            LG_TRY(constrain32(W32, m, X32all, j0, LOBPCG_PH_CONSTRAINT));
            LG_TRY(constrain32(W32, m, X32, m, LOBPCG_PH_UPDATE));
            LG_TRY(applyH32(W32, HW32, m));
            if (nP) {
                // P <- P - X (X^H P), H P likewise (FP32)
                LG_TRY(gemm_cn32(LOBPCG_PH_UPDATE, m, m, X32, P32, G32, m));
                LG_TRY(gemm_nn32(LOBPCG_PH_UPDATE, m, m, -1.0f, X32, G32, m, 1.0f, P32, P32));
                LG_TRY(gemm_nn32(LOBPCG_PH_UPDATE, m, m, -1.0f, HX32, G32, m, 1.0f, HP32, HP32));
            }
            const int nz = (2 + nP) * m, nw = nz - m;
            // step 4: Grams in FP32: T1 = [R W P]^H [W P], T2 = [W P]^H [HW HP]; FP32 pencil; FP32 RR
            LG_TRY(gemm_cn32(LOBPCG_PH_GRAM, nz, nw, Q, W32, S32, nz));
            LG_TRY(gemm_cn32(LOBPCG_PH_GRAM, nw, nw, W32, HW32, A32, nw));
            {
                PhaseScope ps(prof, LOBPCG_PH_RR, 0.0, 0.0, false);
                LG_TRY(assemble_gram_mixed(nz, m, S32, nz, A32, nw, theta, S, A, s));
            }
            LG_TRY(rr_mixed(nz, m));
            // step 5: P = W Lambda + P Gamma, H P likewise (FP32)
            c32 *Qn = Q32[1 - cur], *HQn = HQ32[1 - cur];
            LG_TRY(gemm_nn32(LOBPCG_PH_UPDATE, m, nw, 1.0f, W32, C32 + m, nz, 0.0f, nullptr, col(Qn, 2 * m)));
            LG_TRY(gemm_nn32(LOBPCG_PH_UPDATE, m, nw, 1.0f, HW32, C32 + m, nz, 0.0f, nullptr, col(HQn, 2 * m)));
            // X = X Delta + P, H X = H X Delta + H P: FP64, or, in an early sweep (where X and H X
            // carry FP32 accuracy), from the FP32 copies on the tensor cores
            if (early) {
                LG_TRY(gemm_nn32(LOBPCG_PH_UPDATE, m, m, 1.0f, X32, C32, nz, 1.0f, col(Qn, 2 * m), D32));
                LG_TRY(cast<double, float>(m, D32, Z[1 - cur]));
                LG_TRY(gemm_nn32(LOBPCG_PH_UPDATE, m, m, 1.0f, HX32, C32, nz, 1.0f, col(HQn, 2 * m), D32));
                LG_TRY(cast<double, float>(m, D32, HZ[1 - cur]));
            } else {
                bool small = false;
                LG_TRY(near_identity(m, C, nz, small));
                if (small) {
                    // X_new = X + (X32 (C_X - I) + P), H X likewise (near-identity C_X of a late sweep)
                    LG_TRY(gemm_nn32(LOBPCG_PH_UPDATE, m, m, 1.0f, X32, E32, m, 1.0f, col(Qn, 2 * m), D32));
                    LG_TRY(add_cast_cols(Xb, D32, Z[1 - cur], m));
                    LG_TRY(gemm_nn32(LOBPCG_PH_UPDATE, m, m, 1.0f, HX32, E32, m, 1.0f, col(HQn, 2 * m), D32));
                    LG_TRY(add_cast_cols(HXb, D32, HZ[1 - cur], m));
                } else {
                    LG_TRY(cast<double, float>(m, col(Qn, 2 * m), Tmp));
                    LG_TRY(gemm_nn64(LOBPCG_PH_UPDATE, m, m, 1.0, Xb, C, nz, 1.0, Tmp, Z[1 - cur]));
                    LG_TRY(cast<double, float>(m, col(HQn, 2 * m), Tmp));
                    LG_TRY(gemm_nn64(LOBPCG_PH_UPDATE, m, m, 1.0, HXb, C, nz, 1.0, Tmp, HZ[1 - cur]));
                }
            }
            cur = 1 - cur;
            nP = 1;
            ++iterations;
            if (verbose >= 2) {
                LG_TRY(ritz_values(Z[cur], HZ[cur]));
                trace("mixed", b, it, Z[cur], HZ[cur], m);
            }
        }
        LG_TRY(copy64(col(X, j0), Z[cur], m));
        LG_TRY(copy64(col(HX, j0), HZ[cur], m));
        LG_TRY(cast<float, double>(m, Z[cur], col(X32all, j0)));
        LG_TRY(cast<float, double>(m, HZ[cur], col(HX32all, j0)));
        return LOBPCG_OK;
    }
    // FP32 copies of block b (read by the constraint of later mixed blocks) after an FP64 visit
    int refresh32(int b) {
        LG_TRY(cast<float, double>(m, col(X, b * m), col(X32all, b * m)));
        return cast<float, double>(m, col(HX, b * m), col(HX32all, b * m));
    }
    // Early-sweep block start: constraint against the earlier blocks and the block's Rayleigh-Ritz
    // from the FP32 copies (FP64 diagonals, FP64 eigensolve), rotation of the FP32 copies into
    // Z[1], HZ[1].
    int block_start_early(int b, z64 *Xb, z64 *HXb) {
        const int j0 = b * m;
        if (b > 0) {
            for (int rep = 0; rep < 2; ++rep) {
                LG_TRY(cast<float, double>(m, Xb, X32));
                LG_TRY(gemm_cn32(LOBPCG_PH_CONSTRAINT, j0, m, X32all, X32, G32, j0));
                LG_TRY(gemm_nn32(LOBPCG_PH_CONSTRAINT, m, j0, 1.0f, X32all, G32, j0, 0.0f, nullptr, D32));
                LG_TRY(cast<double, float>(m, D32, Tmp));
                LG_TRY(gemm_nn64_axpy(Xb, Tmp, m));
                LG_TRY(gemm_nn32(LOBPCG_PH_CONSTRAINT, m, j0, 1.0f, HX32all, G32, j0, 0.0f, nullptr, D32));
                LG_TRY(cast<double, float>(m, D32, Tmp));
                LG_TRY(gemm_nn64_axpy(HXb, Tmp, m));
            }
        }
        LG_TRY(cast<float, double>(m, Xb, X32));
        LG_TRY(cast<float, double>(m, HXb, HX32));
        LG_TRY(gemm_cn32(LOBPCG_PH_GRAM, m, m, X32, X32, S32, m));
        LG_TRY(gemm_cn32(LOBPCG_PH_GRAM, m, m, X32, HX32, A32, m));
        {
            PhaseScope ps(prof, LOBPCG_PH_RR, 16.0 * npw * m, cbytes64(2.0 * m), true);
            LG_TRY(assemble_gram_mixed(m, 0, S32, m, A32, m, nullptr, S, A, s));
            LG_TRY(diag_pencil(npw, m, Xb, npw, HXb, npw, S, A, part, s));
        }
        LG_TRY(rr(m, m, drop_tol32));
        {
            PhaseScope ps(prof, LOBPCG_PH_UPDATE, 0.0, 24.0 * m * m, false);
            LG_TRY(copy_cast<float, double>(m, m, C, m, C32, m, s));
        }
        LG_TRY(gemm_nn32(LOBPCG_PH_UPDATE, m, m, 1.0f, X32, C32, m, 0.0f, nullptr, D32));
        LG_TRY(cast<double, float>(m, D32, Z[1]));
        LG_TRY(gemm_nn32(LOBPCG_PH_UPDATE, m, m, 1.0f, HX32, C32, m, 0.0f, nullptr, D32));
        return cast<double, float>(m, D32, HZ[1]);
    }
    // Is the rotation C (leading k x k of ld ldc) the identity up to E = C - I with
    // max|E| * k <= kRotSmall?  Then X C = X + X E can take X E from the FP32 copies on the
    // tensor cores: its error, ~2e-6 of the column 1-norm of E, stays at the FP64 level of X.
    static constexpr double kRotSmall = 1e-4;
    int near_identity(int kk, const z64 *Cm, int ldc, bool &small) {
        float emax = 0.f;
        {
            PhaseScope ps(prof, LOBPCG_PH_UPDATE, 0.0, 24.0 * kk * kk, false);
            LG_TRY(near_identity32(kk, kk, Cm, ldc, E32, kk, dmax, &emax, s));
        }
        small = (double)emax * kk <= kRotSmall;
        return LOBPCG_OK;
    }
    int add_cast_cols(const z64 *Aa, const c32 *Tt, z64 *Out, int cols) {
        PhaseScope ps(prof, LOBPCG_PH_UPDATE, 2.0 * npw * cols, 2.0 * cbytes64(cols) + cbytes32(cols), true);
        return add_cast(npw, cols, Aa, npw, Tt, npw, Out, npw, s);
    }
    int gemm_nn64_axpy(z64 *V, const z64 *D, int cols) {
        PhaseScope ps(prof, LOBPCG_PH_CONSTRAINT, 2.0 * npw * cols, 3.0 * cbytes64(cols), true);
        return axpy_cols(npw, cols, -1.0, D, npw, V, npw, s);
    }
    // Ritz values and residuals to the host.  The all-band Rayleigh-Ritz step must keep all M
    // directions: a dropped one means the bands lost linear independence (breakdown).
    int fetch_results(double *eig_h, double *res_h) {
        int nd_h = 0;
        LG_CUDA_TRY(cudaMemcpyAsync(eig_h, theta, sizeof(double) * M, cudaMemcpyDeviceToHost, s));
        LG_CUDA_TRY(cudaMemcpyAsync(res_h, res, sizeof(double) * M, cudaMemcpyDeviceToHost, s));
        LG_CUDA_TRY(cudaMemcpyAsync(&nd_h, ndrop, sizeof(int), cudaMemcpyDeviceToHost, s));
        LG_CUDA_TRY(cudaStreamSynchronize(s));
        // a device wait that gave up leaves its outputs undefined: report it before judging them
        LG_TRY(tc_check_error());
        if (nd_h > 0)
            return fail(LOBPCG_ERR_BREAKDOWN, "the bands lost linear independence (" + std::to_string(nd_h) +
                                                  " dropped in the all-band Rayleigh-Ritz step)");
        return LOBPCG_OK;
    }
    // Rayleigh-Ritz over all M bands closing a sweep (Sec. 3.2), then FP64 residuals.
    // After block b's visit (X_b final for this sweep): H X_b on the side stream into HXr.
    int side_refresh(int b) {
        Lane &R = *L->side;
        LG_CUDA_TRY(cudaEventRecord(L->ev_main, s));
        LG_CUDA_TRY(cudaStreamWaitEvent(R.stream, L->ev_main, 0));
        if (real) {
            applies64 += (m + 1) / 2;
            return apply_real<double>(c, R, k, col(X, b * m), col(HXr, b * m), m, nullptr, df);
        }
        applies64 += m;
        return apply_H_dev<double>(c, R, k, col(X, b * m), npw, col(HXr, b * m), npw, m, nullptr, df);
    }
    int final_rr(double *eig_h, double *res_h) {
        if (early) return final_rr_early(eig_h, res_h);
        if (mixed && hxr_ready) {
            // FP64 H X for the residual test: the side stream's, computed block by block
            LG_CUDA_TRY(cudaEventRecord(L->ev_side, L->side->stream));
            LG_CUDA_TRY(cudaStreamWaitEvent(s, L->ev_side, 0));
            std::swap(HX, HXr);
            hxr_ready = false;
        } else if (mixed) {
            LG_TRY(applyH64(X, HX, M));
        }
        LG_TRY(gram64(M, X, X, S));
        LG_TRY(gram64(M, X, HX, A));
        LG_TRY(rr(M, M, drop_tol));
        bool small = false;
        if (mixed) {
            LG_TRY(fix_phases(M, M, C, M, s));
            LG_TRY(near_identity(M, C, M, small));
        }
        if (small) {
            // near-identity all-band rotation: X += X32 (C - I), H X likewise
            LG_TRY(cast<float, double>(M, X, X32all));
            LG_TRY(cast<float, double>(M, HX, HX32all));
            LG_TRY(gemm_nn32(LOBPCG_PH_UPDATE, M, M, 1.0f, X32all, E32, M, 0.0f, nullptr, T32));
            LG_TRY(add_cast_cols(X, T32, X, M));
            LG_TRY(gemm_nn32(LOBPCG_PH_UPDATE, M, M, 1.0f, HX32all, E32, M, 0.0f, nullptr, T32));
            LG_TRY(add_cast_cols(HX, T32, HX, M));
        } else {
            LG_TRY(gemm_nn64(LOBPCG_PH_UPDATE, M, M, 1.0, X, C, M, 0.0, nullptr, Tmp));
            LG_TRY(copy64(X, Tmp, M));
            LG_TRY(gemm_nn64(LOBPCG_PH_UPDATE, M, M, 1.0, HX, C, M, 0.0, nullptr, Tmp));
            LG_TRY(copy64(HX, Tmp, M));
        }
        {
            PhaseScope ps(prof, LOBPCG_PH_UPDATE, 8.0 * npw * M, cbytes64(2.0 * M), true);
            LG_TRY(column_resid_norms(npw, M, X, npw, HX, npw, theta, res, part, s));
        }
        if (mixed) {
            LG_TRY(cast<float, double>(M, X, X32all));
            LG_TRY(cast<float, double>(M, HX, HX32all));
        }
        return fetch_results(eig_h, res_h);
    }
    // The same step in an early sweep of the mixed schedule (residuals far above FP32
    // resolution): Grams from the FP32 copies on the tensor cores with FP64 diagonals, FP64
    // eigensolve, rotation of the FP32 copies, no FP64 H refresh (H X is the one the block
    // iterations keep).  X and H X come out with FP32 accuracy, which the FP64 block starts of
    // the later sweeps restore.
    int final_rr_early(double *eig_h, double *res_h) {
        LG_TRY(gemm_cn32(LOBPCG_PH_GRAM, M, M, X32all, X32all, S32, M));
        LG_TRY(gemm_cn32(LOBPCG_PH_GRAM, M, M, X32all, HX32all, A32, M));
        {
            PhaseScope ps(prof, LOBPCG_PH_RR, 16.0 * npw * M, cbytes64(2.0 * M), true);
            LG_TRY(assemble_gram_mixed(M, 0, S32, M, A32, M, nullptr, S, A, s));
            LG_TRY(diag_pencil(npw, M, X, npw, HX, npw, S, A, part, s));
        }
        LG_TRY(rr(M, M, drop_tol32));
        {
            PhaseScope ps(prof, LOBPCG_PH_UPDATE, 0.0, 24.0 * M * M, false);
            LG_TRY(copy_cast<float, double>(M, M, C, M, C32, M, s));
        }
        LG_TRY(gemm_nn32(LOBPCG_PH_UPDATE, M, M, 1.0f, X32all, C32, M, 0.0f, nullptr, T32));
        LG_TRY(cast<double, float>(M, T32, X));
        LG_TRY(copy32(X32all, T32, M));
        LG_TRY(gemm_nn32(LOBPCG_PH_UPDATE, M, M, 1.0f, HX32all, C32, M, 0.0f, nullptr, T32));
        LG_TRY(cast<double, float>(M, T32, HX));
        LG_TRY(copy32(HX32all, T32, M));
        {
            PhaseScope ps(prof, LOBPCG_PH_UPDATE, 8.0 * npw * M, cbytes64(2.0 * M), true);
            LG_TRY(column_resid_norms(npw, M, X, npw, HX, npw, theta, res, part, s));
        }
        return fetch_results(eig_h, res_h);
    }
};

template <typename T>
T *carve(lobpcg_ctx *c, DevBuf &b, size_t count, int &rc) {
    rc = c->alloc.ensure(b, sizeof(T) * std::max<size_t>(count, 1));
    return reinterpret_cast<T *>(b.p);
}

// Mixed schedule: a block whose residuals after the previous sweep are all below this fraction of
// the tolerance takes no inner iterations in the next sweep.
constexpr double kSettledFrac = 1e-2;

struct SolveCounters {
    long long settled = 0;               // mixed block visits without inner iterations
    long long a64 = 0, a32 = 0;          // single-band H applications (FP64, FP32)
    long long visits32 = 0, visits64 = 0;  // block visits per precision
    int iters = 0;                       // Algorithm 1 iterations
};

// Solve one k-point for M bands of which the first Mreq must converge (the rest are buffer bands).
int solve_k(lobpcg_ctx *c, Lane &L, int k, int M, int Mreq, z64 *X, double *eig_h, double *res_h, int &sweeps_done,
            Prof *prof, SolveCounters &cnt, bool real = false) {
    L.clear_graphs();  // buffers may have moved since an earlier solve
    // whatever way this returns, no side-stream work (reading X) outlives it
    struct SideSync {
        Lane &L;
        ~SideSync() {
            if (L.side && L.side->stream) cudaStreamSynchronize(L.side->stream);
        }
    } side_sync{L};
    Solver sv;
    sv.c = c;
    sv.L = &L;
    sv.prof = prof;
    sv.k = k;
    sv.real = real;
    sv.npw = real ? c->kp[k].n_half : c->kp[k].npw;
    sv.kin = real ? c->kp[k].kin_half64 : c->kp[k].kin64;
    sv.M = M;
    sv.m = c->opt.block_size;
    sv.nblk = M / sv.m;
    sv.mixed = c->opt.precision == LOBPCG_MIXED;
    sv.df = c->opt.fp64_gemm >= 2 || (c->opt.fp64_gemm == 0 && sv.mixed);
    L.ew.df = sv.df;  // the Rayleigh-Ritz step's FP64-unit-bound parts likewise
    // the tall FP64-class GEMMs on the tensor cores (exact digit slices); the side lane of the
    // H X refresh follows (its KB projections)
    L.gw.oz = c->opt.fp64_gemm == 3 || (c->opt.fp64_gemm == 0 && sv.mixed);
    sv.X = X;
    sv.s = L.stream;
    sv.drop_tol = 1e-12;
    sv.drop_tol32 = 1e-3;
    if (const char *v = std::getenv("LOBPCG_VERBOSE")) sv.verbose = std::atoi(v);
    const int npw = sv.npw, m = sv.m;
    const int nzmax = std::max(3 * m, M);
    int rc = 0;
    const int zcols = 3 * m;   // a mixed solve visits converged blocks in FP64
    for (int i = 0; i < 2; ++i) {
        sv.Z[i] = carve<z64>(c, L.Zb[i], (size_t)npw * zcols, rc); LG_TRY(rc);
        sv.HZ[i] = carve<z64>(c, L.HZb[i], (size_t)npw * zcols, rc); LG_TRY(rc);
    }
    sv.HX = carve<z64>(c, L.HXall, (size_t)npw * M, rc); LG_TRY(rc);
    if (c->opt.precision == LOBPCG_MIXED) {
        sv.HXr = carve<z64>(c, L.HXr, (size_t)npw * M, rc); LG_TRY(rc);
        LG_TRY(L.make_side(&c->alloc));
        L.side->gw.oz = L.gw.oz;
    }
    sv.Tmp = carve<z64>(c, L.Tmp, (size_t)npw * M, rc); LG_TRY(rc);
    sv.S = carve<z64>(c, L.Gram, (size_t)nzmax * nzmax, rc); LG_TRY(rc);
    sv.A = carve<z64>(c, L.Gram2, (size_t)nzmax * nzmax, rc); LG_TRY(rc);
    sv.C = carve<z64>(c, L.Cbuf, (size_t)nzmax * nzmax, rc); LG_TRY(rc);
    sv.G = carve<z64>(c, L.Gc, (size_t)M * m, rc); LG_TRY(rc);
    sv.theta = carve<double>(c, L.dtheta, nzmax, rc); LG_TRY(rc);
    sv.res = carve<double>(c, L.dres, nzmax, rc); LG_TRY(rc);
    double *w = carve<double>(c, L.dwork, 4 * (size_t)nzmax + 64 + colsum_part_elems(nzmax), rc); LG_TRY(rc);
    sv.work = w;
    sv.ndrop = reinterpret_cast<int *>(w + 4 * (size_t)nzmax);
    sv.part = w + 4 * (size_t)nzmax + 64;  // partial sums of the per-column reductions
    if (sv.mixed) {
        sv.X32all = carve<c32>(c, L.X32all, (size_t)npw * M, rc); LG_TRY(rc);
        sv.HX32all = carve<c32>(c, L.HX32all, (size_t)npw * M, rc); LG_TRY(rc);
        for (int i = 0; i < 2; ++i) {
            sv.Q32[i] = carve<c32>(c, L.Q32[i], (size_t)npw * 3 * m, rc); LG_TRY(rc);
            sv.HQ32[i] = carve<c32>(c, L.HQ32[i], (size_t)npw * 3 * m, rc); LG_TRY(rc);
        }
        sv.X32 = carve<c32>(c, L.Z32, (size_t)npw * m, rc); LG_TRY(rc);
        sv.HX32 = carve<c32>(c, L.HZ32, (size_t)npw * m, rc); LG_TRY(rc);
        sv.D32 = carve<c32>(c, L.D32, (size_t)npw * m, rc); LG_TRY(rc);
        c32 *sm = carve<c32>(c, L.Small32, 3 * (size_t)nzmax * nzmax + (size_t)M * m, rc); LG_TRY(rc);
        sv.S32 = sm;
        sv.A32 = sm + (size_t)nzmax * nzmax;
        sv.C32 = sm + 2 * (size_t)nzmax * nzmax;
        sv.G32 = sm + 3 * (size_t)nzmax * nzmax;
        sv.T32 = carve<c32>(c, L.T32, (size_t)npw * M, rc); LG_TRY(rc);
        sv.E32 = carve<c32>(c, L.E32, (size_t)nzmax * nzmax, rc); LG_TRY(rc);
        sv.dmax = reinterpret_cast<unsigned int *>(w + 4 * (size_t)nzmax + 8);
        // H X of the start vectors, and the FP32 copies the constraint uses
        LG_TRY(sv.applyH64(X, sv.HX, M));
        LG_TRY(sv.cast<float, double>(M, X, sv.X32all));
        LG_TRY(sv.cast<float, double>(M, sv.HX, sv.HX32all));
    }
    sweeps_done = 0;
    double maxr = 0.0;
    // residuals of the previous sweep choose each block's precision in a mixed solve
    std::vector<double> res_prev(M, HUGE_VAL);
    // per block: H X_b holds FP64 accuracy (false after an early visit or an early sweep end)
    std::vector<char> hx64(sv.nblk, 1);
    for (int sw = 0; sw < c->opt.max_sweeps; ++sw) {
        // Early visits (FP32 block start and X updates) only while every band of the block is
        // above mixed_early: bands nearer the FP32 noise of H X (~1e-7 |H|) get W directions
        // made of that noise, and their Rayleigh-Ritz steps then drop most of [W P] and lose
        // the block (seen with 2048 bands, whose lowest blocks converge sweeps before the top).
        std::vector<char> early_b(sv.nblk, 0);
        bool all_early = sv.mixed;
        for (int b = 0; b < sv.nblk; ++b) {
            double rmin = HUGE_VAL;
            for (int i = b * m; i < (b + 1) * m; ++i) rmin = std::min(rmin, res_prev[i]);
            early_b[b] = sv.mixed && c->opt.mixed_early > 0.0 && rmin > c->opt.mixed_early;
            all_early = all_early && early_b[b];
        }
        // a full sweep end needs H X of every block in FP64 class: computed beside the sweep
        const bool side = sv.mixed && !all_early;
        for (int b = 0; b < sv.nblk; ++b) {
            double rmin = HUGE_VAL;
            for (int i = b * m; i < (b + 1) * m; ++i) rmin = std::min(rmin, res_prev[i]);
            sv.early = early_b[b] != 0;
            if (sv.mixed && !sv.early && !hx64[b]) {
                // first full visit after early ones: H X_b in FP64 from X_b (its FP32 noise would
                // dominate the residuals of well converged bands)
                LG_TRY(sv.applyH64(sv.col(X, b * m), sv.col(sv.HX, b * m), m));
                LG_TRY(sv.refresh32(b));
            }
            hx64[b] = !sv.early;
            // A block whose bands all sit far below the tolerance keeps its block start (constraint
            // and the block's Rayleigh-Ritz) but takes no inner iterations: its residuals, hence its
            // W, are rounding noise there, and a Rayleigh-Ritz step on such a basis broke a
            // converged block of the 2048-band cell (residual 3e-12 -> 1 Ha in one iteration).
            double rmax = 0.0;
            for (int i = b * m; i < (b + 1) * m; ++i) rmax = std::max(rmax, res_prev[i]);
            const bool settled = sv.mixed && rmax < kSettledFrac * c->opt.tol;
            if (sv.mixed && !(rmin < c->opt.mixed_switch)) {
                LG_TRY(sv.block_mixed(b, settled ? 0 : c->opt.nline));
                if (settled) ++cnt.settled;
                ++cnt.visits32;
            } else {
                LG_TRY(sv.block64(b));
                if (sv.mixed) LG_TRY(sv.refresh32(b));
                ++cnt.visits64;
            }
            if (side) LG_TRY(sv.side_refresh(b));
        }
        sv.hxr_ready = side;
        // the sweep-end Rayleigh-Ritz runs on the FP32 copies only if every block was early; else
        // it takes the FP64 H X computed beside the sweep
        sv.early = all_early;
        if (all_early) std::fill(hx64.begin(), hx64.end(), 0);
        else std::fill(hx64.begin(), hx64.end(), 1);
        LG_TRY(sv.final_rr(eig_h, res_h));
        if (prof) prof->collect();
        ++sweeps_done;
        maxr = 0.0;
        bool finite = true;
        for (int i = 0; i < Mreq; ++i) {
            finite = finite && std::isfinite(res_h[i]) && std::isfinite(eig_h[i]);
            maxr = std::max(maxr, res_h[i]);
        }
        if (sv.verbose >= 1) fprintf(stderr, "[lobpcg] k=%d sweep=%d max_resid=%.3e\n", k, sw, maxr);
        LG_TRY(tc_check_error());
        if (!finite) return fail(LOBPCG_ERR_BREAKDOWN, "non-finite Ritz value or residual");
        std::copy(res_h, res_h + M, res_prev.begin());
        if (maxr <= c->opt.tol && !sv.early) break;
    }
    cnt.a64 += sv.applies64;
    cnt.a32 += sv.applies32;
    cnt.iters += sv.iterations;
    return maxr <= c->opt.tol ? LOBPCG_OK : LOBPCG_NOT_CONVERGED;
}

// Band-by-band PCG (the method Sec. 3.3 compares LOBPCG with) on one k-point for M bands of
// which the first Mreq must converge: every band in order, kept orthogonal to the bands before
// it, takes nline PCG iterations (pcg.cu); each sweep is closed by the same all-band
// Rayleigh-Ritz step and FP64 residual test as the LOBPCG sweeps.  FP64 schedule: FP64
// everywhere; MIXED: the H applications and GEMMs in the FP64-class engines (double-FP32 FFT
// passes, tensor-core digit-slice GEMMs); the band steps themselves are FP64.
int solve_pcg_k(lobpcg_ctx *c, Lane &L, int k, int M, int Mreq, z64 *X, double *eig_h, double *res_h,
                int &sweeps_done, Prof *prof, SolveCounters &cnt) {
    Solver sv;
    sv.c = c;
    sv.L = &L;
    sv.prof = prof;
    sv.k = k;
    sv.npw = c->kp[k].npw;
    sv.kin = c->kp[k].kin64;
    sv.M = M;
    sv.m = c->opt.block_size;
    sv.nblk = M / sv.m;
    sv.mixed = false;
    sv.df = c->opt.fp64_gemm >= 2 || (c->opt.fp64_gemm == 0 && c->opt.precision == LOBPCG_MIXED);
    L.ew.df = sv.df;
    L.gw.oz = c->opt.fp64_gemm == 3 || (c->opt.fp64_gemm == 0 && c->opt.precision == LOBPCG_MIXED);
    sv.X = X;
    sv.s = L.stream;
    sv.drop_tol = 1e-12;
    sv.drop_tol32 = 1e-3;
    const int npw = sv.npw;
    int rc = 0;
    sv.HX = carve<z64>(c, L.HXall, (size_t)npw * M, rc); LG_TRY(rc);
    sv.Tmp = carve<z64>(c, L.Tmp, (size_t)npw * M, rc); LG_TRY(rc);
    sv.S = carve<z64>(c, L.Gram, (size_t)M * M, rc); LG_TRY(rc);
    sv.A = carve<z64>(c, L.Gram2, (size_t)M * M, rc); LG_TRY(rc);
    sv.C = carve<z64>(c, L.Cbuf, (size_t)M * M, rc); LG_TRY(rc);
    sv.G = carve<z64>(c, L.Gc, (size_t)M, rc); LG_TRY(rc);
    sv.theta = carve<double>(c, L.dtheta, M, rc); LG_TRY(rc);
    sv.res = carve<double>(c, L.dres, M, rc); LG_TRY(rc);
    double *w = carve<double>(c, L.dwork, 4 * (size_t)M + 64 + colsum_part_elems(M), rc); LG_TRY(rc);
    sv.work = w;
    sv.ndrop = reinterpret_cast<int *>(w + 4 * (size_t)M);
    sv.part = w + 4 * (size_t)M + 64;
    z64 *vv = carve<z64>(c, L.pcgv, 6 * (size_t)npw, rc); LG_TRY(rc);
    double *ps = carve<double>(c, L.pcgs, pcg_scratch_doubles(npw, M), rc); LG_TRY(rc);
    PcgBand pb;
    pb.npw = npw;
    pb.s = sv.s;
    pb.kin = c->kp[k].kin64;
    pb.Y = X;
    pb.ldy = npw;
    pb.xi = vv;
    pb.eta = vv + npw;
    pb.d = vv + 2 * (size_t)npw;
    pb.dh = vv + 3 * (size_t)npw;
    pb.hd = vv + 4 * (size_t)npw;
    pcg_carve(pb, ps, npw, M);
    sweeps_done = 0;
    double maxr = 0.0;
    for (int sw = 0; sw < c->opt.max_sweeps; ++sw) {
        for (int n = 0; n < M; ++n) {
            pb.j = n;
            pb.x = sv.col(X, n);
            pb.hx = sv.col(sv.HX, n);
            LG_TRY(pb.prepare_start());
            LG_TRY(sv.applyH64(pb.x, pb.hx, 1));
            LG_TRY(pb.after_hx());
            for (int it = 0; it < c->opt.nline; ++it) {
                LG_TRY(pb.direction(it == 0));
                LG_TRY(sv.applyH64(pb.dh, pb.hd, 1));
                LG_TRY(pb.step());
                ++sv.iterations;
            }
        }
        sv.early = false;
        LG_TRY(sv.final_rr(eig_h, res_h));
        if (prof) prof->collect();
        ++sweeps_done;
        maxr = 0.0;
        bool finite = true;
        for (int i = 0; i < Mreq; ++i) {
            finite = finite && std::isfinite(res_h[i]) && std::isfinite(eig_h[i]);
            maxr = std::max(maxr, res_h[i]);
        }
        if (!finite) return fail(LOBPCG_ERR_BREAKDOWN, "non-finite Ritz value or residual");
        if (maxr <= c->opt.tol) break;
    }
    cnt.a64 += sv.applies64;
    cnt.iters += sv.iterations;
    return maxr <= c->opt.tol ? LOBPCG_OK : LOBPCG_NOT_CONVERGED;
}

int validate_options(const lobpcg_options &o) {
    if (o.block_size < 1) return fail(LOBPCG_ERR_ARG, "block_size must be >= 1");
    if (o.nline < 1) return fail(LOBPCG_ERR_ARG, "nline must be >= 1");
    if (o.max_sweeps < 1) return fail(LOBPCG_ERR_ARG, "max_sweeps must be >= 1");
    if (o.precision != LOBPCG_FP64 && o.precision != LOBPCG_MIXED) return fail(LOBPCG_ERR_ARG, "unknown precision");
    if (!(o.tol > 0.0)) return fail(LOBPCG_ERR_ARG, "tol must be > 0");
    if (3 * o.block_size > 4096) return fail(LOBPCG_ERR_ARG, "block_size too large (3 m must be <= 4096)");
    if (o.nbuf < 0) return fail(LOBPCG_ERR_ARG, "nbuf must be >= 0");
    if (o.gemm_split == 1) return fail(LOBPCG_ERR_UNSUPPORTED, "gemm_split 1 (BF16x3) is not built; use 2 (TF32x3)");
    if (o.gemm_split != 0 && o.gemm_split != 2 && o.gemm_split != 3)
        return fail(LOBPCG_ERR_ARG, "gemm_split must be 0, 2 or 3");
    if (!(o.mixed_switch >= 0.0)) return fail(LOBPCG_ERR_ARG, "mixed_switch must be >= 0");
    if (!(o.mixed_early >= 0.0)) return fail(LOBPCG_ERR_ARG, "mixed_early must be >= 0");
    if (o.fp64_gemm < 0 || o.fp64_gemm > 3) return fail(LOBPCG_ERR_ARG, "fp64_gemm must be 0, 1, 2 or 3");
    if (o.gamma_real != 0 && o.gamma_real != 1) return fail(LOBPCG_ERR_ARG, "gamma_real must be 0 or 1");
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
    opt->timing = 0;
    opt->nbuf = 0;
    opt->mixed_switch = 0.0;
    opt->mixed_early = 1e-3;
    opt->fp64_gemm = 0;
    opt->gamma_real = 0;
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
    const int N = cell->N;
    const size_t N3 = (size_t)N * N * N;
    // every argument is checked before the first device call
    for (size_t i = 0; i < N3; ++i)
        if (!std::isfinite(vloc_r[i])) return fail(LOBPCG_ERR_ARG, "vloc_r has non-finite values");
    for (int i = 0; i < 3 * nk; ++i)
        if (!std::isfinite(kpts[i])) return fail(LOBPCG_ERR_ARG, "non-finite k-point");
    for (int p = 0; p < nproj; ++p)
        if (!std::isfinite(proj_E[p])) return fail(LOBPCG_ERR_ARG, "proj_E has non-finite values");
    c->cell = *cell;
    c->nk = nk;
    c->nproj = nproj;
    // potential: [x][y][z] -> [z][x][y] (FP32 register FFT: [y][x][z]), scaled by 1/N^3
    // (the forward FFT's normalisation)
    std::vector<double> vt(N3);
    std::vector<float> vt32(N3);
    const double inv = 1.0 / (double)N3;
    const bool reg32 = fft_reg_supported(N);
    if (reg32) LG_TRY(fft_reg_prepare());
    for (int x = 0; x < N; ++x)
        for (int y = 0; y < N; ++y)
            for (int z = 0; z < N; ++z) {
                const double v = vloc_r[((size_t)x * N + y) * N + z] * inv;
                vt[((size_t)z * N + x) * N + y] = v;
                vt32[reg32 ? ((size_t)y * N + x) * N + z : ((size_t)z * N + x) * N + y] = (float)v;
            }
    LG_TRY(upload(c, &c->vt64, vt.data(), N3));
    {   // the same table as (hi, lo) FP32 pairs for the double-FP32 passes
        std::vector<float2> vp(N3);
        for (size_t i = 0; i < N3; ++i) {
            const float hi = (float)vt[i];
            vp[i] = make_float2(hi, (float)(vt[i] - (double)hi));
        }
        LG_TRY(upload(c, &c->vtdf, vp.data(), N3));
    }
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
        for (int d = 0; d < 3; ++d) c->kp[k].k[d] = kpts[3 * k + d];
        LG_TRY(build_basis(c, c->kp[k]));
    }
    LG_CUDA_TRY(cudaGetDevice(&c->device));
    LG_TRY(noalloc_prepare());
    LG_CUDA_TRY(cudaEventCreateWithFlags(&c->gate.ev, cudaEventDisableTiming));
    c->lanes.emplace_back(new Lane());
    c->lanes[0]->stream = c->stream;
    c->lanes[0]->bind(&c->alloc, nullptr, 1);
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
    if (!ctx->lanes.empty()) ctx->lanes[0]->stream = ctx->stream;
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

}  // extern "C"

namespace lg {
int ctx_local_view(const lobpcg_ctx *c, int k, LocalView *v) {
    if (!c || !v) return fail(LOBPCG_ERR_ARG, "ctx is NULL");
    if (k < 0 || k >= c->nk) return fail(LOBPCG_ERR_ARG, "k out of range");
    const KPoint &K = c->kp[k];
    v->geom = &K.geom;
    v->plan = &c->plan;
    v->npw = K.npw;
    v->kin64 = K.kin64;
    v->kin32 = K.kin32;
    v->vt64 = c->vt64;
    v->vt32 = c->vt32;
    v->tw64 = c->tw64;
    v->tw32 = c->tw32;
    v->stream = c->stream;
    v->device = c->device;
    return LOBPCG_OK;
}
bool is_device_pointer(const void *p) { return is_device_ptr(p); }
}  // namespace lg

extern "C" {

static int apply_impl(lobpcg_ctx *c, int k, const void *X, void *Y, int nb, int precision) {
    if (k < 0 || k >= c->nk) return fail(LOBPCG_ERR_ARG, "k out of range");
    if (nb < 0) return fail(LOBPCG_ERR_ARG, "nb must be >= 0");
    if (nb == 0) return LOBPCG_OK;
    if (!X || !Y) return fail(LOBPCG_ERR_ARG, "X and Y must not be NULL");
    if (precision != LOBPCG_C128 && precision != LOBPCG_C64 && precision != LOBPCG_C128_DF32 &&
        precision != LOBPCG_C128_TC)
        return fail(LOBPCG_ERR_ARG, "unknown precision");
    const int npw = c->kp[k].npw;
    const size_t esz = precision == LOBPCG_C64 ? sizeof(c32) : sizeof(z64);
    const size_t bytes = esz * (size_t)npw * nb;
    const char *xa = static_cast<const char *>(X), *ya = static_cast<const char *>(Y);
    if (xa < ya + bytes && ya < xa + bytes) return fail(LOBPCG_ERR_ARG, "X and Y overlap");
    const bool dx = is_device_ptr(X), dy = is_device_ptr(Y);
    const void *Xd = X;
    void *Yd = Y;
    Lane &L = *c->lanes[0];
    if (!dx) {
        LG_TRY(c->alloc.ensure(L.stageX, bytes));
        LG_CUDA_TRY(cudaMemcpyAsync(L.stageX.p, X, bytes, cudaMemcpyHostToDevice, c->stream));
        Xd = L.stageX.p;
    }
    if (!dy) {
        LG_TRY(c->alloc.ensure(L.stageY, bytes));
        Yd = L.stageY.p;
    }
    if (precision != LOBPCG_C64) {
        L.gw.oz = precision == LOBPCG_C128_TC;
        const int rc = apply_H_dev<double>(c, L, k, static_cast<const z64 *>(Xd), npw, static_cast<z64 *>(Yd), npw,
                                           nb, nullptr, precision == LOBPCG_C128_DF32 || precision == LOBPCG_C128_TC);
        L.gw.oz = false;
        LG_TRY(rc);
    }
    else
        LG_TRY(apply_H_dev<float>(c, L, k, static_cast<const c32 *>(Xd), npw, static_cast<c32 *>(Yd), npw, nb));
    if (!dy) {
        LG_CUDA_TRY(cudaMemcpyAsync(Y, Yd, bytes, cudaMemcpyDeviceToHost, c->stream));
    }
    if (!dx || !dy) LG_CUDA_TRY(cudaStreamSynchronize(c->stream));
    return LOBPCG_OK;
}

int lobpcg_apply_H(lobpcg_ctx *ctx, int k, const void *X, void *Y, int nb, int precision) {
    if (!ctx) return fail(LOBPCG_ERR_ARG, "ctx is NULL");
    set_gemm_mode(ctx->opt.gemm_split);
    return ret(ctx, apply_impl(ctx, k, X, Y, nb, precision));
}

static int density_impl(lobpcg_ctx *c, int k, const void *X, int nb, const double *f, double *rho, int precision) {
    if (k < 0 || k >= c->nk) return fail(LOBPCG_ERR_ARG, "k out of range");
    if (nb < 0) return fail(LOBPCG_ERR_ARG, "nb must be >= 0");
    if (nb == 0) return LOBPCG_OK;
    if (!X || !f || !rho) return fail(LOBPCG_ERR_ARG, "X, f and rho must not be NULL");
    if (precision != LOBPCG_C128 && precision != LOBPCG_C64 && precision != LOBPCG_C128_DF32)
        return fail(LOBPCG_ERR_ARG, "unknown precision");
    for (int b = 0; b < nb; ++b)
        if (!std::isfinite(f[b])) return fail(LOBPCG_ERR_ARG, "f has non-finite values");
    if (!is_device_ptr(X) || !is_device_ptr(rho)) return fail(LOBPCG_ERR_ARG, "X and rho must be device pointers");
    KPoint &K = c->kp[k];
    const FFTGeom &g = K.geom;
    Lane &L = *c->lanes[0];
    const bool f64 = precision != LOBPCG_C64;
    const size_t cb = f64 ? sizeof(z64) : sizeof(c32);
    const size_t per_band = cb * (size_t)g.Px * g.N * g.N;
    int nbatch = (int)std::max<size_t>(1, c->fft_budget / per_band);
    nbatch = std::min(std::min(nbatch, nb), 65535);
    LG_TRY(c->alloc.ensure(L.T2, per_band * nbatch));
    LG_TRY(c->alloc.ensure(L.occ, (sizeof(double) + sizeof(float)) * (size_t)nb));
    std::vector<float> f32(f, f + nb);
    double *fd = static_cast<double *>(L.occ.p);
    float *ff = reinterpret_cast<float *>(fd + nb);
    LG_CUDA_TRY(cudaMemcpyAsync(fd, f, sizeof(double) * nb, cudaMemcpyHostToDevice, c->stream));
    LG_CUDA_TRY(cudaMemcpyAsync(ff, f32.data(), sizeof(float) * nb, cudaMemcpyHostToDevice, c->stream));
    const double scale = 1.0 / (c->cell.a * c->cell.a * c->cell.a);   // psi = Omega^-1/2 sum c(G) e^{i(k+G).r}
    int rc;
    if (f64)
        rc = fft_density<double>(g, c->plan, static_cast<const z64 *>(X), K.npw, nb, c->tw64, fd, ff, scale, rho,
                                 reinterpret_cast<z64 *>(L.T2.p), nbatch, c->stream, precision == LOBPCG_C128_DF32);
    else
        rc = fft_density<float>(g, c->plan, static_cast<const c32 *>(X), K.npw, nb, c->tw32, fd, ff, scale, rho,
                                reinterpret_cast<c32 *>(L.T2.p), nbatch, c->stream, false);
    LG_TRY(rc);
    // the host copy of f32 must outlive its transfer
    LG_CUDA_TRY(cudaStreamSynchronize(c->stream));
    return LOBPCG_OK;
}

int lobpcg_density(lobpcg_ctx *ctx, int k, const void *X, int nb, const double *f, double *rho, int precision) {
    if (!ctx) return fail(LOBPCG_ERR_ARG, "ctx is NULL");
    return ret(ctx, density_impl(ctx, k, X, nb, f, rho, precision));
}

// Concurrent k-point lanes of one solve (k-points are independent, Sec. 5.2).
// (10 lanes for the 10-k-point cell measured slower than 4: 3.1 s against 2.65 s.)
constexpr int kMaxLanes = 4;

// Autotuner (options.autotune): for each k-point, the FFT scratch budget per band batch (which
// sets how many bands one launch of the FFT passes covers) of the FP32 H application and of the
// FP64-class one, timed with CUDA events on the lane's stream over candidates from 32 to 256 MB
// with nb = the block size.  Once per k-point and handle; its time is reported apart.
static int autotune_k(lobpcg_ctx *c, Lane &L, int k, bool df, int nb) {
    KPoint &K = c->kp[k];
    if (K.tuned) return LOBPCG_OK;
    const int npw = K.npw;
    DevBuf bx, by;
    int rc = c->alloc.ensure(bx, sizeof(z64) * (size_t)npw * nb);
    if (rc == LOBPCG_OK) rc = c->alloc.ensure(by, sizeof(z64) * (size_t)npw * nb);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (rc == LOBPCG_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        rc = fail(LOBPCG_ERR_CUDA, "autotune: event creation failed");
    if (rc == LOBPCG_OK && cudaMemsetAsync(bx.p, 0, sizeof(z64) * (size_t)npw * nb, L.stream) != cudaSuccess)
        rc = fail(LOBPCG_ERR_CUDA, "autotune: memset failed");
    const size_t cands[] = {(size_t)32 << 20, (size_t)64 << 20, (size_t)128 << 20, (size_t)256 << 20};
    for (int pass = 0; pass < 2 && rc == LOBPCG_OK; ++pass) {
        size_t &budget = pass == 0 ? K.fft_budget32 : K.fft_budget64;
        float best = 0.f;
        size_t best_b = 0;
        for (size_t b : cands) {
            budget = b;
            auto run = [&]() {
                if (pass == 0)
                    return apply_H_dev<float>(c, L, k, static_cast<const c32 *>(bx.p), npw, static_cast<c32 *>(by.p),
                                              npw, nb);
                return apply_H_dev<double>(c, L, k, static_cast<const z64 *>(bx.p), npw, static_cast<z64 *>(by.p),
                                           npw, nb, nullptr, df);
            };
            rc = run();  // warm-up (allocates the scratch)
            if (rc != LOBPCG_OK) break;
            cudaEventRecord(e0, L.stream);
            for (int r = 0; r < 3 && rc == LOBPCG_OK; ++r) rc = run();
            cudaEventRecord(e1, L.stream);
            float ms = 0.f;
            if (rc == LOBPCG_OK &&
                (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                rc = fail(LOBPCG_ERR_CUDA, "autotune: timing failed");
            if (rc != LOBPCG_OK) break;
            if (best_b == 0 || ms < best) {
                best = ms;
                best_b = b;
            }
        }
        budget = best_b;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    c->alloc.release(bx);
    c->alloc.release(by);
    if (rc == LOBPCG_OK) K.tuned = true;
    return rc;
}

// One k-point on one lane: stage host vectors, add buffer bands, solve, copy back.
static int solve_one(lobpcg_ctx *c, Lane &L, int k, int M, int nbuf, void *Xk, double *eig_k, double *res_k,
                     int &sw, Prof *prof, SolveCounters &cnt, bool pcg) {
    auto run = [&](int MM, z64 *XX, double *ee, double *rr) {
        return pcg ? solve_pcg_k(c, L, k, MM, M, XX, ee, rr, sw, prof, cnt)
                   : solve_k(c, L, k, MM, M, XX, ee, rr, sw, prof, cnt);
    };
    const bool host = !is_device_ptr(Xk);
    const int npw = c->kp[k].npw;
    const size_t bytes = sizeof(z64) * (size_t)npw * M;
    z64 *Xd = static_cast<z64 *>(Xk);
    if (host) {
        LG_TRY(c->alloc.ensure(L.stageX, bytes));
        Xd = static_cast<z64 *>(L.stageX.p);
        LG_CUDA_TRY(cudaMemcpyAsync(Xd, Xk, bytes, cudaMemcpyHostToDevice, L.stream));
    }
    int rc;
    const KPoint &K = c->kp[k];
    if (!pcg && c->opt.gamma_real && K.gamma) {
        // Gamma real form: the start vectors projected onto it and packed on the half sphere
        // (n_half rows), buffer bands pseudo-random there (G = 0 component real), solved packed,
        // unpacked into the caller's sphere vectors (c(-G) = conj(c(G)))
        const int nz = K.n_half;
        LG_TRY(c->alloc.ensure(L.Xpk, sizeof(z64) * (size_t)nz * (M + nbuf)));
        z64 *Xp = static_cast<z64 *>(L.Xpk.p);
        LG_TRY(gamma_pack_full<double>(nz, M, Xd, npw, K.half, K.mirror, Xp, nz, L.stream));
        if (nbuf > 0) {
            LG_TRY(fill_random(nz, nbuf, Xp + (size_t)nz * M, nz, 0x51ED270Bu + 977u * (unsigned)k, L.stream));
            LG_TRY(zero_imag<double>(1, nbuf, Xp + (size_t)nz * M, nz, L.stream));
        }
        std::vector<double> ebuf(2 * (size_t)(M + nbuf));
        rc = solve_k(c, L, k, M + nbuf, M, Xp, ebuf.data(), ebuf.data() + (M + nbuf), sw, prof, cnt, true);
        if (rc < 0) return rc;
        LG_TRY(gamma_unpack_full<double>(nz, M, Xp, nz, K.half, K.mirror, Xd, npw, L.stream));
        LG_CUDA_TRY(cudaStreamSynchronize(L.stream));
        std::memcpy(eig_k, ebuf.data(), sizeof(double) * M);
        std::memcpy(res_k, ebuf.data() + (M + nbuf), sizeof(double) * M);
    } else if (nbuf > 0) {
        // buffer bands: an internal block of M + nbuf columns, the extra ones pseudo-random
        LG_TRY(c->alloc.ensure(L.Xext, sizeof(z64) * (size_t)npw * (M + nbuf)));
        z64 *Xe = static_cast<z64 *>(L.Xext.p);
        LG_CUDA_TRY(cudaMemcpyAsync(Xe, Xd, bytes, cudaMemcpyDeviceToDevice, L.stream));
        LG_TRY(fill_random(npw, nbuf, Xe + (size_t)npw * M, npw, 0x51ED270Bu + 977u * (unsigned)k, L.stream));
        std::vector<double> ebuf(2 * (size_t)(M + nbuf));
        rc = run(M + nbuf, Xe, ebuf.data(), ebuf.data() + (M + nbuf));
        if (rc < 0) return rc;
        LG_CUDA_TRY(cudaMemcpyAsync(Xd, Xe, bytes, cudaMemcpyDeviceToDevice, L.stream));
        LG_CUDA_TRY(cudaStreamSynchronize(L.stream));
        std::memcpy(eig_k, ebuf.data(), sizeof(double) * M);
        std::memcpy(res_k, ebuf.data() + (M + nbuf), sizeof(double) * M);
    } else {
        rc = run(M, Xd, eig_k, res_k);
        if (rc < 0) return rc;
    }
    if (host) {
        LG_CUDA_TRY(cudaMemcpyAsync(Xk, Xd, bytes, cudaMemcpyDeviceToHost, L.stream));
        LG_CUDA_TRY(cudaStreamSynchronize(L.stream));
    }
    return rc;
}

static int solve_impl(lobpcg_ctx *c, int M, void *const *X, double *eig, double *resid, lobpcg_stats *st,
                      bool pcg = false) {
    if (!X || !eig || !resid) return fail(LOBPCG_ERR_ARG, "X, eig and resid must not be NULL");
    const int m = c->opt.block_size;
    if (M < 1 || M % m) return fail(LOBPCG_ERR_ARG, "nbands must be a positive multiple of block_size");
    for (int k = 0; k < c->nk; ++k) {
        if (!X[k]) return fail(LOBPCG_ERR_ARG, "X[k] is NULL");
        const int nb_extra = c->opt.nbuf > 0 ? ((c->opt.nbuf + m - 1) / m) * m : 0;
        if (M + nb_extra > c->kp[k].npw)
            return fail(LOBPCG_ERR_ARG, "nbands (plus buffer bands) exceeds the plane-wave count");
        if (c->nproj > 0 && !c->kp[k].has_beta) return fail(LOBPCG_ERR_ARG, "projectors missing for a k-point");
    }
    double ms_tune = 0.0;
    bool untuned = false;
    for (int k = 0; k < c->nk; ++k) untuned = untuned || !c->kp[k].tuned;
    if (c->opt.autotune && untuned) {  // first solve of the handle: tune each k-point on lane 0, timed apart
        const auto ta = std::chrono::steady_clock::now();
        if (c->lanes.empty()) {
            std::unique_ptr<Lane> L(new Lane());
            c->lanes.push_back(std::move(L));
        }
        Lane &L0 = *c->lanes[0];
        L0.bind(&c->alloc, nullptr, 1);
        L0.stream = c->stream;
        const bool mixed = c->opt.precision == LOBPCG_MIXED;
        const bool df = c->opt.fp64_gemm >= 2 || (c->opt.fp64_gemm == 0 && mixed);
        L0.gw.oz = c->opt.fp64_gemm == 3 || (c->opt.fp64_gemm == 0 && mixed);
        int rc_t = LOBPCG_OK;
        for (int k = 0; k < c->nk && rc_t == LOBPCG_OK; ++k) rc_t = autotune_k(c, L0, k, df, m);
        L0.gw.oz = false;
        LG_TRY(rc_t);
        ms_tune = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - ta).count();
    }
    const auto t0 = std::chrono::steady_clock::now();
    const long long l0 = launch_count();
    const int nbuf = c->opt.nbuf > 0 ? ((c->opt.nbuf + m - 1) / m) * m : 0;
    // lanes: one per concurrent k-point, each on its own high-priority stream (so that the
    // low-priority side streams of the H X refresh only fill the gaps), all ordered after the work
    // already queued on the handle's stream; lane 0 returns to the handle's stream afterwards
    // as many lanes as k-points (up to kMaxLanes) while their buffers fit: about ten npw x (M +
    // buffer bands) complex128 arrays per lane, against the free memory (2 lanes for two 268k
    // plane-wave k-points of 2304 bands)
    int nl = std::max(1, std::min(c->nk, kMaxLanes));
    {
        size_t free_b = 0, total_b = 0;
        int npw_max = 1;
        for (int k = 0; k < c->nk; ++k) npw_max = std::max(npw_max, c->kp[k].npw);
        const double per_lane = 10.0 * 16.0 * npw_max * (double)(M + nbuf);
        if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess && per_lane > 0.0) {
            const int fit = (int)std::max(1.0, std::floor(0.9 * (double)free_b / per_lane));
            nl = std::max(1, std::min(nl, fit));
        }
    }
    int least = 0, greatest = 0;
    LG_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    if (c->lanes.empty()) c->lanes.push_back(std::unique_ptr<Lane>(new Lane()));
    while ((int)c->lanes.size() < nl) {
        std::unique_ptr<Lane> L(new Lane());
        LG_CUDA_TRY(cudaStreamCreateWithPriority(&L->stream, cudaStreamNonBlocking, greatest));
        L->own_stream = true;
        c->lanes.push_back(std::move(L));
    }
    if (!c->lanes[0]->solve_stream)
        LG_CUDA_TRY(cudaStreamCreateWithPriority(&c->lanes[0]->solve_stream, cudaStreamNonBlocking, greatest));
    for (int l = 0; l < nl; ++l) c->lanes[l]->bind(&c->alloc, nl > 1 ? &c->gate : nullptr, nl);
    c->lanes[0]->stream = c->lanes[0]->solve_stream;
    struct Lane0Back {  // lane 0 serves lobpcg_apply_H on the handle's stream
        lobpcg_ctx *c;
        ~Lane0Back() {
            cudaStreamSynchronize(c->lanes[0]->solve_stream);
            c->lanes[0]->stream = c->stream;
        }
    } lane0_back{c};
    c->gate.used = false;
    LG_CUDA_TRY(cudaEventRecord(c->gate.ev, c->stream));
    for (int l = 0; l < nl; ++l) LG_CUDA_TRY(cudaStreamWaitEvent(c->lanes[l]->stream, c->gate.ev, 0));
    std::vector<Prof> profs(nl);
    std::vector<SolveCounters> cnts(nl);
    std::vector<int> sweeps_k(c->nk, 0), rc_k(c->nk, LOBPCG_OK);
    std::vector<int> lane_rc(nl, LOBPCG_OK);
    std::vector<std::string> lane_err(nl);
    auto run_lane = [&](int l) {
        if (l > 0) cudaSetDevice(c->device);
        set_gemm_mode(c->opt.gemm_split);  // the engine choice is per host thread
        Prof &pr = profs[l];
        pr.on = c->opt.timing != 0;
        pr.s = c->lanes[l]->stream;
        for (int k = l; k < c->nk; k += nl) {
            const int rc = solve_one(c, *c->lanes[l], k, M, nbuf, X[k], eig + (size_t)k * M, resid + (size_t)k * M,
                                     sweeps_k[k], pr.on ? &pr : nullptr, cnts[l], pcg);
            if (rc < 0) {
                lane_rc[l] = rc;
                lane_err[l] = last_fail();
                return;
            }
            rc_k[k] = rc;
        }
        pr.collect();
    };
    if (nl == 1) {
        run_lane(0);
    } else {
        std::vector<std::thread> th;
        for (int l = 1; l < nl; ++l) th.emplace_back(run_lane, l);
        run_lane(0);
        for (auto &t : th) t.join();
        for (int l = 1; l < nl; ++l) LG_CUDA_TRY(cudaStreamSynchronize(c->lanes[l]->stream));
    }
    for (int l = 0; l < nl; ++l)
        if (lane_rc[l] < 0) return fail(lane_rc[l], lane_err[l]);
    int worst = LOBPCG_OK, sweeps = 0;
    double maxr = 0.0;
    SolveCounters cnt;
    for (int l = 0; l < nl; ++l) {
        cnt.a64 += cnts[l].a64;
        cnt.a32 += cnts[l].a32;
        cnt.visits32 += cnts[l].visits32;
        cnt.visits64 += cnts[l].visits64;
        cnt.settled += cnts[l].settled;
        cnt.iters += cnts[l].iters;
    }
    for (int k = 0; k < c->nk; ++k) {
        if (rc_k[k] == LOBPCG_NOT_CONVERGED) worst = LOBPCG_NOT_CONVERGED;
        sweeps = std::max(sweeps, sweeps_k[k]);
        for (int i = 0; i < M; ++i) maxr = std::max(maxr, resid[(size_t)k * M + i]);
    }
    if (st) {
        std::memset(st, 0, sizeof(*st));
        st->sweeps = sweeps;
        st->iterations = cnt.iters;
        st->converged = worst == LOBPCG_OK;
        st->max_resid = maxr;
        st->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        st->band_applies_fp64 = cnt.a64;
        st->band_applies_fp32 = cnt.a32;
        st->block_visits_fp32 = cnt.visits32;
        st->block_visits_fp64 = cnt.visits64;
        st->block_visits_settled = cnt.settled;
        st->ms_autotune = ms_tune;
        st->kernel_launches = launch_count() - l0;
        for (int l = 0; l < nl; ++l)
            for (int p = 0; p < LOBPCG_PH_COUNT; ++p) {
                const Prof &pr = profs[l];
                st->ph_ms[p] += pr.ms[p];
                st->ph_flops[p] += pr.flops[p];
                st->ph_bytes[p] += pr.bytes[p];
                st->ph_calls[p] += pr.calls[p];
                st->ph_fp64_flops[p] += pr.fp64_flops[p];
                st->ph_ms_fp64[p] += pr.ms64[p];
                st->ph_bytes_fp64[p] += pr.bytes64[p];
            }
    }
    return worst;
}

int lobpcg_solve(lobpcg_ctx *ctx, int nbands, void *const *X, double *eig, double *resid, lobpcg_stats *stats) {
    if (!ctx) return fail(LOBPCG_ERR_ARG, "ctx is NULL");
    set_gemm_mode(ctx->opt.gemm_split);
    return ret(ctx, solve_impl(ctx, nbands, X, eig, resid, stats));
}

int lobpcg_solve_pcg(lobpcg_ctx *ctx, int nbands, void *const *X, double *eig, double *resid, lobpcg_stats *stats) {
    if (!ctx) return fail(LOBPCG_ERR_ARG, "ctx is NULL");
    set_gemm_mode(ctx->opt.gemm_split);
    return ret(ctx, solve_impl(ctx, nbands, X, eig, resid, stats, true));
}

int lobpcg_struct_sizes(int64_t *cell, int64_t *options, int64_t *stats) {
    if (cell) *cell = (int64_t)sizeof(lobpcg_cell);
    if (options) *options = (int64_t)sizeof(lobpcg_options);
    if (stats) *stats = (int64_t)sizeof(lobpcg_stats);
    return LOBPCG_OK;
}

long long lobpcg_launch_count(void) { return launch_count(); }

const char *lobpcg_last_error(const lobpcg_ctx *ctx) {
    if (!ctx) return global_error();
    return ctx->err.c_str();
}

void lobpcg_destroy(lobpcg_ctx *ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    for (auto &L : ctx->lanes) {
        if (L->stream) cudaStreamSynchronize(L->stream);
        L->release(ctx->alloc);
    }
    for (auto &b : ctx->owned) ctx->alloc.release(b);
    if (ctx->gate.ev) cudaEventDestroy(ctx->gate.ev);
    delete ctx;
}

}  // extern "C"
