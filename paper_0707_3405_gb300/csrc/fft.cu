// Local-potential application through a zero-padded 3D FFT (Sec. 2.2 item iii,
// Sec. 4.1: the paper applies v_loc with Goedecker's FFT, which skips the
// zero planes of the plane-wave sphere).
//
// The sphere of one k-point occupies Px x-planes and Py y-rows of the N^3 box.
// Three passes per block of bands, each a batched 1D FFT in shared memory:
//   pass A  per (band, x-plane): scatter the plane's coefficients into a
//           Py x N (y, z) tile, inverse z-FFT of the occupied rows, then
//           inverse y-FFT of every z-line; write the plane to T2[b][px][z][y].
//   pass B  per (band, z, y-chunk): inverse x-FFT of the Px occupied planes
//           (zero-padded to N), multiply by V(r) / N^3, forward x-FFT, keep
//           the Px planes.
//   pass C  per (band, x-plane): forward y-FFT, keep the Py rows, forward
//           z-FFT, gather the sphere coefficients and add T(q) x(q).
// T2 holds Px N^2 complex numbers per band: half the box, as the sphere
// radius is a quarter of the box edge.
//
// 1D FFTs: Stockham autosort, mixed radix 8/4/2/5/3, in place in shared
// memory; each stage reads all its inputs into registers before a barrier
// and writes its outputs after it.  Twiddles e^{-2 pi i t/N} come from a
// host-computed FP64 table (rounded to the compute precision).
#include "common.cuh"
#include "df64.cuh"

#include <algorithm>
#include <cmath>
#include <type_traits>

namespace lg {

bool make_fft_plan(int N, FFTPlan &p, bool allow8) {
    p.N = N;
    p.nstage = 0;
    int r = N;
    if (N < 2) return false;
    const int pref[5] = {8, 4, 2, 5, 3};
    for (int f : pref) {
        if (f == 8 && !allow8) continue;
        while (r % f == 0) {
            if (p.nstage >= 12) return false;
            p.radix[p.nstage++] = f;
            r /= f;
        }
    }
    return r == 1;
}

namespace {

template <typename R>
__device__ __forceinline__ cx<R> mul_isg(cx<R> a, int sg) {  // a * (i * sg), sg = +-1
    return sg > 0 ? mkc<R>(-a.y, a.x) : mkc<R>(a.y, -a.x);
}

template <typename R, int RDX>
struct DFT;

template <typename R>
struct DFT<R, 2> {
    static __device__ __forceinline__ void run(cx<R> *v, int) {
        cx<R> a = v[0], b = v[1];
        v[0] = a + b;
        v[1] = a - b;
    }
};

template <typename R>
struct DFT<R, 3> {
    static __device__ __forceinline__ void run(cx<R> *v, int sg) {
        const R s3 = (R)0.86602540378443864676;  // sin(2 pi / 3)
        cx<R> a = v[0], t1 = v[1] + v[2];
        cx<R> t2 = a - (R)0.5 * t1;
        cx<R> t3 = s3 * mul_isg(v[1] - v[2], sg);
        v[0] = a + t1;
        v[1] = t2 + t3;
        v[2] = t2 - t3;
    }
};

template <typename R>
struct DFT<R, 4> {
    static __device__ __forceinline__ void run(cx<R> *v, int sg) {
        cx<R> t0 = v[0] + v[2], t1 = v[0] - v[2];
        cx<R> t2 = v[1] + v[3], t3 = mul_isg(v[1] - v[3], sg);
        v[0] = t0 + t2;
        v[2] = t0 - t2;
        v[1] = t1 + t3;
        v[3] = t1 - t3;
    }
};

template <typename R>
struct DFT<R, 5> {
    static __device__ __forceinline__ void run(cx<R> *v, int sg) {
        const R c1 = (R)0.30901699437494742410;   // cos(2 pi / 5)
        const R c2 = (R)-0.80901699437494742410;  // cos(4 pi / 5)
        const R s1 = (R)0.95105651629515357212;   // sin(2 pi / 5)
        const R s2 = (R)0.58778525229247312917;   // sin(4 pi / 5)
        cx<R> a = v[0];
        cx<R> bpe = v[1] + v[4], bme = v[1] - v[4];
        cx<R> cpd = v[2] + v[3], cmd = v[2] - v[3];
        cx<R> r1 = a + c1 * bpe + c2 * cpd;
        cx<R> r2 = a + c2 * bpe + c1 * cpd;
        cx<R> i1 = mul_isg(s1 * bme + s2 * cmd, sg);
        cx<R> i2 = mul_isg(s2 * bme - s1 * cmd, sg);
        v[0] = a + bpe + cpd;
        v[1] = r1 + i1;
        v[4] = r1 - i1;
        v[2] = r2 + i2;
        v[3] = r2 - i2;
    }
};

template <typename R>
struct DFT<R, 8> {
    static __device__ __forceinline__ void run(cx<R> *v, int sg) {
        const R h = (R)0.70710678118654752440;  // 1/sqrt(2)
        cx<R> e[4] = {v[0], v[2], v[4], v[6]};
        cx<R> o[4] = {v[1], v[3], v[5], v[7]};
        DFT<R, 4>::run(e, sg);
        DFT<R, 4>::run(o, sg);
        // o_p *= e^{sg 2 pi i p / 8}
        o[1] = h * (o[1] + mul_isg(o[1], sg));
        o[2] = mul_isg(o[2], sg);
        o[3] = h * (mul_isg(o[3], sg) - o[3]);
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            v[p] = e[p] + o[p];
            v[p + 4] = e[p] - o[p];
        }
    }
};

// One Stockham stage over `nlines` lines (all butterflies held in registers
// between the two barriers, so the stage can run in place).
// NC > 0: the line length and the stage's Ns are the compile-time NC and NSC (constant index
// arithmetic); NC = 0: the runtime N and Ns.
template <typename R, int RDX, int VPT, int NC = 0, int NSC = 1>
__device__ __forceinline__ void fft_stage(cx<R> *buf, int nlines, int ls, int es, int N_, int Ns_,
                                          const cx<R> *tw, int sg) {
    constexpr int NB = (VPT + RDX - 1) / RDX;
    const int N = NC ? NC : N_;
    const int Ns = NC ? NSC : Ns_;
    const int bpl = N / RDX;
    const int total = nlines * bpl;
    const int tstride = N / (Ns * RDX);
    cx<R> v[NB][RDX];
    int off[NB], kk[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int t = threadIdx.x + b * blockDim.x;
        off[b] = -1;
        kk[b] = 0;
        if (t < total) {
            const int line = t / bpl;
            const int j = t - line * bpl;
            const cx<R> *L = buf + line * ls;
#pragma unroll
            for (int q = 0; q < RDX; ++q) v[b][q] = L[(j + q * bpl) * es];
            const int k = j % Ns;
            kk[b] = k;
            off[b] = line * ls + ((j - k) * RDX + k) * es;
        }
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        if (off[b] >= 0) {
            if (kk[b] != 0) {
#pragma unroll
                for (int q = 1; q < RDX; ++q) {
                    cx<R> w = tw[q * kk[b] * tstride];
                    if (sg > 0) w.y = -w.y;
                    v[b][q] = v[b][q] * w;
                }
            }
            DFT<R, RDX>::run(v[b], sg);
#pragma unroll
            for (int q = 0; q < RDX; ++q) buf[off[b] + q * Ns * es] = v[b][q];
        }
    }
    __syncthreads();
}

constexpr int kThreads = 256;
// Values per thread and stage: 8 (radix up to 8) for FP32 / FP64; the double-FP32 passes hold
// 4 (radix up to 5, no radix-8 stage) so that their pair arithmetic fits in half the registers
// and two blocks share an SM.
template <typename CT>
constexpr int vpt() { return sizeof(CT) == 8 && !std::is_same<CT, double>::value ? 4 : 8; }
template <typename CT>
constexpr bool radix8() { return vpt<CT>() == 8; }
// Threads of the plane passes (A, C): their shared plane tile allows one block per SM, so the
// double-FP32 passes, which fit 128 registers a thread, run 512 threads to keep 16 warps there.
// Pass B likewise: 512 threads take its 16 lines in one group (half the stage barriers).
template <typename CT>
constexpr int plane_threads() { return vpt<CT>() == 4 ? 512 : kThreads; }

// Radix of stage s of the plan make_fft_plan builds for N (0 past the last stage).
constexpr int plan_radix(int N, bool allow8, int s) {
    const int pref[5] = {8, 4, 2, 5, 3};
    int r = N, k = 0;
    for (int i = 0; i < 5; ++i) {
        const int f = pref[i];
        if (f == 8 && !allow8) continue;
        while (r % f == 0) {
            if (k == s) return f;
            r /= f;
            ++k;
        }
    }
    return 0;
}

// The stages of a compile-time plan for line length NC, from stage S on (Ns = NS).
template <typename R, int NC, int S = 0, int NS = 1>
__device__ __forceinline__ void fft_stages_c(cx<R> *b, int nl, int ls, int es, const cx<R> *tw, int sg) {
    constexpr int RDX = plan_radix(NC, radix8<R>(), S);
    if constexpr (RDX != 0) {
        fft_stage<R, RDX, vpt<R>(), NC, NS>(b, nl, ls, es, NC, NS, tw, sg);
        fft_stages_c<R, NC, S + 1, NS * RDX>(b, nl, ls, es, tw, sg);
    }
}

// In-place FFT of `nlines` lines (line stride ls, element stride es) by the whole block.
// sg = -1: forward (e^{-i...}); sg = +1: inverse without 1/N.  NC > 0: the plan of a line of
// NC points unrolled at compile time (plan.N must equal NC); NC = 0: the runtime plan.
template <typename R, int NC = 0>
__device__ void fft_lines(cx<R> *buf, int nlines, int ls, int es, const FFTPlan &plan, const cx<R> *tw, int sg) {
    constexpr int kVPT = vpt<R>();
    const int N = NC ? NC : plan.N;
    if constexpr (NC > 0) {
        int lpg = (int)(blockDim.x * kVPT) / N;
        if (lpg < 1) lpg = 1;
        for (int l0 = 0; l0 < nlines; l0 += lpg)
            fft_stages_c<R, NC>(buf + l0 * ls, min(lpg, nlines - l0), ls, es, tw, sg);
        return;
    }
    int lpg = (int)(blockDim.x * kVPT) / N;
    if (lpg < 1) lpg = 1;
    for (int l0 = 0; l0 < nlines; l0 += lpg) {
        const int nl = min(lpg, nlines - l0);
        cx<R> *b = buf + l0 * ls;
        int Ns = 1;
        for (int s = 0; s < plan.nstage; ++s) {
            const int r = plan.radix[s];
            switch (r) {
                case 8:
                    if constexpr (radix8<R>()) fft_stage<R, 8, kVPT>(b, nl, ls, es, N, Ns, tw, sg);
                    break;
                case 4: fft_stage<R, 4, kVPT>(b, nl, ls, es, N, Ns, tw, sg); break;
                case 2: fft_stage<R, 2, kVPT>(b, nl, ls, es, N, Ns, tw, sg); break;
                case 5: fft_stage<R, 5, kVPT>(b, nl, ls, es, N, Ns, tw, sg); break;
                default: fft_stage<R, 3, kVPT>(b, nl, ls, es, N, Ns, tw, sg); break;
            }
            Ns *= r;
        }
    }
}

// R: storage type of X, Y, V, T and the twiddles; CT: compute type of the transforms and of
// the half-box scratch T2 (double-FP32 for FP64 data on a GPU with few FP64 units).
template <typename CT, typename R>
__device__ __forceinline__ cx<CT> to_ct(cx<R> v) {
    if constexpr (std::is_same<CT, R>::value) return v;
    else return mkc<CT>((CT)v.x, (CT)v.y);
}

template <typename R, typename CT = R, int NC = 0>
__global__ void __launch_bounds__(plane_threads<CT>())
k_pass_a(const cx<R> *__restrict__ X, int ldx, cx<CT> *__restrict__ T2, FFTPlan plan, int Px, int Py, int ny0m,
         const int *__restrict__ plane_begin, const int2 *__restrict__ yrange, const int *__restrict__ gmap,
         const cx<R> *__restrict__ twg, int zc_max) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = NC ? NC : plan.N;
    cx<CT> *tw = reinterpret_cast<cx<CT> *>(smem_raw);
    cx<CT> *A = tw + N;
    cx<CT> *L = A + Py * N;
    const int lsL = N + 1;
    const int px = blockIdx.x, b = blockIdx.y;
    const cx<R> *Xb = X + (size_t)b * ldx;
    const cx<CT> zero = mkc<CT>(0, 0);
    for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = to_ct<CT>(twg[i]);
    for (int i = threadIdx.x; i < Py * N; i += blockDim.x) A[i] = zero;
    __syncthreads();
    const int g0 = plane_begin[px], g1 = plane_begin[px + 1];
    for (int g = g0 + threadIdx.x; g < g1; g += blockDim.x) A[gmap[g]] = to_ct<CT>(Xb[g]);
    __syncthreads();
    const int2 yr = yrange[px];
    fft_lines<CT, NC>(A + yr.x * N, yr.y - yr.x + 1, N, 1, plan, tw, 1);
    cx<CT> *out = T2 + ((size_t)b * Px + px) * (size_t)N * N;  // [z][y]
    for (int z0 = 0; z0 < N; z0 += zc_max) {
        const int nz = min(zc_max, N - z0);
        for (int i = threadIdx.x; i < nz * N; i += blockDim.x) {
            const int zc = i % nz, iy = i / nz;
            int py = iy - ny0m;
            if (py < 0) py += N;
            L[zc * lsL + iy] = (py < Py) ? A[py * N + z0 + zc] : zero;
        }
        __syncthreads();
        fft_lines<CT, NC>(L, nz, lsL, 1, plan, tw, 1);
        for (int i = threadIdx.x; i < nz * N; i += blockDim.x) {
            const int zc = i / N, iy = i - zc * N;
            out[(size_t)(z0 + zc) * N + iy] = L[zc * lsL + iy];
        }
        __syncthreads();
    }
}

template <typename R, typename CT = R, int NC = 0>
__global__ void __launch_bounds__(plane_threads<CT>())
k_pass_b(cx<CT> *__restrict__ T2, FFTPlan plan, int Px, int nx0m, const R *__restrict__ vt,
         const CT *__restrict__ vtc, const cx<R> *__restrict__ twg, int yc) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = NC ? NC : plan.N;
    cx<CT> *tw = reinterpret_cast<cx<CT> *>(smem_raw);
    cx<CT> *L = tw + N;
    const int lsL = N + 1;
    const int y0 = blockIdx.x * yc, z = blockIdx.y, b = blockIdx.z;
    const int ny = min(yc, N - y0);
    const cx<CT> zero = mkc<CT>(0, 0);
    for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = to_ct<CT>(twg[i]);
    for (int i = threadIdx.x; i < ny * lsL; i += blockDim.x) L[i] = zero;
    __syncthreads();
    const size_t NN = (size_t)N * N;
    cx<CT> *base = T2 + (size_t)b * Px * NN + (size_t)z * N + y0;
    for (int i = threadIdx.x; i < Px * ny; i += blockDim.x) {
        const int px = i / ny, yy = i - px * ny;
        int ix = nx0m + px;
        if (ix >= N) ix -= N;
        L[yy * lsL + ix] = base[(size_t)px * NN + yy];
    }
    __syncthreads();
    fft_lines<CT, NC>(L, ny, lsL, 1, plan, tw, 1);
    // V in the compute type: from vtc when given (no conversion), else converted here
    const R *vz = vt + (size_t)z * NN + y0;
    const CT *vcz = vtc ? vtc + (size_t)z * NN + y0 : nullptr;
    for (int i = threadIdx.x; i < ny * N; i += blockDim.x) {
        const int ix = i / ny, yy = i - ix * ny;
        const CT vv = vcz ? vcz[(size_t)ix * N + yy] : (CT)vz[(size_t)ix * N + yy];
        L[yy * lsL + ix] = vv * L[yy * lsL + ix];
    }
    __syncthreads();
    fft_lines<CT, NC>(L, ny, lsL, 1, plan, tw, -1);
    for (int i = threadIdx.x; i < Px * ny; i += blockDim.x) {
        const int px = i / ny, yy = i - px * ny;
        int ix = nx0m + px;
        if (ix >= N) ix -= N;
        base[(size_t)px * NN + yy] = L[yy * lsL + ix];
    }
}

template <typename R, typename CT = R, int NC = 0>
__global__ void __launch_bounds__(plane_threads<CT>())
k_pass_c(const cx<CT> *__restrict__ T2, cx<R> *__restrict__ Y, int ldy, const cx<R> *__restrict__ X, int ldx,
         const R *__restrict__ kin, FFTPlan plan, int Px, int Py, int ny0m, const int *__restrict__ plane_begin,
         const int2 *__restrict__ yrange, const int *__restrict__ gmap, const cx<R> *__restrict__ twg,
         int zc_max) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = NC ? NC : plan.N;
    cx<CT> *tw = reinterpret_cast<cx<CT> *>(smem_raw);
    cx<CT> *A = tw + N;
    cx<CT> *L = A + Py * N;
    const int lsL = N + 1;
    const int px = blockIdx.x, b = blockIdx.y;
    for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = to_ct<CT>(twg[i]);
    __syncthreads();
    const cx<CT> *in = T2 + ((size_t)b * Px + px) * (size_t)N * N;  // [z][y]
    for (int z0 = 0; z0 < N; z0 += zc_max) {
        const int nz = min(zc_max, N - z0);
        for (int i = threadIdx.x; i < nz * N; i += blockDim.x) {
            const int zc = i / N, iy = i - zc * N;
            L[zc * lsL + iy] = in[(size_t)(z0 + zc) * N + iy];
        }
        __syncthreads();
        fft_lines<CT, NC>(L, nz, lsL, 1, plan, tw, -1);
        for (int i = threadIdx.x; i < nz * Py; i += blockDim.x) {
            const int zc = i % nz, py = i / nz;
            int iy = py + ny0m;
            if (iy >= N) iy -= N;
            A[py * N + z0 + zc] = L[zc * lsL + iy];
        }
        __syncthreads();
    }
    const int2 yr = yrange[px];
    fft_lines<CT, NC>(A + yr.x * N, yr.y - yr.x + 1, N, 1, plan, tw, -1);
    const int g0 = plane_begin[px], g1 = plane_begin[px + 1];
    cx<R> *Yb = Y + (size_t)b * ldy;
    const cx<R> *Xb = X + (size_t)b * ldx;
    for (int g = g0 + threadIdx.x; g < g1; g += blockDim.x) {
        cx<CT> v = A[gmap[g]];
        if (kin) v = v + (CT)kin[g] * to_ct<CT>(Xb[g]);
        if constexpr (std::is_same<CT, R>::value) Yb[g] = v;
        else Yb[g] = mkc<R>((R)v.x, (R)v.y);
    }
}

// Density pass (after pass A, Sec. 2.1 first step of the SC loop, by the same FFT as the local
// potential, Sec. 2.2 item iii): per (y chunk, z) block, for the batch's bands in band order,
// inverse x-FFT of the zero-padded lines and acc(x, y, z) += f_b |psi_b|^2 in shared memory; the
// block then adds scale * acc to rho[x][y][z].  No atomics: every grid point belongs to one block.
template <typename R, typename CT = R>
__global__ void __launch_bounds__(kThreads)
k_pass_d(const cx<CT> *__restrict__ T2, FFTPlan plan, int Px, int nx0m, const cx<R> *__restrict__ twg, int yc,
         int nbb, const double *__restrict__ f, double scale, double *__restrict__ rho) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = plan.N;
    cx<CT> *tw = reinterpret_cast<cx<CT> *>(smem_raw);
    cx<CT> *L = tw + N;
    const int lsL = N + 1;
    CT *acc = reinterpret_cast<CT *>(L + (size_t)yc * lsL);
    const int y0 = blockIdx.x * yc, z = blockIdx.y;
    const int ny = min(yc, N - y0);
    const cx<CT> zero = mkc<CT>(0, 0);
    for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = to_ct<CT>(twg[i]);
    for (int i = threadIdx.x; i < ny * N; i += blockDim.x) acc[i] = CT(0);
    const size_t NN = (size_t)N * N;
    for (int b = 0; b < nbb; ++b) {
        for (int i = threadIdx.x; i < ny * lsL; i += blockDim.x) L[i] = zero;
        __syncthreads();
        const cx<CT> *base = T2 + (size_t)b * Px * NN + (size_t)z * N + y0;
        for (int i = threadIdx.x; i < Px * ny; i += blockDim.x) {
            const int px = i / ny, yy = i - px * ny;
            int ix = nx0m + px;
            if (ix >= N) ix -= N;
            L[yy * lsL + ix] = base[(size_t)px * NN + yy];
        }
        __syncthreads();
        fft_lines<CT>(L, ny, lsL, 1, plan, tw, 1);
        const CT fb = CT(f[b]);
        for (int i = threadIdx.x; i < ny * N; i += blockDim.x) {
            const int ix = i / ny, yy = i - ix * ny;
            const cx<CT> v = L[yy * lsL + ix];
            acc[yy * N + ix] += fb * (v.x * v.x + v.y * v.y);
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < ny * N; i += blockDim.x) {
        const int ix = i / ny, yy = i - ix * ny;
        double *dst = rho + ((size_t)ix * N + y0 + yy) * N + z;
        *dst += scale * (double)acc[yy * N + ix];
    }
}

template <typename R>
size_t smem_ac(const FFTGeom &g, int zc) {
    return sizeof(cx<R>) * ((size_t)g.N + (size_t)g.Py * g.N + (size_t)zc * (g.N + 1));
}

int max_dyn_smem() {
    static std::atomic<int> cached{-1};
    int v = cached.load();
    if (v < 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || v <= 0)
            v = 48 * 1024;
        cached.store(v);
    }
    return v;
}

template <typename R>
int pick_zc(const FFTGeom &g) {
    const size_t lim = (size_t)max_dyn_smem();
    int zc = 16;
    while (zc > 1 && smem_ac<R>(g, zc) > lim) zc /= 2;
    if (smem_ac<R>(g, zc) > lim) return 0;
    return zc;
}

}  // namespace

double fft_flops_per_band(const FFTGeom &g) {
    const double N = g.N;
    const double line = 5.0 * N * std::log2(N);
    // pass A: occupied z-lines + Px N y-lines; pass B: 2 N^2 x-lines; pass C as A
    const double lines = 2.0 * (double)g.zlines + 2.0 * g.Px * N + 2.0 * N * N;
    return lines * line + 2.0 * N * N * N + 8.0 * g.npw;
}

template <typename R>
size_t fft_smem_need(const FFTGeom &g) {
    if (std::is_same<R, float>::value && fft_reg_supported(g.N)) {
        const size_t need = fft_reg_smem_need(g);
        return need <= (size_t)max_dyn_smem() ? need : 0;
    }
    const int zc = pick_zc<R>(g);
    return zc ? smem_ac<R>(g, zc) : 0;
}

namespace {

// The three passes over batches of bands; CT is the compute type (see k_pass_a); NC > 0: the
// kernels compiled for that grid edge.
template <typename R, typename CT, int NC>
int fft_passes_n(const FFTGeom &g, const FFTPlan &plan, const cx<R> *X, int ldx, cx<R> *Y, int ldy, int nb,
                 const R *kin, const R *vt, const CT *vtc, const cx<R> *tw, cx<CT> *T2, int nbatch, cudaStream_t s) {
    const int N = g.N;
    const int zc = pick_zc<R>(g);
    if (zc == 0) return fail(LOBPCG_ERR_UNSUPPORTED, "FFT grid too large for shared memory");
    const size_t sm_ac = smem_ac<R>(g, zc);
    const int yc = 16;
    const size_t sm_b = sizeof(cx<R>) * ((size_t)N + (size_t)yc * (N + 1));
    static std::atomic<bool> attr_set{false};
    if (!attr_set.load()) {
        const int lim = max_dyn_smem();
        LG_CUDA_TRY(cudaFuncSetAttribute(k_pass_a<R, CT, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
        LG_CUDA_TRY(cudaFuncSetAttribute(k_pass_b<R, CT, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
        LG_CUDA_TRY(cudaFuncSetAttribute(k_pass_c<R, CT, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
        attr_set.store(true);
    }
    const int ny0m = ((g.ny0 % N) + N) % N;
    const int nx0m = ((g.nx0 % N) + N) % N;
    for (int b0 = 0; b0 < nb; b0 += nbatch) {
        const int nbb = std::min(nbatch, nb - b0);
        const cx<R> *Xb = X + (size_t)b0 * ldx;
        cx<R> *Yb = Y + (size_t)b0 * ldy;
        k_pass_a<R, CT, NC><<<dim3(g.Px, nbb), plane_threads<CT>(), sm_ac, s>>>(Xb, ldx, T2, plan, g.Px, g.Py, ny0m, g.plane_begin,
                                                             g.plane_yrange, g.gmap, tw, zc);
        LG_TRY(check_launch("fft pass A"));
        k_pass_b<R, CT, NC><<<dim3((N + yc - 1) / yc, N, nbb), plane_threads<CT>(), sm_b, s>>>(T2, plan, g.Px, nx0m, vt, vtc, tw, yc);
        LG_TRY(check_launch("fft pass B"));
        k_pass_c<R, CT, NC><<<dim3(g.Px, nbb), plane_threads<CT>(), sm_ac, s>>>(T2, Yb, ldy, Xb, ldx, kin, plan, g.Px, g.Py, ny0m,
                                                             g.plane_begin, g.plane_yrange, g.gmap, tw, zc);
        LG_TRY(check_launch("fft pass C"));
    }
    return LOBPCG_OK;
}

// Grid edges of the benchmark cells get their own double-FP32 kernels (compile-time plan).
template <typename R, typename CT>
int fft_passes(const FFTGeom &g, const FFTPlan &plan, const cx<R> *X, int ldx, cx<R> *Y, int ldy, int nb,
               const R *kin, const R *vt, const CT *vtc, const cx<R> *tw, cx<CT> *T2, int nbatch, cudaStream_t s) {
    if constexpr (std::is_same<CT, df64f>::value) {
        switch (g.N) {
            case 72: return fft_passes_n<R, CT, 72>(g, plan, X, ldx, Y, ldy, nb, kin, vt, vtc, tw, T2, nbatch, s);
            case 96: return fft_passes_n<R, CT, 96>(g, plan, X, ldx, Y, ldy, nb, kin, vt, vtc, tw, T2, nbatch, s);
            case 120: return fft_passes_n<R, CT, 120>(g, plan, X, ldx, Y, ldy, nb, kin, vt, vtc, tw, T2, nbatch, s);
            case 160: return fft_passes_n<R, CT, 160>(g, plan, X, ldx, Y, ldy, nb, kin, vt, vtc, tw, T2, nbatch, s);
            default: break;
        }
    }
    return fft_passes_n<R, CT, 0>(g, plan, X, ldx, Y, ldy, nb, kin, vt, vtc, tw, T2, nbatch, s);
}

// rho += scale sum_b f_b |psi_b|^2 over batches of bands: pass A then the density pass.
template <typename R, typename CT>
int density_passes(const FFTGeom &g, const FFTPlan &plan, const cx<R> *X, int ldx, int nb, const cx<R> *tw,
                   const double *f, double scale, double *rho, cx<CT> *T2, int nbatch, cudaStream_t s) {
    const int N = g.N;
    const int zc = pick_zc<R>(g);
    if (zc == 0) return fail(LOBPCG_ERR_UNSUPPORTED, "FFT grid too large for shared memory");
    const size_t sm_ac = smem_ac<R>(g, zc);
    const int yc = 16;
    const size_t sm_d = sizeof(cx<CT>) * ((size_t)N + (size_t)yc * (N + 1)) + sizeof(CT) * (size_t)yc * N;
    static std::atomic<bool> attr_set{false};
    if (!attr_set.load()) {
        const int lim = max_dyn_smem();
        LG_CUDA_TRY(cudaFuncSetAttribute(k_pass_a<R, CT>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
        LG_CUDA_TRY(cudaFuncSetAttribute(k_pass_d<R, CT>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
        attr_set.store(true);
    }
    if (sm_d > (size_t)max_dyn_smem()) return fail(LOBPCG_ERR_UNSUPPORTED, "density pass exceeds shared memory");
    const int ny0m = ((g.ny0 % N) + N) % N;
    const int nx0m = ((g.nx0 % N) + N) % N;
    for (int b0 = 0; b0 < nb; b0 += nbatch) {
        const int nbb = std::min(nbatch, nb - b0);
        k_pass_a<R, CT><<<dim3(g.Px, nbb), plane_threads<CT>(), sm_ac, s>>>(X + (size_t)b0 * ldx, ldx, T2, plan, g.Px, g.Py,
                                                             ny0m, g.plane_begin, g.plane_yrange, g.gmap, tw, zc);
        LG_TRY(check_launch("density: fft pass A"));
        k_pass_d<R, CT><<<dim3((N + yc - 1) / yc, N), kThreads, sm_d, s>>>(T2, plan, g.Px, nx0m, tw, yc, nbb,
                                                                       f + b0, scale, rho);
        LG_TRY(check_launch("density: x-lines and |psi|^2"));
    }
    return LOBPCG_OK;
}

}  // namespace

template <typename R>
int fft_density(const FFTGeom &g, const FFTPlan &plan, const cx<R> *X, int ldx, int nb, const cx<R> *tw,
                const double *f, const float *f32, double scale, double *rho, cx<R> *T2, int nbatch, cudaStream_t s,
                bool df) {
    if (nb <= 0) return LOBPCG_OK;
    if constexpr (std::is_same<R, float>::value) {
        if (fft_reg_supported(g.N)) return fft_reg_density(g, X, ldx, nb, f32, scale, rho, T2, nbatch, s);
    } else {
        if (df) {
            FFTPlan p4;
            if (!make_fft_plan(g.N, p4, false)) return fail(LOBPCG_ERR_UNSUPPORTED, "FFT plan");
            return density_passes<R, df64f>(g, p4, X, ldx, nb, tw, f, scale, rho, reinterpret_cast<cx<df64f> *>(T2),
                                           nbatch, s);
        }
    }
    (void)f32;
    return density_passes<R, R>(g, plan, X, ldx, nb, tw, f, scale, rho, T2, nbatch, s);
}

template int fft_density<float>(const FFTGeom &, const FFTPlan &, const c32 *, int, int, const c32 *, const double *,
                                const float *, double, double *, c32 *, int, cudaStream_t, bool);
template int fft_density<double>(const FFTGeom &, const FFTPlan &, const z64 *, int, int, const z64 *,
                                 const double *, const float *, double, double *, z64 *, int, cudaStream_t, bool);

template <typename R>
int fft_vloc_apply(const FFTGeom &g, const FFTPlan &plan, const cx<R> *X, int ldx, cx<R> *Y, int ldy, int nb,
                   const R *kin, const R *vt, const cx<R> *tw, cx<R> *T2, int nbatch, cudaStream_t s, bool df,
                   const float2 *vt_pair) {
    if (nb <= 0) return LOBPCG_OK;
    if constexpr (std::is_same<R, float>::value) {
        if (fft_reg_supported(g.N)) return fft_reg_apply(g, X, ldx, Y, ldy, nb, kin, vt, T2, nbatch, s);
    } else {
        if (df) {  // FP64 data transformed in double-FP32 (the half box holds pairs of floats)
            FFTPlan p4;
            if (!make_fft_plan(g.N, p4, false)) return fail(LOBPCG_ERR_UNSUPPORTED, "FFT plan");
            return fft_passes<R, df64f>(g, p4, X, ldx, Y, ldy, nb, kin, vt,
                                        reinterpret_cast<const df64f *>(vt_pair), tw, reinterpret_cast<cx<df64f> *>(T2),
                                       nbatch, s);
        }
    }
    (void)vt_pair;
    return fft_passes<R, R>(g, plan, X, ldx, Y, ldy, nb, kin, vt, nullptr, tw, T2, nbatch, s);
}

template int fft_vloc_apply<float>(const FFTGeom &, const FFTPlan &, const c32 *, int, c32 *, int, int,
                                   const float *, const float *, const c32 *, c32 *, int, cudaStream_t, bool,
                                   const float2 *);
template int fft_vloc_apply<double>(const FFTGeom &, const FFTPlan &, const z64 *, int, z64 *, int, int,
                                    const double *, const double *, const z64 *, z64 *, int, cudaStream_t, bool,
                                    const float2 *);
template size_t fft_smem_need<float>(const FFTGeom &);
template size_t fft_smem_need<double>(const FFTGeom &);

}  // namespace lg
