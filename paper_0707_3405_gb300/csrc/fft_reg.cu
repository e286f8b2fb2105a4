// Register-resident FP32 line FFTs for the local-potential passes (Sec. 4.1:
// v_loc applied through Goedecker's zero-padded 3D FFT; Sec. 2.2 item iii).
//
// Same three passes as the shared-memory engine, with these differences:
//   * A length-N line is held in the registers of T adjacent lanes of one warp
//     (T = 2 or 4; E = N / T points per lane).  With the line split as
//     x[t + T e], each lane first runs an E-point DFT over e entirely in
//     registers (compile-time mixed radix 4/8/3/5/2), multiplies by the
//     W_N^{t k} twiddles, then the T lanes of the line swap values with warp
//     shuffles and finish with T-point DFTs.  The result sits in "block
//     layout": lane t holds outputs (t BK + i) + E k2, BK = ceil(E / T); where
//     T does not divide E (N = 72, 120 on four lanes) the last lane's trailing
//     slots are padding.  The reverse path (block layout in, strided layout
//     out) runs the same steps backwards.
//     No shared memory and no barrier inside a line FFT.
//   * The half-box scratch is laid out T2[b][px][y][z] (z fastest) and the
//     potential V(r) / N^3 as [y][x][z], so that the 32 / T lines of a warp
//     are consecutive z and every global load or store of a warp covers
//     whole 32-byte sectors.
//   * Pass A and pass C keep one x-plane in shared memory (row pitch N + 2,
//     which spreads the rows of a half-warp over all banks) between the z and
//     the y transforms; pass B touches no shared memory at all.
// Twiddles e^{-2 pi i j / N} are computed on the host in FP64, rounded to FP32
// and kept in constant memory; the ones with compile-time indices become
// immediate constant operands.
#include "common.cuh"

#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

namespace lg {

namespace {

// Grid edges with a register plan: T lanes per line (E = N / T points per lane,
// E / T an integer), and the offset of each edge's twiddles in the table.
constexpr int kRegN[] = {8, 12, 16, 20, 24, 36, 48, 64, 72, 96, 120, 128, 160};
constexpr int kNumRegN = sizeof(kRegN) / sizeof(kRegN[0]);
constexpr int tw_off(int N) {
    int off = 0;
    for (int i = 0; i < kNumRegN && kRegN[i] != N; ++i) off += kRegN[i];
    return off;
}
constexpr int kTwTotal = tw_off(-1);
constexpr int kMaxDevices = 64;

template <int N>
struct RP {
    // four lanes per line from N = 64 up (N a multiple of 4), else two
    static constexpr int T = (N % 16 == 0 || (N % 4 == 0 && N >= 64)) ? 4 : 2;
    static constexpr int E = N / T;                 // points per lane (strided layout)
    static constexpr int BK = (E + T - 1) / T;      // block-layout slots per output group
    static constexpr int VS = T * BK;               // register slots per lane (>= E)
    static constexpr int OFF = tw_off(N);
    // resident CTAs per SM the register budget is sized for (fewer for long per-lane lines)
    static constexpr int MINB = (E <= 24) ? 4 : (E <= 40) ? 3 : 2;
    static_assert(N % T == 0, "a line must split over its T lanes");
    static_assert(T == 4 || E % T == 0, "two-lane lines split into two blocks of E / 2 points");
    // block-layout slot i of lane t holds output group t BK + i, which exists for t BK + i < E
    static __device__ __forceinline__ bool slot_ok(int t, int i) { return t * BK + i < E; }
};

__constant__ float2 c_tw[kTwTotal];

using C = cx<float>;

template <int N, bool INV>
__device__ __forceinline__ C twc(int j) {  // W_N^{+-j}, j in [0, N)
    const float2 w = c_tw[RP<N>::OFF + j];
    return mkc<float>(w.x, INV ? -w.y : w.y);
}

template <bool INV>
__device__ __forceinline__ C mul_i(C a) {  // a * (+-i): +i for the inverse sign
    return INV ? mkc<float>(-a.y, a.x) : mkc<float>(a.y, -a.x);
}

// ------------------------------------------------------------- small DFTs
template <int R, bool INV>
struct Base;

template <bool INV>
struct Base<1, INV> {
    static __device__ __forceinline__ void run(C *) {}
};

template <bool INV>
struct Base<2, INV> {
    static __device__ __forceinline__ void run(C *v) {
        const C a = v[0], b = v[1];
        v[0] = a + b;
        v[1] = a - b;
    }
};

template <bool INV>
struct Base<3, INV> {
    static __device__ __forceinline__ void run(C *v) {
        const float s3 = 0.86602540378443864676f;  // sin(2 pi / 3)
        const C a = v[0], t1 = v[1] + v[2];
        const C t2 = a - 0.5f * t1;
        const C t3 = s3 * mul_i<INV>(v[1] - v[2]);
        v[0] = a + t1;
        v[1] = t2 + t3;
        v[2] = t2 - t3;
    }
};

template <bool INV>
struct Base<4, INV> {
    static __device__ __forceinline__ void run(C *v) {
        const C t0 = v[0] + v[2], t1 = v[0] - v[2];
        const C t2 = v[1] + v[3], t3 = mul_i<INV>(v[1] - v[3]);
        v[0] = t0 + t2;
        v[2] = t0 - t2;
        v[1] = t1 + t3;
        v[3] = t1 - t3;
    }
};

template <bool INV>
struct Base<5, INV> {
    static __device__ __forceinline__ void run(C *v) {
        const float c1 = 0.30901699437494742410f;   // cos(2 pi / 5)
        const float c2 = -0.80901699437494742410f;  // cos(4 pi / 5)
        const float s1 = 0.95105651629515357212f;   // sin(2 pi / 5)
        const float s2 = 0.58778525229247312917f;   // sin(4 pi / 5)
        const C a = v[0];
        const C bpe = v[1] + v[4], bme = v[1] - v[4];
        const C cpd = v[2] + v[3], cmd = v[2] - v[3];
        const C r1 = a + c1 * bpe + c2 * cpd;
        const C r2 = a + c2 * bpe + c1 * cpd;
        const C i1 = mul_i<INV>(s1 * bme + s2 * cmd);
        const C i2 = mul_i<INV>(s2 * bme - s1 * cmd);
        v[0] = a + bpe + cpd;
        v[1] = r1 + i1;
        v[4] = r1 - i1;
        v[2] = r2 + i2;
        v[3] = r2 - i2;
    }
};

template <bool INV>
struct Base<8, INV> {
    static __device__ __forceinline__ void run(C *v) {
        const float h = 0.70710678118654752440f;  // 1 / sqrt(2)
        C e[4] = {v[0], v[2], v[4], v[6]};
        C o[4] = {v[1], v[3], v[5], v[7]};
        Base<4, INV>::run(e);
        Base<4, INV>::run(o);
        o[1] = h * (o[1] + mul_i<INV>(o[1]));
        o[2] = mul_i<INV>(o[2]);
        o[3] = h * (mul_i<INV>(o[3]) - o[3]);
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            v[p] = e[p] + o[p];
            v[p + 4] = e[p] - o[p];
        }
    }
};

constexpr bool is_base(int E) { return E == 1 || E == 2 || E == 3 || E == 4 || E == 5 || E == 8; }
constexpr int pick_a(int E) {
    return (E % 4 == 0 && E / 4 > 1) ? 4 : (E % 8 == 0 && E / 8 > 1) ? 8 : (E % 3 == 0 && E / 3 > 1) ? 3
         : (E % 5 == 0 && E / 5 > 1) ? 5 : 2;
}

// E-point DFT of v in registers (Cooley-Tukey, E = A B with n = n1 + A n2, k = k2 + B k1);
// the inner twiddles W_E^{n1 k2} are W_N^{n1 k2 N / E}.
template <int E, int N, bool INV, bool BASE = is_base(E)>
struct RDFT;

template <int E, int N, bool INV>
struct RDFT<E, N, INV, true> {
    static __device__ __forceinline__ void run(C *v) { Base<E, INV>::run(v); }
};

template <int E, int N, bool INV>
struct RDFT<E, N, INV, false> {
    static constexpr int A = pick_a(E), B = E / A;
    static __device__ __forceinline__ void run(C *v) {
#pragma unroll
        for (int n1 = 0; n1 < A; ++n1) {
            C sub[B];
#pragma unroll
            for (int n2 = 0; n2 < B; ++n2) sub[n2] = v[n1 + A * n2];
            RDFT<B, N, INV>::run(sub);
#pragma unroll
            for (int k2 = 0; k2 < B; ++k2)
                v[n1 + A * k2] = (n1 * k2 == 0) ? sub[k2] : sub[k2] * twc<N, INV>(((n1 * k2) % E) * (N / E));
        }
        C out[E];
#pragma unroll
        for (int k2 = 0; k2 < B; ++k2) {
            C a[A];
#pragma unroll
            for (int n1 = 0; n1 < A; ++n1) a[n1] = v[n1 + A * k2];
            RDFT<A, N, INV>::run(a);
#pragma unroll
            for (int k1 = 0; k1 < A; ++k1) out[k2 + B * k1] = a[k1];
        }
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = out[e];
    }
};

__device__ __forceinline__ C shfl_xor_c(C a, int m) {
    return mkc<float>(__shfl_xor_sync(0xffffffffu, a.x, m), __shfl_xor_sync(0xffffffffu, a.y, m));
}

// 4 x 4 transpose across the four lanes t = 0..3 of a line: on return lane t holds, in a[s], the
// value lane s held in a[t].  Two butterfly stages: lanes t and t^1 swap the two elements whose
// index bit 0 differs from bit 0 of t, then lanes t and t^2 swap the two whose bit 1 differs from
// bit 1 of t (12 selects and 4 shuffles per stage).  Pure data movement: the values are those of
// any other exchange, bit for bit.
__device__ __forceinline__ void xpose4(C (&a)[4], int t) {
    const bool b0 = (t & 1) != 0;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const C send = b0 ? a[2 * k] : a[2 * k + 1];
        const C recv = shfl_xor_c(send, 1);
        a[2 * k] = b0 ? recv : a[2 * k];
        a[2 * k + 1] = b0 ? a[2 * k + 1] : recv;
    }
    const bool b1 = (t & 2) != 0;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const C send = b1 ? a[k] : a[k + 2];
        const C recv = shfl_xor_c(send, 2);
        a[k] = b1 ? recv : a[k];
        a[k + 2] = b1 ? a[k + 2] : recv;
    }
}

// Strided -> block: in v[e] = x[t + T e] (e < E); out v[i + BK k2] = X[(t BK + i) + E k2] for the
// slots with t BK + i < E (BK = ceil(E / T); with four lanes and E not a multiple of 4 the last
// lane's trailing slots are padding, exchanged as zeros and never stored).
template <int N, bool INV>
__device__ __forceinline__ void s2b(C *v, int t) {
    constexpr int T = RP<N>::T, E = RP<N>::E, BK = RP<N>::BK, VS = RP<N>::VS;
    RDFT<E, N, INV>::run(v);
    if constexpr (T == 2) {
#pragma unroll
        for (int k = 1; k < E; ++k) v[k] = t ? v[k] * twc<N, INV>(k) : v[k];
        C out[E];
#pragma unroll
        for (int i = 0; i < BK; ++i) {
            const C own = t ? v[BK + i] : v[i];
            const C snd = t ? v[i] : v[BK + i];
            const C rcv = shfl_xor_c(snd, 1);
            const C a = t ? rcv : own, b = t ? own : rcv;
            out[i] = a + b;
            out[i + BK] = a - b;
        }
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = out[e];
    } else if constexpr (T == 4) {
#pragma unroll
        for (int k = 1; k < E; ++k) v[k] = v[k] * twc<N, INV>((t * k) % N);
        const C zero = mkc<float>(0.f, 0.f);
        C out[VS];
#pragma unroll
        for (int i = 0; i < BK; ++i) {
            C w[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) w[q] = (q * BK + i < E) ? v[q * BK + i] : zero;
            xpose4(w, t);   // w[s] = lane s's v[t BK + i]
            Base<4, INV>::run(w);
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) out[i + BK * k2] = w[k2];
        }
#pragma unroll
        for (int e = 0; e < VS; ++e) v[e] = out[e];
    }
}

// Block -> strided: in v[i + BK x2] = x[(t BK + i) + E x2] (valid slots); out v[e] = X[t + T e].
template <int N, bool INV>
__device__ __forceinline__ void b2s(C *v, int t) {
    constexpr int T = RP<N>::T, E = RP<N>::E, BK = RP<N>::BK;
    if constexpr (T == 2) {
        C out[E];
#pragma unroll
        for (int i = 0; i < BK; ++i) {
            const C a = v[i], b = v[i + BK];
            const C u0 = a + b;
            const C u1 = (a - b) * (t ? twc<N, INV>(BK + i) : twc<N, INV>(i));
            const C rcv = shfl_xor_c(t ? u0 : u1, 1);
            const C keep = t ? u1 : u0;
            out[i] = t ? rcv : keep;
            out[BK + i] = t ? keep : rcv;
        }
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = out[e];
    } else if constexpr (T == 4) {
        C out[E];
#pragma unroll
        for (int i = 0; i < BK; ++i) {
            C w[4] = {v[i], v[i + BK], v[i + 2 * BK], v[i + 3 * BK]};
            Base<4, INV>::run(w);
            const int x1 = t * BK + i;   // a padding slot's twiddle index stays inside [0, N)
#pragma unroll
            for (int s = 1; s < 4; ++s) w[s] = w[s] * twc<N, INV>((x1 * s) % N);
            xpose4(w, t);   // w[s] = lane s's w[t]
#pragma unroll
            for (int s = 0; s < 4; ++s)
                if (s * BK + i < E) out[s * BK + i] = w[s];
        }
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = out[e];
    }
    RDFT<E, N, INV>::run(v);
}

constexpr int kWarps = 4;  // warps per CTA

// ------------------------------------------------------------- pass B
// One warp per (band, y, chunk of 32/T consecutive z): inverse x-FFT of the
// Px occupied planes (zero-padded to N), times V(r) / N^3, forward x-FFT,
// keep the Px planes.  T2 is updated in place.
template <int N>
__global__ void __launch_bounds__(32 * kWarps, RP<N>::MINB)
k_rb(C *__restrict__ T2, int Px, int nx0m, const float *__restrict__ vr) {
    constexpr int T = RP<N>::T, E = RP<N>::E, BK = RP<N>::BK, VS = RP<N>::VS, LPW = 32 / T;
    constexpr int NZC = (N + LPW - 1) / LPW;
    const int lane = threadIdx.x & 31;
    const int w = blockIdx.x * kWarps + (threadIdx.x >> 5);
    const int y = w / NZC, zc = w - y * NZC;
    if (y >= N) return;
    const int l = lane / T, t = lane - l * T;
    const int z = zc * LPW + l;
    const bool ok = z < N;
    const size_t NN = (size_t)N * N;
    C *base = T2 + (size_t)blockIdx.y * Px * NN + (size_t)y * N + z;
    C v[VS];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        int px = t + T * e - nx0m;
        px += (px < 0) ? N : 0;
        v[e] = (ok && px < Px) ? base[(size_t)px * NN] : mkc<float>(0.f, 0.f);
    }
    s2b<N, true>(v, t);
    const float *vy = vr + (size_t)y * NN + z;
#pragma unroll
    for (int k2 = 0; k2 < T; ++k2)
#pragma unroll
        for (int i = 0; i < BK; ++i) {
            const int x = t * BK + i + E * k2;
            v[i + BK * k2] = (ok && RP<N>::slot_ok(t, i) ? vy[(size_t)x * N] : 0.f) * v[i + BK * k2];
        }
    b2s<N, false>(v, t);
    if (!ok) return;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        int px = t + T * e - nx0m;
        px += (px < 0) ? N : 0;
        if (px < Px) base[(size_t)px * NN] = v[e];
    }
}

// ------------------------------------------------------------- density pass
// After pass A: one warp per (y, chunk of 32/T consecutive z), looping over the batch's bands in
// band order: inverse x-FFT of the Px occupied planes (zero-padded to N), acc(x) += f_b |psi_b|^2
// (FP32, in the warp's slice of shared memory), then rho[x][y][z] += scale acc (FP64).  Every
// grid point belongs to one lane: no atomics, a fixed summation order.
template <int N>
__global__ void __launch_bounds__(32 * kWarps, RP<N>::MINB)
k_rd(const C *__restrict__ T2, int Px, int nx0m, int nbb, const float *__restrict__ f, double scale,
     double *__restrict__ rho) {
    constexpr int T = RP<N>::T, E = RP<N>::E, BK = RP<N>::BK, VS = RP<N>::VS, LPW = 32 / T;
    constexpr int NZC = (N + LPW - 1) / LPW;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float *acc = reinterpret_cast<float *>(smem_raw) + (size_t)wid * VS * 32;  // [slot][lane]
    const int w = blockIdx.x * kWarps + wid;
    const int y = w / NZC, zc = w - y * NZC;
    if (y >= N) return;
    const int l = lane / T, t = lane - l * T;
    const int z = zc * LPW + l;
    const bool ok = z < N;
    const size_t NN = (size_t)N * N;
#pragma unroll
    for (int e = 0; e < VS; ++e) acc[e * 32 + lane] = 0.f;
    for (int b = 0; b < nbb; ++b) {
        const C *base = T2 + (size_t)b * Px * NN + (size_t)y * N + z;
        C v[VS];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            int px = t + T * e - nx0m;
            px += (px < 0) ? N : 0;
            v[e] = (ok && px < Px) ? base[(size_t)px * NN] : mkc<float>(0.f, 0.f);
        }
        s2b<N, true>(v, t);
        const float fb = f[b];
#pragma unroll
        for (int e = 0; e < VS; ++e) acc[e * 32 + lane] = fmaf(fb, v[e].x * v[e].x + v[e].y * v[e].y, acc[e * 32 + lane]);
    }
    if (!ok) return;
#pragma unroll
    for (int k2 = 0; k2 < T; ++k2)
#pragma unroll
        for (int i = 0; i < BK; ++i) {
            if (!RP<N>::slot_ok(t, i)) continue;
            const int x = t * BK + i + E * k2;
            rho[((size_t)x * N + y) * N + z] += scale * (double)acc[(i + BK * k2) * 32 + lane];
        }
}

// ------------------------------------------------------------- pass A
// One CTA per (band, x-plane): scatter the plane's sphere coefficients into
// the Py x N tile, inverse z-FFT of the occupied rows, inverse y-FFT of every
// z-line (rows outside the sphere are zero), write T2[b][px][y][z].
template <int N>
__global__ void __launch_bounds__(32 * kWarps, RP<N>::MINB)
k_ra(const C *__restrict__ X, int ldx, C *__restrict__ T2, int Px, int Py, int ny0m,
     const int *__restrict__ plane_begin, const int2 *__restrict__ yrange, const int *__restrict__ gmap) {
    constexpr int T = RP<N>::T, E = RP<N>::E, BK = RP<N>::BK, VS = RP<N>::VS, LPW = 32 / T, P = N + 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *S = reinterpret_cast<C *>(smem_raw);
    const int px = blockIdx.x, b = blockIdx.y;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int l = lane / T, t = lane - l * T;
    const C zero = mkc<float>(0.f, 0.f);
    for (int i = threadIdx.x; i < Py * P; i += blockDim.x) S[i] = zero;
    __syncthreads();
    const C *Xb = X + (size_t)b * ldx;
    const int g0 = plane_begin[px], g1 = plane_begin[px + 1];
    // eight coefficients per thread in flight (the loads are independent)
    constexpr int U = 8;
    for (int gb = g0 + threadIdx.x; gb < g1; gb += U * blockDim.x) {
        int gm[U];
        C xv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int g = gb + u * blockDim.x;
            gm[u] = g < g1 ? gmap[g] : -1;
            xv[u] = g < g1 ? Xb[g] : zero;
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (gm[u] >= 0) {
                const int py = gm[u] / N;
                S[py * P + (gm[u] - py * N)] = xv[u];
            }
    }
    __syncthreads();
    // inverse z-FFT of the occupied rows, in place in the tile
    const int2 yr = yrange[px];
    const int nrows = yr.y - yr.x + 1;
    for (int r0 = wid * LPW; r0 < nrows; r0 += kWarps * LPW) {
        const int r = yr.x + r0 + l;
        const bool ok = r0 + l < nrows;
        C *row = S + (ok ? r : yr.x) * P;
        C v[VS];
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = ok ? row[t + T * e] : zero;
        s2b<N, true>(v, t);
        __syncwarp();
        if (ok) {
#pragma unroll
            for (int k2 = 0; k2 < T; ++k2)
#pragma unroll
                for (int i = 0; i < BK; ++i)
                    if (RP<N>::slot_ok(t, i)) row[t * BK + i + E * k2] = v[i + BK * k2];
        }
    }
    __syncthreads();
    // inverse y-FFT of every z-line
    constexpr int NZC = (N + LPW - 1) / LPW;
    C *out = T2 + ((size_t)b * Px + px) * (size_t)N * N;
    for (int zc = wid; zc < NZC; zc += kWarps) {
        const int z = zc * LPW + l;
        const bool ok = z < N;
        C v[VS];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            int py = t + T * e - ny0m;
            py += (py < 0) ? N : 0;
            v[e] = (ok && py < Py) ? S[py * P + z] : zero;
        }
        s2b<N, true>(v, t);
        if (ok) {
#pragma unroll
            for (int k2 = 0; k2 < T; ++k2)
#pragma unroll
                for (int i = 0; i < BK; ++i)
                    if (RP<N>::slot_ok(t, i)) out[(size_t)(t * BK + i + E * k2) * N + z] = v[i + BK * k2];
        }
    }
}

// ------------------------------------------------------------- pass C
// One CTA per (band, x-plane): forward y-FFT of every z-line of T2, keep the
// Py rows of the sphere in the tile, forward z-FFT of the occupied rows,
// gather the sphere coefficients and add T(q) x(q).
template <int N>
__global__ void __launch_bounds__(32 * kWarps, RP<N>::MINB)
k_rc(const C *__restrict__ T2, C *__restrict__ Y, int ldy, const C *__restrict__ X, int ldx,
     const float *__restrict__ kin, int Px, int Py, int ny0m, const int *__restrict__ plane_begin,
     const int2 *__restrict__ yrange, const int *__restrict__ gmap) {
    constexpr int T = RP<N>::T, E = RP<N>::E, BK = RP<N>::BK, VS = RP<N>::VS, LPW = 32 / T, P = N + 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *S = reinterpret_cast<C *>(smem_raw);
    const int px = blockIdx.x, b = blockIdx.y;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int l = lane / T, t = lane - l * T;
    const C zero = mkc<float>(0.f, 0.f);
    constexpr int NZC = (N + LPW - 1) / LPW;
    const C *in = T2 + ((size_t)b * Px + px) * (size_t)N * N;
    for (int zc = wid; zc < NZC; zc += kWarps) {
        const int z = zc * LPW + l;
        const bool ok = z < N;
        C v[VS];
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = ok ? in[(size_t)(t + T * e) * N + z] : zero;
        s2b<N, false>(v, t);
        if (ok) {
#pragma unroll
            for (int k2 = 0; k2 < T; ++k2)
#pragma unroll
                for (int i = 0; i < BK; ++i) {
                    if (!RP<N>::slot_ok(t, i)) continue;
                    int py = t * BK + i + E * k2 - ny0m;
                    py += (py < 0) ? N : 0;
                    if (py < Py) S[py * P + z] = v[i + BK * k2];
                }
        }
    }
    __syncthreads();
    const int2 yr = yrange[px];
    const int nrows = yr.y - yr.x + 1;
    for (int r0 = wid * LPW; r0 < nrows; r0 += kWarps * LPW) {
        const int r = yr.x + r0 + l;
        const bool ok = r0 + l < nrows;
        C *row = S + (ok ? r : yr.x) * P;
        C v[VS];
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = ok ? row[t + T * e] : zero;
        s2b<N, false>(v, t);
        __syncwarp();
        if (ok) {
#pragma unroll
            for (int k2 = 0; k2 < T; ++k2)
#pragma unroll
                for (int i = 0; i < BK; ++i)
                    if (RP<N>::slot_ok(t, i)) row[t * BK + i + E * k2] = v[i + BK * k2];
        }
    }
    __syncthreads();
    const int g0 = plane_begin[px], g1 = plane_begin[px + 1];
    C *Yb = Y + (size_t)b * ldy;
    const C *Xb = X + (size_t)b * ldx;
    // eight coefficients per thread in flight (the loads are independent)
    constexpr int U = 8;
    for (int gb = g0 + threadIdx.x; gb < g1; gb += U * blockDim.x) {
        int gm[U];
        C xv[U];
        float kv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int g = gb + u * blockDim.x;
            const bool in = g < g1;
            gm[u] = in ? gmap[g] : 0;
            xv[u] = (in && kin) ? Xb[g] : zero;
            kv[u] = (in && kin) ? kin[g] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int g = gb + u * blockDim.x;
            if (g < g1) {
                const int py = gm[u] / N;
                Yb[g] = S[py * P + (gm[u] - py * N)] + kv[u] * xv[u];
            }
        }
    }
}

size_t tile_bytes(int N, int Py) { return sizeof(C) * (size_t)Py * (N + 2); }

template <int N>
int run_reg(const FFTGeom &g, const C *X, int ldx, C *Y, int ldy, int nb, const float *kin, const float *vr, C *T2,
            int nbatch, cudaStream_t s) {
    constexpr int LPW = 32 / RP<N>::T;
    constexpr int NZC = (N + LPW - 1) / LPW;
    const size_t sm = tile_bytes(N, g.Py);
    // dynamic shared-memory ceiling: the device maximum, set once (process-wide attribute)
    static std::atomic<bool> attr{false};
    if (!attr.load()) {
        int dev = 0, smem_max = 0;
        LG_CUDA_TRY(cudaGetDevice(&dev));
        LG_CUDA_TRY(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        if (sm > (size_t)smem_max) return fail(LOBPCG_ERR_UNSUPPORTED, "FFT plane tile exceeds shared memory");
        cudaFuncAttributes fa, fc;
        LG_CUDA_TRY(cudaFuncGetAttributes(&fa, k_ra<N>));
        LG_CUDA_TRY(cudaFuncGetAttributes(&fc, k_rc<N>));
        LG_CUDA_TRY(cudaFuncSetAttribute(k_ra<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smem_max - (int)fa.sharedSizeBytes));
        LG_CUDA_TRY(cudaFuncSetAttribute(k_rc<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smem_max - (int)fc.sharedSizeBytes));
        attr.store(true);
    }
    const int ny0m = ((g.ny0 % N) + N) % N;
    const int nx0m = ((g.nx0 % N) + N) % N;
    const int nwb = N * NZC;
    for (int b0 = 0; b0 < nb; b0 += nbatch) {
        const int nbb = std::min(nbatch, nb - b0);
        const C *Xb = X + (size_t)b0 * ldx;
        C *Yb = Y + (size_t)b0 * ldy;
        k_ra<N><<<dim3(g.Px, nbb), 32 * kWarps, sm, s>>>(Xb, ldx, T2, g.Px, g.Py, ny0m, g.plane_begin,
                                                         g.plane_yrange, g.gmap);
        LG_TRY(check_launch("fft pass A (registers)"));
        k_rb<N><<<dim3((nwb + kWarps - 1) / kWarps, nbb), 32 * kWarps, 0, s>>>(T2, g.Px, nx0m, vr);
        LG_TRY(check_launch("fft pass B (registers)"));
        k_rc<N><<<dim3(g.Px, nbb), 32 * kWarps, sm, s>>>(T2, Yb, ldy, Xb, ldx, kin, g.Px, g.Py, ny0m,
                                                         g.plane_begin, g.plane_yrange, g.gmap);
        LG_TRY(check_launch("fft pass C (registers)"));
    }
    return LOBPCG_OK;
}

template <int N>
int run_reg_density(const FFTGeom &g, const C *X, int ldx, int nb, const float *f, double scale, double *rho, C *T2,
                    int nbatch, cudaStream_t s) {
    constexpr int LPW = 32 / RP<N>::T, VS = RP<N>::VS;
    constexpr int NZC = (N + LPW - 1) / LPW;
    const size_t sm = tile_bytes(N, g.Py);
    const size_t smd = sizeof(float) * (size_t)VS * 32 * kWarps;
    static std::atomic<bool> attr{false};
    if (!attr.load()) {
        int dev = 0, smem_max = 0;
        LG_CUDA_TRY(cudaGetDevice(&dev));
        LG_CUDA_TRY(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        if (sm > (size_t)smem_max || smd > (size_t)smem_max)
            return fail(LOBPCG_ERR_UNSUPPORTED, "FFT plane tile exceeds shared memory");
        cudaFuncAttributes fa, fd;
        LG_CUDA_TRY(cudaFuncGetAttributes(&fa, k_ra<N>));
        LG_CUDA_TRY(cudaFuncGetAttributes(&fd, k_rd<N>));
        LG_CUDA_TRY(cudaFuncSetAttribute(k_ra<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smem_max - (int)fa.sharedSizeBytes));
        LG_CUDA_TRY(cudaFuncSetAttribute(k_rd<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smem_max - (int)fd.sharedSizeBytes));
        attr.store(true);
    }
    const int ny0m = ((g.ny0 % N) + N) % N;
    const int nx0m = ((g.nx0 % N) + N) % N;
    const int nwb = N * NZC;
    for (int b0 = 0; b0 < nb; b0 += nbatch) {
        const int nbb = std::min(nbatch, nb - b0);
        k_ra<N><<<dim3(g.Px, nbb), 32 * kWarps, sm, s>>>(X + (size_t)b0 * ldx, ldx, T2, g.Px, g.Py, ny0m,
                                                         g.plane_begin, g.plane_yrange, g.gmap);
        LG_TRY(check_launch("density: fft pass A (registers)"));
        k_rd<N><<<(nwb + kWarps - 1) / kWarps, 32 * kWarps, smd, s>>>(T2, g.Px, nx0m, nbb, f + b0, scale, rho);
        LG_TRY(check_launch("density: x-lines and |psi|^2 (registers)"));
    }
    return LOBPCG_OK;
}

std::mutex g_tw_mu;
bool g_tw_ready[kMaxDevices] = {false};

}  // namespace

bool fft_reg_supported(int N) {
    for (int i = 0; i < kNumRegN; ++i)
        if (kRegN[i] == N) return true;
    return false;
}

int fft_reg_prepare() {
    int dev = 0;
    LG_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(LOBPCG_ERR_UNSUPPORTED, "device index too large");
    std::lock_guard<std::mutex> lk(g_tw_mu);
    if (g_tw_ready[dev]) return LOBPCG_OK;
    std::vector<float2> h(kTwTotal);
    for (int i = 0, off = 0; i < kNumRegN; off += kRegN[i], ++i)
        for (int j = 0; j < kRegN[i]; ++j) {
            const double a = -2.0 * M_PI * (double)j / (double)kRegN[i];
            h[off + j] = make_float2((float)std::cos(a), (float)std::sin(a));
        }
    LG_CUDA_TRY(cudaMemcpyToSymbol(c_tw, h.data(), sizeof(float2) * kTwTotal));
    g_tw_ready[dev] = true;
    return LOBPCG_OK;
}

size_t fft_reg_smem_need(const FFTGeom &g) { return tile_bytes(g.N, g.Py); }

int fft_reg_apply(const FFTGeom &g, const C *X, int ldx, C *Y, int ldy, int nb, const float *kin, const float *vr,
                  C *T2, int nbatch, cudaStream_t s) {
    if (nb <= 0) return LOBPCG_OK;
    switch (g.N) {
#define LG_REG_CASE(n) \
    case n: return run_reg<n>(g, X, ldx, Y, ldy, nb, kin, vr, T2, nbatch, s);
        LG_REG_CASE(8) LG_REG_CASE(12) LG_REG_CASE(16) LG_REG_CASE(20) LG_REG_CASE(24) LG_REG_CASE(36)
        LG_REG_CASE(48) LG_REG_CASE(64) LG_REG_CASE(72) LG_REG_CASE(96) LG_REG_CASE(120) LG_REG_CASE(128)
        LG_REG_CASE(160)
#undef LG_REG_CASE
        default: return fail(LOBPCG_ERR_UNSUPPORTED, "no register FFT for this grid");
    }
}

int fft_reg_density(const FFTGeom &g, const C *X, int ldx, int nb, const float *f, double scale, double *rho, C *T2,
                    int nbatch, cudaStream_t s) {
    if (nb <= 0) return LOBPCG_OK;
    switch (g.N) {
#define LG_REG_CASE(n) \
    case n: return run_reg_density<n>(g, X, ldx, nb, f, scale, rho, T2, nbatch, s);
        LG_REG_CASE(8) LG_REG_CASE(12) LG_REG_CASE(16) LG_REG_CASE(20) LG_REG_CASE(24) LG_REG_CASE(36)
        LG_REG_CASE(48) LG_REG_CASE(64) LG_REG_CASE(72) LG_REG_CASE(96) LG_REG_CASE(120) LG_REG_CASE(128)
        LG_REG_CASE(160)
#undef LG_REG_CASE
        default: return fail(LOBPCG_ERR_UNSUPPORTED, "no register FFT for this grid");
    }
}

}  // namespace lg
