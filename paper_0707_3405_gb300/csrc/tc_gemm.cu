// Complex64 GEMMs on the 5th-generation tensor cores (tcgen05, accumulators in
// TMEM) with split TF32 operands: the projector, Gram, constraint and update
// contractions of Algorithm 1 (Sec. 3.2 and 4.1, zgemm in the paper) on the
// mixed-precision path.
//
// Precision ("3xTF32"): every FP32 operand x is split as x = hi + lo with hi
// and lo rounded to TF32 (10-bit mantissa); a product is hi*hi + hi*lo + lo*hi
// (the lo*lo term is below FP32 resolution), accumulated in FP32 by the tensor
// core.  The relative error per product is about 2^-21, i.e. FP32 class.
//
// Complex arithmetic as one real GEMM per tile (interleaved re/im along K):
//   C = A^H B:  Re C = A'.B', Im C = A'.B'' where A' is a column of A read as
//               [re, im, re, im, ...], B' likewise and B'' = [im, -re, ...].
//               The MMA runs with N = 2 NT: B' rows and B'' rows side by side.
//   D = A B:    D read as a real (2M x n) matrix equals Ahat Bhat with
//               Ahat rows 2g = [re, -im, ...], 2g+1 = [im, re, ...] (along K
//               pairs) and Bhat = B read as real; the producer expands A.
//
// Data path per CTA (256 threads, one tile): the threads load FP32 from HBM
// (coalesced) one stage ahead into registers, split, and store hi / lo into
// 128-byte-swizzled K-major shared tiles (the layout tcgen05 descriptors
// address); thread 0 issues the MMAs of a stage and commits them to that
// stage's mbarrier; the stage is refilled once the barrier shows the MMAs
// done (2-3 stage ring).  The accumulator tile is read back from TMEM by the
// eight warps (warp w reads lane quarter w % 4, column half w / 4).
// Long reductions (A^H B over the plane-wave count) are split over grid.z;
// FP64 partial tiles are summed afterwards in a fixed order (reproducible).
//
// Every mbarrier wait is bounded; a wait that runs out raises a device flag
// (read by tc_check_error) and the CTA stops issuing work, waits (bounded) for
// the MMAs it has in flight, frees its TMEM and returns.
#include "common.cuh"
#include "tc.cuh"

#include <algorithm>

namespace lg {

namespace {

using namespace tc;

constexpr int kThreads = 256;  // 8 warps: all load / split / store; thread 0 issues the MMAs
constexpr int KBC = 16;     // complex K per stage: 32 floats = one 128-byte shared row
constexpr int ROWB = 128;   // bytes per shared row

__device__ int g_tc_err = 0;
// Poll limit of the ring waits (a stage's MMAs done before its refill); the drain wait for the
// MMAs a CTA has issued always takes the full kSpinLimit, so a CTA that gave up never frees
// TMEM or returns while its own MMAs may still run.  Lowered only by tests of the timeout path.
__device__ long long g_tc_spin = kSpinLimit;

// Byte offset of complex element kc (0..15) of row r in a 128-byte-swizzled K-major tile.
__device__ __forceinline__ uint32_t swz(int r, int kc) {
    return (uint32_t)r * 128u + ((((uint32_t)kc >> 1) ^ ((uint32_t)r & 7u)) << 4) + (((uint32_t)kc & 1u) << 3);
}

__device__ __forceinline__ void put_split(unsigned char *hi, unsigned char *lo, uint32_t off, float a, float b) {
    const float ah = to_tf32(a), bh = to_tf32(b);
    *reinterpret_cast<float2 *>(hi + off) = make_float2(ah, bh);
    *reinterpret_cast<float2 *>(lo + off) = make_float2(to_tf32(a - ah), to_tf32(b - bh));
}

__device__ __forceinline__ unsigned char *align1k(unsigned char *p) {
    return reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(p) + 1023) & ~(uintptr_t)1023);
}

// Ring depth: NSF if given, else 3 stages when they fit in 200 KB, else 2.
template <int STAGE, int NSF = 0>
constexpr int n_stages() { return NSF ? NSF : (3 * STAGE <= 200 * 1024 ? 3 : 2); }

template <int STAGE, int NSF = 0>
constexpr size_t smem_bytes() { return (size_t)n_stages<STAGE, NSF>() * STAGE + 1024 + 64; }

// A B with 64 columns: a 2-stage ring (97 KB) lets two CTAs share an SM; the products of the
// block iterations are tall and short (K = 64 .. 192), so a deeper ring never fills anyway.
template <int NN>
constexpr int nn_ring() { return NN == 64 ? 2 : 0; }
template <int NN>
constexpr int nn_ctas_per_sm() { return NN == 64 ? 2 : 1; }

// Issue the 3xTF32 MMAs of one stage (4 K-steps of 8) and commit them to `bar`.
__device__ __forceinline__ void issue_stage(uint32_t tmem, uint32_t a_h, uint32_t a_l, uint32_t b_h, uint32_t b_l,
                                            uint32_t idesc, bool first, uint64_t *bar) {
    fence_after_sync();
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        const uint32_t o = 32u * kk;
        mma_tf32(tmem, make_desc_sw128(a_h + o), make_desc_sw128(b_h + o), idesc, (first && kk == 0) ? 0u : 1u);
        mma_tf32(tmem, make_desc_sw128(a_h + o), make_desc_sw128(b_l + o), idesc, 1u);
        mma_tf32(tmem, make_desc_sw128(a_l + o), make_desc_sw128(b_h + o), idesc, 1u);
    }
    mma_commit(bar);
}

// ------------------------------------------------------------------ C = A^H B
// CTA tile: 128 columns of A (rows i of C) x NT columns of B; K range
// [blockIdx.z * kchunk, +kchunk).  Writes the FP64 partial tile of its split.
template <int NT>
__global__ void __launch_bounds__(kThreads, 1)
k_tc_cn(int m, int n, int K, int kchunk, const c32 *__restrict__ A, int lda, const c32 *__restrict__ B, int ldb,
        z64 *__restrict__ part) {
    constexpr int NR = 2 * NT;  // B' rows then B'' rows
    constexpr int A_BYTES = 128 * ROWB, B_BYTES = NR * ROWB;
    constexpr int STAGE = 2 * A_BYTES + 2 * B_BYTES;
    constexpr int NS = n_stages<STAGE>();
    constexpr uint32_t IDESC = make_idesc_tf32(128, NR);
    extern __shared__ unsigned char smraw[];
    unsigned char *base = align1k(smraw);
    uint64_t *bar = reinterpret_cast<uint64_t *>(base + NS * STAGE);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + NS);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int i0 = blockIdx.x * 128, j0 = blockIdx.y * NT;
    const int kbeg = blockIdx.z * kchunk, kend = min(K, kbeg + kchunk);
    const int nkb = kend > kbeg ? (kend - kbeg + KBC - 1) / KBC : 0;
    if (warp == 0) tmem_alloc(tslot, NR);
    if (tid == 0)
        for (int s = 0; s < NS; ++s) mbar_init(&bar[s], 1);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tslot;
    // Each thread owns NA elements of the A tile and NB of the B tile per stage; the loads of
    // stage kb + 1 are issued before stage kb is split and stored, so they overlap the MMAs.
    constexpr int NA = 128 * KBC / kThreads, NB = NT * KBC / kThreads;
    float2 ra[NA], rb[NB];
    auto load = [&](int kb) {
        const int k0 = kbeg + kb * KBC;
#pragma unroll
        for (int q = 0; q < NA; ++q) {
            const int idx = tid + kThreads * q, r = idx >> 4, kc = idx & 15;
            const int i = i0 + r, k = k0 + kc;
            ra[q] = (i < m && k < kend) ? __ldg(reinterpret_cast<const float2 *>(A + (size_t)i * lda + k))
                                        : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            const int idx = tid + kThreads * q, j = idx >> 4, kc = idx & 15;
            const int k = k0 + kc;
            rb[q] = (j0 + j < n && k < kend) ? __ldg(reinterpret_cast<const float2 *>(B + (size_t)(j0 + j) * ldb + k))
                                             : make_float2(0.f, 0.f);
        }
    };
    int bad = 0, issued = 0;
    if (nkb > 0) load(0);
    for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % NS;
        if (kb >= NS && !mbar_wait(&bar[s], (uint32_t)((kb / NS - 1) & 1), g_tc_spin)) bad = 1;
        unsigned char *sAh = base + s * STAGE, *sAl = sAh + A_BYTES, *sBh = sAl + A_BYTES, *sBl = sBh + B_BYTES;
#pragma unroll
        for (int q = 0; q < NA; ++q) {
            const int idx = tid + kThreads * q;
            put_split(sAh, sAl, swz(idx >> 4, idx & 15), ra[q].x, ra[q].y);
        }
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            const int idx = tid + kThreads * q, j = idx >> 4, kc = idx & 15;
            put_split(sBh, sBl, swz(j, kc), rb[q].x, rb[q].y);
            put_split(sBh, sBl, swz(NT + j, kc), rb[q].y, -rb[q].x);
        }
        if (kb + 1 < nkb) load(kb + 1);
        fence_proxy_async();
        if (__syncthreads_or(bad)) break;
        if (tid == 0)
            issue_stage(tmem, smem_u32(sAh), smem_u32(sAl), smem_u32(sBh), smem_u32(sBl), IDESC, kb == 0, &bar[s]);
        ++issued;
    }
    if (issued > 0) {
        const int kl = issued - 1;
        if (!mbar_wait(&bar[kl % NS], (uint32_t)((kl / NS) & 1))) bad = 1;
    }
    fence_after_sync();
    bad = __syncthreads_or(bad);
    z64 *P = part + (size_t)blockIdx.z * m * n;
    const int quarter = warp & 3, half = warp >> 2;
    const int i = i0 + quarter * 32 + lane;
    const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16);
    if (!bad) {
#pragma unroll 1
        for (int c0 = half * (NT / 2); c0 < (half + 1) * (NT / 2); c0 += 16) {
            float re[16], im[16];
            if (issued > 0) {
                tmem_ld16(trow + (uint32_t)c0, re);
                tmem_ld16(trow + (uint32_t)(NT + c0), im);
            } else {
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) re[jj] = im[jj] = 0.f;
            }
            if (i < m) {
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) {
                    const int j = j0 + c0 + jj;
                    if (j < n) P[(size_t)j * m + i] = mkc((double)re[jj], (double)im[jj]);
                }
            }
        }
    } else if (tid == 0) {
        atomicExch(&g_tc_err, 1);
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, NR);
}

__global__ void k_tc_reduce(int m, int n, int nsplit, float alpha, const z64 *__restrict__ part, float beta,
                            c32 *C, int ldc) {
    const size_t tot = (size_t)m * n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % m), j = (int)(e / m);
        z64 acc = part[e];
        for (int z = 1; z < nsplit; ++z) acc = acc + part[(size_t)z * tot + e];
        z64 v = (double)alpha * acc;
        if (beta != 0.f) v = v + (double)beta * cvt<double, float>(C[(size_t)j * ldc + i]);
        C[(size_t)j * ldc + i] = cvt<float, double>(v);
    }
}

// ------------------------------------------------------------------ D = alpha A B + beta C
// CTA tile: 64 complex rows of A / D (128 real rows) x NN columns of B / D, full K.
template <int NN>
__global__ void __launch_bounds__(kThreads, nn_ctas_per_sm<NN>())
k_tc_nn(int M, int n, int k, float alpha, const c32 *__restrict__ A, int lda, const c32 *__restrict__ B, int ldb,
        float beta, const c32 *C, int ldc, c32 *D, int ldd) {
    constexpr int A_BYTES = 128 * ROWB, B_BYTES = NN * ROWB;
    constexpr int STAGE = 2 * A_BYTES + 2 * B_BYTES;
    constexpr int NS = n_stages<STAGE, nn_ring<NN>()>();
    constexpr uint32_t IDESC = make_idesc_tf32(128, NN);
    extern __shared__ unsigned char smraw[];
    unsigned char *base = align1k(smraw);
    uint64_t *bar = reinterpret_cast<uint64_t *>(base + NS * STAGE);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + NS);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g0 = blockIdx.x * 64, jt0 = blockIdx.y * NN;
    const int nkb = (k + KBC - 1) / KBC;
    if (warp == 0) tmem_alloc(tslot, NN);
    if (tid == 0)
        for (int s = 0; s < NS; ++s) mbar_init(&bar[s], 1);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tslot;
    // producer map for A: each warp step covers 8 consecutive rows g x 4 consecutive K (l);
    // lane bits -> (g low 3, l low 2), warp -> l high 2 of the 16, q -> g high 3 (of 64)
    // with 8 warps: warp & 3 -> l high bits, warp >> 2 -> g offset 32
    const int gl = lane & 7, ll = (lane >> 3) + 4 * (warp & 3), gq = (warp >> 2) * 32;
    constexpr int NA = 4, NB = NN * KBC / kThreads;
    float2 ra[NA], rb[NB];
    auto load = [&](int kb) {
        const int l0 = kb * KBC;
        const int l = l0 + ll;
#pragma unroll
        for (int q = 0; q < NA; ++q) {
            const int g = gq + 8 * q + gl;
            ra[q] = (g0 + g < M && l < k) ? __ldg(reinterpret_cast<const float2 *>(A + (size_t)l * lda + g0 + g))
                                          : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            const int idx = tid + kThreads * q, j = idx >> 4, kc = idx & 15;
            const int lk = l0 + kc;
            rb[q] = (jt0 + j < n && lk < k) ? __ldg(reinterpret_cast<const float2 *>(B + (size_t)(jt0 + j) * ldb + lk))
                                            : make_float2(0.f, 0.f);
        }
    };
    int bad = 0, issued = 0;
    if (nkb > 0) load(0);
    for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % NS;
        if (kb >= NS && !mbar_wait(&bar[s], (uint32_t)((kb / NS - 1) & 1), g_tc_spin)) bad = 1;
        unsigned char *sAh = base + s * STAGE, *sAl = sAh + A_BYTES, *sBh = sAl + A_BYTES, *sBl = sBh + B_BYTES;
#pragma unroll
        for (int q = 0; q < NA; ++q) {
            const int g = gq + 8 * q + gl;
            const float rh = to_tf32(ra[q].x), ih = to_tf32(ra[q].y);
            const float rl = to_tf32(ra[q].x - rh), il = to_tf32(ra[q].y - ih);
            const uint32_t o0 = swz(2 * g, ll), o1 = swz(2 * g + 1, ll);
            *reinterpret_cast<float2 *>(sAh + o0) = make_float2(rh, -ih);
            *reinterpret_cast<float2 *>(sAl + o0) = make_float2(rl, -il);
            *reinterpret_cast<float2 *>(sAh + o1) = make_float2(ih, rh);
            *reinterpret_cast<float2 *>(sAl + o1) = make_float2(il, rl);
        }
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            const int idx = tid + kThreads * q;
            put_split(sBh, sBl, swz(idx >> 4, idx & 15), rb[q].x, rb[q].y);
        }
        if (kb + 1 < nkb) load(kb + 1);
        fence_proxy_async();
        if (__syncthreads_or(bad)) break;
        if (tid == 0)
            issue_stage(tmem, smem_u32(sAh), smem_u32(sAl), smem_u32(sBh), smem_u32(sBl), IDESC, kb == 0, &bar[s]);
        ++issued;
    }
    if (issued > 0) {
        const int kl = issued - 1;
        if (!mbar_wait(&bar[kl % NS], (uint32_t)((kl / NS) & 1))) bad = 1;
    }
    fence_after_sync();
    bad = __syncthreads_or(bad);
    const int quarter = warp & 3, half = warp >> 2;
    const int rho = quarter * 32 + lane;  // real row of the tile: complex row g0 + rho/2, part rho & 1
    const bool row_ok = g0 + (rho >> 1) < M;
    const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16);
    float *Df = reinterpret_cast<float *>(D);
    const float *Cf = reinterpret_cast<const float *>(C);
    if (!bad) {
#pragma unroll 1
        for (int c0 = half * (NN / 2); c0 < (half + 1) * (NN / 2); c0 += 16) {
            // C may be D (in-place accumulate): all 16 loads of the chunk are issued before its stores
            float cv[16], acc[16];
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) {
                const int j = jt0 + c0 + jj;
                cv[jj] = (row_ok && j < n && beta != 0.f) ? Cf[2 * ((size_t)j * ldc + g0) + rho] : 0.f;
            }
            if (issued > 0) {
                tmem_ld16(trow + (uint32_t)c0, acc);
            } else {
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) acc[jj] = 0.f;
            }
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) {
                const int j = jt0 + c0 + jj;
                if (row_ok && j < n) Df[2 * ((size_t)j * ldd + g0) + rho] = fmaf(beta, cv[jj], alpha * acc[jj]);
            }
        }
    } else if (tid == 0) {
        atomicExch(&g_tc_err, 1);
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, NN);
}

template <typename Kern>
int ensure_smem(Kern kern, size_t bytes, std::atomic<bool> &done) {
    if (!done.load()) {
        LG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
        done.store(true);
    }
    return LOBPCG_OK;
}

int num_sms_tc() {
    static std::atomic<int> cached{0};
    int v = cached.load();
    if (!v) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 148;
        cached.store(v);
    }
    return v;
}

template <int NT>
int launch_cn(GemmWork &w, int m, int n, int K, float alpha, const c32 *A, int lda, const c32 *B, int ldb,
              float beta, c32 *C, int ldc, cudaStream_t s) {
    constexpr int STAGE = 2 * 128 * ROWB + 2 * 2 * NT * ROWB;
    constexpr size_t SMEM = smem_bytes<STAGE>();
    static std::atomic<bool> attr{false};
    LG_TRY(ensure_smem(k_tc_cn<NT>, SMEM, attr));
    const int tm = (m + 127) / 128, tn = (n + NT - 1) / NT;
    const int tiles = tm * tn;
    // one CTA per SM (shared memory): split K over the GPU.  Cost model in units of one 16-term
    // stage of a CTA (about a microsecond): whole waves x stages per CTA, plus the FP64 partial
    // tiles written and summed (about 7 MB per stage-time of HBM traffic); the cheapest split
    // with chunks of 256 to 8192 terms wins.
    const int sms = num_sms_tc();
    int kchunk = std::max(KBC, ((K + KBC - 1) / KBC) * KBC);
    double best = 1e300;
    for (int ns = 1; ns <= 4 * sms; ++ns) {
        const int kc = ((K + ns - 1) / ns + KBC - 1) / KBC * KBC;
        if (kc > 8192) continue;
        if (kc < 256 && ns > 1) break;
        const int nsp = (K + kc - 1) / kc;
        const long long ctas = (long long)tiles * nsp;
        const long long waves = (ctas + sms - 1) / sms;
        const double cost = (double)waves * (kc / KBC) + (double)nsp * 32.0 * m * (double)n / 7.2e6;
        if (cost < best) {
            best = cost;
            kchunk = kc;
        }
    }
    kchunk = std::max(kchunk, KBC);
    const int nsplit = (K + kchunk - 1) / kchunk;
    LG_TRY(w.alloc->ensure(w.part, sizeof(z64) * (size_t)nsplit * m * n));
    z64 *part = reinterpret_cast<z64 *>(w.part.p);
    k_tc_cn<NT><<<dim3(tm, tn, nsplit), kThreads, SMEM, s>>>(m, n, K, kchunk, A, lda, B, ldb, part);
    LG_TRY(check_launch("tensor-core gemm A^H B"));
    const size_t tot = (size_t)m * n;
    const int blocks = (int)std::min<size_t>((tot + 255) / 256, 4096);
    k_tc_reduce<<<blocks, 256, 0, s>>>(m, n, nsplit, alpha, part, beta, C, ldc);
    return check_launch("tensor-core gemm reduce");
}

template <int NN>
int launch_nn(int M, int n, int k, float alpha, const c32 *A, int lda, const c32 *B, int ldb, float beta,
              const c32 *C, int ldc, c32 *D, int ldd, cudaStream_t s) {
    constexpr int STAGE = 2 * 128 * ROWB + 2 * NN * ROWB;
    constexpr size_t SMEM = smem_bytes<STAGE, nn_ring<NN>()>();
    static std::atomic<bool> attr{false};
    LG_TRY(ensure_smem(k_tc_nn<NN>, SMEM, attr));
    const dim3 grid((M + 63) / 64, (n + NN - 1) / NN);
    k_tc_nn<NN><<<grid, kThreads, SMEM, s>>>(M, n, k, alpha, A, lda, B, ldb, beta, beta != 0.f ? C : D, ldc, D, ldd);
    return check_launch("tensor-core gemm A B");
}

}  // namespace

int tc_gemm_cn(GemmWork &w, int m, int n, int K, float alpha, const c32 *A, int lda, const c32 *B, int ldb,
               float beta, c32 *C, int ldc, cudaStream_t s) {
    if (m <= 0 || n <= 0) return LOBPCG_OK;
    if (n > 64) return launch_cn<128>(w, m, n, K, alpha, A, lda, B, ldb, beta, C, ldc, s);
    return launch_cn<64>(w, m, n, K, alpha, A, lda, B, ldb, beta, C, ldc, s);
}

int tc_gemm_nn(int M, int n, int k, float alpha, const c32 *A, int lda, const c32 *B, int ldb, float beta,
               const c32 *C, int ldc, c32 *D, int ldd, cudaStream_t s) {
    if (M <= 0 || n <= 0) return LOBPCG_OK;
    if (n > 128) return launch_nn<256>(M, n, k, alpha, A, lda, B, ldb, beta, C, ldc, D, ldd, s);
    if (n > 64) return launch_nn<128>(M, n, k, alpha, A, lda, B, ldb, beta, C, ldc, D, ldd, s);
    return launch_nn<64>(M, n, k, alpha, A, lda, B, ldb, beta, C, ldc, D, ldd, s);
}

int *device_wait_flag() {
    static std::atomic<int *> cached{nullptr};
    int *p = cached.load();
    if (!p) {
        void *q = nullptr;
        if (cudaGetSymbolAddress(&q, g_tc_err) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        p = static_cast<int *>(q);
        cached.store(p);
    }
    return p;
}

int tc_set_spin_limit(long long polls) {
    const long long v = polls < 0 ? kSpinLimit : polls;
    LG_CUDA_TRY(cudaMemcpyToSymbol(g_tc_spin, &v, sizeof(v)));
    return LOBPCG_OK;
}

int tc_check_error() {
    int h = 0;
    LG_CUDA_TRY(cudaMemcpyFromSymbol(&h, g_tc_err, sizeof(int)));
    if (h) {
        const int z = 0;
        LG_CUDA_TRY(cudaMemcpyToSymbol(g_tc_err, &z, sizeof(int)));
        return fail(LOBPCG_ERR_TIMEOUT,
                    "a bounded device wait ran out (tensor-core GEMM mbarrier or tridiagonalisation grid barrier)");
    }
    return oz_check_error();
}

}  // namespace lg
