// FP64-class complex128 GEMMs on the 5th-generation tensor cores (tcgen05, BF16
// operands, FP32 accumulators in TMEM): the tall contractions of the FP64-class
// work of the mixed schedule (all-band Grams, constraint projections and
// updates, block and sweep-end Ritz rotations, the KB projections of the FP64
// H X refresh) -- zgemm in the paper (Sec. 4.1), where it dominates.
//
// Arithmetic (error-free slicing after Ozaki, Ogita, Oishi and Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication", Numer. Algorithms 2012; integer slices with exact
// fixed-point accumulation as in Ootomo, Ozaki and Yokota 2024):
//   * The reduction dimension is cut into chunks of 64 complex terms.  Within a
//     chunk every operand vector (a row of the product's left or right factor)
//     gets one power-of-two scale 2^e with max |x| < 2^e, and each real part is
//     written as x = 2^e sum_{p=1..6} d_p 2^{-8p} + (rest at most 2^{e-49}),
//     with integer digits |d_1| <= 256, |d_p| <= 128: x 2^{48-e} is rounded to
//     an integer from its FP64 bit pattern and peeled into signed base-256
//     digits with integer operations.  Integers of that size are exact BF16
//     numbers.
//   * x y = 2^{e_x + e_y} sum_{p,q} d_p d'_q 2^{-8(p+q)}: the digit products of
//     one "level" l = p + q (l = 2..7; products with p + q > 7 are below 2^-48
//     relative and dropped) are summed by the tensor core into one FP32
//     accumulator.  Each product is at most 2^16 and a level holds at most
//     2^17 per real term, so over the 128 real terms of a chunk every partial
//     sum is an integer below 2^24: FP32 accumulation is exact.
//   * After each chunk the six level accumulators are read from TMEM, scaled by
//     2^{e_x + e_y - 8 l} (exact) and added into a double-FP32 accumulator per
//     output (pairs of FP32 numbers, TwoSum; about 2^-48 relative), which is
//     written out as FP64.
//   Result: error about 2^-44 of sum |x||y| at worst (chunk scales are shared by
//   64 consecutive plane waves), FP64 class, at BF16 tensor throughput / 21.
//
// Complex arithmetic as one real product (re / im interleaved along K):
//   C = A^H B:  rows of the left factor: columns of A as (re, im) pairs; right
//               factor: two rows per column of B, (re, im) and (im, -re);
//               C_ij = P[2j][i] + i P[2j+1][i].
//   D = A B:    left factor: two rows per row of A, (re, -im) and (im, re);
//               right factor: columns of B as (re, im); D_ij = P[j][2i] + i P[j][2i+1].
//
// Data path: a split kernel writes each operand's digits once, as 64-byte-swizzled
// K-major BF16 tiles in the exact order one pipeline stage needs them (six slices
// of a 128- or 64-row tile x 32 K values, contiguous), plus the chunk scales.
// The product kernel (one CTA per output tile and K split, 10 warps) streams the
// stages with one bulk copy per operand (cp.async.bulk into a 3-stage ring,
// mbarrier transaction counts), one thread issues the 42 MMAs of a stage
// (21 slice pairs x 2 K-steps of 16, M = 128, N = 64), and eight warps read the
// six level accumulators after every chunk (tcgen05.ld) and fold them into the
// double-FP32 sums.  Long reductions (A^H B) are split over the GPU and cut
// into K slabs that bound the digit scratch; FP64 partial tiles are summed in
// a fixed order (reproducible).  Every mbarrier wait is bounded; a wait that
// runs out sets a device flag (read by oz_check_error) and the CTA stops,
// waits (bounded) for its copies and MMAs in flight, frees its TMEM and returns.
#include "common.cuh"
#include "tc.cuh"

#include <algorithm>
#include <cmath>

namespace lg {

namespace {

using namespace tc;

constexpr int kSlices = 6;                   // 8-bit digits per real value
constexpr int kLevels = kSlices;             // p + q = 2 .. 7
constexpr int kStageK = 32;                  // real K (BF16) per stage: 64-byte tile rows
constexpr int kChunkStages = 4;              // 128 real K = 64 complex terms per exact chunk
constexpr int kChunkC = kStageK * kChunkStages / 2;
constexpr int TM = 128;                      // left-factor tile rows (MMA M)
constexpr int TQ = 64;                       // right-factor tile rows (MMA N)
constexpr int kTileA = TM * 64;              // bytes of one slice of a left tile stage
constexpr int kTileB = TQ * 64;
constexpr int kStageA = kSlices * kTileA;    // 48 KB
constexpr int kStageB = kSlices * kTileB;    // 24 KB
constexpr int kStageBytes = kStageA + kStageB;
constexpr int kRing = 3;
constexpr int kEpiWarps = 8;
constexpr int kThreads = 32 * (kEpiWarps + 2);   // + producer warp + MMA warp
constexpr int kTmemCols = 512;               // 6 levels x 64 columns used
constexpr size_t kSmem = (size_t)kRing * kStageBytes + 1024 + 256;   // ring + alignment + barriers

// split modes: how a complex vector becomes real rows of a factor
constexpr int kRowsPlain = 0;   // one row (re, im)                     left of A^H B, right of A B
constexpr int kRowsCnB = 1;     // two rows (re, im), (im, -re)         right of A^H B
constexpr int kRowsNnA = 2;     // two rows (re, -im), (im, re)         left of A B

__device__ int g_oz_err = 0;

// Byte offset of BF16 element (r, c) (c < 32) in a 64-byte-swizzled K-major tile:
// the 16-byte chunk c / 8 of row r sits at chunk position (c / 8) ^ ((r / 2) % 4).
__device__ __forceinline__ uint32_t swz64(int r, int c) {
    return (uint32_t)r * 64u + ((((uint32_t)c >> 3) ^ (((uint32_t)r >> 1) & 3u)) << 4) + (((uint32_t)c & 7u) << 1);
}

// Shared-memory matrix descriptor for a 64-byte-swizzled K-major tile: stride between
// 8-row groups 512 bytes, descriptor version 1, swizzle mode 4 (64 bytes).
__device__ __forceinline__ uint64_t make_desc_sw64(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1u << 16;
    d |= (uint64_t)(512u >> 4) << 32;
    d |= (uint64_t)1u << 46;
    d |= (uint64_t)4u << 61;
    return d;
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ float pow2f(int e) {
    if (e >= -126 && e <= 127) return __int_as_float((e + 127) << 23);
    return ldexpf(1.0f, e);
}

// Knuth TwoSum: s + err = a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &err) {
    s = a + b;
    const float bb = s - a;
    err = (a - (s - bb)) + (b - bb);
}

// (hi, lo) += (x, y) in double-FP32 arithmetic, renormalised.
__device__ __forceinline__ void df_add(float &hi, float &lo, float x, float y) {
    float s, e;
    two_sum(hi, x, s, e);
    e += lo + y;
    hi = s + e;
    lo = e - (hi - s);
}

// The six base-256 digits of x relative to the chunk scale 2^e (|x| < 2^e), most significant
// first: F = round(x 2^(48 - e)) is formed exactly from the mantissa with a rounding shift, then
// peeled into signed digits d_6 .. d_2 in [-128, 127] from the low end; the rest, |d_1| <= 256,
// is the top digit.  x = 2^e sum_p d_p 2^(-8p) up to 2^(e-49).  Integer operations only.
__device__ __forceinline__ void digits(double x, int e, float (&d)[kSlices]) {
    const long long bits = __double_as_longlong(x);
    const int b = (int)((bits >> 52) & 0x7FF);
    long long F = 0;
    if (b > 0) {
        const unsigned long long m = (unsigned long long)(bits & 0xFFFFFFFFFFFFFLL) | (1ULL << 52);
        const int sh = 1027 + e - b;                       // >= 5 because |x| < 2^e
        if (sh < 60) F = (long long)((m + (1ULL << (sh - 1))) >> sh);
        if (bits < 0) F = -F;
    }
#pragma unroll
    for (int p = kSlices - 1; p >= 1; --p) {
        const long long dp = ((F + 128) & 0xFF) - 128;
        d[p] = (float)dp;
        F = (F - dp) >> 8;
    }
    d[0] = (float)F;
}

// ------------------------------------------------------------------ split
// One CTA: 32 complex vectors x one chunk (64 complex terms) of the K range
// [k0, k0 + nchunks * 64) of the operand X (element (v, k) at X[v * rs + k * ks]).
// Writes the chunk's digit tiles and the vectors' chunk exponents.
template <int TR, int MODE>
__global__ void __launch_bounds__(256)
k_oz_split(const z64 *__restrict__ X, long long rs, long long ks, int nvec, int K, int k0, int KS,
           unsigned char *__restrict__ T, int *__restrict__ E, int nvec_pad) {
    constexpr int RPC = MODE == kRowsPlain ? 1 : 2;
    __shared__ double2 tile[32][kChunkC + 1];
    __shared__ int ex[32];
    const int v0 = blockIdx.x * 32, chunk = blockIdx.y;
    const int kb = k0 + chunk * kChunkC;
    const int tid = threadIdx.x;
    if (ks == 1) {   // K contiguous: threads along K
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int v = tid / 64 + 4 * i, k = tid % 64;
            const int gv = v0 + v, gk = kb + k;
            double2 a = make_double2(0.0, 0.0);
            if (gv < nvec && gk < K) {
                const z64 z = X[(size_t)gv * rs + (size_t)gk];
                a = make_double2(z.x, z.y);
            }
            tile[v][k] = a;
        }
    } else {         // vectors contiguous: threads along the vectors
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int v = tid % 32, k = tid / 32 + 8 * i;
            const int gv = v0 + v, gk = kb + k;
            double2 a = make_double2(0.0, 0.0);
            if (gv < nvec && gk < K) {
                const z64 z = X[(size_t)gv * rs + (size_t)gk * ks];
                a = make_double2(z.x, z.y);
            }
            tile[v][k] = a;
        }
    }
    __syncthreads();
    // chunk exponent of each vector: 2^e > max |re|, |im| (e = 0 for an all-zero chunk).  Taken from
    // the FP64 exponent fields with integer operations (this GPU's FP64 units are slow): a normal
    // x with biased exponent b has |x| < 2^(b - 1022); subnormals count as zero.
    const int warp = tid >> 5, lane = tid & 31;
    for (int v = warp; v < 32; v += 8) {
        int bmax = 0;
        for (int k = lane; k < kChunkC; k += 32) {
            const int br = (int)((__double_as_longlong(tile[v][k].x) >> 52) & 0x7FF);
            const int bi = (int)((__double_as_longlong(tile[v][k].y) >> 52) & 0x7FF);
            bmax = max(bmax, max(br, bi));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) bmax = max(bmax, __shfl_xor_sync(0xffffffffu, bmax, o));
        if (lane == 0) {
            const int e = bmax > 0 ? bmax - 1022 : 0;
            ex[v] = e;
            if (v0 + v < nvec_pad) E[(size_t)chunk * nvec_pad + v0 + v] = e;
        }
    }
    __syncthreads();
    // digits: 8 elements per thread, integer arithmetic on the FP64 bit patterns
#pragma unroll 1
    for (int i = 0; i < 8; ++i) {
        const int idx = tid + 256 * i;
        const int v = idx / kChunkC, k = idx % kChunkC;
        if (v0 + v >= nvec_pad) continue;
        const double2 a = tile[v][k];
        const int e = ex[v];
        float dr[kSlices], di[kSlices];
        digits(a.x, e, dr);
        digits(a.y, e, di);
        const int kk = 2 * k;                       // real K of the re part within the chunk
        const int stage = chunk * kChunkStages + kk / kStageK, col = kk % kStageK;
#pragma unroll
        for (int sub = 0; sub < RPC; ++sub) {
            const int rr = RPC * (v0 + v) + sub;    // real row
            unsigned char *base = T + ((size_t)(rr / TR) * KS + stage) * (size_t)(kSlices * TR * 64) +
                                  swz64(rr % TR, col);
#pragma unroll
            for (int p = 0; p < kSlices; ++p) {
                float u0 = dr[p], u1 = di[p];
                if (MODE == kRowsCnB && sub == 1) { u0 = di[p]; u1 = -dr[p]; }
                if (MODE == kRowsNnA) {
                    if (sub == 0) { u0 = dr[p]; u1 = -di[p]; }
                    else { u0 = di[p]; u1 = dr[p]; }
                }
                __nv_bfloat162 pr = __floats2bfloat162_rn(u0, u1);   // integers <= 256: exact
                *reinterpret_cast<__nv_bfloat162 *>(base + (size_t)p * TR * 64) = pr;
            }
        }
    }
}

// ------------------------------------------------------------------ product
struct OzArgs {
    const unsigned char *At, *Bt;   // digit tiles of the left / right factor
    const int *EA, *EB;             // chunk exponents [chunk][vector]
    int KS;                         // stages per tile row (4 x chunks of the slab)
    int nvA_pad, nvB_pad;           // padded vector counts of the exponent tables
    int nchunks, cps;               // chunks of the slab, chunks per K split
    int lower;                      // skip tiles with every output column j above every row i
    // mode 0: FP64 partial tiles P[split][q][r] (written, or added to when accumulate)
    double *P;
    int ldp;
    size_t pstride;
    int accumulate;
    // mode 1: D = alpha (product) + beta C for complex rows row0 .. of A B
    int M, n, row0;
    double alpha, beta;
    const z64 *C;
    int ldc;
    z64 *D;
    int ldd;
};

template <int OUT>
__global__ void __launch_bounds__(kThreads, 1) k_oz_mma(OzArgs a) {
    extern __shared__ unsigned char smraw[];
    unsigned char *base = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smraw) + 1023) &
                                                            ~(uintptr_t)1023);
    uint64_t *full = reinterpret_cast<uint64_t *>(base + kRing * kStageBytes);
    uint64_t *empty = full + kRing;
    uint64_t *accf = empty + kRing;
    uint64_t *acce = accf + 1;              // one per level: its accumulator has been read
    uint32_t *tslot = reinterpret_cast<uint32_t *>(acce + kLevels);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tslot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int qt = blockIdx.x, rt = blockIdx.y, z = blockIdx.z;
    if (a.lower) {
        // right rows 64 qt .. are columns j >= 32 qt (two rows per column); left rows are i
        if (32 * qt > TM * rt + TM - 1) return;
    }
    const int c0 = z * a.cps, c1 = min(a.nchunks, c0 + a.cps);
    const int nch = max(0, c1 - c0);
    if (warp == kEpiWarps + 1) tmem_alloc(tslot, kTmemCols);
    if (tid == 0) {
        for (int s = 0; s < kRing; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(accf, 1);
        for (int L = 0; L < kLevels; ++L) mbar_init(&acce[L], kEpiWarps);
        *abort_flag = 0;
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tslot;
    const int nst = nch * kChunkStages;
    if (warp == kEpiWarps) {
        // ---- producer: one bulk copy per factor per stage
        if (lane == 0) {
            int g = 0;
            for (; g < nst && !*abort_flag; ++g) {
                const int s = g % kRing;
                if (g >= kRing && !mbar_wait(&empty[s], (uint32_t)((g / kRing - 1) & 1))) {
                    *abort_flag = 1;
                    break;
                }
                const int stage = c0 * kChunkStages + g;
                unsigned char *sA = base + s * kStageBytes, *sB = sA + kStageA;
                mbar_expect_tx(&full[s], kStageBytes);
                bulk_g2s(sA, a.At + ((size_t)rt * a.KS + stage) * kStageA, kStageA, &full[s]);
                bulk_g2s(sB, a.Bt + ((size_t)qt * a.KS + stage) * kStageB, kStageB, &full[s]);
            }
            // drain: the copies of the last (up to kRing) issued stages must land before exit
            for (int h = max(0, g - kRing); h < g; ++h) mbar_wait(&full[h % kRing], (uint32_t)((h / kRing) & 1));
        }
    } else if (warp == kEpiWarps + 1) {
        // ---- MMA issuer
        if (lane == 0) {
            constexpr uint32_t IDESC = make_idesc_bf16(TM, TQ);
            int g = 0, last_commit = -1;
            bool ok = true;
            for (int ci = 0; ci < nch && ok; ++ci) {
                for (int st = 0; st < kChunkStages; ++st, ++g) {
                    const int s = g % kRing;
                    if (*abort_flag || !mbar_wait(&full[s], (uint32_t)((g / kRing) & 1))) { ok = false; break; }
                    fence_after_sync();
                    const uint32_t sA = smem_u32(base + s * kStageBytes), sB = sA + kStageA;
                    if (st == 0) {
                        // first stage of a chunk, level by level: level L starts (accumulate = 0) as
                        // soon as the epilogue has read level L of the previous chunk, so the reads
                        // and the double-FP32 folding overlap this chunk's MMAs
                        for (int L = 0; L < kLevels && ok; ++L) {
                            if (ci > 0) {
                                if (!mbar_wait(&acce[L], (uint32_t)((ci - 1) & 1))) { ok = false; break; }
                                fence_after_sync();
                            }
                            for (int p = 0; p <= L; ++p)
#pragma unroll
                                for (int kk = 0; kk < 2; ++kk)
                                    mma_bf16(tmem + (uint32_t)(L * TQ), make_desc_sw64(sA + p * kTileA + kk * 32),
                                             make_desc_sw64(sB + (L - p) * kTileB + kk * 32), IDESC,
                                             (p | kk) ? 1u : 0u);
                        }
                        if (!ok) break;
                    } else {
#pragma unroll
                        for (int kk = 0; kk < 2; ++kk)
#pragma unroll
                            for (int p = 0; p < kSlices; ++p)
#pragma unroll
                                for (int q = 0; q < kSlices - p; ++q)
                                    mma_bf16(tmem + (uint32_t)((p + q) * TQ), make_desc_sw64(sA + p * kTileA + kk * 32),
                                             make_desc_sw64(sB + q * kTileB + kk * 32), IDESC, 1u);
                    }
                    mma_commit(&empty[s]);
                    last_commit = s;
                }
                if (ok) mma_commit(accf);
            }
            if (!ok) {
                *abort_flag = 1;
                atomicExch(&g_oz_err, 1);
                // wait (bounded) for the MMAs already issued before the CTA frees its TMEM
                if (last_commit >= 0) {
                    const int h = g - 1;
                    mbar_wait(&empty[h % kRing], (uint32_t)((h / kRing) & 1));
                }
            }
        }
    } else {
        // ---- epilogue: eight warps, warp w reads TMEM lanes 32 (w % 4) .., columns 32 (w / 4) ..
        const int wq = warp & 3, h = warp >> 2;
        const int row = wq * 32 + lane;
        const uint32_t taddr = tmem + ((uint32_t)(wq * 32) << 16) + (uint32_t)(h * 32);
        float ah[32], al[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) ah[j] = al[j] = 0.f;
        const int rr = rt * TM + row;                      // real left row
        const int rpcA = OUT == 0 ? 1 : 2, rpcB = OUT == 0 ? 2 : 1;
        bool ok = true;
        for (int ci = 0; ci < nch; ++ci) {
            if (*abort_flag || !mbar_wait(accf, (uint32_t)(ci & 1))) { ok = false; break; }
            fence_after_sync();
            const int c = c0 + ci;
            const int er = a.EA[(size_t)c * a.nvA_pad + rr / rpcA];
            // chunk sum per column as a double-FP32 pair: levels 0-2 through TwoSum into (ch, cl);
            // levels 3-5 (at most 2^-16 of the chunk's scale) added into cl, whose FP32 rounding
            // then stays below 2^-40 of that scale
            float ch[32], cl[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) ch[j] = cl[j] = 0.f;
#pragma unroll
            for (int L = 0; L < kLevels; ++L) {
                const float sc = pow2f(-8 * (L + 2));
#pragma unroll
                for (int cg = 0; cg < 2; ++cg) {
                    float v[16];
                    tmem_ld16(taddr + (uint32_t)(L * TQ + cg * 16), v);
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int jj = cg * 16 + j;
                        if (L < 3) {
                            float s, e;
                            two_sum(ch[jj], v[j] * sc, s, e);
                            ch[jj] = s;
                            cl[jj] += e;
                        } else {
                            cl[jj] = fmaf(v[j], sc, cl[jj]);
                        }
                    }
                }
                // level L of this chunk is in registers: its accumulator may take the next chunk
                fence_before_sync();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acce[L]);
            }
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int qq = qt * TQ + h * 32 + j;
                const float S = pow2f(er + a.EB[(size_t)c * a.nvB_pad + qq / rpcB]);
                df_add(ah[j], al[j], ch[j] * S, cl[j] * S);
            }
        }
        if (!ok) {
            *abort_flag = 1;
            atomicExch(&g_oz_err, 1);
        } else if (OUT == 0) {
            double *P = a.P + (size_t)z * a.pstride;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int qq = qt * TQ + h * 32 + j;
                const double val = (double)ah[j] + (double)al[j];
                double *dst = P + (size_t)qq * a.ldp + rr;
                *dst = a.accumulate ? *dst + val : val;
            }
        } else {
            const int i = rr >> 1, part = rr & 1;
            const int gi = a.row0 + i;
            if (i < a.M) {
                double *Dd = reinterpret_cast<double *>(a.D);
                const double *Cd = reinterpret_cast<const double *>(a.C);
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int jj = qt * TQ + h * 32 + j;
                    if (jj < a.n) {
                        double val = a.alpha * ((double)ah[j] + (double)al[j]);
                        if (a.beta != 0.0) val += a.beta * Cd[2 * ((size_t)jj * a.ldc + gi) + part];
                        Dd[2 * ((size_t)jj * a.ldd + gi) + part] = val;
                    }
                }
            }
        }
    }
    fence_before_sync();
    __syncthreads();
    if (warp == kEpiWarps + 1) tmem_dealloc(tmem, kTmemCols);
}

// C = alpha (P-assembled A^H B) + beta C, P[split][q][r] with q = 2 j + (0: re, 1: im).
__global__ void k_oz_finish_cn(int m, int n, int nsplit, const double *__restrict__ P, int ldp, size_t pstride,
                               double alpha, double beta, z64 *C, int ldc, int lower) {
    const size_t tot = (size_t)m * n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % m), j = (int)(e / m);
        if (lower && i < j) continue;
        double re = 0.0, im = 0.0;
        for (int zz = 0; zz < nsplit; ++zz) {
            re += P[zz * pstride + (size_t)(2 * j) * ldp + i];
            im += P[zz * pstride + (size_t)(2 * j + 1) * ldp + i];
        }
        z64 v = mkc(alpha * re, alpha * im);
        if (beta != 0.0) v = v + beta * C[(size_t)j * ldc + i];
        C[(size_t)j * ldc + i] = v;
    }
}

int ensure_attr() {
    static std::atomic<bool> done0{false}, done1{false};
    if (!done0.load()) {
        LG_CUDA_TRY(cudaFuncSetAttribute(k_oz_mma<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem));
        done0.store(true);
    }
    if (!done1.load()) {
        LG_CUDA_TRY(cudaFuncSetAttribute(k_oz_mma<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem));
        done1.store(true);
    }
    return LOBPCG_OK;
}

int num_sms() {
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

inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

// Digits of nvec vectors over K range [k0, k0 + nchunks * 64) into tiles of TR real rows.
template <int TR, int MODE>
int split(const z64 *X, long long rs, long long ks, int nvec, int K, int k0, int nchunks, unsigned char *T, int *E,
          int nvec_pad, cudaStream_t s) {
    const int KS = nchunks * kChunkStages;
    k_oz_split<TR, MODE><<<dim3((nvec_pad + 31) / 32, nchunks), 256, 0, s>>>(X, rs, ks, nvec, K, k0, KS, T, E,
                                                                             nvec_pad);
    return check_launch("FP64-class tensor-core GEMM: operand digits");
}

// Scratch budget of the digit tiles of one slab (bytes).
constexpr size_t kSlabBytes = (size_t)768 << 20;

}  // namespace

// C = alpha A^H B + beta C, complex128, A: K x m (lda), B: K x n (ldb), C: m x n (ldc).
// lower: only entries i >= j are written (and tiles wholly above the diagonal skipped).
int oz_gemm_cn(GemmWork &w, int m, int n, int K, double alpha, const z64 *A, int lda, const z64 *B, int ldb,
               double beta, z64 *C, int ldc, cudaStream_t s, bool lower) {
    if (m <= 0 || n <= 0) return LOBPCG_OK;
    LG_TRY(ensure_attr());
    const int mA = round_up(m, TM);            // left real rows (one per column of A)
    const int qB = round_up(2 * n, TQ);        // right real rows (two per column of B)
    const int nvA = mA, nvB = qB / 2;          // padded vector counts
    const int Kc = std::max(1, (K + kChunkC - 1) / kChunkC);   // chunks of the whole reduction
    // slab: chunks whose digits fit the scratch budget
    const size_t per_chunk = (size_t)kChunkStages * ((size_t)(mA / TM) * kStageA + (size_t)(qB / TQ) * kStageB);
    const int slab = std::max(1, std::min(Kc, (int)(kSlabBytes / per_chunk)));
    const int tm = mA / TM, tq = qB / TQ;
    long long tiles = 0;
    for (int rt = 0; rt < tm; ++rt)
        for (int qt = 0; qt < tq; ++qt)
            if (!lower || 32 * qt <= TM * rt + TM - 1) ++tiles;
    const int want = std::max(1, (int)((2LL * num_sms() + tiles - 1) / tiles));
    int cps = std::max(1, (slab + want - 1) / want);
    const int nsplit = (slab + cps - 1) / cps;
    LG_TRY(w.alloc->ensure(w.oz_a, per_chunk * slab));
    LG_TRY(w.alloc->ensure(w.oz_e, sizeof(int) * (size_t)slab * (nvA + nvB)));
    LG_TRY(w.alloc->ensure(w.oz_p, sizeof(double) * (size_t)nsplit * qB * mA));
    unsigned char *At = static_cast<unsigned char *>(w.oz_a.p);
    unsigned char *Bt = At + (size_t)slab * kChunkStages * tm * kStageA;
    int *EA = static_cast<int *>(w.oz_e.p), *EB = EA + (size_t)slab * nvA;
    double *P = static_cast<double *>(w.oz_p.p);
    for (int cb = 0, first = 1; cb < Kc; cb += slab, first = 0) {
        const int nc = std::min(slab, Kc - cb);
        const int k0 = cb * kChunkC;
        LG_TRY((split<TM, kRowsPlain>(A, lda, 1, m, K, k0, nc, At, EA, nvA, s)));
        LG_TRY((split<TQ, kRowsCnB>(B, ldb, 1, n, K, k0, nc, Bt, EB, nvB, s)));
        OzArgs a{};
        a.At = At;
        a.Bt = Bt;
        a.EA = EA;
        a.EB = EB;
        a.KS = nc * kChunkStages;
        a.nvA_pad = nvA;
        a.nvB_pad = nvB;
        a.nchunks = nc;
        a.cps = cps;
        a.lower = lower ? 1 : 0;
        a.P = P;
        a.ldp = mA;
        a.pstride = (size_t)qB * mA;
        a.accumulate = first ? 0 : 1;
        k_oz_mma<0><<<dim3(tq, tm, nsplit), kThreads, kSmem, s>>>(a);
        LG_TRY(check_launch("FP64-class tensor-core GEMM A^H B"));
    }
    const size_t tot = (size_t)m * n;
    const int blocks = (int)std::min<size_t>((tot + 255) / 256, 4096);
    k_oz_finish_cn<<<blocks, 256, 0, s>>>(m, n, nsplit, P, mA, (size_t)qB * mA, alpha, beta, C, ldc,
                                          lower ? 1 : 0);
    return check_launch("FP64-class tensor-core GEMM: partial sums");
}

// D = alpha A B + beta C, complex128, A: M x k (lda), B: k x n (ldb), C, D: M x n.
int oz_gemm_nn(GemmWork &w, int M, int n, int k, double alpha, const z64 *A, int lda, const z64 *B, int ldb,
               double beta, const z64 *C, int ldc, z64 *D, int ldd, cudaStream_t s) {
    if (M <= 0 || n <= 0) return LOBPCG_OK;
    LG_TRY(ensure_attr());
    const int Kc = std::max(1, (k + kChunkC - 1) / kChunkC);
    const int qB = round_up(n, TQ);
    const int nvB = qB;
    // slab of complex rows of A (two real rows each): a multiple of 64 rows (one left tile)
    const size_t per_row = (size_t)2 * Kc * kChunkStages * kSlices * 64;   // bytes of digits per complex row
    int rows = (int)std::min<size_t>((size_t)round_up(M, TM / 2), std::max<size_t>(TM / 2, kSlabBytes / per_row));
    rows = std::max(TM / 2, rows / (TM / 2) * (TM / 2));
    const int nvA = rows;
    const size_t bytesA = (size_t)(2 * rows / TM) * Kc * kChunkStages * kStageA;
    const size_t bytesB = (size_t)(qB / TQ) * Kc * kChunkStages * kStageB;
    LG_TRY(w.alloc->ensure(w.oz_a, bytesA + bytesB));
    LG_TRY(w.alloc->ensure(w.oz_e, sizeof(int) * (size_t)Kc * (nvA + nvB)));
    unsigned char *At = static_cast<unsigned char *>(w.oz_a.p), *Bt = At + bytesA;
    int *EA = static_cast<int *>(w.oz_e.p), *EB = EA + (size_t)Kc * nvA;
    LG_TRY((split<TQ, kRowsPlain>(B, ldb, 1, n, k, 0, Kc, Bt, EB, nvB, s)));
    for (int r0 = 0; r0 < M; r0 += rows) {
        const int mr = std::min(rows, M - r0);
        LG_TRY((split<TM, kRowsNnA>(A + r0, 1, lda, mr, k, 0, Kc, At, EA, nvA, s)));
        OzArgs a{};
        a.At = At;
        a.Bt = Bt;
        a.EA = EA;
        a.EB = EB;
        a.KS = Kc * kChunkStages;
        a.nvA_pad = nvA;
        a.nvB_pad = nvB;
        a.nchunks = Kc;
        a.cps = Kc;
        a.M = mr;
        a.n = n;
        a.row0 = r0;
        a.alpha = alpha;
        a.beta = beta;
        a.C = beta != 0.0 ? C : D;
        a.ldc = beta != 0.0 ? ldc : ldd;
        a.D = D;
        a.ldd = ldd;
        const int tm = (2 * mr + TM - 1) / TM;
        k_oz_mma<1><<<dim3(qB / TQ, tm, 1), kThreads, kSmem, s>>>(a);
        LG_TRY(check_launch("FP64-class tensor-core GEMM A B"));
    }
    return LOBPCG_OK;
}

int oz_check_error() {
    int h = 0;
    LG_CUDA_TRY(cudaMemcpyFromSymbol(&h, g_oz_err, sizeof(int)));
    if (h) {
        const int zero = 0;
        LG_CUDA_TRY(cudaMemcpyToSymbol(g_oz_err, &zero, sizeof(int)));
        return fail(LOBPCG_ERR_TIMEOUT, "a bounded device wait ran out (FP64-class tensor-core GEMM)");
    }
    return LOBPCG_OK;
}

}  // namespace lg
