// Allocation-free variant of the local-potential H application.
//
// Some callers cannot call cudaMalloc while they run: code that executes
// inside another framework's memory pool or under a strict device-memory
// budget, real-time loops that must not touch the allocator (allocation can
// synchronise the device), and processes that forbid further allocation after
// start-up.  lobpcg_apply_local_noalloc computes Y = (T + V_loc) X with the
// same three FFT passes as lobpcg_apply_H but keeps its intermediate
// half-box in a fixed file-scope device array instead of library-allocated
// scratch, and calls no allocating routine.
//
// The array is kNoAllocScratchBytes (32 MiB) per device, held by every GPU
// that loads the library until the process exits.  Host code cannot use the
// array's name as a device address, so the first call on each device, with
// that device current, looks the address up with cudaGetSymbolAddress and
// keeps it; that first call should therefore come before any stream capture.
// All calls share the array: calls that overlap on the GPU (different
// streams, or different handles at once) race on it.  Every element of the
// half-box is written before it is read within a call, so nothing carried
// over from an earlier call is used.
#include "common.cuh"

#include <algorithm>
#include <mutex>

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

void *g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

// Device address of the scratch array on the current device (looked up once per device).
int scratch_address(void **out) {
    int dev = 0;
    LG_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return lg::fail(LOBPCG_ERR_UNSUPPORTED, "device index too large");
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        LG_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return LOBPCG_OK;
}

}  // namespace

using namespace lg;

extern "C" {

int lobpcg_apply_local_noalloc(lobpcg_ctx *ctx, int k, const void *X, void *Y, int nb, int precision) {
    if (!ctx) return fail(LOBPCG_ERR_ARG, "ctx is NULL");
    LocalView v;
    LG_TRY(ctx_local_view(ctx, k, &v));
    if (nb < 0) return fail(LOBPCG_ERR_ARG, "nb must be >= 0");
    if (nb == 0) return LOBPCG_OK;
    if (!X || !Y) return fail(LOBPCG_ERR_ARG, "X and Y must not be NULL");
    if (precision != LOBPCG_C128 && precision != LOBPCG_C64) return fail(LOBPCG_ERR_ARG, "unknown precision");
    if (!is_device_pointer(X) || !is_device_pointer(Y))
        return fail(LOBPCG_ERR_ARG, "X and Y must be device pointers (no staging without allocation)");
    const size_t esz = precision == LOBPCG_C128 ? sizeof(z64) : sizeof(c32);
    const size_t bytes = esz * (size_t)v.npw * nb;
    const char *xa = static_cast<const char *>(X), *ya = static_cast<const char *>(Y);
    if (xa < ya + bytes && ya < xa + bytes) return fail(LOBPCG_ERR_ARG, "X and Y overlap");
    const FFTGeom &g = *v.geom;
    const size_t per_band = esz * (size_t)g.Px * g.N * g.N;
    if (per_band > kNoAllocScratchBytes)
        return fail(LOBPCG_ERR_ARG, "one band's FFT half-box (" + std::to_string(per_band) +
                                        " bytes) exceeds the no-alloc scratch of " +
                                        std::to_string(kNoAllocScratchBytes) + " bytes");
    void *scratch = nullptr;
    LG_TRY(scratch_address(&scratch));
    const int nbatch = (int)std::min<size_t>(std::min<size_t>(kNoAllocScratchBytes / per_band, (size_t)nb), 65535);
    if (precision == LOBPCG_C128)
        return fft_vloc_apply<double>(g, *v.plan, static_cast<const z64 *>(X), v.npw, static_cast<z64 *>(Y), v.npw,
                                      nb, v.kin64, v.vt64, v.tw64, static_cast<z64 *>(scratch), nbatch, v.stream);
    return fft_vloc_apply<float>(g, *v.plan, static_cast<const c32 *>(X), v.npw, static_cast<c32 *>(Y), v.npw, nb,
                                 v.kin32, v.vt32, v.tw32, static_cast<c32 *>(scratch), nbatch, v.stream);
}

}  // extern "C"
