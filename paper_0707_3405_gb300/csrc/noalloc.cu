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
// array's name as a device address: lobpcg_create, with the handle's device
// current, looks the address up once per device with cudaGetSymbolAddress and
// keeps it.  That lookup is also what loads this file's device module (the
// library is built without relocatable device code, so each source file is a
// module of its own, and CUDA loads modules lazily), i.e. where the 32 MiB are
// actually reserved; doing it at create keeps that reservation out of the
// allocation-free call.  A call therefore needs the handle's device to be the
// current one (else LOBPCG_ERR_ARG).
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

namespace lg {
// Called by lobpcg_create on the handle's device: loads this module and records the
// scratch address, so that lobpcg_apply_local_noalloc itself does no set-up.
int noalloc_prepare() {
    void *p = nullptr;
    return scratch_address(&p);
}
}  // namespace lg

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
    int dev = -1;
    LG_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != v.device)
        return fail(LOBPCG_ERR_ARG, "the current device is not the handle's device (" + std::to_string(dev) +
                                        " vs " + std::to_string(v.device) + ")");
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
