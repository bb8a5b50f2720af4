// rll_learn_update_noalloc: the end-of-pass learning step without any
// device allocation.
//
// Who needs it: callers that must not call cudaMalloc while they run -- a
// host that has handed all device memory to its own pool or allocator, a
// process that runs under an allocation budget enforced outside CUDA, or a
// loop that must not synchronise (the growable workspace of rll_learn_update
// synchronises and calls cudaFree/cudaMalloc the first time it grows).
//
// How: the radix-sort buffers live in one file-scope device array of fixed
// size. Every GPU that loads this library holds that array until the process
// exits. Its device address is looked up once per device (the first call of
// the entry point on a device does that set-up, so make that first call
// before any stream capture) and kept for the life of the process: it does
// not survive a cudaDeviceReset of that device, after which this entry point
// must not be called again in the same process. All calls share the array and it keeps the
// previous call's contents; whatever must start at zero (the per-pass digit
// totals, the touched-cell count) is cleared by the call itself. Calls whose
// work overlaps on the GPU (other streams, other host threads) race on the
// array: serialise them.
#include <cuda_runtime.h>

#include <mutex>

#include "rll_device.cuh"
#include "rll_internal.h"

namespace {

// Largest record count one call accepts.
constexpr int64_t kNoAllocMaxRecords = int64_t(1) << 20;

// Sort scratch for kNoAllocMaxRecords records (the sort's own formula).
constexpr size_t kNoAllocScratchBytes = rll::sort_scratch_bytes_for(kNoAllocMaxRecords);

static __device__ __align__(256) unsigned char g_learn_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_learn_scratch on `device` (current), looked up once.
int scratch_for(rll_ctx* ctx, void** out)
{
    if (ctx->device < 0 || ctx->device >= kMaxDevices) return rll::fail(ctx, RLL_E_INVALID, "device index too large");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[ctx->device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_learn_scratch);
        if (e != cudaSuccess) return rll::check_cuda(ctx, e, "cudaGetSymbolAddress(learn scratch)");
        g_scratch_ptr[ctx->device] = p;
    }
    *out = g_scratch_ptr[ctx->device];
    return RLL_OK;
}

}  // namespace

extern "C" int rll_learn_update_noalloc(rll_ctx* ctx, rll_grid* grid, const uint32_t* rec_key, const float* rec_val,
                                        int64_t n_records)
{
    if (!ctx) return RLL_E_INVALID;
    if (!grid) return rll::fail(ctx, RLL_E_INVALID, "grid is NULL");
    if (n_records < 0) return rll::fail(ctx, RLL_E_INVALID, "n_records < 0");
    if (n_records > kNoAllocMaxRecords)
        return rll::fail(ctx, RLL_E_INVALID,
                         "rll_learn_update_noalloc takes at most 1048576 records per call (use rll_learn_update)");
    if (n_records > 0 && (!rec_key || !rec_val)) return rll::fail(ctx, RLL_E_INVALID, "NULL records");
    rll::DeviceGuard dev(ctx->device);
    void* scratch = nullptr;
    const int rc = scratch_for(ctx, &scratch);
    if (rc != RLL_OK) return rc;
    return rll::learn_update_with_scratch(ctx, grid, rec_key, rec_val, n_records, scratch, kNoAllocScratchBytes);
}
