// xpr_tile_bin_noalloc: the tile-binning entry point for callers that cannot allocate device memory.
//
// xpr_tile_bin needs a small scratch buffer for its prefix sum (one 8-byte partial sum per 4096
// primitives plus the total).  Some callers cannot hand one over: a process whose device memory is
// owned entirely by another framework's pool (a cudaMalloc there fails or evicts someone else's
// data), or a latency-critical loop that must not call cudaMalloc/cudaFree because those can
// synchronise the whole device and stall every other stream.  This variant takes its scratch from
// a file-scope __device__ array instead, so the caller passes only inputs and outputs.
//
// The array lives in the library's module: every GPU that loads libxpr.so holds it (131,328 bytes)
// until the process exits.  Host code cannot use the array's name as a device address, so the
// first call on each device looks the address up with cudaGetSymbolAddress while that device is
// current and caches it; that first call should therefore come before any stream capture.
#include <mutex>

#include "xpr_internal.cuh"

namespace xpr {
namespace {

// Largest primitive count served: the scan keeps ceil(n / 4096) partial sums plus its total.
constexpr int64_t kNoAllocMaxN = int64_t(1) << 26;  // 67,108,864 primitives
constexpr size_t kNoAllocScratchBytes = 131328;     // = scan_partials_bytes(kNoAllocMaxN)
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_bin_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {};

int scratch_for_current_device(void **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(XPR_ERR_CUDA, "xpr_tile_bin_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices)
        return fail(XPR_ERR_INVALID, "xpr_tile_bin_noalloc: device ordinal %d beyond %d", dev, kMaxDevices);
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_scratch_ptr[dev] == nullptr) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_bin_scratch);
        if (e != cudaSuccess || p == nullptr)
            return fail(XPR_ERR_CUDA, "xpr_tile_bin_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return XPR_OK;
}

}  // namespace
}  // namespace xpr

using namespace xpr;

extern "C" int xpr_tile_bin_noalloc(const float *rec, const int32_t *bbox, const int32_t *tile_count,
                                    const int32_t *isect_count, const int32_t *order, int64_t n,
                                    const XprCamera *cam, const XprConfig *cfg, int32_t *offsets, uint64_t *keys,
                                    uint32_t *tiles, uint32_t *vals, int64_t capacity, int64_t *n_isect,
                                    void *stream) {
    if (n > kNoAllocMaxN)
        return fail(XPR_ERR_INVALID, "xpr_tile_bin_noalloc: n = %lld exceeds the static-scratch limit of %lld "
                    "primitives; use xpr_tile_bin with a caller-provided workspace", (long long)n,
                    (long long)kNoAllocMaxN);
    if (xpr_tile_bin_workspace(n) > kNoAllocScratchBytes)
        return fail(XPR_ERR_INTERNAL, "xpr_tile_bin_noalloc: static scratch too small for n = %lld", (long long)n);
    void *ws = nullptr;
    int s = scratch_for_current_device(&ws);
    if (s != XPR_OK) return s;
    return xpr_tile_bin(rec, bbox, tile_count, isect_count, order, n, cam, cfg, offsets, keys, tiles, vals, capacity,
                        n_isect, ws, kNoAllocScratchBytes, stream);
}
