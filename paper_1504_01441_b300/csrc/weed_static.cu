// hdrreg_weed_static: the weeding step (row a6) for callers that cannot
// allocate device memory, with its scratch in a fixed array of this library
// instead of a caller-provided workspace.
//
// The scratch is a file-scope __device__ array, so every GPU that loads the
// library holds it (about 160 KB) until the process exits. In host code the
// array's name is only a host-side stand-in, never a device address: the
// device address is obtained once per device with cudaGetSymbolAddress (with
// that device current) and cached; that set-up runs inside the first call made
// on each device, so that first call should be made before any stream capture.
// All calls share the one array and leave their contents in it; every value the
// kernels read is written by the same call first, so nothing needs clearing.
// Calls whose kernels overlap on the GPU (different streams, or different host
// threads, on one device) race on the array and must be serialized by the caller.
#include <mutex>

#include "hdrreg_internal.cuh"

namespace hdrreg {
namespace {

constexpr size_t align256(size_t v) { return (v + 255) / 256 * 256; }

// Same carve-up as weed_ws_bytes(): tile list, count, FP32 coordinates.
constexpr size_t kStaticTiles = HDRREG_WEED_STATIC_MAX_TILES;
constexpr size_t kStaticBytes = align256(kStaticTiles * 4) + 256 + align256(kStaticTiles * 16);

__device__ __align__(256) unsigned char g_weed_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of g_weed_scratch on the current device (looked up once per device).
hdrreg_status scratch_address(void** out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(HDRREG_E_CUDA, "weed_static: cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices)
        return fail(HDRREG_E_UNSUPPORTED, "weed_static: device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_weed_scratch);
        if (e != cudaSuccess || !p)
            return fail(HDRREG_E_CUDA, "weed_static: cudaGetSymbolAddress: %s",
                        cudaGetErrorString(e));
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return HDRREG_OK;
}

}  // namespace
}  // namespace hdrreg

using namespace hdrreg;

extern "C" hdrreg_status hdrreg_weed_static(const int32_t* corner_xy, const int32_t* match_xy,
                                            const uint8_t* valid, int n, int w, int h,
                                            const hdrreg_params* p, uint64_t seed,
                                            int iter_begin, int iter_end, uint32_t* mask_bits,
                                            void* stream)
{
    hdrreg_status st = hdrreg_validate_params(p);
    if (st) return st;
    if (n < 0 || n > HDRREG_WEED_STATIC_MAX_TILES)
        return fail(HDRREG_E_INVALID_ARG,
                    "weed_static: n = %d tiles; the static scratch holds at most %d (use "
                    "hdrreg_weed with a workspace for more)",
                    n, HDRREG_WEED_STATIC_MAX_TILES);
    if (n > 0 && (!corner_xy || !match_xy || !valid || !mask_bits))
        return fail(HDRREG_E_INVALID_ARG, "weed_static: NULL pointer");
    if (w < 1 || h < 1 || w > 16384 || h > 16384)
        return fail(HDRREG_E_INVALID_ARG, "weed_static: bad size %dx%d", w, h);
    if (iter_begin < 0 || iter_end < iter_begin)
        return fail(HDRREG_E_INVALID_ARG, "weed_static: bad iteration range [%d, %d)",
                    iter_begin, iter_end);
    if (n == 0) return HDRREG_OK;
    if (weed_ws_bytes(n) > kStaticBytes)
        return fail(HDRREG_E_UNSUPPORTED, "weed_static: scratch layout exceeds the static array");
    void* scratch = nullptr;
    if ((st = scratch_address(&scratch))) return st;
    launch_weed(corner_xy, match_xy, valid, n, w, h, p->weed_eps, p->weed_delta_min,
                p->weed_delta_div, seed, iter_begin, iter_end, mask_bits,
                weed_ws_carve(scratch, n), static_cast<cudaStream_t>(stream));
    return launch_status("weed_static");
}
