// C ABI of the hdrreg library: argument validation, workspace layout, the step
// calls and the fused per-stack pipeline (rows a1-a11), all stream-ordered and
// free of host synchronization so a whole call can be captured in a CUDA graph.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "hdrreg_internal.cuh"

namespace hdrreg {

static thread_local std::string g_last_error;

void set_error(const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
}

hdrreg_status fail(hdrreg_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

static std::atomic<unsigned long long> g_launches{0};

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// cudaFuncSetAttribute is a host-side setting per device; do it once per
// (device, kernel) and size so that calls made during stream capture only enqueue.
void ensure_smem(const void* kernel, size_t bytes)
{
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> done;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    size_t& cur = done[{dev, kernel}];
    if (bytes > cur) {
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        cur = bytes;
    }
}

hdrreg_status launch_status(const char* what)
{
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(HDRREG_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
    return HDRREG_OK;
}

static int num_levels(int w, int h, int levels_max, int min_size)
{
    int L = 1;
    while (L < levels_max) {
        const int lw = w >> L, lh = h >> L;
        if (lw < min_size || lh < min_size) break;
        L++;
    }
    return L;
}

static bool bad_dims(int w, int h) { return w < 1 || h < 1 || w > 16384 || h > 16384; }

static SearchGeom make_geom(int w, int h, const hdrreg_params* p)
{
    SearchGeom g;
    g.w = w;
    g.h = h;
    g.tile = p->tile;
    g.radius = p->radius;
    g.patch_half = p->patch_half;
    g.grid_half = p->grid_half;
    g.quad = p->quad;
    g.step = p->tile / 16 > 1 ? p->tile / 16 : 1;
    g.ntx = w / p->tile;
    g.nty = h / p->tile;
    g.corner_thr = (long long)p->corner_thresh * p->quad * p->quad;
    g.threads = p->search_threads ? p->search_threads : 128;
    return g;
}

// ------------------------------------------------------- fused workspace
struct Layout {
    size_t total = 0;
    size_t add(size_t bytes)
    {
        const size_t o = total;
        total += align_up(bytes > 0 ? bytes : 1, 256);
        return o;
    }
};

struct FusedLayout {
    int L = 1, n0 = 0, nsrc = 1;
    size_t ref_lv[kMaxLevels], src_lv[kMaxLevels];
    size_t corner, match, cost, valid, mask, H, fit_st, done, weed, hist, luts, flow, fu, fv;
    bool learned = false;  // level-0 search by the predictor (row a-L)
    int wq = 0, hq = 0, pho = 0, pwo = 0;
    size_t xq = 0, pred = 0, cnn = 0, fellback = 0;
    size_t wy[kMaxSources], wu[kMaxSources], wv[kMaxSources], refn[kMaxSources],
        clip[kMaxSources];
    size_t q = 0, fuse = 0;  // output_mode != 0
    size_t total;
    FusedLayout(int w, int h, int ns, const hdrreg_params* p)
    {
        Layout lay;
        nsrc = ns;
        L = num_levels(w, h, p->levels_max, p->min_level_size);
        n0 = (w / p->tile) * (h / p->tile);
        for (int l = 0; l < kMaxLevels; l++) ref_lv[l] = src_lv[l] = 0;
        for (int l = 0; l < L; l++) {
            ref_lv[l] = lay.add((size_t)(w >> l) * (h >> l));
            src_lv[l] = lay.add((size_t)(w >> l) * (h >> l));
        }
        const size_t nn = n0 > 0 ? n0 : 1;
        corner = lay.add(nn * 8);
        match = lay.add(nn * 8);
        cost = lay.add(nn * 4);
        valid = lay.add(nn);
        mask = lay.add((nn / 32 + 1) * 4);
        H = lay.add((size_t)(kMaxLevels + 2) * 9 * 8);
        fit_st = lay.add(kMaxLevels * 4);
        done = lay.add((kMaxLevels + 1) * 4);  // completion counters + predictor status word
        weed = lay.add(weed_ws_bytes(n0));
        hist = lay.add(2 * 256 * 4);
        luts = lay.add((size_t)kMaxSources * 512);
        flow = lay.add(flow_ws_bytes(w, h));
        fu = lay.add((size_t)flow_pitch(w) * h * 4);  // flow planes at the flow's padded pitch
        fv = lay.add((size_t)flow_pitch(w) * h * 4);
        // one network output cell per 32 x 32 tile (8 x 8 quarter-resolution pixels)
        learned = p->predictor != nullptr && L >= 3 && p->tile == 32 && (w >> 2) >= 8 &&
                  (h >> 2) >= 8;
        if (learned) {
            wq = w >> 2;
            hq = h >> 2;
            cnn_out_dims(hq, wq, &pho, &pwo);
            learned = pho >= h / 32 && pwo >= w / 32;
        }
        if (learned) {
            xq = lay.add((size_t)wq * hq * 4);
            pred = lay.add((size_t)pho * pwo * 8);
            cnn = lay.add(cnn_infer_ws_bytes(1, hq, wq));
            fellback = lay.add(nn);
        }
        for (int k = 0; k < ns; k++) {
            wy[k] = lay.add((size_t)w * h * 4);
            wu[k] = lay.add((size_t)(w / 2) * (h / 2) * 4);
            wv[k] = lay.add((size_t)(w / 2) * (h / 2) * 4);
            refn[k] = lay.add((size_t)w * h);
            clip[k] = lay.add((size_t)w * h);
        }
        q = fuse = 0;
        if (p->output_mode != 0) {  // exposure fusion: the SSIM maps and the pyramids
            q = lay.add((size_t)ns * w * h * 4);
            fuse = lay.add(fuse_ws_bytes(w, h, ns + 1, true));
        }
        total = lay.total;
    }
};

__global__ void __launch_bounds__(256) k_diag(const double* H0, const uint8_t* valid,
                                              const uint32_t* mask, int n, const int32_t* fit_st,
                                              int levels, const uint8_t* fell_back,
                                              const int* flow_err, hdrreg_diag* d)
{
    __shared__ int sv, sk, sf;
    if (threadIdx.x == 0) {
        sv = 0;
        sk = 0;
        sf = 0;
    }
    __syncthreads();
    int v = 0, k = 0, f = 0;
    // the 0/1 flags 16 at a time (one round trip per thread at 5 MP), the rest one by one
    const bool vec = ((uintptr_t)valid & 15u) == 0 && ((uintptr_t)fell_back & 15u) == 0;
    const int n16 = vec ? n / 16 : 0;
    for (int i = threadIdx.x; i < n16; i += blockDim.x) {
        const uint4 a = reinterpret_cast<const uint4*>(valid)[i];
        v = __dp4a((int)a.x, 0x01010101, v);
        v = __dp4a((int)a.y, 0x01010101, v);
        v = __dp4a((int)a.z, 0x01010101, v);
        v = __dp4a((int)a.w, 0x01010101, v);
        if (fell_back) {
            const uint4 b = reinterpret_cast<const uint4*>(fell_back)[i];
            f = __dp4a((int)b.x, 0x01010101, f);
            f = __dp4a((int)b.y, 0x01010101, f);
            f = __dp4a((int)b.z, 0x01010101, f);
            f = __dp4a((int)b.w, 0x01010101, f);
        }
    }
    for (int t = 16 * n16 + threadIdx.x; t < n; t += blockDim.x) {
        v += valid[t];
        if (fell_back) f += fell_back[t];
    }
    for (int wi = threadIdx.x; wi < (n + 31) / 32; wi += blockDim.x) {
        const int bits = n - 32 * wi < 32 ? n - 32 * wi : 32;
        k += __popc(mask[wi] & (bits == 32 ? ~0u : (1u << bits) - 1u));
    }
    v = __reduce_add_sync(0xffffffffu, v);
    k = __reduce_add_sync(0xffffffffu, k);
    f = __reduce_add_sync(0xffffffffu, f);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&sv, v);
        atomicAdd(&sk, k);
        atomicAdd(&sf, f);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 0; i < 9; i++) d->H0[i] = H0[i];
        d->levels = levels;
        d->tiles = n;
        d->valid = sv;
        d->kept = sk;
        int bits = 0;
        for (int l = 0; l < levels; l++) bits |= (fit_st[l] != 0) << l;
        d->fit_status = bits;
        d->fallbacks = fell_back ? sf : -1;
        d->flow_status = (flow_err && *flow_err) ? 1 : 0;
        d->reserved = 0;
    }
}

}  // namespace hdrreg

using namespace hdrreg;

extern "C" {

const char* hdrreg_last_error(void) { return g_last_error.c_str(); }

const char* hdrreg_version(void) { return "hdrreg 0.1 (sm_103a)"; }

unsigned long long hdrreg_launch_count(void) { return g_launches.load(); }

void hdrreg_params_default(hdrreg_params* p)
{
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->tile = 32;
    p->radius = 10;
    p->patch_half = 10;
    p->levels_max = 5;
    p->min_level_size = 100;
    p->grid_half = 4;
    p->quad = 10;
    p->corner_thresh = 2;
    p->weed_iters = 512;
    p->weed_delta_min = 8;
    p->weed_delta_div = 20;
    p->norm_mode = HDRREG_NORM_HISTEQ;
    p->dt_iters = 3;
    p->ssim_radius = 5;
    p->propagate_full = 0;
    p->weed_eps = 1.5;
    p->sigma_s = 400.0;
    p->sigma_r = 0.5;
    p->ssim_sigma = 1.5;
    p->we_sigma = 0.2;
    p->flow_eps = 1e-20;
    p->weed_seed = 0x1504014410ull;
    p->predictor = nullptr;
    p->fallback_cost = 0u;
}

void hdrreg_params_paper(hdrreg_params* p)
{
    if (!p) return;
    hdrreg_params_default(p);
    p->propagate_full = 1;
}

hdrreg_status hdrreg_validate_params(const hdrreg_params* p)
{
    if (!p) return fail(HDRREG_E_INVALID_ARG, "params is NULL");
    if (p->tile < 8 || p->tile > 128 || (p->tile & 1))
        return fail(HDRREG_E_INVALID_ARG, "tile must be even and in [8, 128] (got %d)", p->tile);
    if (p->radius < 1 || p->radius > 15)
        return fail(HDRREG_E_INVALID_ARG, "radius must be in [1, 15] (got %d)", p->radius);
    if (p->patch_half < 1 || p->patch_half > 15)
        return fail(HDRREG_E_INVALID_ARG, "patch_half must be in [1, 15] (got %d)", p->patch_half);
    if (p->levels_max < 1 || p->levels_max > kMaxLevels)
        return fail(HDRREG_E_INVALID_ARG, "levels_max must be in [1, %d]", kMaxLevels);
    if (p->min_level_size < 1) return fail(HDRREG_E_INVALID_ARG, "min_level_size must be >= 1");
    const int step = p->tile / 16 > 1 ? p->tile / 16 : 1;
    if (p->grid_half < 0 || p->grid_half > 8 || p->grid_half * step > p->tile / 2 - 1)
        return fail(HDRREG_E_INVALID_ARG,
                    "grid_half must be in [0, 8] with grid_half*max(1,T/16) < T/2 (got %d)",
                    p->grid_half);
    if (p->quad < 1 || p->quad > 32) return fail(HDRREG_E_INVALID_ARG, "quad must be in [1, 32]");
    if (p->corner_thresh < 0) return fail(HDRREG_E_INVALID_ARG, "corner_thresh must be >= 0");
    if (p->weed_iters < 0 || p->weed_iters > 65536)
        return fail(HDRREG_E_INVALID_ARG, "weed_iters must be in [0, 65536]");
    if (p->weed_delta_min < 0 || p->weed_delta_div < 1)
        return fail(HDRREG_E_INVALID_ARG, "weed_delta_min >= 0 and weed_delta_div >= 1 required");
    if (p->norm_mode != HDRREG_NORM_RATIO && p->norm_mode != HDRREG_NORM_HISTEQ)
        return fail(HDRREG_E_INVALID_ARG, "unknown norm_mode %d", p->norm_mode);
    if (p->dt_iters < 1 || p->dt_iters > 8)
        return fail(HDRREG_E_INVALID_ARG, "dt_iters must be in [1, 8]");
    if (p->ssim_radius != kSsimRadius)
        return fail(HDRREG_E_INVALID_ARG, "ssim_radius must be %d", kSsimRadius);
    if (p->predictor && (p->predictor_refine < 0 || p->predictor_refine > p->radius))
        return fail(HDRREG_E_INVALID_ARG, "predictor_refine must be in [0, radius]");
    if (p->search_threads != 0 && p->search_threads != 64 && p->search_threads != 128 &&
        p->search_threads != 256)
        return fail(HDRREG_E_INVALID_ARG, "search_threads must be 0, 64, 128 or 256");
    if (p->propagate_full != 0 && p->propagate_full != 1)
        return fail(HDRREG_E_INVALID_ARG, "propagate_full must be 0 or 1");
    if (p->output_mode < 0 || p->output_mode > 2)
        return fail(HDRREG_E_INVALID_ARG, "output_mode must be 0, 1 or 2");
    if (!(p->weed_eps > 0) || !(p->sigma_s > 0) || !(p->sigma_r > 0) || !(p->ssim_sigma > 0) ||
        !(p->we_sigma > 0) || !(p->flow_eps >= 0))
        return fail(HDRREG_E_INVALID_ARG,
                    "weed_eps, sigma_s, sigma_r, ssim_sigma, we_sigma must be > 0, flow_eps >= 0");
    return HDRREG_OK;
}

int hdrreg_num_levels(int w, int h, const hdrreg_params* p)
{
    if (!p || bad_dims(w, h)) return 0;
    return num_levels(w, h, p->levels_max, p->min_level_size);
}

int hdrreg_num_tiles(int w, int h, int tile)
{
    if (tile < 1 || w < 0 || h < 0) return 0;
    return (w / tile) * (h / tile);
}

// ------------------------------------------------------------------- a1
size_t hdrreg_normalize_workspace_size(int mode)
{
    return mode == HDRREG_NORM_HISTEQ ? 2 * 256 * 4 : 0;
}

hdrreg_status hdrreg_normalize_exposure(const uint8_t* ref_y, const uint8_t* src_y, int w, int h,
                                        int mode, int ratio_num, int ratio_den, uint8_t* ref_n,
                                        uint8_t* src_n, uint8_t* luts, void* workspace,
                                        size_t ws_bytes, void* stream)
{
    if (!ref_y || !src_y || !ref_n || !src_n)
        return fail(HDRREG_E_INVALID_ARG, "normalize: NULL plane");
    if (bad_dims(w, h)) return fail(HDRREG_E_INVALID_ARG, "normalize: bad size %dx%d", w, h);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t n = (size_t)w * h;
    if (mode == HDRREG_NORM_RATIO) {
        if (ratio_num < 1 || ratio_den < 1)
            return fail(HDRREG_E_INVALID_ARG, "normalize: ratio must be positive (%d/%d)",
                        ratio_num, ratio_den);
        const bool ref_darker = ratio_num >= ratio_den;
        LutSpec la{nullptr, 1, 1}, lb{nullptr, 1, 1};
        if (ref_darker) la = LutSpec{nullptr, ratio_num, ratio_den};
        else lb = LutSpec{nullptr, ratio_den, ratio_num};
        launch_lut2(ref_y, src_y, ref_n, src_n, n, la, lb, s);
        if (luts) launch_write_luts(la, lb, luts, s);
        return launch_status("normalize(ratio)");
    }
    if (mode != HDRREG_NORM_HISTEQ) return fail(HDRREG_E_INVALID_ARG, "normalize: unknown mode");
    if (!workspace || ws_bytes < hdrreg_normalize_workspace_size(mode))
        return fail(HDRREG_E_WORKSPACE, "normalize(histeq): workspace of %zu bytes required",
                    hdrreg_normalize_workspace_size(mode));
    if (!luts) return fail(HDRREG_E_INVALID_ARG, "normalize(histeq): luts buffer required");
    uint32_t* hist = static_cast<uint32_t*>(workspace);
    cudaMemsetAsync(hist, 0, 2 * 256 * 4, s);
    launch_histograms(ref_y, src_y, n, hist, s);
    launch_histeq_luts(hist, n, luts, s);
    launch_lut2(ref_y, src_y, ref_n, src_n, n, LutSpec{luts, 1, 1}, LutSpec{luts + 256, 1, 1}, s);
    return launch_status("normalize(histeq)");
}

// ------------------------------------------------------------------- a2
size_t hdrreg_pyramid_bytes(int w, int h, int levels)
{
    size_t b = 0;
    for (int l = 1; l < levels; l++) b += (size_t)(w >> l) * (h >> l);
    return b;
}

hdrreg_status hdrreg_build_pyramid(const uint8_t* level0, int w, int h, int levels, uint8_t* pyr,
                                   void* stream)
{
    if (!level0 || (levels > 1 && !pyr)) return fail(HDRREG_E_INVALID_ARG, "pyramid: NULL");
    if (bad_dims(w, h)) return fail(HDRREG_E_INVALID_ARG, "pyramid: bad size");
    if (levels < 1 || levels > kMaxLevels)
        return fail(HDRREG_E_INVALID_ARG, "pyramid: levels must be in [1, %d]", kMaxLevels);
    if (levels == 1) return HDRREG_OK;
    uint8_t* lv[kMaxLevels] = {nullptr};
    size_t off = 0;
    for (int l = 1; l < levels; l++) {
        lv[l] = pyr + off;
        off += (size_t)(w >> l) * (h >> l);
    }
    launch_pyramid(level0, w, h, levels, LutSpec{nullptr, 1, 1}, nullptr, lv,
                   static_cast<cudaStream_t>(stream));
    return launch_status("pyramid");
}

// ---------------------------------------------------------------- a3-a5
hdrreg_status hdrreg_local_search(const uint8_t* ref_n, const uint8_t* src_n, int w, int h,
                                  const double* H, const hdrreg_params* p, int32_t* corner_xy,
                                  int32_t* match_xy, uint32_t* cost, uint8_t* valid, void* stream)
{
    hdrreg_status st = hdrreg_validate_params(p);
    if (st) return st;
    if (!ref_n || !src_n || !H || !corner_xy || !match_xy || !cost || !valid)
        return fail(HDRREG_E_INVALID_ARG, "local_search: NULL pointer");
    if (bad_dims(w, h)) return fail(HDRREG_E_INVALID_ARG, "local_search: bad size %dx%d", w, h);
    const SearchGeom g = make_geom(w, h, p);
    launch_local_search(ref_n, src_n, H, g, corner_xy, match_xy, cost, valid,
                        static_cast<cudaStream_t>(stream));
    return launch_status("local_search");
}

// -------------------------------------------------------------------- a6
size_t hdrreg_weed_workspace_size(int n) { return weed_ws_bytes(n); }

hdrreg_status hdrreg_weed(const int32_t* corner_xy, const int32_t* match_xy, const uint8_t* valid,
                          int n, int w, int h, const hdrreg_params* p, uint64_t seed,
                          int iter_begin, int iter_end, uint32_t* mask_bits, void* workspace,
                          size_t ws_bytes, void* stream)
{
    hdrreg_status st = hdrreg_validate_params(p);
    if (st) return st;
    if (n < 0 || n > (1 << 20)) return fail(HDRREG_E_INVALID_ARG, "weed: n out of range");
    if (n > 0 && (!corner_xy || !match_xy || !valid || !mask_bits))
        return fail(HDRREG_E_INVALID_ARG, "weed: NULL pointer");
    if (bad_dims(w, h)) return fail(HDRREG_E_INVALID_ARG, "weed: bad size");
    if (iter_begin < 0 || iter_end < iter_begin)
        return fail(HDRREG_E_INVALID_ARG, "weed: bad iteration range [%d, %d)", iter_begin,
                    iter_end);
    if (n == 0) return HDRREG_OK;
    if (!workspace || ws_bytes < weed_ws_bytes(n))
        return fail(HDRREG_E_WORKSPACE, "weed: workspace of %zu bytes required", weed_ws_bytes(n));
    launch_weed(corner_xy, match_xy, valid, n, w, h, p->weed_eps, p->weed_delta_min,
                p->weed_delta_div, seed, iter_begin, iter_end, mask_bits,
                weed_ws_carve(workspace, n), static_cast<cudaStream_t>(stream));
    return launch_status("weed");
}

// -------------------------------------------------------------------- a7
hdrreg_status hdrreg_fit_homography(const int32_t* corner_xy, const int32_t* match_xy,
                                    const uint32_t* mask_bits, int n, int w, int h,
                                    const double* H_prev, double* H_out, int32_t* status,
                                    void* stream)
{
    if (n < 0 || n > (1 << 20)) return fail(HDRREG_E_INVALID_ARG, "fit: n out of range");
    if (!H_prev || !H_out || (n > 0 && (!corner_xy || !match_xy || !mask_bits)))
        return fail(HDRREG_E_INVALID_ARG, "fit: NULL pointer");
    if (bad_dims(w, h)) return fail(HDRREG_E_INVALID_ARG, "fit: bad size");
    launch_fit(corner_xy, match_xy, mask_bits, n, w, h, H_prev, H_out, status,
               static_cast<cudaStream_t>(stream));
    return launch_status("fit");
}

int hdrreg_weed_fit_supported(int n) { return n >= 0 && n <= (1 << 20) && weed_level_fits(n); }

hdrreg_status hdrreg_weed_fit(const int32_t* corner_xy, const int32_t* match_xy,
                              const uint8_t* valid, int n, int w, int h, const hdrreg_params* p,
                              uint64_t seed, int iter_begin, int iter_end, uint32_t* mask_bits,
                              const double* H_prev, double* H_out, int32_t* status,
                              uint32_t* counter, void* stream)
{
    hdrreg_status st = hdrreg_validate_params(p);
    if (st) return st;
    if (n < 0 || n > (1 << 20)) return fail(HDRREG_E_INVALID_ARG, "weed_fit: n out of range");
    if (!mask_bits || !H_prev || !H_out || !counter || (n > 0 && (!corner_xy || !match_xy || !valid)))
        return fail(HDRREG_E_INVALID_ARG, "weed_fit: NULL pointer");
    if (bad_dims(w, h)) return fail(HDRREG_E_INVALID_ARG, "weed_fit: bad size");
    if (iter_begin < 0 || iter_end < iter_begin)
        return fail(HDRREG_E_INVALID_ARG, "weed_fit: bad iteration range [%d, %d)", iter_begin,
                    iter_end);
    if (!weed_level_fits(n))
        return fail(HDRREG_E_UNSUPPORTED,
                    "weed_fit: %d tiles do not fit the shared-memory plan (%zu bytes > %zu)", n,
                    weed_level_smem_bytes(n), kWeedLevelSmemMax);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (n > 0) cudaMemsetAsync(mask_bits, 0, (size_t)((n + 31) / 32) * 4, s);
    WeedLevelArgs a{corner_xy, match_xy, valid, n, w, h, p->weed_eps, p->weed_delta_min,
                    p->weed_delta_div, seed, iter_begin, iter_end, mask_bits, H_prev, H_out,
                    status, counter};
    launch_weed_level(a, s);
    return launch_status("weed_fit");
}

// -------------------------------------------------------------------- a8
size_t hdrreg_flow_workspace_size(int w, int h)
{
    if (bad_dims(w, h)) return 0;
    return flow_ws_bytes(w, h);
}

hdrreg_status hdrreg_flow_upsample(const uint8_t* guide_n, int w, int h, const int32_t* corner_xy,
                                   const int32_t* match_xy, const uint32_t* mask_bits, int n,
                                   const double* H, const hdrreg_params* p, float* flow_u,
                                   float* flow_v, void* workspace, size_t ws_bytes, void* stream)
{
    hdrreg_status st = hdrreg_validate_params(p);
    if (st) return st;
    if (!guide_n || !flow_u || !flow_v || (!p->propagate_full && !H))
        return fail(HDRREG_E_INVALID_ARG, "flow: NULL pointer");
    if (bad_dims(w, h)) return fail(HDRREG_E_INVALID_ARG, "flow: bad size");
    if (n != (w / p->tile) * (h / p->tile))
        return fail(HDRREG_E_INVALID_ARG, "flow: n (%d) must equal the tile count %d", n,
                    (w / p->tile) * (h / p->tile));
    if (n > 0 && (!corner_xy || !match_xy || !mask_bits))
        return fail(HDRREG_E_INVALID_ARG, "flow: NULL match arrays");
    if (!flow_supported(w, h))
        return fail(HDRREG_E_UNSUPPORTED, "flow: %dx%d exceeds the on-chip strip capacity", w, h);
    if (!workspace || ws_bytes < flow_ws_bytes(w, h))
        return fail(HDRREG_E_WORKSPACE, "flow: workspace of %zu bytes required",
                    flow_ws_bytes(w, h));
    FlowCorners fc{corner_xy, match_xy, mask_bits, H, w / p->tile, h / p->tile, p->tile,
                   p->propagate_full};
    launch_flow(guide_n, w, h, fc, p->sigma_s, p->sigma_r, p->dt_iters, p->flow_eps, flow_u,
                flow_v, w, workspace, static_cast<cudaStream_t>(stream));
    return launch_status("flow");
}

// -------------------------------------------------------------------- a9
hdrreg_status hdrreg_warp(const hdrreg_frame* src, int w, int h, const double* H,
                          const float* flow_u, const float* flow_v, const hdrreg_planes_f32* out,
                          uint8_t* clip_out, void* stream)
{
    if (!src || !src->y || !H || !flow_u || !flow_v || !out || !out->y)
        return fail(HDRREG_E_INVALID_ARG, "warp: NULL pointer");
    if (bad_dims(w, h)) return fail(HDRREG_E_INVALID_ARG, "warp: bad size");
    const bool chroma = src->u && src->v && out->u && out->v;
    if (chroma && ((w & 1) || (h & 1)))
        return fail(HDRREG_E_INVALID_ARG, "warp: YUV420 needs even width and height");
    launch_warp(src->y, chroma ? src->u : nullptr, chroma ? src->v : nullptr, w, h, H, flow_u,
                flow_v, w, out->y, chroma ? out->u : nullptr, chroma ? out->v : nullptr, clip_out,
                static_cast<cudaStream_t>(stream));
    return launch_status("warp");
}

// ---------------------------------------------------------------- a10-a11
static hdrreg_status merge_src_dev(const hdrreg_merge_src& m, int mode, bool chroma,
                                   MergeSrcDev& d)
{
    if (!m.y || !m.ref_n) return fail(HDRREG_E_INVALID_ARG, "merge: NULL source plane");
    if (chroma && (!m.u || !m.v)) return fail(HDRREG_E_INVALID_ARG, "merge: NULL chroma plane");
    if (m.ratio_num < 1 || m.ratio_den < 1)
        return fail(HDRREG_E_INVALID_ARG, "merge: ratio must be positive");
    if (mode == HDRREG_NORM_HISTEQ && !m.src_lut)
        return fail(HDRREG_E_INVALID_ARG, "merge: HISTEQ needs the source LUT");
    d.y = m.y;
    d.u = m.u;
    d.v = m.v;
    d.ref_n = m.ref_n;
    d.lut = m.src_lut;
    d.inv_ratio = (float)((double)m.ratio_den / (double)m.ratio_num);
    d.gain = m.ratio_num < m.ratio_den ? (float)((double)m.ratio_den / (double)m.ratio_num) : 1.f;
    d.mode = mode;
    d.clip = m.clip;
    d.clip_sign = 0;
    return HDRREG_OK;
}

hdrreg_status hdrreg_merge(const hdrreg_frame* ref, int w, int h, int nsrc,
                           const hdrreg_merge_src* srcs, const hdrreg_params* p,
                           const hdrreg_planes_f32* out, float* q_out, void* stream)
{
    hdrreg_status st = hdrreg_validate_params(p);
    if (st) return st;
    if (!ref || !ref->y || !out || !out->y || !srcs)
        return fail(HDRREG_E_INVALID_ARG, "merge: NULL pointer");
    if (nsrc < 1 || nsrc > kMaxSources)
        return fail(HDRREG_E_INVALID_ARG, "merge: nsrc must be in [1, %d]", kMaxSources);
    if (bad_dims(w, h)) return fail(HDRREG_E_INVALID_ARG, "merge: bad size");
    const bool chroma = ref->u && ref->v && out->u && out->v;
    if (chroma && ((w & 1) || (h & 1)))
        return fail(HDRREG_E_INVALID_ARG, "merge: YUV420 needs even width and height");
    MergeSrcDev d[kMaxSources];
    for (int k = 0; k < nsrc; k++)
        if ((st = merge_src_dev(srcs[k], p->norm_mode, chroma, d[k]))) return st;
    launch_merge(ref->y, chroma ? ref->u : nullptr, chroma ? ref->v : nullptr, w, h, nsrc, d,
                 p->ssim_sigma, p->we_sigma, out->y, chroma ? out->u : nullptr,
                 chroma ? out->v : nullptr, q_out, static_cast<cudaStream_t>(stream));
    return launch_status("merge");
}

// ------------------------------------------------------------ fused a1-a11
size_t hdrreg_register_merge_workspace_size(int w, int h, int nsrc, const hdrreg_params* p)
{
    if (!p || bad_dims(w, h) || nsrc < 1 || nsrc > kMaxSources) return 0;
    return FusedLayout(w, h, nsrc, p).total;
}

}  // extern "C"

namespace hdrreg {

// Argument checks of one fused call (everything but the workspace).
static hdrreg_status rm_validate(const hdrreg_frame* ref, int w, int h, int nsrc,
                                 const hdrreg_frame* srcs, const int* ratio_num,
                                 const int* ratio_den, const hdrreg_params* p,
                                 const hdrreg_planes_f32* out)
{
    hdrreg_status st = hdrreg_validate_params(p);
    if (st) return st;
    if (!ref || !ref->y || !srcs || !ratio_num || !ratio_den || !out || !out->y)
        return fail(HDRREG_E_INVALID_ARG, "register_merge: NULL pointer");
    if (nsrc < 1 || nsrc > kMaxSources)
        return fail(HDRREG_E_INVALID_ARG, "register_merge: nsrc must be in [1, %d]", kMaxSources);
    if (bad_dims(w, h)) return fail(HDRREG_E_INVALID_ARG, "register_merge: bad size %dx%d", w, h);
    const bool chroma = ref->u && ref->v && out->u && out->v;
    if (chroma && ((w & 1) || (h & 1)))
        return fail(HDRREG_E_INVALID_ARG, "register_merge: YUV420 needs even width and height");
    for (int k = 0; k < nsrc; k++) {
        if (!srcs[k].y || (chroma && (!srcs[k].u || !srcs[k].v)))
            return fail(HDRREG_E_INVALID_ARG, "register_merge: NULL source %d plane", k);
        if (ratio_num[k] < 1 || ratio_den[k] < 1)
            return fail(HDRREG_E_INVALID_ARG, "register_merge: ratio %d must be positive", k);
    }
    if (!flow_supported(w, h))
        return fail(HDRREG_E_UNSUPPORTED, "register_merge: %dx%d exceeds the flow strip capacity",
                    w, h);
    return HDRREG_OK;
}

// Where the stage-major batch keeps one stack's merge inputs until its merge launch:
// per source the normalized reference, the warped planes (clip flags in the luma's sign
// bit) and the equalization LUTs; rm_enqueue fills md.
struct StagedOut {
    uint8_t* refn[kMaxSources];
    float* wy[kMaxSources];
    float* wu[kMaxSources];
    float* wv[kMaxSources];
    uint8_t* luts;  // 512 bytes per source
    MergeSrcDev md[kMaxSources];
};

// Enqueue the whole path for one validated stack on stream s, using the workspace
// laid out by `lay`. With `so` the merge inputs go to so's buffers and the merge is left
// to the caller (so->md describes its sources).
static hdrreg_status rm_enqueue(const hdrreg_frame* ref, int w, int h, int nsrc,
                                const hdrreg_frame* srcs, const int* ratio_num,
                                const int* ratio_den, const hdrreg_params* p,
                                const FusedLayout& lay, void* workspace,
                                const hdrreg_planes_f32* out, hdrreg_diag* diag, cudaStream_t s,
                                StagedOut* so = nullptr)
{
    hdrreg_status st = HDRREG_OK;
    const bool chroma = ref->u && ref->v && out->u && out->v;
    uint8_t* base = static_cast<uint8_t*>(workspace);
    auto at = [&](size_t off) { return base + off; };
    int32_t* corner = reinterpret_cast<int32_t*>(at(lay.corner));
    int32_t* match = reinterpret_cast<int32_t*>(at(lay.match));
    uint32_t* cost = reinterpret_cast<uint32_t*>(at(lay.cost));
    uint8_t* valid = at(lay.valid);
    uint32_t* mask = reinterpret_cast<uint32_t*>(at(lay.mask));
    double* Hs = reinterpret_cast<double*>(at(lay.H));
    int32_t* fit_st = reinterpret_cast<int32_t*>(at(lay.fit_st));
    unsigned* done = reinterpret_cast<unsigned*>(at(lay.done));
    const WeedWs wws = weed_ws_carve(at(lay.weed), lay.n0);
    uint32_t* hist = reinterpret_cast<uint32_t*>(at(lay.hist));
    float* fu = reinterpret_cast<float*>(at(lay.fu));
    float* fv = reinterpret_cast<float*>(at(lay.fv));
    const int L = lay.L;
    const size_t npx = (size_t)w * h;
    MergeSrcDev md[kMaxSources];

    for (int k = 0; k < nsrc; k++) {
        // ---- a1 + a2: normalized level 0 (or an alias of the input) and the pyramids
        LutSpec lr{nullptr, 1, 1}, ls{nullptr, 1, 1};
        uint8_t* luts_k = so ? so->luts + 512 * k : at(lay.luts) + 512 * k;
        uint8_t* refn_k = so ? so->refn[k] : at(lay.refn[k]);
        bool ref_identity = true, src_identity = true;
        float gain = 1.f;
        if (p->norm_mode == HDRREG_NORM_RATIO) {
            if (ratio_num[k] > ratio_den[k]) {
                lr = LutSpec{nullptr, ratio_num[k], ratio_den[k]};
                ref_identity = false;
            } else if (ratio_num[k] < ratio_den[k]) {
                ls = LutSpec{nullptr, ratio_den[k], ratio_num[k]};
                src_identity = false;
                gain = (float)((double)ratio_den[k] / (double)ratio_num[k]);
            }
        } else {
            cudaMemsetAsync(hist, 0, 2 * 256 * 4, s);
            launch_histograms(ref->y, srcs[k].y, npx, hist, s);
            launch_histeq_luts(hist, npx, luts_k, s);
            lr = LutSpec{luts_k, 1, 1};
            ls = LutSpec{luts_k + 256, 1, 1};
            ref_identity = src_identity = false;
        }
        const uint8_t* ref0 = ref_identity ? ref->y : refn_k;
        const uint8_t* src0 = src_identity ? srcs[k].y : at(lay.src_lv[0]);
        {
            uint8_t* rl[kMaxLevels] = {nullptr};
            uint8_t* sl[kMaxLevels] = {nullptr};
            for (int l = 1; l < L; l++) {
                rl[l] = at(lay.ref_lv[l]);
                sl[l] = at(lay.src_lv[l]);
            }
            const uint8_t* ins[2] = {ref->y, srcs[k].y};
            const LutSpec luts[2] = {lr, ls};
            uint8_t* outs0[2] = {ref_identity ? nullptr : refn_k,
                                 src_identity ? nullptr : at(lay.src_lv[0])};
            uint8_t* const* lvs[2] = {rl, sl};
            launch_pyramid2(ins, w, h, L, luts, outs0, lvs, 2, s);
        }
        // ---- a3..a7 from the coarsest level to level 0
        launch_set_identity(Hs + 9 * L, s, done, kMaxLevels + 1);
        for (int l = L - 1; l >= 0; l--) {
            const int lw = w >> l, lh = h >> l;
            const uint8_t* rl = l == 0 ? ref0 : at(lay.ref_lv[l]);
            const uint8_t* sl = l == 0 ? src0 : at(lay.src_lv[l]);
            const SearchGeom g = make_geom(lw, lh, p);
            const int n = g.ntx * g.nty;
            if (l == 0 && lay.learned) {
                // learned level-0 search: network input at quarter resolution (level 2),
                // prediction per tile, SSD check with fallback to the full search
                launch_predictor_input(at(lay.ref_lv[2]), at(lay.src_lv[2]), lay.wq, lay.hq,
                                       Hs + 9, at(lay.xq), s);
                if (!cnn_infer(p->predictor, reinterpret_cast<const __nv_bfloat16*>(at(lay.xq)), 1,
                               lay.hq, lay.wq, reinterpret_cast<float*>(at(lay.pred)),
                               at(lay.cnn), reinterpret_cast<int*>(done + kMaxLevels), s))
                    return fail(HDRREG_E_UNSUPPORTED, "register_merge: tensor-core product not available");
                const PredSearch ps{reinterpret_cast<const float*>(at(lay.pred)), lay.pwo,
                                    p->predictor_refine, p->fallback_cost, at(lay.fellback)};
                launch_local_search(rl, sl, Hs + 9, g, corner, match, cost, valid, s, mask, &ps);
            } else {
                launch_local_search(rl, sl, Hs + 9 * (l + 1), g, corner, match, cost, valid, s,
                                    mask);  // also zeroes the level's mask words
            }
            if (weed_level_fits(n)) {
                WeedLevelArgs a{corner, match, valid, n, lw, lh, p->weed_eps, p->weed_delta_min,
                                p->weed_delta_div, p->weed_seed + (uint64_t)l, 0, p->weed_iters,
                                mask, Hs + 9 * (l + 1), Hs + 9 * l, fit_st + l, done + l};
                launch_weed_level(a, s);
            } else {
                launch_weed(corner, match, valid, n, lw, lh, p->weed_eps, p->weed_delta_min,
                            p->weed_delta_div, p->weed_seed + (uint64_t)l, 0, p->weed_iters,
                            mask, wws, s);
                launch_fit(corner, match, mask, n, lw, lh, Hs + 9 * (l + 1), Hs + 9 * l,
                           fit_st + l, s);
            }
        }
        // ---- a8: dense flow guided by the normalized reference
        const double* Hw = Hs;
        if (p->propagate_full) {
            launch_set_identity(Hs + 9 * (kMaxLevels + 1), s);
            Hw = Hs + 9 * (kMaxLevels + 1);
        }
        FlowCorners fc{corner, match, mask, Hs, w / p->tile, h / p->tile, p->tile,
                       p->propagate_full};
        launch_flow(ref0, w, h, fc, p->sigma_s, p->sigma_r, p->dt_iters, p->flow_eps, fu, fv,
                    flow_pitch(w), at(lay.flow), s);
        // ---- a9: warp the source frame
        float* wy = so ? so->wy[k] : reinterpret_cast<float*>(at(lay.wy[k]));
        float* wu = so ? so->wu[k] : reinterpret_cast<float*>(at(lay.wu[k]));
        float* wv = so ? so->wv[k] : reinterpret_cast<float*>(at(lay.wv[k]));
        // the merge alone reads the warped luma: its clip flags ride in the sign bit; the
        // exposure fusion reads the planes too, so there they get a plane of their own
        const bool clip_sign = p->output_mode == 0;
        uint8_t* clip = clip_sign ? nullptr : at(lay.clip[k]);
        launch_warp(srcs[k].y, chroma ? srcs[k].u : nullptr, chroma ? srcs[k].v : nullptr, w, h,
                    Hw, fu, fv, flow_pitch(w), wy, chroma ? wu : nullptr, chroma ? wv : nullptr,
                    clip, s, clip_sign);
        if (diag) {
            note_launch();
            k_diag<<<1, 256, 0, s>>>(Hs, valid, mask, lay.n0, fit_st, L,
                                     lay.learned ? at(lay.fellback) : nullptr,
                                     flow_error_word(at(lay.flow), w, h), diag + k);
        }
        md[k].y = wy;
        md[k].u = chroma ? wu : nullptr;
        md[k].v = chroma ? wv : nullptr;
        md[k].ref_n = ref0;
        md[k].lut = p->norm_mode == HDRREG_NORM_HISTEQ ? luts_k + 256 : nullptr;
        md[k].inv_ratio = (float)((double)ratio_den[k] / (double)ratio_num[k]);
        md[k].gain = gain;
        md[k].mode = p->norm_mode;
        md[k].clip = clip;
        md[k].clip_sign = clip_sign ? 1 : 0;
        if (so) so->md[k] = md[k];
        if ((st = launch_status("register_merge(register)"))) return st;
    }
    if (so) return HDRREG_OK;  // the caller merges
    // ---- a10 + a11 (with output_mode != 0 the merge also leaves the SSIM maps, which the
    //      exposure fusion of Sec. 2.5 then uses; its result replaces the merge's)
    float* qmaps = p->output_mode ? reinterpret_cast<float*>(at(lay.q)) : nullptr;
    launch_merge(ref->y, chroma ? ref->u : nullptr, chroma ? ref->v : nullptr, w, h, nsrc, md,
                 p->ssim_sigma, p->we_sigma, out->y, chroma ? out->u : nullptr,
                 chroma ? out->v : nullptr, qmaps, s);
    if (p->output_mode) {
        FuseSrcDev fs[kMaxSources];
        for (int k = 0; k < nsrc; k++)
            fs[k] = FuseSrcDev{md[k].y, md[k].u, md[k].v, qmaps + (size_t)k * w * h};
        launch_fuse(ref->y, chroma ? ref->u : nullptr, chroma ? ref->v : nullptr, w, h, nsrc, fs,
                    p->output_mode == 1, p->we_sigma, out->y, chroma ? out->u : nullptr,
                    chroma ? out->v : nullptr, at(lay.fuse), s);
    }
    return launch_status("register_merge(merge)");
}

// Streams and events of the batched call, created once per device on its first
// batched call and kept for the process lifetime.
struct LaneSet {
    cudaStream_t stream[HDRREG_MAX_LANES];
    cudaEvent_t fork, join[HDRREG_MAX_LANES];
    bool ready = false;
};

// The lane streams and events are shared by every batched call of a device: one
// batched enqueue at a time per process.
static std::mutex lane_enqueue_mu;

static hdrreg_status lane_set(LaneSet** out)
{
    static std::mutex mu;
    static std::map<int, LaneSet> sets;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(HDRREG_E_CUDA, "batch: cudaGetDevice: %s", cudaGetErrorString(e));
    std::lock_guard<std::mutex> lock(mu);
    LaneSet& ls = sets[dev];
    if (!ls.ready) {
        e = cudaEventCreateWithFlags(&ls.fork, cudaEventDisableTiming);
        for (int i = 0; i < HDRREG_MAX_LANES && e == cudaSuccess; i++) {
            e = cudaStreamCreateWithFlags(&ls.stream[i], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ls.join[i], cudaEventDisableTiming);
        }
        if (e != cudaSuccess)
            return fail(HDRREG_E_CUDA, "batch: creating lane streams: %s", cudaGetErrorString(e));
        ls.ready = true;
    }
    *out = &ls;
    return HDRREG_OK;
}

}  // namespace hdrreg

extern "C" {

hdrreg_status hdrreg_register_merge(const hdrreg_frame* ref, int w, int h, int nsrc,
                                    const hdrreg_frame* srcs, const int* ratio_num,
                                    const int* ratio_den, const hdrreg_params* p,
                                    void* workspace, size_t ws_bytes,
                                    const hdrreg_planes_f32* out, hdrreg_diag* diag,
                                    void* stream)
{
    hdrreg_status st = rm_validate(ref, w, h, nsrc, srcs, ratio_num, ratio_den, p, out);
    if (st) return st;
    const FusedLayout lay(w, h, nsrc, p);
    if (!workspace || ws_bytes < lay.total)
        return fail(HDRREG_E_WORKSPACE, "register_merge: workspace of %zu bytes required",
                    lay.total);
    return rm_enqueue(ref, w, h, nsrc, srcs, ratio_num, ratio_den, p, lay, workspace, out, diag,
                      static_cast<cudaStream_t>(stream));
}

hdrreg_status hdrreg_gemm_bf16(const void* A, int lda, const void* B, int ldb, int M, int N,
                               int K, float* C, int ldc, int32_t* status, void* stream)
{
    if (!A || !B || !C || !status) return fail(HDRREG_E_INVALID_ARG, "gemm: NULL pointer");
    if (M < 1 || N < 1 || K < 1 || lda < K || ldb < K || ldc < N)
        return fail(HDRREG_E_INVALID_ARG, "gemm: bad sizes M=%d N=%d K=%d lda=%d ldb=%d ldc=%d", M,
                    N, K, lda, ldb, ldc);
    if (!gemm_supported(A, lda, B, ldb))
        return fail(HDRREG_E_UNSUPPORTED,
                    "gemm: operands must be 16-byte aligned with lda, ldb multiples of 8");
    GemmEpi e{kEpiF32, C, nullptr, nullptr, ldc, 0};
    if (!launch_gemm_bf16(A, lda, B, ldb, M, N, K, 1, e, status, static_cast<cudaStream_t>(stream)))
        return fail(HDRREG_E_UNSUPPORTED, "gemm: tensor map creation failed");
    return launch_status("gemm_bf16");
}

hdrreg_status hdrreg_predictor_input(const uint8_t* ref_q, const uint8_t* src_q, int w, int h,
                                     const double* H, uint16_t* x_out, void* stream)
{
    if (!ref_q || !src_q || !H || !x_out)
        return fail(HDRREG_E_INVALID_ARG, "predictor_input: NULL pointer");
    if (bad_dims(w, h)) return fail(HDRREG_E_INVALID_ARG, "predictor_input: bad size %dx%d", w, h);
    launch_predictor_input(ref_q, src_q, w, h, H, x_out, static_cast<cudaStream_t>(stream));
    return launch_status("predictor_input");
}

hdrreg_status hdrreg_tile_labels(const int32_t* corner_xy, const int32_t* match_xy,
                                 const uint8_t* valid, int n, int w, int h, const double* H,
                                 float* label, void* stream)
{
    if (n < 0 || n > (1 << 20)) return fail(HDRREG_E_INVALID_ARG, "tile_labels: n out of range");
    if (n > 0 && (!corner_xy || !match_xy || !valid || !H || !label))
        return fail(HDRREG_E_INVALID_ARG, "tile_labels: NULL pointer");
    if (bad_dims(w, h)) return fail(HDRREG_E_INVALID_ARG, "tile_labels: bad size");
    launch_tile_labels(corner_xy, match_xy, valid, n, w, h, H, label,
                       static_cast<cudaStream_t>(stream));
    return launch_status("tile_labels");
}

hdrreg_status hdrreg_predictor_crops(const uint16_t* x_full, int wq, int hq, const float* label_full,
                                     const uint8_t* valid_full, int ntx, int nty,
                                     const int32_t* origins, int n, int crop_tiles,
                                     float label_bound, uint16_t* x_out, float* label_out,
                                     uint8_t* valid_out, void* stream)
{
    if (!x_full || !label_full || !valid_full || !origins || !x_out || !label_out || !valid_out)
        return fail(HDRREG_E_INVALID_ARG, "predictor_crops: NULL pointer");
    if (n < 1 || n > 65535 || crop_tiles < 1 || crop_tiles > 64 || bad_dims(wq, hq) || ntx < 1 ||
        nty < 1)
        return fail(HDRREG_E_INVALID_ARG, "predictor_crops: bad sizes");
    launch_predictor_crops(x_full, wq, hq, label_full, valid_full, ntx, nty, origins, n,
                           crop_tiles, label_bound, x_out, label_out, valid_out,
                           static_cast<cudaStream_t>(stream));
    return launch_status("predictor_crops");
}

hdrreg_status hdrreg_local_search_predicted(const uint8_t* ref_n, const uint8_t* src_n, int w,
                                            int h, const double* H, const hdrreg_params* p,
                                            const float* pred, int pred_rows, int pred_ld,
                                            int refine, uint32_t fallback_cost,
                                            int32_t* corner_xy, int32_t* match_xy,
                                            uint32_t* cost, uint8_t* valid, uint8_t* fell_back,
                                            void* stream)
{
    hdrreg_status st = hdrreg_validate_params(p);
    if (st) return st;
    if (!ref_n || !src_n || !H || !pred || !corner_xy || !match_xy || !cost || !valid)
        return fail(HDRREG_E_INVALID_ARG, "local_search_predicted: NULL pointer");
    if (bad_dims(w, h)) return fail(HDRREG_E_INVALID_ARG, "local_search_predicted: bad size");
    const SearchGeom g = make_geom(w, h, p);
    if (pred_ld < g.ntx || pred_rows < g.nty)
        return fail(HDRREG_E_INVALID_ARG,
                    "local_search_predicted: prediction grid %d x %d smaller than the %d x %d tiles",
                    pred_rows, pred_ld, g.nty, g.ntx);
    if (refine < 0 || refine > p->radius)
        return fail(HDRREG_E_INVALID_ARG, "local_search_predicted: refine must be in [0, radius]");
    const PredSearch ps{pred, pred_ld, refine, fallback_cost, fell_back};
    launch_local_search(ref_n, src_n, H, g, corner_xy, match_xy, cost, valid,
                        static_cast<cudaStream_t>(stream), nullptr, &ps);
    return launch_status("local_search_predicted");
}

static bool cnn_bad_dims(int n, int h, int w)
{
    return n < 1 || h < 8 || w < 8 || h > 4096 || w > 4096 || (long long)n * h * w > (1LL << 24);
}

size_t hdrreg_cnn_workspace_size(int n, int h, int w)
{
    return cnn_bad_dims(n, h, w) ? 0 : cnn_ws_bytes(n, h, w);
}

int hdrreg_cnn_out_dims(int h, int w, int* ho, int* wo)
{
    if (!ho || !wo || cnn_bad_dims(1, h, w)) return 1;
    cnn_out_dims(h, w, ho, wo);
    return 0;
}

hdrreg_status hdrreg_cnn_forward(const float* theta, const uint16_t* x, int n, int h, int w,
                                 float* out, void* workspace, size_t ws_bytes, int32_t* status,
                                 void* stream)
{
    if (!theta || !x || !out || !status) return fail(HDRREG_E_INVALID_ARG, "cnn_forward: NULL pointer");
    if (cnn_bad_dims(n, h, w))
        return fail(HDRREG_E_INVALID_ARG, "cnn_forward: bad batch %d x %d x %d", n, h, w);
    if (!workspace || ws_bytes < cnn_ws_bytes(n, h, w))
        return fail(HDRREG_E_WORKSPACE, "cnn_forward: workspace of %zu bytes required",
                    cnn_ws_bytes(n, h, w));
    if (!cnn_forward(theta, reinterpret_cast<const __nv_bfloat16*>(x), n, h, w, out, workspace,
                     status, static_cast<cudaStream_t>(stream)))
        return fail(HDRREG_E_UNSUPPORTED, "cnn_forward: tensor-core product not available");
    return launch_status("cnn_forward");
}

size_t hdrreg_cnn_infer_workspace_size(int n, int h, int w)
{
    return cnn_bad_dims(n, h, w) ? 0 : cnn_infer_ws_bytes(n, h, w);
}

hdrreg_status hdrreg_cnn_infer(const float* theta, const uint16_t* x, int n, int h, int w,
                               float* out, void* workspace, size_t ws_bytes, int32_t* status,
                               void* stream)
{
    if (!theta || !x || !out || !status) return fail(HDRREG_E_INVALID_ARG, "cnn_infer: NULL pointer");
    if (cnn_bad_dims(n, h, w))
        return fail(HDRREG_E_INVALID_ARG, "cnn_infer: bad batch %d x %d x %d", n, h, w);
    if (!workspace || ws_bytes < cnn_infer_ws_bytes(n, h, w))
        return fail(HDRREG_E_WORKSPACE, "cnn_infer: workspace of %zu bytes required",
                    cnn_infer_ws_bytes(n, h, w));
    if (((uintptr_t)x & 3u) || ((uintptr_t)workspace & 255u))
        return fail(HDRREG_E_INVALID_ARG, "cnn_infer: x must be 4-byte, workspace 256-byte aligned");
    if (!cnn_infer(theta, reinterpret_cast<const __nv_bfloat16*>(x), n, h, w, out, workspace,
                   status, static_cast<cudaStream_t>(stream)))
        return fail(HDRREG_E_UNSUPPORTED, "cnn_infer: no convolution kernel for a layer");
    return launch_status("cnn_infer");
}

hdrreg_status hdrreg_cnn_backward(const float* theta, const uint16_t* x, int n, int h, int w,
                                  const float* out, const float* label, const uint8_t* valid,
                                  float* grad, float* loss, void* workspace, size_t ws_bytes,
                                  int32_t* status, void* stream)
{
    if (!theta || !x || !out || !label || !valid || !grad || !loss || !status)
        return fail(HDRREG_E_INVALID_ARG, "cnn_backward: NULL pointer");
    if (cnn_bad_dims(n, h, w))
        return fail(HDRREG_E_INVALID_ARG, "cnn_backward: bad batch %d x %d x %d", n, h, w);
    if (!workspace || ws_bytes < cnn_ws_bytes(n, h, w))
        return fail(HDRREG_E_WORKSPACE, "cnn_backward: workspace of %zu bytes required",
                    cnn_ws_bytes(n, h, w));
    if (!cnn_backward(theta, reinterpret_cast<const __nv_bfloat16*>(x), n, h, w, out, label, valid,
                      grad, loss, workspace, status, static_cast<cudaStream_t>(stream)))
        return fail(HDRREG_E_UNSUPPORTED, "cnn_backward: tensor-core product not available");
    return launch_status("cnn_backward");
}

hdrreg_status hdrreg_cnn_activation(const void* workspace, int n, int h, int w, int layer,
                                    const uint16_t** ptr, int* rows, int* cols)
{
    if (!workspace || !ptr || !rows || !cols)
        return fail(HDRREG_E_INVALID_ARG, "cnn_activation: NULL pointer");
    if (cnn_bad_dims(n, h, w))
        return fail(HDRREG_E_INVALID_ARG, "cnn_activation: bad batch %d x %d x %d", n, h, w);
    const void* p = cnn_activation(workspace, n, h, w, layer, rows, cols);
    if (!p) return fail(HDRREG_E_INVALID_ARG, "cnn_activation: layer %d stores no activation", layer);
    *ptr = static_cast<const uint16_t*>(p);
    return HDRREG_OK;
}

hdrreg_status hdrreg_cnn_adam(float* theta, float* m, float* v, const float* grad, int step,
                              float lr, void* stream)
{
    if (!theta || !m || !v || !grad) return fail(HDRREG_E_INVALID_ARG, "cnn_adam: NULL pointer");
    if (step < 1 || !(lr > 0)) return fail(HDRREG_E_INVALID_ARG, "cnn_adam: step >= 1, lr > 0");
    cnn_adam(theta, m, v, grad, step, lr, static_cast<cudaStream_t>(stream));
    return launch_status("cnn_adam");
}

size_t hdrreg_register_merge_batch_workspace_size(int w, int h, int nsrc, int lanes,
                                                  const hdrreg_params* p)
{
    if (!p || bad_dims(w, h) || nsrc < 1 || nsrc > kMaxSources || lanes < 1 ||
        lanes > HDRREG_MAX_LANES)
        return 0;
    return (size_t)lanes * align_up(FusedLayout(w, h, nsrc, p).total, 256);
}

hdrreg_status hdrreg_register_merge_batch(const hdrreg_stack* stacks, int count, int w, int h,
                                          int nsrc, int lanes, const hdrreg_params* p,
                                          void* workspace, size_t ws_bytes, void* stream)
{
    if (count < 0 || (count > 0 && !stacks))
        return fail(HDRREG_E_INVALID_ARG, "register_merge_batch: bad stack array");
    if (lanes < 1 || lanes > HDRREG_MAX_LANES)
        return fail(HDRREG_E_INVALID_ARG, "register_merge_batch: lanes must be in [1, %d]",
                    HDRREG_MAX_LANES);
    for (int i = 0; i < count; i++) {
        const hdrreg_stack& k = stacks[i];
        hdrreg_status st =
            rm_validate(k.ref, w, h, nsrc, k.srcs, k.ratio_num, k.ratio_den, p, &k.out);
        if (st) return fail(st, "register_merge_batch: stack %d: %s", i, hdrreg_last_error());
    }
    const size_t per = align_up(FusedLayout(w, h, nsrc, p).total, 256);
    if (!workspace || ws_bytes < per * lanes)
        return fail(HDRREG_E_WORKSPACE, "register_merge_batch: workspace of %zu bytes required",
                    per * lanes);
    if (count == 0) return HDRREG_OK;
    const FusedLayout lay(w, h, nsrc, p);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int used = count < lanes ? count : lanes;
    if (used == 1) {
        for (int i = 0; i < count; i++) {
            const hdrreg_stack& k = stacks[i];
            hdrreg_status st = rm_enqueue(k.ref, w, h, nsrc, k.srcs, k.ratio_num, k.ratio_den, p,
                                          lay, workspace, &k.out, k.diag, s);
            if (st) return st;
        }
        return HDRREG_OK;
    }
    LaneSet* ls = nullptr;
    hdrreg_status st = lane_set(&ls);
    if (st) return st;
    std::lock_guard<std::mutex> lock(lane_enqueue_mu);
    cudaError_t e = cudaEventRecord(ls->fork, s);
    for (int j = 0; j < used && e == cudaSuccess; j++) e = cudaStreamWaitEvent(ls->stream[j], ls->fork, 0);
    if (e != cudaSuccess)
        return fail(HDRREG_E_CUDA, "register_merge_batch: fork: %s", cudaGetErrorString(e));
    for (int i = 0; i < count; i++) {
        const int j = i % used;
        const hdrreg_stack& k = stacks[i];
        st = rm_enqueue(k.ref, w, h, nsrc, k.srcs, k.ratio_num, k.ratio_den, p, lay,
                        static_cast<uint8_t*>(workspace) + per * j, &k.out, k.diag,
                        ls->stream[j]);
        if (st) break;
    }
    for (int j = 0; j < used; j++) {  // join every lane, also after an error
        cudaError_t e1 = cudaEventRecord(ls->join[j], ls->stream[j]);
        cudaError_t e2 = cudaStreamWaitEvent(s, ls->join[j], 0);
        if (!st && (e1 != cudaSuccess || e2 != cudaSuccess))
            st = fail(HDRREG_E_CUDA, "register_merge_batch: join: %s",
                      cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
    }
    return st;
}

// -------------------------------------------------------------------- f1
size_t hdrreg_fuse_workspace_size(int w, int h, int nsrc, int chroma)
{
    if (bad_dims(w, h) || nsrc < 1 || nsrc > kMaxSources) return 0;
    return fuse_ws_bytes(w, h, nsrc + 1, chroma != 0);
}

hdrreg_status hdrreg_fuse(const hdrreg_frame* ref, int w, int h, int nsrc,
                          const hdrreg_fuse_src* srcs, int use_contrast, double we_sigma,
                          hdrreg_planes_f32* out, void* workspace, size_t ws_bytes, void* stream)
{
    if (!ref || !ref->y || !srcs || !out || !out->y)
        return fail(HDRREG_E_INVALID_ARG, "fuse: NULL pointer");
    if (bad_dims(w, h)) return fail(HDRREG_E_INVALID_ARG, "fuse: bad size %dx%d", w, h);
    if (nsrc < 1 || nsrc > kMaxSources)
        return fail(HDRREG_E_INVALID_ARG, "fuse: nsrc must be in [1, %d]", kMaxSources);
    if (!(we_sigma > 0)) return fail(HDRREG_E_INVALID_ARG, "fuse: we_sigma must be > 0");
    const bool chroma = ref->u && ref->v && out->u && out->v;
    if (chroma && ((w & 1) || (h & 1)))
        return fail(HDRREG_E_INVALID_ARG, "fuse: YUV420 needs even width and height");
    FuseSrcDev fs[kMaxSources];
    for (int k = 0; k < nsrc; k++) {
        if (!srcs[k].y || !srcs[k].q || (chroma && (!srcs[k].u || !srcs[k].v)))
            return fail(HDRREG_E_INVALID_ARG, "fuse: NULL plane of source %d", k);
        fs[k] = FuseSrcDev{srcs[k].y, srcs[k].u, srcs[k].v, srcs[k].q};
    }
    const size_t need = fuse_ws_bytes(w, h, nsrc + 1, chroma);
    if (!workspace || ws_bytes < need)
        return fail(HDRREG_E_WORKSPACE, "fuse: workspace of %zu bytes required", need);
    launch_fuse(ref->y, chroma ? ref->u : nullptr, chroma ? ref->v : nullptr, w, h, nsrc, fs,
                use_contrast != 0, we_sigma, out->y, chroma ? out->u : nullptr,
                chroma ? out->v : nullptr, workspace, static_cast<cudaStream_t>(stream));
    return launch_status("fuse");
}

// Per-lane layout of the host-staged batch: the fused workspace, then device copies of
// one stack's input planes, its FP32 output planes and its diagnostics.
struct HostStage {
    size_t fused, in_y[kMaxSources + 1], in_u[kMaxSources + 1], in_v[kMaxSources + 1];
    size_t out_y, out_u, out_v, diag, total;
    HostStage(int w, int h, int nsrc, const hdrreg_params* p)
    {
        Layout L;
        fused = L.add(FusedLayout(w, h, nsrc, p).total);
        const size_t luma = (size_t)w * h, chr = (size_t)(w / 2) * (h / 2);
        for (int k = 0; k <= nsrc; k++) {
            in_y[k] = L.add(luma);
            in_u[k] = L.add(chr);
            in_v[k] = L.add(chr);
        }
        out_y = L.add(luma * 4);
        out_u = L.add(chr * 4);
        out_v = L.add(chr * 4);
        diag = L.add(sizeof(hdrreg_diag) * nsrc);
        total = align_up(L.total, 256);
    }
};

size_t hdrreg_register_merge_host_workspace_size(int w, int h, int nsrc, int lanes,
                                                 const hdrreg_params* p)
{
    if (!p || hdrreg_validate_params(p) || bad_dims(w, h) || nsrc < 1 || nsrc > kMaxSources ||
        lanes < 1 || lanes > HDRREG_MAX_LANES)
        return 0;
    return HostStage(w, h, nsrc, p).total * lanes;
}

hdrreg_status hdrreg_register_merge_host(const hdrreg_stack* stacks, int count, int w, int h,
                                         int nsrc, int lanes, const hdrreg_params* p,
                                         void* workspace, size_t ws_bytes, void* stream)
{
    if (count < 0 || (count > 0 && !stacks))
        return fail(HDRREG_E_INVALID_ARG, "register_merge_host: bad stack array");
    if (lanes < 1 || lanes > HDRREG_MAX_LANES)
        return fail(HDRREG_E_INVALID_ARG, "register_merge_host: lanes must be in [1, %d]",
                    HDRREG_MAX_LANES);
    for (int i = 0; i < count; i++) {
        const hdrreg_stack& k = stacks[i];
        hdrreg_status st =
            rm_validate(k.ref, w, h, nsrc, k.srcs, k.ratio_num, k.ratio_den, p, &k.out);
        if (st) return fail(st, "register_merge_host: stack %d: %s", i, hdrreg_last_error());
    }
    const HostStage hs(w, h, nsrc, p);
    if (!workspace || ws_bytes < hs.total * lanes)
        return fail(HDRREG_E_WORKSPACE, "register_merge_host: workspace of %zu bytes required",
                    hs.total * lanes);
    if (count == 0) return HDRREG_OK;
    const FusedLayout lay(w, h, nsrc, p);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int used = count < lanes ? count : lanes;
    LaneSet* ls = nullptr;
    hdrreg_status st = lane_set(&ls);
    if (st) return st;
    const size_t luma = (size_t)w * h, chr = (size_t)(w / 2) * (h / 2);
    std::lock_guard<std::mutex> lock(lane_enqueue_mu);
    cudaError_t e = cudaEventRecord(ls->fork, s);
    for (int j = 0; j < used && e == cudaSuccess; j++) e = cudaStreamWaitEvent(ls->stream[j], ls->fork, 0);
    if (e != cudaSuccess)
        return fail(HDRREG_E_CUDA, "register_merge_host: fork: %s", cudaGetErrorString(e));
    for (int i = 0; i < count && !st; i++) {
        const int j = i % used;
        const hdrreg_stack& k = stacks[i];
        cudaStream_t q = ls->stream[j];
        uint8_t* lb = static_cast<uint8_t*>(workspace) + hs.total * j;
        const bool chroma = k.ref->u && k.ref->v && k.out.u && k.out.v;
        hdrreg_frame dref, dsrc[kMaxSources];
        auto put = [&](size_t off, const uint8_t* host, size_t n) -> const uint8_t* {
            if (!host) return nullptr;
            if (e == cudaSuccess) e = cudaMemcpyAsync(lb + off, host, n, cudaMemcpyHostToDevice, q);
            return lb + off;
        };
        dref.y = put(hs.in_y[0], k.ref->y, luma);
        dref.u = chroma ? put(hs.in_u[0], k.ref->u, chr) : nullptr;
        dref.v = chroma ? put(hs.in_v[0], k.ref->v, chr) : nullptr;
        for (int m = 0; m < nsrc; m++) {
            dsrc[m].y = put(hs.in_y[m + 1], k.srcs[m].y, luma);
            dsrc[m].u = chroma ? put(hs.in_u[m + 1], k.srcs[m].u, chr) : nullptr;
            dsrc[m].v = chroma ? put(hs.in_v[m + 1], k.srcs[m].v, chr) : nullptr;
        }
        if (e != cudaSuccess) {
            st = fail(HDRREG_E_CUDA, "register_merge_host: copy in: %s", cudaGetErrorString(e));
            break;
        }
        const hdrreg_planes_f32 dout{reinterpret_cast<float*>(lb + hs.out_y),
                                     chroma ? reinterpret_cast<float*>(lb + hs.out_u) : nullptr,
                                     chroma ? reinterpret_cast<float*>(lb + hs.out_v) : nullptr};
        hdrreg_diag* ddiag = reinterpret_cast<hdrreg_diag*>(lb + hs.diag);
        st = rm_enqueue(&dref, w, h, nsrc, dsrc, k.ratio_num, k.ratio_den, p, lay, lb + hs.fused,
                        &dout, ddiag, q);
        if (st) break;
        e = cudaMemcpyAsync(k.out.y, dout.y, luma * 4, cudaMemcpyDeviceToHost, q);
        if (chroma && e == cudaSuccess)
            e = cudaMemcpyAsync(k.out.u, dout.u, chr * 4, cudaMemcpyDeviceToHost, q);
        if (chroma && e == cudaSuccess)
            e = cudaMemcpyAsync(k.out.v, dout.v, chr * 4, cudaMemcpyDeviceToHost, q);
        if (k.diag && e == cudaSuccess)
            e = cudaMemcpyAsync(k.diag, ddiag, sizeof(hdrreg_diag) * nsrc, cudaMemcpyDeviceToHost, q);
        if (e != cudaSuccess)
            st = fail(HDRREG_E_CUDA, "register_merge_host: copy out: %s", cudaGetErrorString(e));
    }
    for (int j = 0; j < used; j++) {  // join every lane, also after an error
        cudaError_t e1 = cudaEventRecord(ls->join[j], ls->stream[j]);
        cudaError_t e2 = cudaStreamWaitEvent(s, ls->join[j], 0);
        if (!st && (e1 != cudaSuccess || e2 != cudaSuccess))
            st = fail(HDRREG_E_CUDA, "register_merge_host: join: %s",
                      cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
    }
    return st;
}

// Lane plan of a multi-shape batch: longest first onto the least-loaded lane; per lane
// the workspace of its largest stack (offsets into one buffer).
struct MultiPlan {
    std::vector<int> lane_of;
    std::vector<size_t> lane_off;
    size_t total = 0;
    int used = 0;
};

static MultiPlan plan_multi(const hdrreg_stack_ex* st, int count, int lanes)
{
    MultiPlan mp;
    mp.lane_of.assign(count, 0);
    std::vector<int> order(count);
    for (int i = 0; i < count; i++) order[i] = i;
    auto work = [&](int i) { return (double)st[i].w * st[i].h * st[i].nsrc; };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work(a) > work(b); });
    const int L = count < lanes ? count : lanes;
    std::vector<double> load(L, 0.0);
    std::vector<size_t> need(L, 0);
    for (int i : order) {
        int best = 0;
        for (int j = 1; j < L; j++)
            if (load[j] < load[best]) best = j;
        mp.lane_of[i] = best;
        load[best] += work(i);
        const size_t b = align_up(FusedLayout(st[i].w, st[i].h, st[i].nsrc, st[i].p).total, 256);
        need[best] = need[best] > b ? need[best] : b;
    }
    mp.lane_off.assign(L, 0);
    for (int j = 0; j < L; j++) {
        mp.lane_off[j] = mp.total;
        mp.total += need[j];
    }
    mp.used = L;
    return mp;
}

size_t hdrreg_register_merge_multi_workspace_size(const hdrreg_stack_ex* stacks, int count,
                                                  int lanes)
{
    if (!stacks || count < 1 || lanes < 1 || lanes > HDRREG_MAX_LANES) return 0;
    for (int i = 0; i < count; i++)
        if (!stacks[i].p || bad_dims(stacks[i].w, stacks[i].h) || stacks[i].nsrc < 1 ||
            stacks[i].nsrc > kMaxSources)
            return 0;
    return plan_multi(stacks, count, lanes).total;
}

hdrreg_status hdrreg_register_merge_multi(const hdrreg_stack_ex* stacks, int count, int lanes,
                                          void* workspace, size_t ws_bytes, void* stream)
{
    if (count < 0 || (count > 0 && !stacks))
        return fail(HDRREG_E_INVALID_ARG, "register_merge_multi: bad stack array");
    if (lanes < 1 || lanes > HDRREG_MAX_LANES)
        return fail(HDRREG_E_INVALID_ARG, "register_merge_multi: lanes must be in [1, %d]",
                    HDRREG_MAX_LANES);
    for (int i = 0; i < count; i++) {
        const hdrreg_stack_ex& k = stacks[i];
        hdrreg_status st = rm_validate(k.s.ref, k.w, k.h, k.nsrc, k.s.srcs, k.s.ratio_num,
                                       k.s.ratio_den, k.p, &k.s.out);
        if (st) return fail(st, "register_merge_multi: stack %d: %s", i, hdrreg_last_error());
    }
    if (count == 0) return HDRREG_OK;
    const MultiPlan mp = plan_multi(stacks, count, lanes);
    if (!workspace || ws_bytes < mp.total)
        return fail(HDRREG_E_WORKSPACE, "register_merge_multi: workspace of %zu bytes required",
                    mp.total);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint8_t* base = static_cast<uint8_t*>(workspace);
    auto run = [&](int i, cudaStream_t q) {
        const hdrreg_stack_ex& k = stacks[i];
        const FusedLayout lay(k.w, k.h, k.nsrc, k.p);
        return rm_enqueue(k.s.ref, k.w, k.h, k.nsrc, k.s.srcs, k.s.ratio_num, k.s.ratio_den, k.p,
                          lay, base + mp.lane_off[mp.lane_of[i]], &k.s.out, k.s.diag, q);
    };
    if (mp.used == 1) {
        for (int i = 0; i < count; i++) {
            hdrreg_status st = run(i, s);
            if (st) return st;
        }
        return HDRREG_OK;
    }
    LaneSet* ls = nullptr;
    hdrreg_status st = lane_set(&ls);
    if (st) return st;
    std::lock_guard<std::mutex> lock(lane_enqueue_mu);
    cudaError_t e = cudaEventRecord(ls->fork, s);
    for (int j = 0; j < mp.used && e == cudaSuccess; j++)
        e = cudaStreamWaitEvent(ls->stream[j], ls->fork, 0);
    if (e != cudaSuccess)
        return fail(HDRREG_E_CUDA, "register_merge_multi: fork: %s", cudaGetErrorString(e));
    for (int i = 0; i < count && !st; i++) st = run(i, ls->stream[mp.lane_of[i]]);
    for (int j = 0; j < mp.used; j++) {
        cudaError_t e1 = cudaEventRecord(ls->join[j], ls->stream[j]);
        cudaError_t e2 = cudaStreamWaitEvent(s, ls->join[j], 0);
        if (!st && (e1 != cudaSuccess || e2 != cudaSuccess))
            st = fail(HDRREG_E_CUDA, "register_merge_multi: join: %s",
                      cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
    }
    return st;
}

}  // extern "C"

namespace hdrreg {

// Per-stack blocks of the stage-major batch: the merge inputs of every source.
struct StagedPlan {
    MultiPlan mp;
    std::vector<size_t> off;  // per stack: start of its block (after the lane workspaces)
    size_t total = 0;
};

static size_t staged_block(int w, int h, int nsrc)
{
    const size_t cpx = (size_t)(w / 2) * (h / 2);
    return (size_t)nsrc * (align_up((size_t)w * h * 4, 256) + 2 * align_up(cpx * 4, 256) +
                           align_up((size_t)w * h, 256)) + 512 * (size_t)nsrc;
}

static StagedPlan plan_staged(const hdrreg_stack_ex* st, int count, int lanes)
{
    StagedPlan sp;
    sp.mp = plan_multi(st, count, lanes);
    sp.total = sp.mp.total;
    sp.off.assign(count, 0);
    for (int i = 0; i < count; i++) {
        sp.off[i] = sp.total;
        sp.total += align_up(staged_block(st[i].w, st[i].h, st[i].nsrc), 256);
    }
    return sp;
}

static StagedOut staged_out(uint8_t* b, int w, int h, int nsrc)
{
    StagedOut so{};
    const size_t cpx = (size_t)(w / 2) * (h / 2);
    for (int k = 0; k < nsrc; k++) {
        so.wy[k] = reinterpret_cast<float*>(b);
        b += align_up((size_t)w * h * 4, 256);
        so.wu[k] = reinterpret_cast<float*>(b);
        b += align_up(cpx * 4, 256);
        so.wv[k] = reinterpret_cast<float*>(b);
        b += align_up(cpx * 4, 256);
        so.refn[k] = b;
        b += align_up((size_t)w * h, 256);
    }
    so.luts = b;
    return so;
}

}  // namespace hdrreg

extern "C" {

size_t hdrreg_register_merge_staged_workspace_size(const hdrreg_stack_ex* stacks, int count,
                                                   int lanes)
{
    if (!hdrreg_register_merge_multi_workspace_size(stacks, count, lanes)) return 0;
    return plan_staged(stacks, count, lanes).total;
}

hdrreg_status hdrreg_register_merge_staged(const hdrreg_stack_ex* stacks, int count, int lanes,
                                           void* workspace, size_t ws_bytes, void* stream)
{
    if (count < 0 || (count > 0 && !stacks))
        return fail(HDRREG_E_INVALID_ARG, "register_merge_staged: bad stack array");
    if (lanes < 1 || lanes > HDRREG_MAX_LANES)
        return fail(HDRREG_E_INVALID_ARG, "register_merge_staged: lanes must be in [1, %d]",
                    HDRREG_MAX_LANES);
    for (int i = 0; i < count; i++) {
        const hdrreg_stack_ex& k = stacks[i];
        hdrreg_status st = rm_validate(k.s.ref, k.w, k.h, k.nsrc, k.s.srcs, k.s.ratio_num,
                                       k.s.ratio_den, k.p, &k.s.out);
        if (st) return fail(st, "register_merge_staged: stack %d: %s", i, hdrreg_last_error());
        if (k.p->output_mode != 0)
            return fail(HDRREG_E_UNSUPPORTED,
                        "register_merge_staged: stack %d asks for the exposure fusion", i);
    }
    if (count == 0) return HDRREG_OK;
    const StagedPlan sp = plan_staged(stacks, count, lanes);
    if (!workspace || ws_bytes < sp.total)
        return fail(HDRREG_E_WORKSPACE, "register_merge_staged: workspace of %zu bytes required",
                    sp.total);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint8_t* base = static_cast<uint8_t*>(workspace);
    std::vector<StagedOut> so(count);
    for (int i = 0; i < count; i++)
        so[i] = staged_out(base + sp.off[i], stacks[i].w, stacks[i].h, stacks[i].nsrc);
    auto run = [&](int i, cudaStream_t q) {
        const hdrreg_stack_ex& k = stacks[i];
        const FusedLayout lay(k.w, k.h, k.nsrc, k.p);
        return rm_enqueue(k.s.ref, k.w, k.h, k.nsrc, k.s.srcs, k.s.ratio_num, k.s.ratio_den, k.p,
                          lay, base + sp.mp.lane_off[sp.mp.lane_of[i]], &k.s.out, k.s.diag, q,
                          &so[i]);
    };
    hdrreg_status st = HDRREG_OK;
    if (sp.mp.used == 1) {
        for (int i = 0; i < count && !st; i++) st = run(i, s);
    } else {
        LaneSet* ls = nullptr;
        if ((st = lane_set(&ls))) return st;
        std::lock_guard<std::mutex> lock(lane_enqueue_mu);
        cudaError_t e = cudaEventRecord(ls->fork, s);
        for (int j = 0; j < sp.mp.used && e == cudaSuccess; j++)
            e = cudaStreamWaitEvent(ls->stream[j], ls->fork, 0);
        if (e != cudaSuccess)
            return fail(HDRREG_E_CUDA, "register_merge_staged: fork: %s", cudaGetErrorString(e));
        for (int i = 0; i < count && !st; i++) st = run(i, ls->stream[sp.mp.lane_of[i]]);
        for (int j = 0; j < sp.mp.used; j++) {
            cudaError_t e1 = cudaEventRecord(ls->join[j], ls->stream[j]);
            cudaError_t e2 = cudaStreamWaitEvent(s, ls->join[j], 0);
            if (!st && (e1 != cudaSuccess || e2 != cudaSuccess))
                st = fail(HDRREG_E_CUDA, "register_merge_staged: join: %s",
                          cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
        }
    }
    if (st) return st;
    // every stack's merge in persistent launches over all their tiles
    std::vector<MergeJob> jobs(count);
    for (int i = 0; i < count; i++) {
        const hdrreg_stack_ex& k = stacks[i];
        const bool chroma = k.s.ref->u && k.s.ref->v && k.s.out.u && k.s.out.v;
        MergeJob& J = jobs[i];
        J.ref_y = k.s.ref->y;
        J.ref_u = chroma ? k.s.ref->u : nullptr;
        J.ref_v = chroma ? k.s.ref->v : nullptr;
        J.w = k.w;
        J.h = k.h;
        J.nsrc = k.nsrc;
        for (int q = 0; q < k.nsrc; q++) J.srcs[q] = so[i].md[q];
        J.ssim_sigma = k.p->ssim_sigma;
        J.we_sigma = k.p->we_sigma;
        J.oy = k.s.out.y;
        J.ou = chroma ? k.s.out.u : nullptr;
        J.ov = chroma ? k.s.out.v : nullptr;
    }
    launch_merge_many(jobs.data(), count, s);
    return launch_status("register_merge_staged(merge)");
}

}  // extern "C"
