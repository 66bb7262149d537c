// Internal declarations of the hdrreg CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hdrreg.h"

namespace hdrreg {

// ---------------------------------------------------------------- host errors
void set_error(const char* fmt, ...);
hdrreg_status fail(hdrreg_status st, const char* fmt, ...);
hdrreg_status launch_status(const char* what);
void note_launch();                                  // counts kernels this library enqueues
void ensure_smem(const void* kernel, size_t bytes);  // raise the dynamic smem limit once

constexpr int kMaxLevels = 8;
constexpr int kSsimRadius = 5;

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// ----------------------------------------------------- binary64, one rounding
// Every FP64 step whose result decides an integer (search centre, inlier flag)
// or feeds the level homography is written with explicit round-to-nearest
// intrinsics, so the compiler cannot contract a*b+c into an FMA and the value
// is the IEEE result of the written order.
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double ddiv(double a, double b) { return __ddiv_rn(a, b); }

// normalized coordinate of Eq. 3: (2v - (extent - 1)) / w
__device__ __forceinline__ double norm_coord(int v, int extent, double W)
{
    return ddiv((double)(2 * v - (extent - 1)), W);
}

// H (reference -> source, normalized) applied to pixel (x, y) of a w x h level;
// returns the source position in pixels of that level. True if D > 0.
__device__ inline bool project_px(const double* H, int x, int y, int w, int h, double& xs,
                                  double& ys)
{
    const double W = (double)w;
    const double xn = norm_coord(x, w, W);
    const double yn = norm_coord(y, h, W);
    const double X = dadd(dadd(dmul(H[0], xn), dmul(H[1], yn)), H[2]);
    const double Y = dadd(dadd(dmul(H[3], xn), dmul(H[4], yn)), H[5]);
    const double D = dadd(dadd(dmul(H[6], xn), dmul(H[7], yn)), H[8]);
    const double xsn = ddiv(X, D);
    const double ysn = ddiv(Y, D);
    xs = dmul(dadd(dmul(xsn, W), (double)(w - 1)), 0.5);
    ys = dmul(dadd(dmul(ysn, W), (double)(h - 1)), 0.5);
    return D > 0.0;
}

// Rounded search centre of Eq. 3, clamped into the level; the corner itself if
// the projection is unusable.
__device__ inline void search_center(const double* H, int x, int y, int w, int h, int& cx, int& cy)
{
    double xs, ys;
    const bool ok = project_px(H, x, y, w, h, xs, ys);
    if (!ok || !isfinite(xs) || !isfinite(ys)) {
        cx = x;
        cy = y;
        return;
    }
    double tx = floor(dadd(xs, 0.5)), ty = floor(dadd(ys, 0.5));
    tx = fmin(fmax(tx, 0.0), (double)(w - 1));
    ty = fmin(fmax(ty, 0.0), (double)(h - 1));
    cx = (int)tx;
    cy = (int)ty;
}

// SplitMix64 (Steele, Lea, Flood 2014) as a counter-based stream.
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t k)
{
    uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// 4 distinct indices in [0, nv) for weeding iteration `it`: draws 16*it + t,
// index = (hi32(draw) * nv) >> 32, duplicates rejected, at most 16 draws.
__device__ inline bool weed_sample(uint64_t seed, long long it, int nv, int pick[4])
{
    int np = 0;
    for (int t = 0; t < 16 && np < 4; t++) {
        const uint64_t z = splitmix64_at(seed, (uint64_t)it * 16u + (uint64_t)t);
        const int j = (int)(((z >> 32) * (uint64_t)nv) >> 32);
        bool dup = false;
        for (int k = 0; k < np; k++) dup |= (pick[k] == j);
        if (!dup) pick[np++] = j;
    }
    return np == 4;
}

// Gaussian elimination with partial pivoting on an 8x8 system (first row of
// largest |a_ik| is the pivot); each pivot is inverted once, factors are
// a_ik * (1/a_kk), back substitution subtracts in increasing column order and
// multiplies by the stored reciprocal; each operation one binary64 rounding.
// Returns 0, or 1 if a pivot magnitude is below tol.
__device__ inline int solve8(double (&A)[8][8], double (&b)[8], double (&x)[8], double tol)
{
    double inv[8];
    for (int k = 0; k < 8; k++) {
        int piv = k;
        double best = fabs(A[k][k]);
        for (int i = k + 1; i < 8; i++) {
            const double v = fabs(A[i][k]);
            if (v > best) {
                best = v;
                piv = i;
            }
        }
        if (!(best >= tol)) return 1;
        if (piv != k) {
            for (int j = 0; j < 8; j++) {
                const double t = A[k][j];
                A[k][j] = A[piv][j];
                A[piv][j] = t;
            }
            const double t = b[k];
            b[k] = b[piv];
            b[piv] = t;
        }
        inv[k] = ddiv(1.0, A[k][k]);
        for (int i = k + 1; i < 8; i++) {
            const double f = dmul(A[i][k], inv[k]);
            for (int j = k + 1; j < 8; j++) A[i][j] = dsub(A[i][j], dmul(f, A[k][j]));
            b[i] = dsub(b[i], dmul(f, b[k]));
        }
    }
    for (int k = 7; k >= 0; k--) {
        double s = b[k];
        for (int j = k + 1; j < 8; j++) s = dsub(s, dmul(A[k][j], x[j]));
        x[k] = dmul(s, inv[k]);
    }
    return 0;
}

// Smallest power of two >= w: the scale S of the coordinates x~ = (2x - (w-1)) / S
// in which the weeding and level-fit systems are solved (the division is exact).
__host__ __device__ inline int pow2_scale(int w)
{
    int s = 1;
    while (s < w) s <<= 1;
    return s;
}

// Division-free inlier predicate of the weeding filter for a homography written in
// the S-scaled coordinates: reprojection of p within eps pixels of q, multiplied
// through by (2D)^2 with D > 0. x, y: S-scaled corner; qxc = 2 q_x - (w-1), qyc.
__device__ __forceinline__ bool is_inlier(const double* H, double x, double y, double qxc,
                                          double qyc, double S, double eps2x)
{
    const double X = dadd(dadd(dmul(H[0], x), dmul(H[1], y)), H[2]);
    const double Y = dadd(dadd(dmul(H[3], x), dmul(H[4], y)), H[5]);
    const double D = dadd(dadd(dmul(H[6], x), dmul(H[7], y)), H[8]);
    const double ex = dsub(dmul(X, S), dmul(qxc, D));
    const double ey = dsub(dmul(Y, S), dmul(qyc, D));
    const double lhs = dadd(dmul(ex, ex), dmul(ey, ey));
    const double t = dmul(eps2x, D);
    return D > 0.0 && lhs <= dmul(t, t);
}

// ------------------------------------------------- asynchronous global->shared
// cp.async copies land in shared memory without a register round trip, so a
// thread can keep all of its staging copies in flight at once.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// ----------------------------------------------------------------- launchers
struct LutSpec {         // a per-frame 8-bit map: device table, or round(v*gn/gd) clipped
    const uint8_t* dev;  // 256 entries, or nullptr
    int gn, gd;
};

void launch_lut2(const uint8_t* a, const uint8_t* b, uint8_t* an, uint8_t* bn, size_t n,
                 LutSpec la, LutSpec lb, cudaStream_t s);
void launch_write_luts(LutSpec a, LutSpec b, uint8_t* luts, cudaStream_t s);
void launch_pyramid2(const uint8_t* const in0[2], int w, int h, int levels, const LutSpec lut[2],
                     uint8_t* const out0[2], uint8_t* const* const lv[2], int nframes,
                     cudaStream_t s);
void launch_histograms(const uint8_t* a, const uint8_t* b, size_t n, uint32_t* hist,
                       cudaStream_t s);
void launch_histeq_luts(const uint32_t* hist, size_t n, uint8_t* luts, cudaStream_t s);
// level 0 (optionally remapped by `lut` into out0) and levels 1..levels-1
void launch_pyramid(const uint8_t* in0, int w, int h, int levels, LutSpec lut, uint8_t* out0,
                    uint8_t* const* out_levels, cudaStream_t s);

struct SearchGeom {
    int w, h, tile, radius, patch_half, grid_half, quad, step, ntx, nty;
    long long corner_thr;
};
void launch_local_search(const uint8_t* ref, const uint8_t* src, const double* H,
                         const SearchGeom& g, int32_t* corner_xy, int32_t* match_xy,
                         uint32_t* cost, uint8_t* valid, cudaStream_t s);

struct WeedWs {  // workspace of the weeding step
    int32_t* list;      // n: valid tile indices in tile order
    int32_t* count;     // 1: number of valid tiles
    double* coords;     // 4n: x~, y~, x_qc, y_qc per valid match (binary64, exact)
    float4* coords32;   // n: x~, y~, x_qc / S, y_qc / S (FP32, exact for w < 2^23)
};
size_t weed_ws_bytes(int n);
WeedWs weed_ws_carve(void* base, int n);
void launch_weed(const int32_t* corner_xy, const int32_t* match_xy, const uint8_t* valid, int n,
                 int w, int h, double eps, int delta_min, int delta_div, uint64_t seed, int it0,
                 int it1, uint32_t* mask, const WeedWs& ws, cudaStream_t s);
void launch_fit(const int32_t* corner_xy, const int32_t* match_xy, const uint32_t* mask, int n,
                int w, int h, const double* H_prev, double* H_out, int32_t* status,
                cudaStream_t s);
void launch_set_identity(double* H, cudaStream_t s);

struct FlowCorners {  // sparse input of the first row pass
    const int32_t* corner_xy;
    const int32_t* match_xy;
    const uint32_t* mask;
    const double* H;
    int ntx, nty, tile;
    int full;  // propagate q - p instead of q - H(p)
};
struct DtLut {  // per-iteration link weights a_i^(1 + (sigma_s/sigma_r) d / 255), d = 0..255
    float w[256];
};
DtLut make_dt_lut(double sigma_s, double sigma_r, int iters, int i);
bool flow_fast_supported(int w, int h, const uint8_t* guide, const float* fu, const float* fv);
size_t flow_fast_extra_bytes(int w, int h);
bool launch_flow_fast(const uint8_t* guide, int w, int h, const FlowCorners& fc, const DtLut* luts,
                      int iters, double flow_eps, float* flow_u, float* flow_v, float* P0,
                      float* P1, float* P2, int* err, void* extra, cudaStream_t s);
size_t flow_ws_bytes(int w, int h);
void launch_flow(const uint8_t* guide, int w, int h, const FlowCorners& fc, double sigma_s,
                 double sigma_r, int iters, double flow_eps, float* flow_u, float* flow_v,
                 void* ws, cudaStream_t s);
int flow_supported(int w, int h);

void launch_warp(const uint8_t* src_y, const uint8_t* src_u, const uint8_t* src_v, int w, int h,
                 const double* H, const float* fu, const float* fv, float* oy, float* ou,
                 float* ov, cudaStream_t s);

struct MergeSrcDev {
    const float* y;
    const float* u;
    const float* v;
    const uint8_t* ref_n;
    const uint8_t* lut;  // HISTEQ: source LUT (device) or nullptr
    float inv_ratio;     // 1 / r_k
    float gain;          // RATIO: gain of the source frame
    int mode;
};
constexpr int kMaxSources = 4;
void launch_merge(const uint8_t* ref_y, const uint8_t* ref_u, const uint8_t* ref_v, int w, int h,
                  int nsrc, const MergeSrcDev* srcs, double ssim_sigma, double we_sigma,
                  float* oy, float* ou, float* ov, float* q_out, cudaStream_t s);

}  // namespace hdrreg
