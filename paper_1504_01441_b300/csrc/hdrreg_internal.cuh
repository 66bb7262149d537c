// Internal declarations of the hdrreg CUDA library (sm_103a).
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
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

__host__ __device__ inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

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

// The search centre of search_center from an FP32 evaluation with a certified
// interval: hf = (float)H, ha = |hf|. The FP32 values X, Y, D are within
// 4.01u (|h0 xn| + |h1 yn| + |h2|) of the exact ones (rounding of H and of xn, two
// FMAs; u = 2^-24), bounded here by 6u plus a tiny absolute term, which also covers
// the binary64 evaluation's own (2^-29 times smaller) error. The ratio and the pixel
// position are then bracketed with directed rounding and widened by 2^-20 of their
// magnitude, far beyond the binary64 rounding of the remaining steps. If both ends
// of the bracket round and clamp to the same pixel, that pixel is the binary64
// result; the function returns false when the bracket straddles a rounding boundary
// or a value is not finite, and the caller evaluates search_center in binary64.
__device__ __forceinline__ bool center_bracket(float num, float e_num, float Dlo, float Dhi,
                                               int extent, float W, int& out)
{
    const float nlo = __fadd_rd(num, -e_num), nhi = __fadd_ru(num, e_num);
    const float rlo = nlo >= 0.f ? __fdiv_rd(nlo, Dhi) : __fdiv_rd(nlo, Dlo);
    const float rhi = nhi >= 0.f ? __fdiv_ru(nhi, Dlo) : __fdiv_ru(nhi, Dhi);
    const float em1 = (float)(extent - 1);
    const float xlo = 0.5f * __fmaf_rd(rlo, W, em1), xhi = 0.5f * __fmaf_ru(rhi, W, em1);
    if (!isfinite(xlo) || !isfinite(xhi)) return false;
    const float m = 9.5367432e-7f * (fabsf(xlo) + fabsf(xhi) + W);  // 2^-20
    float tlo = floorf(__fadd_rd(__fadd_rd(xlo, -m), 0.5f));
    float thi = floorf(__fadd_ru(__fadd_ru(xhi, m), 0.5f));
    tlo = fminf(fmaxf(tlo, 0.f), em1);
    thi = fminf(fmaxf(thi, 0.f), em1);
    if (tlo != thi) return false;
    out = (int)tlo;
    return true;
}

__device__ inline bool search_center_f32(const float* hf, const float* ha, int x, int y, int w,
                                         int h, int& cx, int& cy)
{
    const float W = (float)w;
    const float xn = __fdiv_rn((float)(2 * x - (w - 1)), W);
    const float yn = __fdiv_rn((float)(2 * y - (h - 1)), W);
    const float ax = fabsf(xn), ay = fabsf(yn);
    const float X = fmaf(hf[0], xn, fmaf(hf[1], yn, hf[2]));
    const float Y = fmaf(hf[3], xn, fmaf(hf[4], yn, hf[5]));
    const float D = fmaf(hf[6], xn, fmaf(hf[7], yn, hf[8]));
    const float g = 6.0f * 5.9604645e-8f, tiny = 1e-30f;
    const float eX = fmaf(g, fmaf(ha[0], ax, fmaf(ha[1], ay, ha[2])), tiny);
    const float eY = fmaf(g, fmaf(ha[3], ax, fmaf(ha[4], ay, ha[5])), tiny);
    const float eD = fmaf(g, fmaf(ha[6], ax, fmaf(ha[7], ay, ha[8])), tiny);
    if (!isfinite(X) || !isfinite(Y) || !isfinite(D) || !isfinite(eX) || !isfinite(eY) ||
        !isfinite(eD))
        return false;
    if (__fadd_ru(D, eD) <= 0.f) {  // the binary64 denominator is not positive
        cx = x;
        cy = y;
        return true;
    }
    const float Dlo = __fadd_rd(D, -eD), Dhi = __fadd_ru(D, eD);
    if (!(Dlo > 0.f)) return false;
    int tx, ty;
    if (!center_bracket(X, eX, Dlo, Dhi, w, W, tx)) return false;
    if (!center_bracket(Y, eY, Dlo, Dhi, h, W, ty)) return false;
    cx = tx;
    cy = ty;
    return true;
}

// SplitMix64 (Steele, Lea, Flood 2014) as a counter-based stream.
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t k)
{
    uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

constexpr unsigned kFull = 0xffffffffu;

// 4 distinct indices in [0, nv) for weeding iteration `it`, drawn as in Sec. 2.3:
// draws 16*it + t (t = 0..15), index = (hi32(draw) * nv) >> 32, a draw equal to an
// earlier one rejected, the first four survivors kept. Warp-collective: lanes
// 0..15 evaluate the 16 draws at once; a draw survives iff no earlier draw has its
// value (an earlier equal draw is either kept or equal to a kept one). Returns
// false (all lanes) if fewer than four distinct draws; otherwise lane k of every
// quad (lane & 3 == k) receives pick k.
__device__ inline bool weed_sample_warp(uint64_t seed, long long it, int nv, int& pick)
{
    const int lane = threadIdx.x & 31;
    int j = -1;
    if (lane < 16) {
        const uint64_t z = splitmix64_at(seed, (uint64_t)it * 16u + (uint64_t)lane);
        j = (int)(((z >> 32) * (uint64_t)nv) >> 32);
    }
    bool first = lane < 16;
#pragma unroll
    for (int s = 0; s < 15; s++) {
        const int js = __shfl_sync(kFull, j, s);
        if (s < lane && js == j) first = false;
    }
    const unsigned fb = __ballot_sync(kFull, first);
    if (__popc(fb) < 4) return false;
    pick = __shfl_sync(kFull, j, (int)__fns(fb, 0, (lane & 3) + 1));
    return true;
}

// The binary64 value m * 2^-e, exact for |m| < 2^53 and a normal result, built
// with integer operations only; a zero result is -0.0 when neg_zero is set.
__device__ __forceinline__ double exact_scaled(long long m, int e, bool neg_zero = false)
{
    if (m == 0) return neg_zero ? -0.0 : 0.0;
    const unsigned long long sgn = m < 0 ? 0x8000000000000000ull : 0ull;
    const unsigned long long a = m < 0 ? 0ull - (unsigned long long)m : (unsigned long long)m;
    const int lz = __clzll((long long)a);
    const unsigned long long frac = ((a << lz) << 1) >> 12;  // drop the leading one
    const unsigned long long ex = (unsigned long long)(1023 + 63 - lz - e);
    return __longlong_as_double((long long)(sgn | (ex << 52) | frac));
}

// Gaussian elimination on four independent 8x8 systems in one warp, the same
// arithmetic as the sequential algorithm: partial pivoting (first row of largest
// |a_ik|; a NaN diagonal fails, other NaN rows never win), one reciprocal per
// pivot, factors a_ik * (1/a_kk), updates a_ij - f a_kj, then back substitution by
// columns (x_k = b_k * (1/a_kk), then b_i -= a_ik x_k for every row i above), every
// operation one binary64 rounding. Lane layout: system g = lane >> 3, row r =
// lane & 7; a[0..7] = A[r][0..7], a[8] = b[r]. Each step is one warp instruction for
// all four systems, which matters on a part whose binary64 pipe costs a full warp
// issue per instruction whatever the number of active lanes. Pivot magnitudes are
// compared as integers (|v| as bits is monotone for non-NaN values). Returns, per
// lane, 0 with x[] = its system's solution, or 1 if a pivot magnitude of its system
// is below tol (tol > 0); systems never interact.
__device__ inline int solve8_rows(double (&a)[9], double (&x)[8], double tol)
{
    constexpr long long kAbs = 0x7FFFFFFFFFFFFFFFLL, kInf = 0x7FF0000000000000LL;
    const int lane = threadIdx.x & 31, r = lane & 7, base = lane & ~7;
    const long long tol_bits = __double_as_longlong(tol);
    double inv[8];
    int bad = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) {
        long long key = __double_as_longlong(a[k]) & kAbs;
        const int nan = key > kInf;
        bad |= __shfl_sync(kFull, nan, base + k);
        if (r < k || nan) key = -1;
        int idx = r;
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            const long long k2 = __shfl_xor_sync(kFull, key, o);
            const int i2 = __shfl_xor_sync(kFull, idx, o);
            if (k2 > key || (k2 == key && i2 < idx)) {
                key = k2;
                idx = i2;
            }
        }
        bad |= key < tol_bits;
        const int src = r == k ? base + idx : (r == idx ? base + k : lane);  // swap rows k, idx
#pragma unroll
        for (int j = k; j < 9; j++) a[j] = __shfl_sync(kFull, a[j], src);
        inv[k] = __drcp_rn(__shfl_sync(kFull, a[k], base + k));
        const double f = dmul(a[k], inv[k]);
#pragma unroll
        for (int j = k + 1; j < 9; j++) {
            const double nv = dsub(a[j], dmul(f, __shfl_sync(kFull, a[j], base + k)));
            if (r > k) a[j] = nv;
        }
    }
#pragma unroll
    for (int k = 7; k >= 0; k--) {
        x[k] = dmul(__shfl_sync(kFull, a[8], base + k), inv[k]);
        const double nv = dsub(a[8], dmul(a[k], x[k]));
        if (r < k) a[8] = nv;
    }
    return bad;
}

// One row of the 4-point DLT system of a weeding iteration (lane layout of
// solve8_rows): rows 2k, 2k+1 of sample k are
//   [x~, y~, 1, 0, 0, 0, -x~ u~, -y~ u~ | u~],  [0, 0, 0, x~, y~, 1, -x~ v~, -y~ v~ | v~]
// with x~ = xc / S, u~ = qxc / S (centred integers, S = 2^lg). Every entry is an
// exact binary64 value, so it is built from integers; the products' zero signs
// follow binary64 multiplication and negation.
__device__ __forceinline__ void dlt4_row(int r, int xc, int yc, int qxc, int qyc, int lg,
                                         double (&a)[9])
{
    const bool odd = r & 1;
    const int q = odd ? qyc : qxc;
    const double xs = exact_scaled(xc, lg), ys = exact_scaled(yc, lg);
    a[0] = odd ? 0.0 : xs;
    a[1] = odd ? 0.0 : ys;
    a[2] = odd ? 0.0 : 1.0;
    a[3] = odd ? xs : 0.0;
    a[4] = odd ? ys : 0.0;
    a[5] = odd ? 1.0 : 0.0;
    a[6] = exact_scaled(-(long long)xc * (long long)q, 2 * lg, !((xc < 0) ^ (q < 0)));
    a[7] = exact_scaled(-(long long)yc * (long long)q, 2 * lg, !((yc < 0) ^ (q < 0)));
    a[8] = exact_scaled(q, lg);
}

// Round-to-nearest-even binary64 value of the integer v, times 2^-e, with integer
// operations. For |v| < 2^85 this equals (double)(v >> 32) * 2^32 + (double)(v mod
// 2^32) (the first product is exact there, the sum the only rounding) scaled by the
// exact power of two. Returns false (nothing written) for larger |v|.
__device__ __forceinline__ bool i128_rn_scaled(__int128 v, int e, double& out)
{
    if (v == 0) {
        out = 0.0;
        return true;
    }
    const bool neg = v < 0;
    const unsigned __int128 a = neg ? (unsigned __int128)(-v) : (unsigned __int128)v;
    if ((a >> 84) != 0) return false;
    const unsigned long long hi = (unsigned long long)(a >> 64), lo = (unsigned long long)a;
    const int msb = hi ? 127 - __clzll((long long)hi) : 63 - __clzll((long long)lo);
    unsigned long long mant;
    int ex = msb;
    if (msb <= 52) {
        mant = lo << (52 - msb);
    } else {
        const int sh = msb - 52;
        mant = (unsigned long long)(a >> sh);
        const unsigned __int128 rem = a & ((((unsigned __int128)1) << sh) - 1);
        const unsigned __int128 half = ((unsigned __int128)1) << (sh - 1);
        if (rem > half || (rem == half && (mant & 1ull))) {
            mant++;
            if (mant >> 53) {
                mant >>= 1;
                ex++;
            }
        }
    }
    const unsigned long long bits = (neg ? 0x8000000000000000ull : 0ull) |
                                    ((unsigned long long)(ex + 1023 - e) << 52) |
                                    (mant & 0x000FFFFFFFFFFFFFull);
    out = __longlong_as_double((long long)bits);
    return true;
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

// cuTensorMapEncodeTiled from the driver (resolved once; nullptr if unavailable)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();

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
    int threads;  // threads per tile CTA of the search: 64, 128 or 256
};
// Learned level-0 search (row a-L): predicted displacement per tile and the fallback rule.
struct PredSearch {
    const float* pred;  // FP32 pairs, cell (ty, tx) at 2 * (ty * pred_ld + tx); nullptr: plain
    int pred_ld;
    int refine;         // offsets [-refine, refine]^2 around the rounded prediction
    uint32_t fallback_cost;
    uint8_t* fell_back;  // optional: 1 where the tile fell back to the full search
};
// mask_zero (optional): the level's weeding mask, zeroed word by word on the way
void launch_local_search(const uint8_t* ref, const uint8_t* src, const double* H,
                         const SearchGeom& g, int32_t* corner_xy, int32_t* match_xy,
                         uint32_t* cost, uint8_t* valid, cudaStream_t s,
                         uint32_t* mask_zero = nullptr, const PredSearch* pred = nullptr);
void launch_tile_labels(const int32_t* corner_xy, const int32_t* match_xy, const uint8_t* valid,
                        int n, int w, int h, const double* H, float* label, cudaStream_t s);
void launch_predictor_crops(const void* x_full, int wq, int hq, const float* label_full,
                            const uint8_t* valid_full, int ntx, int nty, const int32_t* origins,
                            int n, int ct, float bound, void* x_out, float* label_out,
                            uint8_t* valid_out, cudaStream_t s);
void launch_predictor_input(const uint8_t* ref_q, const uint8_t* src_q, int w, int h,
                            const double* H, void* out, cudaStream_t s);

struct WeedWs {  // workspace of the weeding step
    int32_t* list;      // n: valid tile indices in tile order
    int32_t* count;     // 1: number of valid tiles
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

// Weeding + level fit of one level in one launch (matches staged in shared memory).
struct WeedLevelArgs {
    const int32_t* corner_xy;
    const int32_t* match_xy;
    const uint8_t* valid;
    int n, w, h;
    double eps;
    int delta_min, delta_div;
    uint64_t seed;
    int it0, it1;
    uint32_t* mask;        // zero on entry; receives the union of accepted inlier sets
    const double* H_prev;  // fit: coarser level's homography (kept if the fit fails)
    double* H_out;
    int32_t* status;       // 0 fitted, 1 fewer than 4 matches, 2 singular
    unsigned* done;        // completion counter, zero on entry and left zero
};
// Dynamic shared memory of the one-launch weeding: up to 11,625 level tiles (a 4000 x
// 3000 frame at T = 32); larger levels take the workspace path.
constexpr size_t kWeedLevelSmemMax = 204 * 1024;
size_t weed_level_smem_bytes(int n);
bool weed_level_fits(int n);
void launch_weed_level(const WeedLevelArgs& a, cudaStream_t s);
void launch_set_identity(double* H, cudaStream_t s, unsigned* counters = nullptr,
                         int ncounters = 0);

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
bool flow_fast_supported(int w, int h);  // sizes only; pitches and alignment checked by the caller
size_t flow_fast_extra_bytes(int w, int h);
bool launch_flow_fast(const uint8_t* guide, int gpitch, int w, int h, const FlowCorners& fc,
                      const DtLut* luts, int iters, double flow_eps, float* flow_u, float* flow_v,
                      int fpitch, float* P0, float* P1, float* P2, int ppitch, int* err,
                      void* extra, cudaStream_t s);
size_t flow_ws_bytes(int w, int h);
int flow_pitch(int w);  // padded pitch (elements) of the flow's internal planes
// The flow's error word inside its workspace (set by a bounded wait that ran out; zeroed
// by every flow call).
int* flow_error_word(void* ws, int w, int h);
void launch_flow(const uint8_t* guide, int w, int h, const FlowCorners& fc, double sigma_s,
                 double sigma_r, int iters, double flow_eps, float* flow_u, float* flow_v,
                 int fpitch, void* ws, cudaStream_t s);
int flow_supported(int w, int h);

void launch_warp(const uint8_t* src_y, const uint8_t* src_u, const uint8_t* src_v, int w, int h,
                 const double* H, const float* fu, const float* fv, int fpitch, float* oy,
                 float* ou, float* ov, uint8_t* clip, cudaStream_t s, bool clip_sign = false);

struct MergeSrcDev {
    const float* y;
    const float* u;
    const float* v;
    const uint8_t* ref_n;
    const uint8_t* lut;  // HISTEQ: source LUT (device) or nullptr
    float inv_ratio;     // 1 / r_k
    float gain;          // RATIO: gain of the source frame
    int mode;
    const uint8_t* clip;  // w x h flags of samples that draw on a pixel at 0 or 255, or nullptr
    int clip_sign;        // 1: y carries the flag in its sign bit (the fused path's own planes)
};
constexpr int kMaxSources = 4;

// Exposure fusion (fuse.cu, row f1): a registered source's warped planes and SSIM map.
struct FuseSrcDev {
    const float* y;
    const float* u;
    const float* v;
    const float* q;
};
size_t fuse_ws_bytes(int w, int h, int nframes, bool chroma);
void launch_fuse(const uint8_t* ref_y, const uint8_t* ref_u, const uint8_t* ref_v, int w, int h,
                 int nsrc, const FuseSrcDev* srcs, int use_contrast, double we_sigma, float* oy,
                 float* ou, float* ov, void* ws, cudaStream_t s);
void launch_merge(const uint8_t* ref_y, const uint8_t* ref_u, const uint8_t* ref_v, int w, int h,
                  int nsrc, const MergeSrcDev* srcs, double ssim_sigma, double we_sigma,
                  float* oy, float* ou, float* ov, float* q_out, cudaStream_t s);
// One stack's merge for launch_merge_many (the stage-major batch schedule).
struct MergeJob {
    const uint8_t* ref_y;
    const uint8_t* ref_u;
    const uint8_t* ref_v;
    int w, h, nsrc;
    MergeSrcDev srcs[kMaxSources];
    double ssim_sigma, we_sigma;
    float* oy;
    float* ou;
    float* ov;
};
constexpr int kMergeBatchStacks = 48;  // stacks per persistent merge launch (parameter space)
void launch_merge_many(const MergeJob* jobs, int count, cudaStream_t s);

// ------------------------------------------ tensor-core GEMM (row a-L)
// C[M x N] = A[M x K] * B[N x K]^T, bf16 K-major operands (16-byte aligned, ld % 8 == 0),
// FP32 accumulation; the epilogue writes FP32 (per K split at out + split * split_stride),
// FP32 + bias, or bf16 max(0, acc + bias).
enum { kEpiF32 = 0, kEpiBiasF32 = 1, kEpiBiasReluBf16 = 2 };
struct GemmEpi {
    int mode;
    float* out;
    __nv_bfloat16* out_bf16;
    const float* bias;
    int ldc;
    size_t split_stride;
};
int gemm_bn_for(int N);
bool gemm_supported(const void* A, int lda, const void* B, int ldb);
int gemm_splits_used(int K, int splits);
bool launch_gemm_bf16(const void* A, int lda, const void* B, int ldb, int M, int N, int K,
                      int splits, const GemmEpi& epi, int* err, cudaStream_t s);

// ------------------------------------------- learned predictor (row a-L)
// Implicit-GEMM 3x3 convolution (conv_tc.cu): x bf16 [n][h][w][cin] (cin = padded channel
// count, a multiple of 8), W FP32 [cout][3][3][cin_src] (cin_src <= cin; channels past
// cin_src weigh 0), bias FP32 [cout], out bf16 [M][cout] = relu(conv + bias), M = n*ho*wo.
// wimg must hold the packed weights (launch_pack_conv) when the convolution runs.
struct ConvArgs {
    const __nv_bfloat16* x;
    int h, w, ho, wo, M;
    const float* W;
    int cin_src, cin, stride, cout;
    const float* bias;
    __nv_bfloat16* out;
    int* err;
    void* wimg;  // conv_wimg_size(cin, cout) bytes, 16-byte aligned: the packed weights
};
bool launch_conv3x3(const ConvArgs& a, cudaStream_t s);  // false: no kernel for this shape
size_t conv_wimg_size(int cin, int cout);
// The weight images (wimg) of up to 8 layers in one launch, before the convolutions.
struct ConvPack {
    const float* W[8];
    void* img[8];
    int cin[8], cin_src[8], cout[8];
    int layers;
};
void launch_pack_conv(const ConvPack& p, cudaStream_t s);

size_t cnn_params();
size_t cnn_infer_ws_bytes(int n, int h, int w);
bool cnn_infer(const float* theta, const __nv_bfloat16* x, int n, int h, int w, float* out,
               void* ws, int* err, cudaStream_t s);
size_t cnn_ws_bytes(int n, int h, int w, bool train = true);  // train = false: forward only
const void* cnn_activation(const void* ws, int n, int h, int w, int layer, int* rows, int* cols);
void cnn_out_dims(int h, int w, int* ho, int* wo);
bool cnn_forward(const float* theta, const __nv_bfloat16* x, int n, int h, int w, float* out,
                 void* ws, int* err, cudaStream_t s);
bool cnn_backward(const float* theta, const __nv_bfloat16* x, int n, int h, int w, const float* out,
                  const float* label, const uint8_t* valid, float* grad, float* loss, void* ws,
                  int* err, cudaStream_t s);
void cnn_adam(float* theta, float* m, float* v, const float* grad, int step, float lr,
              cudaStream_t s);

}  // namespace hdrreg
