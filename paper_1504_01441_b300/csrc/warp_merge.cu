// Rows a9-a11: bilinear warp of the source onto the reference grid
// (Sec. 2.4), SSIM consistency mask (Sec. 2.5, Wang et al. 2004) and the
// weighted irradiance merge (Sec. 2.5 weights, Sec. 3.1 irradiance map).
//
// Warp: one thread per 2x2 luma block (= one chroma pixel of YUV420). The
// homography is evaluated as a displacement H(p) - p from FP32 coefficients
// prepared once per CTA in binary64, so the bilinear fraction is computed from
// small numbers (no 2600-px absolute coordinates in FP32).
// Merge: persistent CTAs (three per SM) walk 32x32 luma tiles, each with a 5-pixel
// halo staged in shared memory; the five Gaussian moments are separable (row pass,
// column pass). To
// avoid the FP32 cancellation of E[x^2] - mu^2, each row segment's moments are
// taken about its own centre pixel and the column pass re-centres them exactly
// onto the output pixel, so flat windows only ever sum small numbers. The two
// images' moment chains run side by side as packed FP32x2 operations (each
// component rounds as its scalar form would).
#include <math.h>

#include <cmath>

#include "hdrreg_internal.cuh"

namespace hdrreg {

namespace {

struct WarpCoef {  // dx = (a0 u + a1 v + a2 - u E/2) / D, E = c0 u + c1 v, D = E + c2
    float a0, a1, a2, b0, b1, b2, c0, c1, c2;
};

__device__ __forceinline__ void prep_coef(const double* H, int w, WarpCoef& c)
{
    const double W = (double)w;
    c.a0 = (float)((H[0] - H[8]) * 0.5);
    c.a1 = (float)(H[1] * 0.5);
    c.a2 = (float)(H[2] * W * 0.5);
    c.b0 = (float)(H[3] * 0.5);
    c.b1 = (float)((H[4] - H[8]) * 0.5);
    c.b2 = (float)(H[5] * W * 0.5);
    c.c0 = (float)(H[6] / W);
    c.c1 = (float)(H[7] / W);
    c.c2 = (float)H[8];
}

__device__ __forceinline__ void h_disp(const WarpCoef& c, int x, int y, int w, int h, float& dx,
                                       float& dy)
{
    const float u = (float)(2 * x - (w - 1)), v = (float)(2 * y - (h - 1));
    const float E = fmaf(c.c0, u, c.c1 * v);
    const float D = E + c.c2;
    if (!(D > 0.f)) {
        dx = 0.f;
        dy = 0.f;
        return;
    }
    const float nx = fmaf(c.a0, u, fmaf(c.a1, v, c.a2)) - 0.5f * u * E;
    const float ny = fmaf(c.b0, u, fmaf(c.b1, v, c.b2)) - 0.5f * v * E;
    const float r = __frcp_rn(D);  // one reciprocal for both components
    dx = nx * r;
    dy = ny * r;
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// The four taps of a bilinear sample at (x + t_x, y + t_y) (integer x, y, small offsets t):
// (ix, iy), (ix + 1, iy), (ix, iy + 1), (ix + 1, iy + 1) with clamp-to-edge reads, and the
// fractions. Frames hold fewer than 2^31 pixels, so offsets are 32-bit; samples whose
// footprint lies inside the frame (almost all) skip the clamps.
struct Taps {
    unsigned a, b, c, d;
    float fx, fy;
};

__device__ __forceinline__ Taps taps_at(const uint8_t* __restrict__ img, int w, int h, int x,
                                        int y, float tx, float ty)
{
    const float fx0 = floorf(tx), fy0 = floorf(ty);
    Taps t;
    t.fx = tx - fx0;
    t.fy = ty - fy0;
    const int ix = x + (int)fx0, iy = y + (int)fy0;
    if ((unsigned)ix < (unsigned)(w - 1) && (unsigned)iy < (unsigned)(h - 1)) {
        const uint8_t* p = img + (iy * w + ix);
        t.a = __ldg(p);
        t.b = __ldg(p + 1);
        t.c = __ldg(p + w);
        t.d = __ldg(p + w + 1);
    } else {
        const int xa = clampi(ix, 0, w - 1), xb = clampi(ix + 1, 0, w - 1);
        const int ra = clampi(iy, 0, h - 1) * w, rb = clampi(iy + 1, 0, h - 1) * w;
        t.a = __ldg(img + ra + xa);
        t.b = __ldg(img + ra + xb);
        t.c = __ldg(img + rb + xa);
        t.d = __ldg(img + rb + xb);
    }
    return t;
}

__device__ __forceinline__ float lerp_taps(const Taps& t)
{
    const float a = (float)t.a, b = (float)t.b, c = (float)t.c, d = (float)t.d;
    const float top = fmaf(t.fx, b - a, a);
    const float bot = fmaf(t.fx, d - c, c);
    return fmaf(t.fy, bot - top, top);
}

__device__ __forceinline__ float bilerp(const uint8_t* __restrict__ img, int w, int h, int x, int y,
                                        float tx, float ty)
{
    return lerp_taps(taps_at(img, w, h, x, y, tx, ty));
}

// The same sample, plus whether it draws on a clipped pixel: a tap at 0 or 255 with a
// nonzero weight -- (ix, iy) always, (ix + 1, iy) when fx > 0, (ix, iy + 1) when
// fy > 0, (ix + 1, iy + 1) when both are.
__device__ __forceinline__ float bilerp_clip(const uint8_t* __restrict__ img, int w, int h, int x,
                                             int y, float tx, float ty, bool& clipped)
{
    const Taps t = taps_at(img, w, h, x, y, tx, ty);
    const bool right = t.fx > 0.f, below = t.fy > 0.f;
    auto sat = [](unsigned v) { return v - 1u >= 254u; };  // v == 0 or v == 255
    clipped = sat(t.a) || (right && sat(t.b)) || (below && (sat(t.c) || (right && sat(t.d))));
    return lerp_taps(t);
}

// kVec: the flow pitch and the width are even and the planes 8-byte aligned, so each
// row pair of a 2x2 block moves as one float2 (flows in, warped luma out) and its two
// clip flags as one 16-bit word.
template <bool kVec>
__global__ void __launch_bounds__(256, 5) k_warp(const uint8_t* __restrict__ sy,
                                              const uint8_t* __restrict__ su,
                                              const uint8_t* __restrict__ sv, int w, int h,
                                              const double* __restrict__ H,
                                              const float* __restrict__ fu,
                                              const float* __restrict__ fv, int fpitch,
                                              float* __restrict__ oy, float* __restrict__ ou,
                                              float* __restrict__ ov,
                                              uint8_t* __restrict__ clip, int clip_sign)
{
    // The coefficients take a chain of binary64 operations (one thread, the others
    // waiting), so the grid is sized to the resident CTAs and each CTA strides over
    // many blocks: the chain runs once per CTA, not once per 256 blocks.
    __shared__ WarpCoef cs;
    if (threadIdx.x == 0) prep_coef(H, w, cs);
    __syncthreads();
    const WarpCoef c = cs;
    const int bw = (w + 1) / 2, bh = (h + 1) / 2;
    const int nb = bw * bh;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < nb; idx += gridDim.x * blockDim.x) {
    const int bx = idx % bw, by = idx / bw;
    const int x = 2 * bx;
    const bool two = x + 1 < w;  // the block's right column exists
    float stx = 0.f, sty = 0.f;
#pragma unroll
    for (int j = 0; j < 2; j++) {
        const int y = 2 * by + j;
        if (y >= h) continue;
        const size_t o = (size_t)y * w + x, of = (size_t)y * fpitch + x;
        float f[2][2];  // [u, v][column]
        if (kVec) {
            const float2 a = __ldg(reinterpret_cast<const float2*>(fu + of));
            const float2 b = __ldg(reinterpret_cast<const float2*>(fv + of));
            f[0][0] = a.x; f[0][1] = a.y; f[1][0] = b.x; f[1][1] = b.y;
        } else {
            f[0][0] = fu[of];
            f[1][0] = fv[of];
            f[0][1] = two ? fu[of + 1] : 0.f;
            f[1][1] = two ? fv[of + 1] : 0.f;
        }
        float z[2];
        bool cl[2] = {false, false};
#pragma unroll
        for (int i = 0; i < 2; i++) {
            z[i] = 0.f;
            if (i == 1 && !two) continue;
            float dx, dy;
            h_disp(c, x + i, y, w, h, dx, dy);
            const float tx = dx + f[0][i], ty = dy + f[1][i];
            stx += tx;
            sty += ty;
            z[i] = bilerp_clip(sy, w, h, x + i, y, tx, ty, cl[i]);
            // clip_sign: the flag travels in the sign bit of the (non-negative) sample
            if (clip_sign && cl[i]) z[i] = __int_as_float(__float_as_int(z[i]) | (int)0x80000000);
        }
        if (kVec) {
            *reinterpret_cast<float2*>(oy + o) = make_float2(z[0], z[1]);
            if (clip)
                *reinterpret_cast<uint16_t*>(clip + o) =
                    (uint16_t)((cl[0] ? 1u : 0u) | (cl[1] ? 256u : 0u));
        } else {
            oy[o] = z[0];
            if (clip) clip[o] = cl[0] ? 1 : 0;
            if (two) {
                oy[o + 1] = z[1];
                if (clip) clip[o + 1] = cl[1] ? 1 : 0;
            }
        }
    }
    if (su && ou) {
        const int cw = w / 2, ch = h / 2;
        if (bx < cw && by < ch) {
            const float tx = stx * 0.125f, ty = sty * 0.125f;  // mean offset / 2
            const size_t o = (size_t)by * cw + bx;
            ou[o] = bilerp(su, cw, ch, bx, by, tx, ty);
            ov[o] = bilerp(sv, cw, ch, bx, by, tx, ty);
        }
    }
    }
}

// Network input of the learned search (row a-L) at quarter resolution: the reference
// and the source sampled at H(p) (the displacement form above), both mapped to
// (v - 127.5) / 127.5 and stored as a bfloat16 pair per pixel.
__global__ void __launch_bounds__(256) k_predictor_input(const uint8_t* __restrict__ ref_q,
                                                         const uint8_t* __restrict__ src_q, int w,
                                                         int h, const double* __restrict__ H,
                                                         __nv_bfloat162* __restrict__ out)
{
    __shared__ WarpCoef cs;
    if (threadIdx.x == 0) prep_coef(H, w, cs);
    __syncthreads();
    const WarpCoef c = cs;
    const long long n = (long long)w * h;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % w), y = (int)(i / w);
        float dx, dy;
        h_disp(c, x, y, w, h, dx, dy);
        const float v = bilerp(src_q, w, h, x, y, dx, dy);
        const float r = (float)ref_q[i];
        out[i] = __floats2bfloat162_rn((r - 127.5f) / 127.5f, (v - 127.5f) / 127.5f);
    }
}

// ----------------------------------------------------------------- merge
constexpr int kTile = 32;
constexpr int kHalo = kSsimRadius;
constexpr int kIn = kTile + 2 * kHalo;  // 42

struct MergeArgs {
    MergeSrcDev src[kMaxSources];
    float g[2 * kSsimRadius + 1];
    float gsum;  // sum of the FP32 taps (1 up to rounding)
    float s0;    // total weight of a window as the column pass accumulates it: fma of each
                 // tap with gsum, taps in order
    float we_k;  // 1 / (2 sigma^2)
    int nsrc;
};

// The exponent lies in [-k/4, 0] (k = 12.5 at sigma 0.2), where the fast exponential's
// error is a few units in the last place: far below the merge's 1e-4 parity rule.
__device__ __forceinline__ float well_exposed(float z, float k)
{
    const float t = z * (1.f / 255.f) - 0.5f;
    return __expf(-(t * t) * k);
}

__device__ __forceinline__ float norm_map(const MergeSrcDev& s, float z)
{
    if (s.mode == 0) return fminf(255.f, s.gain * z);
    const float f0 = floorf(z);
    int i0 = (int)f0;
    if (i0 >= 255) return (float)s.lut[255];
    float f = z - f0;
    if (i0 < 0) {
        i0 = 0;
        f = z;
    }
    const float a = (float)s.lut[i0], b = (float)s.lut[i0 + 1];
    return fmaf(f, b - a, a);
}

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

__device__ __forceinline__ void cp_async16(void* dst, const void* src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}

// Raw inputs of one (tile, source) unit, staged ahead of their use. Columns: Rn holds
// ref_n at x0 - 16 .. x0 + 47, Ys the warped source luma at x0 - 8 .. x0 + 39, both for
// rows y0 - 5 .. y0 + 36; Ry the reference luma of the tile; Ru, Rv, Su, Sv the tile's
// 16 x 16 chroma of the reference and of the warped source.
struct alignas(16) MergeStage {
    uint8_t Rn[kIn][64];
    float Ys[kIn][48];
    uint8_t Ry[kTile][kTile];
    uint8_t Ru[kTile / 2][kTile / 2], Rv[kTile / 2][kTile / 2];
    float Su[kTile / 2][kTile / 2], Sv[kTile / 2][kTile / 2];
};

struct MergeSmem {
    MergeStage st[2];
    float2 XY[kIn][kIn];   // the reference (X) and the normalized warped source (Y)
    float2 H1[kIn][kTile];  // (sum g a, sum g b) of each row segment
    float2 H2[kIn][kTile];  // (sum g a^2, sum g b^2)
    float H11[kIn][kTile + 1];  // sum g a b
    float Wk[kTile][kTile + 1];
};

// Tile t of a row-major grid tiles_x wide: (t mod tiles_x, t / tiles_x) from the FP32
// reciprocal `inv` = 1 / tiles_x and one correction step (exact for t < 2^23).
__device__ __forceinline__ void tile_xy(int t, int tiles_x, float inv, int& bx, int& by)
{
    int q = __float2int_rz((float)t * inv);
    int r = t - q * tiles_x;
    if (r < 0) {
        q--;
        r += tiles_x;
    } else if (r >= tiles_x) {
        q++;
        r -= tiles_x;
    }
    bx = r;
    by = q;
}

// Stage unit (tile t, source k): 16-byte async copies for interior tiles when every
// plane allows them, else plain loads with clamp-to-edge (and the same layout).
__device__ __forceinline__ void merge_stage(MergeStage& S, const MergeArgs& args,
                                            const uint8_t* __restrict__ ref_y,
                                            const uint8_t* __restrict__ ref_u,
                                            const uint8_t* __restrict__ ref_v, int w, int h,
                                            bool chroma, int tiles_x, float inv_tiles_x, int t,
                                            int k, bool async_ok)
{
    const int tid = threadIdx.x;
    int bx, by;
    tile_xy(t, tiles_x, inv_tiles_x, bx, by);
    const int x0 = bx * kTile, y0 = by * kTile;
    const MergeSrcDev& s = args.src[k];
    const int cw = w / 2, ch = h / 2, cx0 = x0 / 2, cy0 = y0 / 2;
    const bool interior = async_ok && x0 >= 16 && x0 + 48 <= w && y0 >= kHalo &&
                          y0 + kTile + kHalo <= h;
    if (interior) {
        // Rn: 42 rows x 4 chunks; Ys: 42 rows x 12 chunks
        for (int i = tid; i < kIn * 4; i += 256) {
            const int r = i >> 2, c = i & 3;
            cp_async16(&S.Rn[r][c * 16], s.ref_n + (size_t)(y0 - kHalo + r) * w + x0 - 16 + c * 16);
        }
        for (int i = tid; i < kIn * 12; i += 256) {
            const int r = i / 12, c = i - r * 12;
            cp_async16(&S.Ys[r][c * 4], s.y + (size_t)(y0 - kHalo + r) * w + x0 - 8 + c * 4);
        }
        if (k == 0 && tid < 64) {
            const int r = tid >> 1, c = tid & 1;
            cp_async16(&S.Ry[r][c * 16], ref_y + (size_t)(y0 + r) * w + x0 + c * 16);
        }
        if (chroma) {
            if (k == 0 && tid < 32) {
                const int r = tid & 15;
                const uint8_t* src = (tid < 16 ? ref_u : ref_v) + (size_t)(cy0 + r) * cw + cx0;
                cp_async16(tid < 16 ? &S.Ru[r][0] : &S.Rv[r][0], src);
            }
            if (tid >= 64 && tid < 192) {
                const int q = tid - 64, pl = q >> 6, r = (q >> 2) & 15, c = q & 3;
                const float* src = (pl ? s.v : s.u) + (size_t)(cy0 + r) * cw + cx0 + c * 4;
                cp_async16(pl ? &S.Sv[r][c * 4] : &S.Su[r][c * 4], src);
            }
        }
        return;
    }
    for (int i = tid; i < kIn * 64; i += 256) {
        const int r = i >> 6, c = i & 63;
        const int gy = clampi(y0 - kHalo + r, 0, h - 1), gx = clampi(x0 - 16 + c, 0, w - 1);
        S.Rn[r][c] = s.ref_n[(size_t)gy * w + gx];
    }
    for (int i = tid; i < kIn * 48; i += 256) {
        const int r = i / 48, c = i - r * 48;
        const int gy = clampi(y0 - kHalo + r, 0, h - 1), gx = clampi(x0 - 8 + c, 0, w - 1);
        S.Ys[r][c] = s.y[(size_t)gy * w + gx];
    }
    if (k == 0)
        for (int i = tid; i < kTile * kTile; i += 256) {
            const int r = i >> 5, c = i & 31;
            const int gy = y0 + r < h ? y0 + r : h - 1, gx = x0 + c < w ? x0 + c : w - 1;
            S.Ry[r][c] = ref_y[(size_t)gy * w + gx];
        }
    if (chroma && cw > 0 && ch > 0) {
        const int r = tid >> 4, c = tid & 15;
        const int gy = cy0 + r < ch ? cy0 + r : ch - 1, gx = cx0 + c < cw ? cx0 + c : cw - 1;
        const size_t o = (size_t)gy * cw + gx;
        if (k == 0) {
            S.Ru[r][c] = ref_u[o];
            S.Rv[r][c] = ref_v[o];
        }
        S.Su[r][c] = s.u[o];
        S.Sv[r][c] = s.v[o];
    }
}

// One stack's merge as the kernel sees it: its planes, sizes, sources and weights.
struct MergeStackDev {
    const uint8_t* ref_y;
    const uint8_t* ref_u;  // nullptr: luma only
    const uint8_t* ref_v;
    float* oy;
    float* ou;
    float* ov;
    float* q_out;          // optional SSIM maps (nsrc planes of w x h)
    int w, h, tiles_x;
    float inv_tiles_x;     // 1 / tiles_x
    int item_begin;        // first item (32 x 32 tile) of this stack in the launch's item list
    int async_ok;          // every plane allows 16-byte asynchronous row copies
    MergeArgs a;
};

// The stacks of one launch; their tiles are numbered consecutively, stack after stack.
template <int NS>
struct MergeBatch {
    int nstacks, nitems;
    MergeStackDev st[NS];
};

template <int NS>
__device__ __forceinline__ int stack_of(const MergeBatch<NS>& B, int item)
{
    int s = 0;
    while (s + 1 < B.nstacks && B.st[s + 1].item_begin <= item) s++;
    return s;
}

// Persistent CTAs over (tile, source) units: items (tiles of any stack of the launch)
// i = blockIdx.x + j * gridDim.x, and within an item every source of its stack in order;
// the next unit's inputs are staged (async copies) while the current one computes. Three
// CTAs fit an SM: 80 registers a thread (the launch bound) and 74 KB of shared memory,
// each thread keeping its four output rows' luma sums in registers.
template <int NS>
__global__ void __launch_bounds__(256, 3) k_merge(const __grid_constant__ MergeBatch<NS> B)
{
    extern __shared__ __align__(16) uint8_t merge_smem[];
    MergeSmem& M = *reinterpret_cast<MergeSmem*>(merge_smem);
    const int tid = threadIdx.x;
    const float2 neg1 = f2(-1.f, -1.f);
    const float C1 = (0.01f * 255.f) * (0.01f * 255.f), C2 = (0.03f * 255.f) * (0.03f * 255.f);
    // this thread's 4 luma pixels: (tx, ty + 8 k); its chroma pixel: (tid % 16, tid / 16)
    const int tx = tid % kTile, ty0 = tid / kTile;
    const int ccx = tid % 16, ccy = tid / 16;

    int item = blockIdx.x;
    if (item >= B.nitems) return;
    int si = stack_of(B, item), k = 0, buf = 0;
    {
        const MergeStackDev& D = B.st[si];
        merge_stage(M.st[0], D.a, D.ref_y, D.ref_u, D.ref_v, D.w, D.h,
                    D.ref_u != nullptr && D.ou != nullptr, D.tiles_x, D.inv_tiles_x,
                    item - D.item_begin, 0,
                    D.async_ok);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    // this thread's sums over the sources: chroma, and luma for rows 4 ty0 .. 4 ty0 + 3 of
    // column tx (the rows its column pass computes)
    float cnu = 0.f, cnv = 0.f, cden = 0.f;
    float ns_acc[4] = {0.f, 0.f, 0.f, 0.f}, ds_acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (;;) {
        // the unit after this one: the next source of the item, or the CTA's next item
        int nitem = item, nsi = si, nk = k + 1;
        if (nk >= B.st[si].a.nsrc) {
            nitem = item + gridDim.x;
            nk = 0;
            nsi = nitem < B.nitems ? stack_of(B, nitem) : si;
        }
        const bool more = nitem < B.nitems;
        if (more) {
            const MergeStackDev& Dn = B.st[nsi];
            merge_stage(M.st[buf ^ 1], Dn.a, Dn.ref_y, Dn.ref_u, Dn.ref_v, Dn.w, Dn.h,
                        Dn.ref_u != nullptr && Dn.ou != nullptr, Dn.tiles_x, Dn.inv_tiles_x,
                        nitem - Dn.item_begin,
                        nk, Dn.async_ok);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group 1;" ::: "memory");
        __syncthreads();
        const MergeStackDev& D = B.st[si];
        const MergeArgs& args = D.a;
        const uint8_t* __restrict__ ref_y = D.ref_y;
        float* __restrict__ oy = D.oy;
        float* __restrict__ ou = D.ou;
        float* __restrict__ ov = D.ov;
        float* __restrict__ q_out = D.q_out;
        const int w = D.w, h = D.h, ns = args.nsrc;
        const bool chroma = D.ref_u != nullptr && ou != nullptr;
        const int cw = w / 2, ch = h / 2;
        const int t = item - D.item_begin;
        int tbx, tby;
        tile_xy(t, D.tiles_x, D.inv_tiles_x, tbx, tby);
        const int x0 = tbx * kTile, y0 = tby * kTile;
        const float2 gsum2 = f2(args.gsum, args.gsum);
        const float2 s02 = f2(args.s0, args.s0);
        (void)ref_y;
        const MergeStage& S = M.st[buf];
        const MergeSrcDev& s = args.src[k];
        const int cx = x0 / 2 + ccx, cy = y0 / 2 + ccy;
        const bool c_ok = chroma && cx < cw && cy < ch;
        if (k == 0) {  // the reference's own weights open the sums
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int ly = 4 * ty0 + q;
                const int x = x0 + tx, y = y0 + ly;
                float nu = 0.f, de = 0.f;
                if (x < w && y < h) {
                    const float z = (float)S.Ry[ly][tx];
                    de = well_exposed(z, args.we_k);
                    nu = de * z;
                }
                ns_acc[q] = nu;
                ds_acc[q] = de;
                M.Wk[ly][tx] = de;
            }
        }
        // two neighbours per step (rows have an even length, so a pair never straddles two
        // rows), stored as one 16-byte write
        static_assert(kIn % 2 == 0, "XY pairs");
        for (int i = tid; i < kIn * kIn / 2; i += 256) {
            const int yy = i / (kIn / 2), xx = 2 * (i - yy * (kIn / 2));
            const float za = S.Ys[yy][xx + 3], zb = S.Ys[yy][xx + 4];
            const float na = norm_map(s, s.clip_sign ? fabsf(za) : za);
            const float nb = norm_map(s, s.clip_sign ? fabsf(zb) : zb);
            *reinterpret_cast<float4*>(&M.XY[yy][xx]) =
                make_float4((float)S.Rn[yy][xx + 11], na, (float)S.Rn[yy][xx + 12], nb);
        }
        __syncthreads();
        if (k == 0) {
            cnu = cnv = cden = 0.f;
            if (c_ok) {
                const int lx = 2 * ccx, ly = 2 * ccy;
                const float wb =
                    ((M.Wk[ly][lx] + M.Wk[ly][lx + 1]) + (M.Wk[ly + 1][lx] + M.Wk[ly + 1][lx + 1])) * 0.25f;
                cnu = wb * ((float)S.Ru[ccy][ccx] - 128.f);
                cnv = wb * ((float)S.Rv[ccy][ccx] - 128.f);
                cden = wb;
            }
        }
        // Row pass: moments of each 11-tap row segment about its own centre pixel
        // (a = x - x_c, b = y - y_c): M1 = sum g (a, b), M2 = sum g (a^2, b^2), M11 = sum g a b.
        // Two neighbouring segments per step share one 12-element window, read as six
        // 16-byte loads; each keeps its own sums in tap order.
        static_assert(kTile % 2 == 0 && 2 * kHalo + 2 == 12, "row pass window");
        for (int i = tid; i < kIn * kTile / 2; i += 256) {
            const int yy = i / (kTile / 2), xx = 2 * (i - yy * (kTile / 2));
            float2 r[12];
            const float4* src = reinterpret_cast<const float4*>(&M.XY[yy][xx]);
#pragma unroll
            for (int q = 0; q < 6; q++) {
                const float4 t = src[q];
                r[2 * q] = f2(t.x, t.y);
                r[2 * q + 1] = f2(t.z, t.w);
            }
            const float2 c0 = r[kHalo], c1 = r[kHalo + 1];
            float2 m1a = f2(0.f, 0.f), m2a = f2(0.f, 0.f), m1b = f2(0.f, 0.f), m2b = f2(0.f, 0.f);
            float m11a = 0.f, m11b = 0.f;
#pragma unroll
            for (int d = 0; d <= 2 * kHalo; d++) {
                if (d == kHalo) continue;  // the centre tap's deviations are exactly zero
                const float2 g2 = f2(args.g[d], args.g[d]);
                const float2 aba = __ffma2_rn(c0, neg1, r[d]);
                const float2 abb = __ffma2_rn(c1, neg1, r[d + 1]);
                const float2 gaba = __fmul2_rn(g2, aba);
                const float2 gabb = __fmul2_rn(g2, abb);
                m1a = __fadd2_rn(m1a, gaba);
                m1b = __fadd2_rn(m1b, gabb);
                m2a = __ffma2_rn(gaba, aba, m2a);
                m2b = __ffma2_rn(gabb, abb, m2b);
                m11a = fmaf(gaba.x, aba.y, m11a);
                m11b = fmaf(gabb.x, abb.y, m11b);
            }
            *reinterpret_cast<float4*>(&M.H1[yy][xx]) = make_float4(m1a.x, m1a.y, m1b.x, m1b.y);
            *reinterpret_cast<float4*>(&M.H2[yy][xx]) = make_float4(m2a.x, m2a.y, m2b.x, m2b.y);
            M.H11[yy][xx] = m11a;
            M.H11[yy][xx + 1] = m11b;
        }
        __syncthreads();
        // Column pass: a thread takes four consecutive output rows 4 ty0 .. 4 ty0 + 3 of
        // column tx. Each of the 14 staged rows they span is read once, its moments are
        // re-centred from its centre c_r onto the value c_t of the thread's first output
        // pixel (delta = c_r - c_t: sum g (a + delta)^k expands exactly), and added, in tap
        // order, to every output whose window holds it. The four sums are then re-centred
        // once more, from c_t onto each output's own value, with the same expansion and
        // the window's total weight S0. Every centre is a pixel inside the output's window
        // (c_t at most three rows away), so flat windows only ever sum small numbers.
        constexpr int kQ = 4, kSpan = kQ + 2 * kHalo;
        const int lyb = kQ * ty0;
        const float2 ct = M.XY[lyb + kHalo][tx + kHalo];
        float2 a1[kQ], a2[kQ];
        float a11[kQ];
#pragma unroll
        for (int q = 0; q < kQ; q++) {
            a1[q] = f2(0.f, 0.f);
            a2[q] = f2(0.f, 0.f);
            a11[q] = 0.f;
        }
#pragma unroll
        for (int rr = 0; rr < kSpan; rr++) {
            const float2 xy = M.XY[lyb + rr][tx + kHalo];
            const float2 m1 = M.H1[lyb + rr][tx];
            const float2 m2 = M.H2[lyb + rr][tx];
            const float m11 = M.H11[lyb + rr][tx];
            const float2 dd = __ffma2_rn(ct, neg1, xy);
            const float2 r1 = __ffma2_rn(dd, gsum2, m1);
            const float2 r2 = __ffma2_rn(dd, __fadd2_rn(m1, r1), m2);
            const float r11 = m11 + fmaf(dd.y, m1.x, dd.x * r1.y);
#pragma unroll
            for (int q = 0; q < kQ; q++) {
                const int d = rr - q;
                if (d < 0 || d > 2 * kHalo) continue;
                const float2 g2 = f2(args.g[d], args.g[d]);
                a1[q] = __ffma2_rn(g2, r1, a1[q]);
                a2[q] = __ffma2_rn(g2, r2, a2[q]);
                a11[q] = fmaf(args.g[d], r11, a11[q]);
            }
        }
#pragma unroll
        for (int q = 0; q < kQ; q++) {
            const int ly = lyb + q;
            const int x = x0 + tx, y = y0 + ly;
            const float2 c = M.XY[ly + kHalo][tx + kHalo];
            // from c_t onto c: delta = c_t - c
            const float2 dq = __ffma2_rn(c, neg1, ct);
            const float2 b1 = __ffma2_rn(dq, s02, a1[q]);
            const float2 b2 = __ffma2_rn(dq, __fadd2_rn(a1[q], b1), a2[q]);
            const float b11 = a11[q] + fmaf(dq.y, a1[q].x, dq.x * b1.y);
            a1[q] = b1;
            const float vx = b2.x - b1.x * b1.x, vy = b2.y - b1.y * b1.y,
                        cxy = b11 - b1.x * b1.y;
            const float ux = c.x + a1[q].x, uy = c.y + a1[q].y;
            // the denominator lies in [C1 C2, 2^33): the fast quotient is within 2 ulp
            const float ssim = __fdividef((2.f * ux * uy + C1) * (2.f * cxy + C2),
                                          (ux * ux + uy * uy + C1) * (vx + vy + C2));
            const float qv = ssim > 0.f ? ssim : 0.f;
            float wk = 0.f;
            if (x < w && y < h) {
                const float zs = S.Ys[ly + kHalo][tx + 8];
                const float z = s.clip_sign ? fabsf(zs) : zs;
                // a sample that draws on a pixel at 0 or 255 carries no irradiance
                const bool clipped = s.clip_sign ? signbit(zs)
                                     : (s.clip ? __ldg(s.clip + (size_t)y * w + x) != 0
                                               : (z <= 0.f || z >= 255.f));
                wk = clipped ? 0.f : well_exposed(z, args.we_k) * qv;
                ns_acc[q] = fmaf(wk, z * s.inv_ratio, ns_acc[q]);
                ds_acc[q] += wk;
                if (q_out) q_out[(size_t)k * w * h + (size_t)y * w + x] = qv;
            }
            M.Wk[ly][tx] = wk;
        }
        __syncthreads();
        if (c_ok) {
            const int lx = 2 * ccx, ly = 2 * ccy;
            const float wb =
                ((M.Wk[ly][lx] + M.Wk[ly][lx + 1]) + (M.Wk[ly + 1][lx] + M.Wk[ly + 1][lx + 1])) * 0.25f;
            cnu = fmaf(wb, (S.Su[ccy][ccx] - 128.f) * s.inv_ratio, cnu);
            cnv = fmaf(wb, (S.Sv[ccy][ccx] - 128.f) * s.inv_ratio, cnv);
            cden += wb;
        }
        if (k == ns - 1) {
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int x = x0 + tx, y = y0 + 4 * ty0 + q;
                // D holds the reference's own weight (at least exp(-k/4)) and at most
                // nsrc + 1: the fast quotient is within 2 ulp
                if (x < w && y < h) oy[(size_t)y * w + x] = __fdividef(ns_acc[q], ds_acc[q]);
            }
            if (c_ok) {
                const size_t o = (size_t)cy * cw + cx;
                ou[o] = __fdividef(cnu, cden);
                ov[o] = __fdividef(cnv, cden);
            }
        }
        __syncthreads();  // the staging buffer and the sums are reused by the next unit
        if (!more) break;
        item = nitem;
        si = nsi;
        k = nk;
        buf ^= 1;
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
}

}  // namespace

void launch_warp(const uint8_t* src_y, const uint8_t* src_u, const uint8_t* src_v, int w, int h,
                 const double* H, const float* fu, const float* fv, int fpitch, float* oy,
                 float* ou, float* ov, uint8_t* clip, cudaStream_t s, bool clip_sign)
{
    const long long nb = (long long)((w + 1) / 2) * ((h + 1) / 2);
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    auto al8 = [](const void* p) { return p == nullptr || ((uintptr_t)p & 7u) == 0; };
    const bool vec = (w % 2) == 0 && (fpitch % 2) == 0 && al8(fu) && al8(fv) && al8(oy) &&
                     (clip == nullptr || ((uintptr_t)clip & 1u) == 0);
    const void* fn = vec ? (const void*)k_warp<true> : (const void*)k_warp<false>;
    // the grid is the resident CTAs: each strides over many blocks, so the binary64
    // coefficient chain runs once per CTA
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, 0) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    const long long need = (nb + 255) / 256, cap = (long long)per_sm * sms;
    const int grid = (int)(need < cap ? need : cap);
    note_launch();
    if (vec)
        k_warp<true><<<grid, 256, 0, s>>>(src_y, src_u, src_v, w, h, H, fu, fv, fpitch, oy, ou, ov,
                                          clip, clip_sign ? 1 : 0);
    else
        k_warp<false><<<grid, 256, 0, s>>>(src_y, src_u, src_v, w, h, H, fu, fv, fpitch, oy, ou,
                                           ov, clip, clip_sign ? 1 : 0);
}

void launch_predictor_input(const uint8_t* ref_q, const uint8_t* src_q, int w, int h,
                            const double* H, void* out, cudaStream_t s)
{
    const long long n = (long long)w * h;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long g = (n + 255) / 256;
    if (g > 8LL * sms) g = 8LL * sms;  // one binary64 coefficient chain per resident CTA
    note_launch();
    k_predictor_input<<<(int)g, 256, 0, s>>>(ref_q, src_q, w, h, H,
                                             static_cast<__nv_bfloat162*>(out));
}

// The weights and flags of one stack's merge.
static MergeStackDev merge_stack(const uint8_t* ref_y, const uint8_t* ref_u, const uint8_t* ref_v,
                                 int w, int h, int nsrc, const MergeSrcDev* srcs,
                                 double ssim_sigma, double we_sigma, float* oy, float* ou,
                                 float* ov, float* q_out)
{
    MergeStackDev D;
    MergeArgs& a = D.a;
    a.nsrc = nsrc;
    for (int k = 0; k < nsrc; k++) a.src[k] = srcs[k];
    double gs[2 * kSsimRadius + 1], tot = 0.0;
    for (int d = -kSsimRadius; d <= kSsimRadius; d++) {
        gs[d + kSsimRadius] = exp(-(double)(d * d) / (2.0 * ssim_sigma * ssim_sigma));
        tot += gs[d + kSsimRadius];
    }
    double fsum = 0.0;
    for (int d = 0; d <= 2 * kSsimRadius; d++) {
        a.g[d] = (float)(gs[d] / tot);
        fsum += (double)a.g[d];
    }
    a.gsum = (float)fsum;
    a.s0 = 0.f;
    for (int d = 0; d <= 2 * kSsimRadius; d++) a.s0 = std::fma(a.g[d], a.gsum, a.s0);
    a.we_k = (float)(1.0 / (2.0 * we_sigma * we_sigma));
    bool async_ok = (w % 32) == 0;  // 16-byte rows for u8 luma and chroma planes
    auto al = [](const void* p) { return p == nullptr || ((uintptr_t)p & 15u) == 0; };
    async_ok = async_ok && al(ref_y) && al(ref_u) && al(ref_v);
    for (int k = 0; k < nsrc; k++)
        async_ok = async_ok && al(srcs[k].y) && al(srcs[k].u) && al(srcs[k].v) && al(srcs[k].ref_n);
    D.ref_y = ref_y;
    D.ref_u = ref_u;
    D.ref_v = ref_v;
    D.oy = oy;
    D.ou = ou;
    D.ov = ov;
    D.q_out = q_out;
    D.w = w;
    D.h = h;
    D.tiles_x = (w + kTile - 1) / kTile;
    D.inv_tiles_x = 1.f / (float)D.tiles_x;
    D.item_begin = 0;
    D.async_ok = async_ok ? 1 : 0;
    return D;
}

static int merge_grid(int nitems)
{
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return nitems < 3 * sms ? nitems : 3 * sms;  // the resident CTAs: three per SM
}

void launch_merge(const uint8_t* ref_y, const uint8_t* ref_u, const uint8_t* ref_v, int w, int h,
                  int nsrc, const MergeSrcDev* srcs, double ssim_sigma, double we_sigma,
                  float* oy, float* ou, float* ov, float* q_out, cudaStream_t s)
{
    MergeBatch<1> B;
    B.nstacks = 1;
    B.st[0] = merge_stack(ref_y, ref_u, ref_v, w, h, nsrc, srcs, ssim_sigma, we_sigma, oy, ou, ov,
                          q_out);
    B.nitems = B.st[0].tiles_x * ((h + kTile - 1) / kTile);
    const size_t smem = sizeof(MergeSmem);
    ensure_smem((const void*)k_merge<1>, smem);
    note_launch();
    k_merge<1><<<merge_grid(B.nitems), 256, smem, s>>>(B);
}

// Several stacks' merges in persistent launches of up to kMergeBatchStacks stacks each.
void launch_merge_many(const MergeJob* jobs, int count, cudaStream_t s)
{
    const size_t smem = sizeof(MergeSmem);
    ensure_smem((const void*)k_merge<kMergeBatchStacks>, smem);
    for (int first = 0; first < count; first += kMergeBatchStacks) {
        MergeBatch<kMergeBatchStacks> B;
        B.nstacks = count - first < kMergeBatchStacks ? count - first : kMergeBatchStacks;
        B.nitems = 0;
        for (int j = 0; j < B.nstacks; j++) {
            const MergeJob& J = jobs[first + j];
            B.st[j] = merge_stack(J.ref_y, J.ref_u, J.ref_v, J.w, J.h, J.nsrc, J.srcs, J.ssim_sigma,
                                  J.we_sigma, J.oy, J.ou, J.ov, nullptr);
            B.st[j].item_begin = B.nitems;
            B.nitems += B.st[j].tiles_x * ((J.h + kTile - 1) / kTile);
        }
        note_launch();
        k_merge<kMergeBatchStacks><<<merge_grid(B.nitems), 256, smem, s>>>(B);
    }
}

}  // namespace hdrreg
