// Row f1: error-tolerant exposure fusion (Sec. 2.5): the exposure fusion of Mertens et
// al. (2007) with the SSIM map of every registered source as a fourth weight.
//
// Weights (luma, per frame k): W_k = C_k * WE(Z_k) * Q_k + 1e-12 (C_k omitted when the
// contrast factor is off), C_k = |4 I - the 4 neighbours| of I = Z / 255 with replicated
// edges, WE(z) = exp(-(z/255 - 0.5)^2 / (2 sigma^2)), Q_k the SSIM map (1 for the
// reference); normalized over the frames. Chroma uses the 2x2 means of the normalized
// luma weights. Burt-Adelson pyramids: REDUCE filters with [1 4 6 4 1]/16 along x, then
// y (coordinates clamped) and keeps even samples; EXPAND interpolates (output 2k:
// (c[k-1] + 6 c[k] + c[k+1]) / 8, output 2k+1: (c[k] + c[k+1]) / 2, clamped), along x
// then y. Blend R^l = sum_k G{W_k}^l (G{I_k}^l - EXPAND(G{I_k}^{l+1})) (the top level
// without the EXPAND term), collapse O^l = R^l + EXPAND(O^{l+1}) in place, output 255 O.
//
// One thread per output pixel in every kernel (x from the block column, y = blockIdx.y);
// the planes of a level go in one launch (blockIdx.z = plane). All buffers live in the
// caller's workspace.
#include <math.h>

#include "hdrreg_internal.cuh"

namespace hdrreg {

namespace {

constexpr int kMaxPlanes = 16;

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// Level-0 luma weights of NF frames (frame 0 = the reference); the level-0 images are
// not stored: the later kernels read the frames themselves.
struct FuseL0 {
    const uint8_t* ref_y;
    const float* y[kMaxSources];
    const float* q[kMaxSources];
    float* gw[kMaxSources + 1];  // normalized weights
    int use_contrast;
    float we_k;  // 1 / (2 sigma^2)
};

// |4 z - (xl + xr) - (u + d)| / 255, the contrast of Sec. 2.5 in DN. On a linear ramp of a
// warped (FP32) frame the exact value is 0, and the weights are then normalized against the
// 1e-12 floor, so a plain FP32 evaluation (rounding error ~1e-5 DN) would decide them. The
// sum is therefore formed without error (Knuth's two-sum), the difference 4 z - hi is exact
// where it cancels (Sterbenz), and one rounding remains. For byte frames every step is exact
// in FP32 already.
__device__ __forceinline__ float two_sum(float a, float b, float& e)
{
    const float s = a + b, bb = s - a;
    e = (a - (s - bb)) + (b - bb);
    return s;
}

__device__ __forceinline__ float contrast_dn(float zc, float xl, float xr, float u, float d, bool exact)
{
    if (exact) return fabsf(fmaf(4.f, zc, -((xl + xr) + (u + d))));
    float e0, e1, e2;
    const float a = two_sum(xl, xr, e0), b = two_sum(u, d, e1);
    const float hi = two_sum(a, b, e2);
    const float lo = (e0 + e1) + e2;
    return fabsf(fmaf(4.f, zc, -hi) - lo);
}

template <typename T>
__device__ __forceinline__ float weight_of(const T* __restrict__ z, size_t i, int x, int y, int w,
                                           int h, const FuseL0& a)
{
    const float zc = (float)z[i];
    const float t = zc * (1.f / 255.f) - 0.5f;
    float wk = expf(-(t * t) * a.we_k);
    if (a.use_contrast) {
        const int xl = x > 0 ? x - 1 : 0, xr = x + 1 < w ? x + 1 : w - 1;
        const int yu = y > 0 ? y - 1 : 0, yd = y + 1 < h ? y + 1 : h - 1;
        const size_t r = (size_t)y * w;
        wk *= contrast_dn(zc, (float)z[r + xl], (float)z[r + xr], (float)z[(size_t)yu * w + x],
                          (float)z[(size_t)yd * w + x], sizeof(T) == 1) *
              (1.f / 255.f);
    }
    return wk;
}

template <int NF>
__global__ void __launch_bounds__(256) k_fuse_level0(FuseL0 a, int w, int h)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x < w) {
        const size_t i = (size_t)y * w + x;
        float wv[NF];
        wv[0] = weight_of(a.ref_y, i, x, y, w, h, a) + 1e-12f;
        float tot = wv[0];
#pragma unroll
        for (int f = 1; f < NF; f++) {
            wv[f] = weight_of(a.y[f - 1], i, x, y, w, h, a) * a.q[f - 1][i] + 1e-12f;
            tot += wv[f];
        }
        const float inv = 1.f / tot;
#pragma unroll
        for (int f = 0; f < NF; f++) a.gw[f][i] = wv[f] * inv;
    }
}

// The same weights for four consecutive pixels x4 .. x4 + 3 of row y (w a multiple of 4,
// rows 4-element aligned): vector loads of the row and of its neighbours, the left and
// right neighbours of the group as single loads; each pixel's arithmetic is weight_of's.
__device__ __forceinline__ void load4(const uint8_t* __restrict__ p, float (&v)[4])
{
    const uchar4 c = *reinterpret_cast<const uchar4*>(p);
    v[0] = (float)c.x;
    v[1] = (float)c.y;
    v[2] = (float)c.z;
    v[3] = (float)c.w;
}

__device__ __forceinline__ void load4(const float* __restrict__ p, float (&v)[4])
{
    const float4 c = *reinterpret_cast<const float4*>(p);
    v[0] = c.x;
    v[1] = c.y;
    v[2] = c.z;
    v[3] = c.w;
}

template <typename T>
__device__ __forceinline__ void weights4(const T* __restrict__ z, int x4, int y, int w, int h,
                                         const FuseL0& a, float (&wk)[4])
{
    const size_t r = (size_t)y * w;
    float c[4];
    load4(z + r + x4, c);
#pragma unroll
    for (int j = 0; j < 4; j++) {
        const float t = c[j] * (1.f / 255.f) - 0.5f;
        wk[j] = expf(-(t * t) * a.we_k);
    }
    if (a.use_contrast) {
        const int yu = y > 0 ? y - 1 : 0, yd = y + 1 < h ? y + 1 : h - 1;
        float u[4], d[4];
        load4(z + (size_t)yu * w + x4, u);
        load4(z + (size_t)yd * w + x4, d);
        const float lft = (float)z[r + (x4 > 0 ? x4 - 1 : 0)];
        const float rgt = (float)z[r + (x4 + 4 < w ? x4 + 4 : w - 1)];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const float xl = j == 0 ? lft : c[j - 1], xr = j == 3 ? rgt : c[j + 1];
            wk[j] *= contrast_dn(c[j], xl, xr, u[j], d[j], sizeof(T) == 1) * (1.f / 255.f);
        }
    }
}

template <int NF>
__global__ void __launch_bounds__(256) k_fuse_level0_v4(FuseL0 a, int w, int h)
{
    const int x4 = 4 * (blockIdx.x * blockDim.x + threadIdx.x), y = blockIdx.y;
    if (x4 >= w) return;
    const size_t i = (size_t)y * w + x4;
    float wv[NF][4], tot[4];
    weights4(a.ref_y, x4, y, w, h, a, wv[0]);
#pragma unroll
    for (int j = 0; j < 4; j++) {
        wv[0][j] = wv[0][j] + 1e-12f;
        tot[j] = wv[0][j];
    }
#pragma unroll
    for (int f = 1; f < NF; f++) {
        float q[4];
        weights4(a.y[f - 1], x4, y, w, h, a, wv[f]);
        load4(a.q[f - 1] + i, q);
#pragma unroll
        for (int j = 0; j < 4; j++) {
            wv[f][j] = wv[f][j] * q[j] + 1e-12f;
            tot[j] += wv[f][j];
        }
    }
    float inv[4];
#pragma unroll
    for (int j = 0; j < 4; j++) inv[j] = 1.f / tot[j];
#pragma unroll
    for (int f = 0; f < NF; f++)
        *reinterpret_cast<float4*>(a.gw[f] + i) =
            make_float4(wv[f][0] * inv[0], wv[f][1] * inv[1], wv[f][2] * inv[2], wv[f][3] * inv[3]);
}

// Level-0 chroma weights: 2x2 means of the normalized luma weights.
struct FuseC0 {
    const float* gw_luma[kMaxSources + 1];
    float* gw[kMaxSources + 1];
    int nf;
};

template <int NF>
__global__ void __launch_bounds__(256) k_fuse_chroma0(FuseC0 a, int w, int cw, int ch)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x < cw) {
        const size_t i = (size_t)y * cw + x;
        const size_t o = (size_t)(2 * y) * w + 2 * x;
#pragma unroll
        for (int f = 0; f < NF; f++) {
            const float* g = a.gw_luma[f];
            a.gw[f][i] = ((g[o] + g[o + 1]) + (g[o + w] + g[o + w + 1])) * 0.25f;
        }
    }
}

// REDUCE of every plane of a level: x first (five rows), then y. T = uint8_t reads a raw
// frame (value = (v + off) * scale), T = float a stored level (off 0, scale 1).
template <typename T>
struct PlaneSetT {
    const T* in[kMaxPlanes];
    float* out[kMaxPlanes];
};

// One thread per 2 x 2 block of outputs: the block's 7 x 7 input window is read once, each
// input row filtered along x for both output columns, then along y for both output rows
// (per output, the sums and their order are those of the one-output form).
template <typename T>
__global__ void __launch_bounds__(256) k_fuse_reduce(PlaneSetT<T> p, int wi, int hi, int wo, int ho,
                                                     float off, float scale)
{
    const float g[5] = {1.f / 16.f, 4.f / 16.f, 6.f / 16.f, 4.f / 16.f, 1.f / 16.f};
    const T* in = p.in[blockIdx.z];
    float* out = p.out[blockIdx.z];
    const int bx = blockIdx.x * blockDim.x + threadIdx.x, by = blockIdx.y;
    if (2 * bx >= wo) return;
    int xs[7];
#pragma unroll
    for (int j = 0; j < 7; j++) xs[j] = clampi(4 * bx + j - 2, 0, wi - 1);
    float s0[7], s1[7];  // row sums for output columns 2 bx and 2 bx + 1
#pragma unroll
    for (int rr = 0; rr < 7; rr++) {
        const T* row = in + (size_t)clampi(4 * by + rr - 2, 0, hi - 1) * wi;
        float v[7];
#pragma unroll
        for (int j = 0; j < 7; j++) v[j] = ((float)row[xs[j]] + off) * scale;
        float a = 0.f, b = 0.f;
#pragma unroll
        for (int j = 0; j < 5; j++) {
            a = fmaf(g[j], v[j], a);
            b = fmaf(g[j], v[j + 2], b);
        }
        s0[rr] = a;
        s1[rr] = b;
    }
#pragma unroll
    for (int dy = 0; dy < 2; dy++) {
        const int y = 2 * by + dy;
        if (y >= ho) break;
#pragma unroll
        for (int dx = 0; dx < 2; dx++) {
            const int x = 2 * bx + dx;
            if (x >= wo) break;
            float acc = 0.f;
#pragma unroll
            for (int r = 0; r < 5; r++) acc = fmaf(g[r], dx ? s1[r + 2 * dy] : s0[r + 2 * dy], acc);
            out[(size_t)y * wo + x] = acc;
        }
    }
}

// REDUCE of a stored plane at output pixel (x, y) (same arithmetic as k_fuse_reduce).
__device__ __forceinline__ float reduce_at(const float* __restrict__ in, int wi, int hi, int x, int y)
{
    const float g[5] = {1.f / 16.f, 4.f / 16.f, 6.f / 16.f, 4.f / 16.f, 1.f / 16.f};
    int xs[5];
#pragma unroll
    for (int j = 0; j < 5; j++) xs[j] = clampi(2 * x + j - 2, 0, wi - 1);
    float acc = 0.f;
#pragma unroll
    for (int r = 0; r < 5; r++) {
        const float* row = in + (size_t)clampi(2 * y + r - 2, 0, hi - 1) * wi;
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < 5; j++) s = fmaf(g[j], (row[xs[j]] + 0.f) * 1.f, s);
        acc = fmaf(g[r], s, acc);
    }
    return acc;
}

// EXPAND of the coarse plane c (wc x hc) at fine pixel (x, y): along x, then y.
__device__ __forceinline__ float expand_at(const float* __restrict__ c, int wc, int hc, int x, int y)
{
    const int kx = x >> 1, ky = y >> 1;
    auto row = [&](int r) {
        const float* cr = c + (size_t)clampi(r, 0, hc - 1) * wc;
        if (x & 1) return (cr[clampi(kx, 0, wc - 1)] + cr[clampi(kx + 1, 0, wc - 1)]) * 0.5f;
        return (cr[clampi(kx - 1, 0, wc - 1)] + 6.f * cr[clampi(kx, 0, wc - 1)] +
                cr[clampi(kx + 1, 0, wc - 1)]) * 0.125f;
    };
    if (y & 1) return (row(ky) + row(ky + 1)) * 0.5f;
    return (row(ky - 1) + 6.f * row(ky) + row(ky + 1)) * 0.125f;
}

// The 3 x 3 coarse neighbourhood (clamped) of coarse pixel (kx, ky), and EXPAND at the
// four fine pixels (2 kx + dx, 2 ky + dy) from it, e[dy][dx]: the same sums as expand_at,
// shared by the four pixels of a 2 x 2 block.
__device__ __forceinline__ void nbr3(const float* __restrict__ c, int wc, int hc, int kx, int ky,
                                     float (&n)[3][3])
{
    const int x0 = clampi(kx - 1, 0, wc - 1), x1 = clampi(kx, 0, wc - 1), x2 = clampi(kx + 1, 0, wc - 1);
#pragma unroll
    for (int r = 0; r < 3; r++) {
        const float* cr = c + (size_t)clampi(ky - 1 + r, 0, hc - 1) * wc;
        n[r][0] = cr[x0];
        n[r][1] = cr[x1];
        n[r][2] = cr[x2];
    }
}

__device__ __forceinline__ void expand4(const float (&n)[3][3], float (&e)[2][2])
{
    float ev[3], od[3];  // each coarse row interpolated to an even and to an odd fine x
#pragma unroll
    for (int r = 0; r < 3; r++) {
        ev[r] = (n[r][0] + 6.f * n[r][1] + n[r][2]) * 0.125f;
        od[r] = (n[r][1] + n[r][2]) * 0.5f;
    }
    e[0][0] = (ev[0] + 6.f * ev[1] + ev[2]) * 0.125f;
    e[0][1] = (od[0] + 6.f * od[1] + od[2]) * 0.125f;
    e[1][0] = (ev[1] + ev[2]) * 0.5f;
    e[1][1] = (od[1] + od[2]) * 0.5f;
}

// Launch grid of the 2 x 2-block kernels: one thread per block of a w x h level.
dim3 grid_blocks(int w, int h)
{
    const int bw = (w + 1) / 2, bh = (h + 1) / 2;
    return dim3((unsigned)((bw + 255) / 256), (unsigned)bh, 1u);
}

// The finest level in one pass: O^0 = sum_f W_f (I_f - EXPAND(I_f^1)) + EXPAND(O^1) with
// I_f read from the frames ((v + off) / 255); out = 255 O^0. Without a level 1 (single
// level) O^0 = sum_f W_f I_f.
struct FinalArgs {
    const uint8_t* ref;        // frame 0
    const float* src[kMaxSources];
    const float* gw[kMaxSources + 1];
    const float* gi1[kMaxSources + 1];  // level-1 images, or nullptr
    const float* o1;                    // level-1 output, or nullptr
    float* out;
    float off;
    int nf;
};

// One thread per 2 x 2 block of fine pixels: the EXPANDs of the block share one 3 x 3
// coarse neighbourhood per plane.
template <int NF>
__global__ void __launch_bounds__(256) k_fuse_final0(FinalArgs a, int w, int h, int wc, int hc)
{
    const int bx = blockIdx.x * blockDim.x + threadIdx.x, by = blockIdx.y;
    if (2 * bx >= w) return;
    float e[NF + 1][2][2];
#pragma unroll
    for (int f = 0; f <= NF; f++) {
        const float* c = f < NF ? a.gi1[f] : a.o1;
        if (c) {
            float n[3][3];
            nbr3(c, wc, hc, bx, by, n);
            expand4(n, e[f]);
        }
    }
#pragma unroll
    for (int dy = 0; dy < 2; dy++) {
        const int y = 2 * by + dy;
        if (y >= h) break;
#pragma unroll
        for (int dx = 0; dx < 2; dx++) {
            const int x = 2 * bx + dx;
            if (x >= w) break;
            const size_t i = (size_t)y * w + x;
            float acc = 0.f;
#pragma unroll
            for (int f = 0; f < NF; f++) {
                float v = ((f == 0 ? (float)a.ref[i] : a.src[f == 0 ? 0 : f - 1][i]) + a.off) *
                          (1.f / 255.f);
                if (a.gi1[f]) v -= e[f][dy][dx];
                acc = fmaf(a.gw[f][i], v, acc);
            }
            if (a.o1) acc += e[NF][dy][dx];
            a.out[i] = acc * 255.f;
        }
    }
}

struct BlendArgs {
    const float* gw[kMaxSources + 1];
    const float* gi[kMaxSources + 1];
    const float* gi_up[kMaxSources + 1];  // the next (coarser) level, or nullptr at the top
    float* r;
    int nf;
};

// One thread per 2 x 2 block (the EXPANDs share one coarse neighbourhood per frame).
__global__ void __launch_bounds__(256) k_fuse_blend(BlendArgs a, int w, int h, int wc, int hc)
{
    const int bx = blockIdx.x * blockDim.x + threadIdx.x, by = blockIdx.y;
    if (2 * bx >= w) return;
    float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
    for (int f = 0; f < a.nf; f++) {
        float e[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
        if (a.gi_up[f]) {
            float n[3][3];
            nbr3(a.gi_up[f], wc, hc, bx, by, n);
            expand4(n, e);
        }
#pragma unroll
        for (int dy = 0; dy < 2; dy++) {
            const int y = 2 * by + dy;
            if (y >= h) break;
#pragma unroll
            for (int dx = 0; dx < 2; dx++) {
                const int x = 2 * bx + dx;
                if (x >= w) break;
                const size_t i = (size_t)y * w + x;
                float lap = a.gi[f][i];
                if (a.gi_up[f]) lap -= e[dy][dx];
                acc[dy][dx] = fmaf(a.gw[f][i], lap, acc[dy][dx]);
            }
        }
    }
#pragma unroll
    for (int dy = 0; dy < 2; dy++) {
        const int y = 2 * by + dy;
        if (y >= h) break;
#pragma unroll
        for (int dx = 0; dx < 2; dx++) {
            const int x = 2 * bx + dx;
            if (x >= w) break;
            a.r[(size_t)y * w + x] = acc[dy][dx];
        }
    }
}

// O^l = R^l + EXPAND(O^{l+1}) (up = nullptr: O = R), in place in r; the finest level is
// written scaled to out.
__global__ void __launch_bounds__(256) k_fuse_collapse(float* __restrict__ r,
                                                       const float* __restrict__ up, int w, int h,
                                                       int wc, int hc, float* __restrict__ out,
                                                       float scale)
{
    const int bx = blockIdx.x * blockDim.x + threadIdx.x, by = blockIdx.y;
    if (2 * bx >= w) return;
    float e[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
    if (up) {
        float n[3][3];
        nbr3(up, wc, hc, bx, by, n);
        expand4(n, e);
    }
#pragma unroll
    for (int dy = 0; dy < 2; dy++) {
        const int y = 2 * by + dy;
        if (y >= h) break;
#pragma unroll
        for (int dx = 0; dx < 2; dx++) {
            const int x = 2 * bx + dx;
            if (x >= w) break;
            const size_t i = (size_t)y * w + x;
            const float o = up ? r[i] + e[dy][dx] : r[i];
            if (out) out[i] = o * scale;
            else r[i] = o;
        }
    }
}

// Pyramid sizes: level l is ceil(w / 2^l) x ceil(h / 2^l).
constexpr int kMaxLv = 24;
struct PyrDev {
    int L;
    int W[kMaxLv], Hh[kMaxLv];
    size_t off[kMaxLv];
};

// Every level from Lc up in one CTA (the coarse levels are a few thousand pixels): the
// remaining REDUCEs of the image and weight pyramids, the blends, and the collapse down
// to level Lc (left in r at level Lc). Same arithmetic as the per-level kernels.
struct CoarseArgs {
    PyrDev P;
    float* img[3 * (kMaxSources + 1)];  // nf * nref image pyramids (frame-major)
    float* wts[kMaxSources + 1];
    float* r[2];                        // nref result pyramids
    int nf, nref, Lc;
};

__global__ void __launch_bounds__(1024) k_fuse_coarse(CoarseArgs a)
{
    const PyrDev& P = a.P;
    const int nimg = a.nf * a.nref;
    for (int l = a.Lc; l + 1 < P.L; l++) {  // REDUCE l -> l + 1, all planes
        const int wo = P.W[l + 1], ho = P.Hh[l + 1], n = wo * ho;
        for (int e = threadIdx.x; e < (nimg + a.nf) * n; e += blockDim.x) {
            const int pl = e / n, i = e - pl * n, x = i % wo, y = i / wo;
            float* base = pl < nimg ? a.img[pl] : a.wts[pl - nimg];
            base[P.off[l + 1] + i] = reduce_at(base + P.off[l], P.W[l], P.Hh[l], x, y);
        }
        __syncthreads();
    }
    for (int l = a.Lc; l < P.L; l++) {  // blends
        const int w = P.W[l], h = P.Hh[l], n = w * h;
        const bool top = l + 1 >= P.L;
        const int wc = top ? 1 : P.W[l + 1], hc = top ? 1 : P.Hh[l + 1];
        for (int e = threadIdx.x; e < a.nref * n; e += blockDim.x) {
            const int j = e / n, i = e - j * n, x = i % w, y = i / w;
            float acc = 0.f;
            for (int f = 0; f < a.nf; f++) {
                const float* g = a.img[f * a.nref + j];
                float lap = g[P.off[l] + i];
                if (!top) lap -= expand_at(g + P.off[l + 1], wc, hc, x, y);
                acc = fmaf(a.wts[f][P.off[l] + i], lap, acc);
            }
            a.r[j][P.off[l] + i] = acc;
        }
    }
    __syncthreads();
    for (int l = P.L - 2; l >= a.Lc; l--) {  // collapse down to Lc
        const int w = P.W[l], h = P.Hh[l], n = w * h;
        for (int e = threadIdx.x; e < a.nref * n; e += blockDim.x) {
            const int j = e / n, i = e - j * n, x = i % w, y = i / w;
            float* r = a.r[j];
            r[P.off[l] + i] += expand_at(r + P.off[l + 1], P.W[l + 1], P.Hh[l + 1], x, y);
        }
        __syncthreads();
    }
}

dim3 grid2(int w, int h, int z = 1) { return dim3((unsigned)((w + 255) / 256), (unsigned)h, (unsigned)z); }

int fuse_levels(int w, int h)
{
    int m = w < h ? w : h, l = 0;
    while ((2 << l) <= m) l++;  // floor(log2(m))
    return l > 0 ? l : 1;
}

constexpr int kCoarsePixels = 2048;  // levels at most this size go to k_fuse_coarse

struct Pyr {
    int L, Lc;  // levels; the first level handled by k_fuse_coarse
    int W[kMaxLv], Hh[kMaxLv];
    size_t off[kMaxLv], total;  // floats per plane pyramid, offset of each level
    Pyr(int w, int h)
    {
        L = fuse_levels(w, h);
        total = 0;
        for (int l = 0; l < L; l++) {
            W[l] = l == 0 ? w : (W[l - 1] + 1) / 2;
            Hh[l] = l == 0 ? h : (Hh[l - 1] + 1) / 2;
            off[l] = total;
            total += align_up((size_t)W[l] * Hh[l], 64);
        }
        Lc = L;  // level 0 is always the per-level kernels' (the frames are read there)
        for (int l = 1; l < L; l++)
            if ((long long)W[l] * Hh[l] <= kCoarsePixels) {
                Lc = l;
                break;
            }
    }
    PyrDev dev() const
    {
        PyrDev d{};
        d.L = L;
        for (int l = 0; l < L; l++) {
            d.W[l] = W[l];
            d.Hh[l] = Hh[l];
            d.off[l] = off[l];
        }
        return d;
    }
};

}  // namespace

size_t fuse_ws_bytes(int w, int h, int nf, bool chroma)
{
    const Pyr pl(w, h);
    size_t n = (size_t)(2 * nf + 1) * pl.total;
    if (chroma) {
        const Pyr pc(w / 2, h / 2);
        n += (size_t)(3 * nf + 2) * pc.total;
    }
    return n * 4 + 256;
}

// Blend levels 1..L-1 and collapse them to level 1 (gi, gw: pyramids whose level 0 holds
// the weights only), then the finest level in one pass from the frames.
static void blend_channel(const Pyr& P, int nf, float* const* gi, float* const* gw, float* r,
                          const uint8_t* ref, const float* const* src, float off, float* out,
                          cudaStream_t s)
{
    // levels Lc.. are already blended and collapsed (k_fuse_coarse)
    for (int l = 1; l < P.Lc; l++) {
        BlendArgs b{};
        b.nf = nf;
        for (int f = 0; f < nf; f++) {
            b.gw[f] = gw[f] + P.off[l];
            b.gi[f] = gi[f] + P.off[l];
            b.gi_up[f] = l + 1 < P.L ? gi[f] + P.off[l + 1] : nullptr;
        }
        b.r = r + P.off[l];
        const int wc = l + 1 < P.L ? P.W[l + 1] : 1, hc = l + 1 < P.L ? P.Hh[l + 1] : 1;
        note_launch();
        k_fuse_blend<<<grid_blocks(P.W[l], P.Hh[l]), 256, 0, s>>>(b, P.W[l], P.Hh[l], wc, hc);
    }
    for (int l = (P.Lc < P.L ? P.Lc : P.L) - 1 - (P.Lc < P.L ? 0 : 1); l >= 1; l--) {
        note_launch();
        k_fuse_collapse<<<grid_blocks(P.W[l], P.Hh[l]), 256, 0, s>>>(
            r + P.off[l], r + P.off[l + 1], P.W[l], P.Hh[l], P.W[l + 1], P.Hh[l + 1], nullptr, 1.f);
    }
    FinalArgs fa{};
    fa.ref = ref;
    fa.nf = nf;
    fa.off = off;
    fa.out = out;
    fa.o1 = P.L > 1 ? r + P.off[1] : nullptr;
    for (int f = 0; f < nf; f++) {
        fa.gw[f] = gw[f];
        fa.gi1[f] = P.L > 1 ? gi[f] + P.off[1] : nullptr;
        if (f > 0) fa.src[f - 1] = src[f - 1];
    }
    const dim3 g = grid_blocks(P.W[0], P.Hh[0]);
    const int wc = P.L > 1 ? P.W[1] : 1, hc = P.L > 1 ? P.Hh[1] : 1;
    note_launch();
    switch (nf) {
    case 2: k_fuse_final0<2><<<g, 256, 0, s>>>(fa, P.W[0], P.Hh[0], wc, hc); break;
    case 3: k_fuse_final0<3><<<g, 256, 0, s>>>(fa, P.W[0], P.Hh[0], wc, hc); break;
    case 4: k_fuse_final0<4><<<g, 256, 0, s>>>(fa, P.W[0], P.Hh[0], wc, hc); break;
    default: k_fuse_final0<5><<<g, 256, 0, s>>>(fa, P.W[0], P.Hh[0], wc, hc); break;
    }
}

template <typename T>
static void reduce_planes(const Pyr& P, int l, const T* const* in, float* const* out, int np,
                          float off, float scale, cudaStream_t s)
{
    for (int b = 0; b < np; b += kMaxPlanes) {
        const int cnt = np - b < kMaxPlanes ? np - b : kMaxPlanes;
        PlaneSetT<T> ps{};
        for (int k = 0; k < cnt; k++) {
            ps.in[k] = in[b + k];
            ps.out[k] = out[b + k];
        }
        note_launch();
        dim3 g = grid_blocks(P.W[l + 1], P.Hh[l + 1]);
        g.z = (unsigned)cnt;
        k_fuse_reduce<T><<<g, 256, 0, s>>>(
            ps, P.W[l], P.Hh[l], P.W[l + 1], P.Hh[l + 1], off, scale);
    }
}

// Level 1 of the images from the frames, then every stored pyramid level by level.
static void build_pyramids(const Pyr& P, int nf, const uint8_t* const* ref_planes, int nref,
                           const float* const* src_planes, float* const* img, float* const* wts,
                           float off, cudaStream_t s)
{
    if (P.L < 2) return;
    float* o1[3 * (kMaxSources + 1)];
    // images: planes per frame are consecutive in img (frame-major, nref planes per frame)
    for (int k = 0; k < nref; k++) o1[k] = img[k] + P.off[1];
    reduce_planes<uint8_t>(P, 0, ref_planes, o1, nref, off, 1.f / 255.f, s);
    const int nsp = (nf - 1) * nref;
    for (int k = 0; k < nsp; k++) o1[k] = img[nref + k] + P.off[1];
    reduce_planes<float>(P, 0, src_planes, o1, nsp, off, 1.f / 255.f, s);
    const float* wi[kMaxSources + 1];
    float* wo[kMaxSources + 1];
    for (int f = 0; f < nf; f++) {
        wi[f] = wts[f];
        wo[f] = wts[f] + P.off[1];
    }
    reduce_planes<float>(P, 0, wi, wo, nf, 0.f, 1.f, s);
    const int np = nf * nref + nf;
    for (int l = 1; l + 1 < P.L && l < P.Lc; l++) {
        const float* in[3 * (kMaxSources + 1) + kMaxSources + 1];
        float* out[3 * (kMaxSources + 1) + kMaxSources + 1];
        for (int k = 0; k < nf * nref; k++) {
            in[k] = img[k] + P.off[l];
            out[k] = img[k] + P.off[l + 1];
        }
        for (int f = 0; f < nf; f++) {
            in[nf * nref + f] = wts[f] + P.off[l];
            out[nf * nref + f] = wts[f] + P.off[l + 1];
        }
        reduce_planes<float>(P, l, in, out, np, 0.f, 1.f, s);
    }
}

// The coarse levels of one channel group (nref result pyramids r) in one CTA.
static void coarse_levels(const Pyr& P, int nf, int nref, float* const* img, float* const* wts,
                          float* const* r, cudaStream_t s)
{
    if (P.Lc >= P.L) return;
    CoarseArgs c{};
    c.P = P.dev();
    c.nf = nf;
    c.nref = nref;
    c.Lc = P.Lc;
    for (int k = 0; k < nf * nref; k++) c.img[k] = img[k];
    for (int f = 0; f < nf; f++) c.wts[f] = wts[f];
    for (int j = 0; j < nref; j++) c.r[j] = r[j];
    note_launch();
    k_fuse_coarse<<<1, 1024, 0, s>>>(c);
}

void launch_fuse(const uint8_t* ref_y, const uint8_t* ref_u, const uint8_t* ref_v, int w, int h,
                 int nsrc, const FuseSrcDev* srcs, int use_contrast, double we_sigma, float* oy,
                 float* ou, float* ov, void* ws, cudaStream_t s)
{
    const int nf = nsrc + 1;
    const bool chroma = ref_u && ref_v && ou && ov;
    const Pyr pl(w, h);
    float* base = static_cast<float*>(ws);
    float* gw[kMaxSources + 1];
    float* gi[kMaxSources + 1];
    for (int f = 0; f < nf; f++) {
        gw[f] = base + (size_t)f * pl.total;
        gi[f] = base + (size_t)(nf + f) * pl.total;
    }
    float* rl = base + (size_t)(2 * nf) * pl.total;
    FuseL0 a{};
    a.ref_y = ref_y;
    a.use_contrast = use_contrast;
    a.we_k = (float)(1.0 / (2.0 * we_sigma * we_sigma));
    const float* sy[kMaxSources];
    for (int k = 0; k < nsrc; k++) {
        a.y[k] = srcs[k].y;
        a.q[k] = srcs[k].q;
        sy[k] = srcs[k].y;
    }
    for (int f = 0; f < nf; f++) a.gw[f] = gw[f];
    // four pixels per thread where every row of every plane starts 16-byte aligned (4 for
    // the reference bytes)
    bool v4 = (w % 4) == 0 && ((uintptr_t)ref_y % 4) == 0;
    for (int k = 0; k < nsrc; k++)
        v4 = v4 && ((uintptr_t)a.y[k] % 16) == 0 && ((uintptr_t)a.q[k] % 16) == 0;
    for (int f = 0; f < nf; f++) v4 = v4 && ((uintptr_t)a.gw[f] % 16) == 0;
    note_launch();
    if (v4) {
        const dim3 g((unsigned)((w / 4 + 255) / 256), (unsigned)h);
        switch (nf) {
        case 2: k_fuse_level0_v4<2><<<g, 256, 0, s>>>(a, w, h); break;
        case 3: k_fuse_level0_v4<3><<<g, 256, 0, s>>>(a, w, h); break;
        case 4: k_fuse_level0_v4<4><<<g, 256, 0, s>>>(a, w, h); break;
        default: k_fuse_level0_v4<5><<<g, 256, 0, s>>>(a, w, h); break;
        }
    } else {
        switch (nf) {
        case 2: k_fuse_level0<2><<<grid2(w, h), 256, 0, s>>>(a, w, h); break;
        case 3: k_fuse_level0<3><<<grid2(w, h), 256, 0, s>>>(a, w, h); break;
        case 4: k_fuse_level0<4><<<grid2(w, h), 256, 0, s>>>(a, w, h); break;
        default: k_fuse_level0<5><<<grid2(w, h), 256, 0, s>>>(a, w, h); break;
        }
    }
    const uint8_t* ry[1] = {ref_y};
    build_pyramids(pl, nf, ry, 1, sy, gi, gw, 0.f, s);
    coarse_levels(pl, nf, 1, gi, gw, &rl, s);
    blend_channel(pl, nf, gi, gw, rl, ref_y, sy, 0.f, oy, s);
    if (!chroma) return;
    const int cw = w / 2, ch = h / 2;
    const Pyr pc(cw, ch);
    float* cbase = rl + pl.total;
    float* cw_[kMaxSources + 1];
    float* cimg[2 * (kMaxSources + 1)];  // frame-major: (u, v) of frame 0, then of frame 1 ...
    for (int f = 0; f < nf; f++) {
        cw_[f] = cbase + (size_t)f * pc.total;
        cimg[2 * f] = cbase + (size_t)(nf + 2 * f) * pc.total;
        cimg[2 * f + 1] = cbase + (size_t)(nf + 2 * f + 1) * pc.total;
    }
    float* ru = cbase + (size_t)(3 * nf) * pc.total;
    float* rv = ru + pc.total;
    FuseC0 c{};
    c.nf = nf;
    for (int f = 0; f < nf; f++) {
        c.gw_luma[f] = gw[f];
        c.gw[f] = cw_[f];
    }
    note_launch();
    switch (nf) {
    case 2: k_fuse_chroma0<2><<<grid2(cw, ch), 256, 0, s>>>(c, w, cw, ch); break;
    case 3: k_fuse_chroma0<3><<<grid2(cw, ch), 256, 0, s>>>(c, w, cw, ch); break;
    case 4: k_fuse_chroma0<4><<<grid2(cw, ch), 256, 0, s>>>(c, w, cw, ch); break;
    default: k_fuse_chroma0<5><<<grid2(cw, ch), 256, 0, s>>>(c, w, cw, ch); break;
    }
    const uint8_t* ruv[2] = {ref_u, ref_v};
    const float* suv[2 * kMaxSources];
    const float* su[kMaxSources];
    const float* sv[kMaxSources];
    for (int k = 0; k < nsrc; k++) {
        suv[2 * k] = srcs[k].u;
        suv[2 * k + 1] = srcs[k].v;
        su[k] = srcs[k].u;
        sv[k] = srcs[k].v;
    }
    build_pyramids(pc, nf, ruv, 2, suv, cimg, cw_, -128.f, s);
    float* ruv_r[2] = {ru, rv};
    coarse_levels(pc, nf, 2, cimg, cw_, ruv_r, s);
    float* cu_[kMaxSources + 1];
    float* cv_[kMaxSources + 1];
    for (int f = 0; f < nf; f++) {
        cu_[f] = cimg[2 * f];
        cv_[f] = cimg[2 * f + 1];
    }
    blend_channel(pc, nf, cu_, cw_, ru, ref_u, su, -128.f, ou, s);
    blend_channel(pc, nf, cv_, cw_, rv, ref_v, sv, -128.f, ov, s);
}

}  // namespace hdrreg
