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
        const float s = ((float)z[r + xl] + (float)z[r + xr]) +
                        ((float)z[(size_t)yu * w + x] + (float)z[(size_t)yd * w + x]);
        wk *= fabsf(fmaf(4.f, zc, -s)) * (1.f / 255.f);
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

template <typename T>
__global__ void __launch_bounds__(256) k_fuse_reduce(PlaneSetT<T> p, int wi, int hi, int wo, int ho,
                                                     float off, float scale)
{
    const float g[5] = {1.f / 16.f, 4.f / 16.f, 6.f / 16.f, 4.f / 16.f, 1.f / 16.f};
    const T* in = p.in[blockIdx.z];
    float* out = p.out[blockIdx.z];
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x < wo) {
        const size_t i = (size_t)y * wo + x;
        int xs[5];
#pragma unroll
        for (int j = 0; j < 5; j++) xs[j] = clampi(2 * x + j - 2, 0, wi - 1);
        float acc = 0.f;
#pragma unroll
        for (int r = 0; r < 5; r++) {
            const T* row = in + (size_t)clampi(2 * y + r - 2, 0, hi - 1) * wi;
            float s = 0.f;
#pragma unroll
            for (int j = 0; j < 5; j++) s = fmaf(g[j], ((float)row[xs[j]] + off) * scale, s);
            acc = fmaf(g[r], s, acc);
        }
        out[i] = acc;
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

template <int NF>
__global__ void __launch_bounds__(256) k_fuse_final0(FinalArgs a, int w, int h, int wc, int hc)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x < w) {
        const size_t i = (size_t)y * w + x;
        float acc = 0.f;
#pragma unroll
        for (int f = 0; f < NF; f++) {
            float v = ((f == 0 ? (float)a.ref[i] : a.src[f == 0 ? 0 : f - 1][i]) + a.off) *
                      (1.f / 255.f);
            if (a.gi1[f]) v -= expand_at(a.gi1[f], wc, hc, x, y);
            acc = fmaf(a.gw[f][i], v, acc);
        }
        if (a.o1) acc += expand_at(a.o1, wc, hc, x, y);
        a.out[i] = acc * 255.f;
    }
}

struct BlendArgs {
    const float* gw[kMaxSources + 1];
    const float* gi[kMaxSources + 1];
    const float* gi_up[kMaxSources + 1];  // the next (coarser) level, or nullptr at the top
    float* r;
    int nf;
};

__global__ void __launch_bounds__(256) k_fuse_blend(BlendArgs a, int w, int h, int wc, int hc)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x < w) {
        const size_t i = (size_t)y * w + x;
        float acc = 0.f;
        for (int f = 0; f < a.nf; f++) {
            float lap = a.gi[f][i];
            if (a.gi_up[f]) lap -= expand_at(a.gi_up[f], wc, hc, x, y);
            acc = fmaf(a.gw[f][i], lap, acc);
        }
        a.r[i] = acc;
    }
}

// O^l = R^l + EXPAND(O^{l+1}) (up = nullptr: O = R), in place in r; the finest level is
// written scaled to out.
__global__ void __launch_bounds__(256) k_fuse_collapse(float* __restrict__ r,
                                                       const float* __restrict__ up, int w, int h,
                                                       int wc, int hc, float* __restrict__ out,
                                                       float scale)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x < w) {
        const size_t i = (size_t)y * w + x;
        const float o = up ? r[i] + expand_at(up, wc, hc, x, y) : r[i];
        if (out) out[i] = o * scale;
        else r[i] = o;
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
        k_fuse_blend<<<grid2(P.W[l], P.Hh[l]), 256, 0, s>>>(b, P.W[l], P.Hh[l], wc, hc);
    }
    for (int l = (P.Lc < P.L ? P.Lc : P.L) - 1 - (P.Lc < P.L ? 0 : 1); l >= 1; l--) {
        note_launch();
        k_fuse_collapse<<<grid2(P.W[l], P.Hh[l]), 256, 0, s>>>(
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
    const dim3 g = grid2(P.W[0], P.Hh[0]);
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
        k_fuse_reduce<T><<<grid2(P.W[l + 1], P.Hh[l + 1], cnt), 256, 0, s>>>(
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
    note_launch();
    switch (nf) {
    case 2: k_fuse_level0<2><<<grid2(w, h), 256, 0, s>>>(a, w, h); break;
    case 3: k_fuse_level0<3><<<grid2(w, h), 256, 0, s>>>(a, w, h); break;
    case 4: k_fuse_level0<4><<<grid2(w, h), 256, 0, s>>>(a, w, h); break;
    default: k_fuse_level0<5><<<grid2(w, h), 256, 0, s>>>(a, w, h); break;
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
