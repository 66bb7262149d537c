// Row a-L: the learned tile-displacement predictor -- forward pass, backward pass,
// masked mean-squared loss and Adam, with every convolution on the tensor cores.
//
// Network (NHWC, bf16 storage, FP32 accumulation): a fixed feature stage (the two
// inputs a, b and a local SSD cost volume -(a(p) - b(p + o))^2, o in [-2, 2]^2: 27
// channels), then eight 3x3 convolutions with zero padding 1 -- 27->16, 16->16, 16->32
// (stride 2), 32->32, 32->48 (stride 2), 48->48, 48->64 (stride 2), 64->64 -- each with
// bias and ReLU, then a 1x1 head 64->2 (bias, no activation). Parameters: one FP32 vector, per layer W[cout][ky][kx][cin] then
// b[cout]. A convolution is the product im2col(x) [M x 9 cin] * W^T (gemm_tc.cu); the
// data gradient is dY * W gathered back by col2im; the weight gradient is
// im2col(x)^T * dY over all M output pixels (K split across CTAs, partial sums added
// in a fixed order so results are deterministic).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <utility>

#include "hdrreg_internal.cuh"

namespace hdrreg {

namespace {

struct LayerSpec {
    int cin, cout, k, stride, relu;
};
constexpr int kNL = 9;
constexpr int kCorr = 2;                                   // cost-volume offsets [-2, 2]^2
constexpr int kFeat = 2 + (2 * kCorr + 1) * (2 * kCorr + 1);  // 27 feature channels
constexpr LayerSpec kNet[kNL] = {{kFeat, 16, 3, 1, 1}, {16, 16, 3, 1, 1}, {16, 32, 3, 2, 1},
                                 {32, 32, 3, 1, 1}, {32, 48, 3, 2, 1}, {48, 48, 3, 1, 1},
                                 {48, 64, 3, 2, 1}, {64, 64, 3, 1, 1}, {64, 2, 1, 1, 0}};

int round_up(int v, int m) { return (v + m - 1) / m * m; }
int kdim(const LayerSpec& L) { return L.k * L.k * L.cin; }
int kpad(const LayerSpec& L) { return round_up(kdim(L), 8); }
int cpad(const LayerSpec& L) { return round_up(L.cout, 16); }
int osz(int n, const LayerSpec& L) { return (n + 2 * (L.k / 2) - L.k) / L.stride + 1; }

// ------------------------------------------------------------------ kernels
// Fixed feature stage: per pixel a, b and -(a(p) - b(p + o))^2 for o = (u, v) in
// [-2, 2]^2 (row-major in v, then u; b = 0 outside). With bfloat16 inputs in [-1, 1] the
// difference and its square are exact in FP32, so only the final rounding to bfloat16
// remains. Grid: x over columns, y over rows, z over images.
__global__ void k_features(const __nv_bfloat162* __restrict__ x, int h, int w,
                           __nv_bfloat16* __restrict__ f)
{
    const int xx = blockIdx.x * blockDim.x + threadIdx.x, yy = blockIdx.y, b = blockIdx.z;
    if (xx >= w) return;
    const __nv_bfloat162* img = x + (size_t)b * h * w;
    const float2 ab = __bfloat1622float2(img[(size_t)yy * w + xx]);
    __nv_bfloat16* o = f + ((size_t)b * h * w + (size_t)yy * w + xx) * kFeat;
    o[0] = __float2bfloat16_rn(ab.x);
    o[1] = __float2bfloat16_rn(ab.y);
    int c = 2;
#pragma unroll
    for (int v = -kCorr; v <= kCorr; v++) {
        const int ys = yy + v;
        const bool rin = ys >= 0 && ys < h;
#pragma unroll
        for (int u = -kCorr; u <= kCorr; u++, c++) {
            const int xs = xx + u;
            const float bb = (rin && xs >= 0 && xs < w) ? __high2float(img[(size_t)ys * w + xs]) : 0.f;
            const float d = ab.x - bb;
            o[c] = __float2bfloat16_rn(-(d * d));
        }
    }
}

// The same features with the channels padded to 32 (27..31 zero): one 64-byte pixel,
// written as four 16-byte vectors (the layout the implicit-GEMM convolution gathers).
constexpr int kFeatPad = 32;
__global__ void k_features32(const __nv_bfloat162* __restrict__ x, int h, int w,
                             __nv_bfloat16* __restrict__ f)
{
    const int xx = blockIdx.x * blockDim.x + threadIdx.x, yy = blockIdx.y, b = blockIdx.z;
    if (xx >= w) return;
    const __nv_bfloat162* img = x + (size_t)b * h * w;
    const float2 ab = __bfloat1622float2(img[(size_t)yy * w + xx]);
    float v[kFeatPad];
    v[0] = ab.x;
    v[1] = ab.y;
    int c = 2;
#pragma unroll
    for (int dv = -kCorr; dv <= kCorr; dv++) {
        const int ys = yy + dv;
        const bool rin = ys >= 0 && ys < h;
#pragma unroll
        for (int u = -kCorr; u <= kCorr; u++, c++) {
            const int xs = xx + u;
            const float bb = (rin && xs >= 0 && xs < w) ? __high2float(img[(size_t)ys * w + xs]) : 0.f;
            const float d = ab.x - bb;
            v[c] = -(d * d);
        }
    }
#pragma unroll
    for (int k = kFeat; k < kFeatPad; k++) v[k] = 0.f;
    uint4* o = reinterpret_cast<uint4*>(f + ((size_t)b * h * w + (size_t)yy * w + xx) * kFeatPad);
#pragma unroll
    for (int q = 0; q < kFeatPad / 8; q++) {
        uint32_t p[4];
#pragma unroll
        for (int e = 0; e < 4; e++) {
            const __nv_bfloat162 t = __floats2bfloat162_rn(v[8 * q + 2 * e], v[8 * q + 2 * e + 1]);
            p[e] = *reinterpret_cast<const uint32_t*>(&t);
        }
        o[q] = make_uint4(p[0], p[1], p[2], p[3]);
    }
}

// The 1x1 head: out[m][o] = b[o] + sum_c bf16(W[o][c]) act[m][c], o = 0, 1 (FP32 sums).
__global__ void k_head(const __nv_bfloat16* __restrict__ act, long long M, const float* __restrict__ W,
                       const float* __restrict__ bias, float* __restrict__ out)
{
    constexpr int C = 64;
    __shared__ float ws[2 * C];
    if (threadIdx.x < 2 * C) ws[threadIdx.x] = __bfloat162float(__float2bfloat16_rn(W[threadIdx.x]));
    __syncthreads();
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < M;
         m += (long long)gridDim.x * blockDim.x) {
        const uint4* a = reinterpret_cast<const uint4*>(act + m * C);
        float s0 = 0.f, s1 = 0.f;
#pragma unroll
        for (int q = 0; q < C / 8; q++) {
            const uint4 u = a[q];
            const uint32_t wds[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&wds[e]));
                const int c = 8 * q + 2 * e;
                s0 = fmaf(f.x, ws[c], s0);
                s0 = fmaf(f.y, ws[c + 1], s0);
                s1 = fmaf(f.x, ws[C + c], s1);
                s1 = fmaf(f.y, ws[C + c + 1], s1);
            }
        }
        out[2 * m] = s0 + bias[0];
        out[2 * m + 1] = s1 + bias[1];
    }
}

// col[m][k] for output pixel m = (b, i, j) and k = (ky * K + kx) * cin + ci: the input
// value at (s i + ky - p, s j + kx - p, ci), 0 outside the image and for k >= K*K*cin.
// One thread per (output pixel, tap) copies the tap's cin contiguous channels (16-byte
// vectors when cin is a multiple of 8); the thread of the last tap also zeroes the K tail.
// Block (16, 16): x = tap (<= 16 taps), y = one of 16 output pixels.
__global__ void k_im2col(const __nv_bfloat16* __restrict__ x, int h, int w, int cin, int ksz,
                         int stride, int ho, int wo, int kp, int Mtot,
                         __nv_bfloat16* __restrict__ col)
{
    const int taps = ksz * ksz, pad = ksz / 2;
    const int m = blockIdx.x * blockDim.y + threadIdx.y;
    const int tap = threadIdx.x;
    if (m >= Mtot || tap >= taps) return;
    const int j = m % wo, t = m / wo, i = t % ho, b = t / ho;
    const int ky = tap / ksz, kx = tap - ky * ksz;
    const int yy = stride * i + ky - pad, xx = stride * j + kx - pad;
    __nv_bfloat16* dst = col + (size_t)m * kp + tap * cin;
    const bool in = yy >= 0 && yy < h && xx >= 0 && xx < w;
    const __nv_bfloat16* src = x + (((size_t)b * h + (in ? yy : 0)) * w + (in ? xx : 0)) * cin;
    if ((cin & 7) == 0 && (kp & 7) == 0) {
        const uint4 z = make_uint4(0, 0, 0, 0);
        for (int c = 0; c < cin; c += 8)
            *reinterpret_cast<uint4*>(dst + c) = in ? *reinterpret_cast<const uint4*>(src + c) : z;
    } else {
        const __nv_bfloat16 z = __float2bfloat16_rn(0.f);
        for (int c = 0; c < cin; c++) dst[c] = in ? src[c] : z;
    }
    if (tap == taps - 1)
        for (int k = taps * cin; k < kp; k++) col[(size_t)m * kp + k] = __float2bfloat16_rn(0.f);
}

// out[c][r] = in[r][c] for an R x C bf16 matrix (row strides ld_in, ld_out); 32 x 32 tiles.
__global__ void k_transpose_bf16(const __nv_bfloat16* __restrict__ in, int R, int Cc, int ld_in,
                                 __nv_bfloat16* __restrict__ out, int ld_out)
{
    __shared__ __nv_bfloat16 t[32][33];
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int r = r0 + k, c = c0 + threadIdx.x;
        t[k][threadIdx.x] = (r < R && c < Cc) ? in[(long long)r * ld_in + c] : __float2bfloat16_rn(0.f);
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int c = c0 + k, r = r0 + threadIdx.x;
        if (c < Cc && r < R) out[(long long)c * ld_out + r] = t[threadIdx.x][k];
    }
}

// Parameters -> GEMM operands: Wb[co][k] (k = (ky, kx, ci), zero past K and past cout) and
// Wt[k][co] (co padded to cp).
__global__ void k_pack_weights(const float* __restrict__ W, int cout, int K, int kp, int cp,
                               __nv_bfloat16* __restrict__ Wb, __nv_bfloat16* __restrict__ Wt)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < cp * kp; e += gridDim.x * blockDim.x) {
        const int co = e / kp, k = e % kp;
        const float v = (co < cout && k < K) ? W[(size_t)co * K + k] : 0.f;
        Wb[e] = __float2bfloat16_rn(v);
        if (k < K) Wt[(size_t)k * cp + co] = __float2bfloat16_rn(v);
    }
}

// dx[b, y, x, ci] = sum over taps (ky, kx) with an output pixel (i, j) that read (y, x):
// s i + ky - p = y, s j + kx - p = x; then times the ReLU mask of the previous layer's
// output (act > 0) and rounded to bf16 (the next output gradient).
__global__ void k_col2im_mask(const float* __restrict__ dcol, int n, int h, int w, int cin,
                              int ksz, int stride, int ho, int wo,
                              const __nv_bfloat16* __restrict__ act, __nv_bfloat16* __restrict__ dy)
{
    const long long total = (long long)n * h * w * cin;
    const int pad = ksz / 2, K = ksz * ksz * cin;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int ci = (int)(e % cin);
        const long long p = e / cin;
        const int xx = (int)(p % w), yy = (int)((p / w) % h), b = (int)(p / ((long long)w * h));
        float acc = 0.f;
        for (int ky = 0; ky < ksz; ky++) {
            const int ys = yy + pad - ky;
            if (ys < 0 || ys % stride) continue;
            const int i = ys / stride;
            if (i >= ho) continue;
            for (int kx = 0; kx < ksz; kx++) {
                const int xs = xx + pad - kx;
                if (xs < 0 || xs % stride) continue;
                const int j = xs / stride;
                if (j >= wo) continue;
                const long long m = ((long long)b * ho + i) * wo + j;
                acc += dcol[m * K + (ky * ksz + kx) * cin + ci];
            }
        }
        const float a = __bfloat162float(act[e]);
        dy[e] = __float2bfloat16_rn(a > 0.f ? acc : 0.f);
    }
}

// ReLU mask and bf16 rounding for a 1x1 layer (the data gradient needs no gather).
__global__ void k_mask_bf16(const float* __restrict__ g, const __nv_bfloat16* __restrict__ act,
                            long long count, __nv_bfloat16* __restrict__ dy)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
         e += (long long)gridDim.x * blockDim.x) {
        const float a = __bfloat162float(act[e]);
        dy[e] = __float2bfloat16_rn(a > 0.f ? g[e] : 0.f);
    }
}

// db[co] = sum_m dy[m][co] (one CTA per output channel, fixed summation order).
__global__ void k_bias_grad(const __nv_bfloat16* __restrict__ dy, long long M, int ld,
                            float* __restrict__ db)
{
    __shared__ float red[32];
    const int co = blockIdx.x;
    float s = 0.f;
    for (long long m = threadIdx.x; m < M; m += blockDim.x) s += __bfloat162float(dy[m * ld + co]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < blockDim.x / 32 ? red[threadIdx.x] : 0.f;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
        if (threadIdx.x == 0) db[co] = v;
    }
}

// dW[co][k] = sum over splits of part[s][k][co] (k < K), in split order.
__global__ void k_splitk_reduce(const float* __restrict__ part, int splits, size_t stride, int K,
                                int cout, int ldp, float* __restrict__ dW)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < K * cout; e += gridDim.x * blockDim.x) {
        const int co = e / K, k = e % K;
        float s = 0.f;
        for (int q = 0; q < splits; q++) s += part[q * stride + (size_t)k * ldp + co];
        dW[e] = s;
    }
}

// Loss = sum over valid cells |out - label|^2 / max(n_valid, 1); dy = bf16(2 (out - label) /
// n_valid) at valid cells, 0 elsewhere (row stride ld >= 2, padding columns zero).
__global__ void __launch_bounds__(1024) k_loss(const float* __restrict__ out,
                                               const float* __restrict__ label,
                                               const uint8_t* __restrict__ valid, int cells, int ld,
                                               __nv_bfloat16* __restrict__ dy, float* __restrict__ loss)
{
    __shared__ float red[32];
    __shared__ float s_nv;
    float c = 0.f;
    for (int i = threadIdx.x; i < cells; i += blockDim.x) c += valid[i] ? 1.f : 0.f;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int k = 0; k < (int)(blockDim.x / 32); k++) t += red[k];
        s_nv = t > 1.f ? t : 1.f;
    }
    __syncthreads();
    const float nv = s_nv;
    float l = 0.f;
    for (int i = threadIdx.x; i < cells; i += blockDim.x) {
        const bool v = valid[i] != 0;
        for (int q = 0; q < ld; q++) {
            float g = 0.f;
            if (q < 2 && v) {
                const float d = out[2 * i + q] - label[2 * i + q];
                l = fmaf(d, d, l);
                g = 2.f * d / nv;
            }
            dy[(size_t)i * ld + q] = __float2bfloat16_rn(g);
        }
    }
    __syncthreads();
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(kFull, l, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int k = 0; k < (int)(blockDim.x / 32); k++) t += red[k];
        *loss = t / nv;
    }
}

// Adam (Kingma and Ba 2015) with bias correction at step t >= 1.
__global__ void k_adam(float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, int count, float lr, float b1, float b2,
                       float eps, float c1, float c2)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

int grid_for(long long n, int threads = 256)
{
    long long g = (n + threads - 1) / threads;
    return (int)(g < 4096 ? (g > 0 ? g : 1) : 4096);
}

}  // namespace

// ------------------------------------------------------------ workspace
struct CnnLayout {
    int n = 0, h = 0, w = 0;
    int H[kNL + 1], Wd[kNL + 1];  // spatial size at the input of layer i (i = kNL: output)
    long long M[kNL];             // output pixels of layer i
    size_t wb[kNL], wt[kNL], col[kNL], act[kNL];
    size_t feat, colT, dyT, dxcol, dy0, dy1, part, gW, total;
    int splits_max = 64;
    // train = false: the forward pass only (no backward scratch)
    CnnLayout(int n_, int h_, int w_, bool train = true)
    {
        n = n_;
        h = h_;
        w = w_;
        H[0] = h;
        Wd[0] = w;
        for (int i = 0; i < kNL; i++) {
            H[i + 1] = osz(H[i], kNet[i]);
            Wd[i + 1] = osz(Wd[i], kNet[i]);
            M[i] = (long long)n * H[i + 1] * Wd[i + 1];
        }
        size_t o = 0;
        auto add = [&](size_t bytes) {
            const size_t r = o;
            o += align_up(bytes > 0 ? bytes : 1, 256);
            return r;
        };
        long long Mmax = 0, MKmax = 0, colTmax = 0, dyTmax = 0, partmax = 0;
        for (int i = 0; i < kNL; i++) {
            const LayerSpec& L = kNet[i];
            wb[i] = add((size_t)cpad(L) * kpad(L) * 2);
            wt[i] = add((size_t)kdim(L) * cpad(L) * 2);
            col[i] = L.k == 1 ? 0 : add((size_t)M[i] * kpad(L) * 2);
            act[i] = L.relu ? add((size_t)M[i] * L.cout * 2) : 0;
            Mmax = M[i] > Mmax ? M[i] : Mmax;
            MKmax = std::max<long long>(MKmax, M[i] * kdim(L));
            colTmax = std::max<long long>(colTmax, (long long)kpad(L) * round_up((int)M[i], 8));
            dyTmax = std::max<long long>(dyTmax, (long long)cpad(L) * round_up((int)M[i], 8));
            partmax = std::max<long long>(partmax, (long long)splits_max * kpad(L) * cpad(L));
        }
        feat = add((size_t)n * h * w * kFeat * 2);
        colT = dyT = dxcol = dy0 = dy1 = part = gW = 0;
        if (train) {
            colT = add((size_t)colTmax * 2);
            dyT = add((size_t)dyTmax * 2);
            dxcol = add((size_t)MKmax * 4);
            dy0 = add((size_t)Mmax * 64 * 2);
            dy1 = add((size_t)Mmax * 64 * 2);
            part = add((size_t)partmax * 4);
            gW = add((size_t)64 * 576 * 4);
        }
        total = o;
    }
};

size_t cnn_params()
{
    size_t t = 0;
    for (int i = 0; i < kNL; i++) t += (size_t)kdim(kNet[i]) * kNet[i].cout + kNet[i].cout;
    return t;
}

size_t cnn_ws_bytes(int n, int h, int w, bool train) { return CnnLayout(n, h, w, train).total; }

// Device address of layer `layer`'s stored output (bf16 [M][cout]; layer kNL - 1 = the 1x1
// head has none) or of the feature stage (layer -1, bf16 [n][h][w][27]) inside a workspace.
const void* cnn_activation(const void* ws, int n, int h, int w, int layer, int* rows, int* cols)
{
    const CnnLayout lay(n, h, w);
    const uint8_t* base = static_cast<const uint8_t*>(ws);
    if (layer == -1) {
        *rows = n * h * w;
        *cols = kFeat;
        return base + lay.feat;
    }
    if (layer < 0 || layer >= kNL || !kNet[layer].relu) return nullptr;
    *rows = (int)lay.M[layer];
    *cols = kNet[layer].cout;
    return base + lay.act[layer];
}

void cnn_out_dims(int h, int w, int* ho, int* wo)
{
    CnnLayout L(1, h, w);
    *ho = L.H[kNL];
    *wo = L.Wd[kNL];
}

static size_t param_offset(int layer)
{
    size_t o = 0;
    for (int i = 0; i < layer; i++) o += (size_t)kdim(kNet[i]) * kNet[i].cout + kNet[i].cout;
    return o;
}

// Forward: x [n][h][w][2] bf16 -> out [n][ho][wo][2] FP32; keeps im2col matrices and
// activations in the workspace for cnn_backward.
bool cnn_forward(const float* theta, const __nv_bfloat16* x, int n, int h, int w, float* out,
                 void* ws, int* err, cudaStream_t s)
{
    const CnnLayout lay(n, h, w);
    uint8_t* base = static_cast<uint8_t*>(ws);
    __nv_bfloat16* feat = reinterpret_cast<__nv_bfloat16*>(base + lay.feat);
    note_launch();
    k_features<<<dim3((w + 127) / 128, h, n), 128, 0, s>>>(
        reinterpret_cast<const __nv_bfloat162*>(x), h, w, feat);
    const __nv_bfloat16* in = feat;
    for (int i = 0; i < kNL; i++) {
        const LayerSpec& L = kNet[i];
        const int K = kdim(L), kp = kpad(L), cp = cpad(L);
        __nv_bfloat16* Wb = reinterpret_cast<__nv_bfloat16*>(base + lay.wb[i]);
        __nv_bfloat16* Wt = reinterpret_cast<__nv_bfloat16*>(base + lay.wt[i]);
        const size_t po = param_offset(i);
        note_launch();
        k_pack_weights<<<grid_for((long long)cp * kp), 256, 0, s>>>(theta + po, L.cout, K, kp, cp, Wb,
                                                                     Wt);
        const __nv_bfloat16* A = in;
        int lda = L.cin;
        if (L.k != 1) {
            __nv_bfloat16* col = reinterpret_cast<__nv_bfloat16*>(base + lay.col[i]);
            note_launch();
            k_im2col<<<(unsigned)((lay.M[i] + 15) / 16), dim3(16, 16), 0, s>>>(
                in, lay.H[i], lay.Wd[i], L.cin, L.k, L.stride, lay.H[i + 1], lay.Wd[i + 1], kp,
                (int)lay.M[i], col);
            A = col;
            lda = kp;
        }
        const float* bias = theta + po + (size_t)K * L.cout;
        GemmEpi e{};
        if (L.relu) {
            __nv_bfloat16* act = reinterpret_cast<__nv_bfloat16*>(base + lay.act[i]);
            e = GemmEpi{kEpiBiasReluBf16, nullptr, act, bias, L.cout, 0};
            in = act;
        } else {
            e = GemmEpi{kEpiBiasF32, out, nullptr, bias, L.cout, 0};
        }
        if (!launch_gemm_bf16(A, lda, Wb, kp, (int)lay.M[i], L.cout, kp, 1, e, err, s)) return false;
    }
    return true;
}

// Inference workspace: the padded features and one activation buffer per ReLU layer.
struct InferLayout {
    size_t feat, act[kNL], wimg[kNL], total;
    int H[kNL + 1], Wd[kNL + 1];
    long long M[kNL];
    InferLayout(int n, int h, int w)
    {
        H[0] = h;
        Wd[0] = w;
        size_t o = 0;
        auto add = [&](size_t bytes) {
            const size_t r = o;
            o += align_up(bytes > 0 ? bytes : 1, 256);
            return r;
        };
        feat = add((size_t)n * h * w * kFeatPad * 2);
        for (int i = 0; i < kNL; i++) {
            H[i + 1] = osz(H[i], kNet[i]);
            Wd[i + 1] = osz(Wd[i], kNet[i]);
            M[i] = (long long)n * H[i + 1] * Wd[i + 1];
            act[i] = kNet[i].relu ? add((size_t)M[i] * kNet[i].cout * 2) : 0;
            wimg[i] = kNet[i].k == 3 ? add(conv_wimg_size(i == 0 ? kFeatPad : kNet[i].cin,
                                                          kNet[i].cout))
                                     : 0;
        }
        total = o;
    }
};

size_t cnn_infer_ws_bytes(int n, int h, int w) { return InferLayout(n, h, w).total; }

// Forward pass for inference: features (32 padded channels), eight implicit-GEMM 3x3
// convolutions, the 1x1 head. No im2col matrix, no packed weights (the convolution
// kernels round the FP32 parameters to bfloat16 as they stage them).
bool cnn_infer(const float* theta, const __nv_bfloat16* x, int n, int h, int w, float* out,
               void* ws, int* err, cudaStream_t s)
{
    const InferLayout lay(n, h, w);
    uint8_t* base = static_cast<uint8_t*>(ws);
    __nv_bfloat16* feat = reinterpret_cast<__nv_bfloat16*>(base + lay.feat);
    note_launch();
    k_features32<<<dim3((w + 127) / 128, h, n), 128, 0, s>>>(
        reinterpret_cast<const __nv_bfloat162*>(x), h, w, feat);
    ConvPack pk{};
    for (int i = 0; i < kNL; i++) {
        if (kNet[i].k != 3) continue;
        const int l = pk.layers++;
        pk.W[l] = theta + param_offset(i);
        pk.img[l] = base + lay.wimg[i];
        pk.cin[l] = i == 0 ? kFeatPad : kNet[i].cin;
        pk.cin_src[l] = kNet[i].cin;
        pk.cout[l] = kNet[i].cout;
    }
    launch_pack_conv(pk, s);
    const __nv_bfloat16* in = feat;
    int cin_pad = kFeatPad;
    for (int i = 0; i < kNL; i++) {
        const LayerSpec& L = kNet[i];
        const size_t po = param_offset(i);
        const float* bias = theta + po + (size_t)kdim(L) * L.cout;
        if (L.k == 3) {
            __nv_bfloat16* act = reinterpret_cast<__nv_bfloat16*>(base + lay.act[i]);
            const ConvArgs a{in, lay.H[i], lay.Wd[i], lay.H[i + 1], lay.Wd[i + 1], (int)lay.M[i],
                             theta + po, L.cin, cin_pad, L.stride, L.cout, bias, act, err,
                             base + lay.wimg[i]};
            if (!launch_conv3x3(a, s)) return false;
            in = act;
            cin_pad = L.cout;
        } else {
            note_launch();
            k_head<<<grid_for(lay.M[i]), 256, 0, s>>>(in, lay.M[i], theta + po, bias, out);
        }
    }
    return true;
}

// Loss and gradient w.r.t. theta for the activations of the preceding cnn_forward.
bool cnn_backward(const float* theta, const __nv_bfloat16* x, int n, int h, int w, const float* out,
                  const float* label, const uint8_t* valid, float* grad, float* loss, void* ws,
                  int* err, cudaStream_t s)
{
    const CnnLayout lay(n, h, w);
    uint8_t* base = static_cast<uint8_t*>(ws);
    auto bf = [&](size_t off) { return reinterpret_cast<__nv_bfloat16*>(base + off); };
    __nv_bfloat16* dy = bf(lay.dy0);
    __nv_bfloat16* dyn = bf(lay.dy1);
    const int last = kNL - 1;
    const int cp_last = cpad(kNet[last]);
    note_launch();
    k_loss<<<1, 1024, 0, s>>>(out, label, valid, (int)lay.M[last], cp_last, dy, loss);
    int dy_ld = cp_last;
    for (int i = last; i >= 0; i--) {
        const LayerSpec& L = kNet[i];
        const int K = kdim(L), kp = kpad(L), cp = cpad(L);
        const long long M = lay.M[i];
        const int Mp = round_up((int)M, 8);
        const size_t po = param_offset(i);
        float* gW = grad + po;
        float* gb = grad + po + (size_t)K * L.cout;
        note_launch();
        k_bias_grad<<<L.cout, 1024, 0, s>>>(dy, M, dy_ld, gb);
        // weight gradient: dW^T [K x cout] = col^T [kp x M] * dY^T [cp x M]^T
        const __nv_bfloat16* colsrc = L.k == 1 ? (i > 0 ? bf(lay.act[i - 1]) : bf(lay.feat))
                                               : bf(lay.col[i]);
        const int col_ld = L.k == 1 ? L.cin : kp;
        const int rowsA = L.k == 1 ? L.cin : kp;
        dim3 tb(32, 8);
        note_launch();
        k_transpose_bf16<<<dim3((rowsA + 31) / 32, (unsigned)((M + 31) / 32)), tb, 0, s>>>(
            colsrc, (int)M, rowsA, col_ld, bf(lay.colT), Mp);
        note_launch();
        k_transpose_bf16<<<dim3((cp + 31) / 32, (unsigned)((M + 31) / 32)), tb, 0, s>>>(
            dy, (int)M, cp, dy_ld, bf(lay.dyT), Mp);
        const int tiles = ((rowsA + 127) / 128) * ((L.cout + gemm_bn_for(L.cout) - 1) / gemm_bn_for(L.cout));
        int splits = (148 + tiles - 1) / tiles;
        const int kchunks = (int)((M + 63) / 64);
        if (splits > kchunks) splits = kchunks;
        if (splits > lay.splits_max) splits = lay.splits_max;
        if (splits < 1) splits = 1;
        const int used = gemm_splits_used((int)M, splits);
        const size_t pstride = (size_t)kp * cp;
        GemmEpi e{kEpiF32, reinterpret_cast<float*>(base + lay.part), nullptr, nullptr, cp, pstride};
        if (!launch_gemm_bf16(bf(lay.colT), Mp, bf(lay.dyT), Mp, rowsA, L.cout, (int)M, splits, e,
                              err, s))
            return false;
        note_launch();
        k_splitk_reduce<<<grid_for((long long)K * L.cout), 256, 0, s>>>(
            reinterpret_cast<float*>(base + lay.part), used, pstride, K, L.cout, cp, gW);
        if (i == 0) break;
        // data gradient: dcol [M x K] = dY [M x cout] * Wt [K x cout]^T, gathered to the input
        float* dcol = reinterpret_cast<float*>(base + lay.dxcol);
        GemmEpi ed{kEpiF32, dcol, nullptr, nullptr, K, 0};
        if (!launch_gemm_bf16(dy, dy_ld, bf(lay.wt[i]), cp, (int)M, K, cp, 1, ed, err, s))
            return false;
        const __nv_bfloat16* prev_act = bf(lay.act[i - 1]);
        if (L.k == 1) {
            note_launch();
            k_mask_bf16<<<grid_for(M * L.cin), 256, 0, s>>>(dcol, prev_act, M * L.cin, dyn);
        } else {
            const long long cnt = (long long)n * lay.H[i] * lay.Wd[i] * L.cin;
            note_launch();
            k_col2im_mask<<<grid_for(cnt), 256, 0, s>>>(dcol, n, lay.H[i], lay.Wd[i], L.cin, L.k,
                                                        L.stride, lay.H[i + 1], lay.Wd[i + 1],
                                                        prev_act, dyn);
        }
        std::swap(dy, dyn);
        dy_ld = L.cin;
    }
    return true;
}

void cnn_adam(float* theta, float* m, float* v, const float* grad, int step, float lr,
              cudaStream_t s)
{
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = (float)(1.0 - pow(0.9, step)), c2 = (float)(1.0 - pow(0.999, step));
    note_launch();
    k_adam<<<grid_for((long long)cnn_params()), 256, 0, s>>>(theta, m, v, grad, (int)cnn_params(),
                                                             lr, b1, b2, 1e-8f, c1, c2);
}

}  // namespace hdrreg
