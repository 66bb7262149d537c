// Rows a9-a11: bilinear warp of the source onto the reference grid
// (Sec. 2.4), SSIM consistency mask (Sec. 2.5, Wang et al. 2004) and the
// weighted irradiance merge (Sec. 2.5 weights, Sec. 3.1 irradiance map).
//
// Warp: one thread per 2x2 luma block (= one chroma pixel of YUV420). The
// homography is evaluated as a displacement H(p) - p from FP32 coefficients
// prepared once per CTA in binary64, so the bilinear fraction is computed from
// small numbers (no 2600-px absolute coordinates in FP32).
// Merge: one CTA per 32x32 luma tile with a 5-pixel halo staged in shared
// memory; the five Gaussian moments are separable (row pass, column pass). To
// avoid the FP32 cancellation of E[x^2] - mu^2, each row segment's moments are
// taken about its own centre pixel and the column pass re-centres them exactly
// onto the output pixel, so flat windows only ever sum small numbers. The two
// images' moment chains run side by side as packed FP32x2 operations (each
// component rounds as its scalar form would).
#include <math.h>

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
    dx = nx / D;
    dy = ny / D;
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// bilinear sample at (x + t_x, y + t_y) with integer x, y and small offsets t
__device__ __forceinline__ float bilerp(const uint8_t* __restrict__ img, int w, int h, int x, int y,
                                        float tx, float ty)
{
    const float fx0 = floorf(tx), fy0 = floorf(ty);
    const float fx = tx - fx0, fy = ty - fy0;
    const int ix = x + (int)fx0, iy = y + (int)fy0;
    const int xa = clampi(ix, 0, w - 1), xb = clampi(ix + 1, 0, w - 1);
    const size_t ra = (size_t)clampi(iy, 0, h - 1) * w, rb = (size_t)clampi(iy + 1, 0, h - 1) * w;
    const float a = __ldg(img + ra + xa), b = __ldg(img + ra + xb);
    const float c = __ldg(img + rb + xa), d = __ldg(img + rb + xb);
    const float top = fmaf(fx, b - a, a);
    const float bot = fmaf(fx, d - c, c);
    return fmaf(fy, bot - top, top);
}

__global__ void __launch_bounds__(256) k_warp(const uint8_t* __restrict__ sy,
                                              const uint8_t* __restrict__ su,
                                              const uint8_t* __restrict__ sv, int w, int h,
                                              const double* __restrict__ H,
                                              const float* __restrict__ fu,
                                              const float* __restrict__ fv, float* __restrict__ oy,
                                              float* __restrict__ ou, float* __restrict__ ov)
{
    __shared__ WarpCoef cs;
    if (threadIdx.x == 0) prep_coef(H, w, cs);
    __syncthreads();
    const WarpCoef c = cs;
    const int bw = (w + 1) / 2, bh = (h + 1) / 2;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= bw * bh) return;
    const int bx = idx % bw, by = idx / bw;
    float stx = 0.f, sty = 0.f;
    for (int j = 0; j < 2; j++)
        for (int i = 0; i < 2; i++) {
            const int x = 2 * bx + i, y = 2 * by + j;
            if (x >= w || y >= h) continue;
            const size_t o = (size_t)y * w + x;
            float dx, dy;
            h_disp(c, x, y, w, h, dx, dy);
            const float tx = dx + fu[o], ty = dy + fv[o];
            stx += tx;
            sty += ty;
            oy[o] = bilerp(sy, w, h, x, y, tx, ty);
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
    float we_k;  // 1 / (2 sigma^2)
    int nsrc;
};

__device__ __forceinline__ float well_exposed(float z, float k)
{
    const float t = z * (1.f / 255.f) - 0.5f;
    return expf(-(t * t) * k);
}

// 0 at 0 and 255, linear to 1 over the 2 DN next to either end: clipped samples
// carry no irradiance and the weight stays continuous in the sample value.
__device__ __forceinline__ float clip_taper(float z)
{
    const float d = fminf(z, 255.f - z) * 0.5f;
    return fminf(fmaxf(d, 0.f), 1.f);
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

__global__ void __launch_bounds__(256, 3) k_merge(const uint8_t* __restrict__ ref_y,
                                               const uint8_t* __restrict__ ref_u,
                                               const uint8_t* __restrict__ ref_v, int w, int h,
                                               MergeArgs args, float* __restrict__ oy,
                                               float* __restrict__ ou, float* __restrict__ ov,
                                               float* __restrict__ q_out)
{
    // the reference (X) and the normalized warped source (Y) interleaved: every step of the
    // two moment chains is one packed FP32x2 instruction
    __shared__ float2 XY[kIn][kIn];
    __shared__ float2 H1[kIn][kTile];   // (sum g a, sum g b) of each row segment
    __shared__ float2 H2[kIn][kTile];   // (sum g a^2, sum g b^2)
    __shared__ float H11[kIn][kTile + 1];  // sum g a b
    __shared__ float Wk[kTile][kTile + 1];
    __shared__ float Ns[kTile][kTile + 1], Ds[kTile][kTile + 1], Zs[kTile][kTile + 1];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int x0 = blockIdx.x * kTile, y0 = blockIdx.y * kTile;
    const bool chroma = ref_u != nullptr && ou != nullptr;
    const int cw = w / 2, ch = h / 2;
    const float2 neg1 = f2(-1.f, -1.f);
    const float2 gsum2 = f2(args.gsum, args.gsum);

    // this thread's 4 luma pixels: (tx, ty + 8 k); its chroma pixel: (tid % 16, tid / 16)
    const int tx = tid % kTile, ty0 = tid / kTile;
    // per-pixel numerator / denominator of the merge live in shared memory (this thread's
    // own entries only), so the column pass loop keeps no arrays in registers
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const int x = x0 + tx, y = y0 + ty0 + 8 * k;
        float nu = 0.f, de = 0.f;
        if (x < w && y < h) {
            const float z = (float)ref_y[(size_t)y * w + x];
            const float wr = well_exposed(z, args.we_k);
            nu = wr * z;
            de = wr;
        }
        Ns[ty0 + 8 * k][tx] = nu;
        Ds[ty0 + 8 * k][tx] = de;
        Wk[ty0 + 8 * k][tx] = de;
    }
    const int cx = x0 / 2 + tid % 16, cy = y0 / 2 + tid / 16;
    const bool c_ok = chroma && cx < cw && cy < ch && (tid % 16) < kTile / 2;
    float cnu = 0.f, cnv = 0.f, cden = 0.f;
    __syncthreads();
    if (c_ok) {
        const int lx = 2 * (tid % 16), ly = 2 * (tid / 16);
        const float wb = ((Wk[ly][lx] + Wk[ly][lx + 1]) + (Wk[ly + 1][lx] + Wk[ly + 1][lx + 1])) * 0.25f;
        const size_t o = (size_t)cy * cw + cx;
        cnu = wb * ((float)ref_u[o] - 128.f);
        cnv = wb * ((float)ref_v[o] - 128.f);
        cden = wb;
    }

    for (int k = 0; k < args.nsrc; k++) {
        const MergeSrcDev s = args.src[k];
        // every global load of this source up front (one round trip): the 42 x 42 halo
        // (warp w: rows w + 8 r, columns lane and lane + 32), this thread's own 4 source
        // pixels, its chroma pixel
        uint8_t hr[12];
        float hy[12];
#pragma unroll
        for (int q = 0; q < 12; q++) {
            const int yy = warp + 8 * (q >> 1), xx = lane + 32 * (q & 1);
            hr[q] = 0;
            hy[q] = 0.f;
            if (yy < kIn && xx < kIn) {
                const int gy = clampi(y0 - kHalo + yy, 0, h - 1);
                const int gx = clampi(x0 - kHalo + xx, 0, w - 1);
                const size_t o = (size_t)gy * w + gx;
                hr[q] = s.ref_n[o];
                hy[q] = s.y[o];
            }
        }
#pragma unroll
        for (int kk = 0; kk < 4; kk++) {
            const int x = x0 + tx, y = y0 + ty0 + 8 * kk;
            Zs[ty0 + 8 * kk][tx] = (x < w && y < h) ? s.y[(size_t)y * w + x] : 0.f;
        }
        float su = 0.f, sv = 0.f;
        if (c_ok) {
            const size_t o = (size_t)cy * cw + cx;
            su = s.u[o];
            sv = s.v[o];
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 12; q++) {
            const int yy = warp + 8 * (q >> 1), xx = lane + 32 * (q & 1);
            if (yy < kIn && xx < kIn) XY[yy][xx] = f2((float)hr[q], norm_map(s, hy[q]));
        }
        __syncthreads();
        // Row pass: moments of each 11-tap row segment about its own centre pixel
        // (a = x - x_c, b = y - y_c): M1 = sum g (a, b), M2 = sum g (a^2, b^2), M11 = sum g a b.
        for (int i = tid; i < kIn * kTile; i += 256) {
            const int yy = i / kTile, xx = i % kTile;
            const float2 c = XY[yy][xx + kHalo];
            float2 m1 = f2(0.f, 0.f), m2 = f2(0.f, 0.f);
            float m11 = 0.f;
#pragma unroll
            for (int d = 0; d <= 2 * kHalo; d++) {
                const float2 g2 = f2(args.g[d], args.g[d]);
                const float2 ab = __ffma2_rn(c, neg1, XY[yy][xx + d]);
                const float2 gab = __fmul2_rn(g2, ab);
                m1 = __fadd2_rn(m1, gab);
                m2 = __ffma2_rn(gab, ab, m2);
                m11 = fmaf(gab.x, ab.y, m11);
            }
            H1[yy][xx] = m1;
            H2[yy][xx] = m2;
            H11[yy][xx] = m11;
        }
        __syncthreads();
        const float C1 = (0.01f * 255.f) * (0.01f * 255.f), C2 = (0.03f * 255.f) * (0.03f * 255.f);
#pragma unroll 1
        for (int kk = 0; kk < 4; kk++) {
            const int ly = ty0 + 8 * kk;
            const int x = x0 + tx, y = y0 + ly;
            // Column pass: re-centre every row's moments from its centre c_r onto the output
            // pixel's value c (delta = c_r - c): sum g (a + delta)^k expands exactly, so the
            // window moments stay small numbers wherever the window is flat.
            const float2 c = XY[ly + kHalo][tx + kHalo];
            float2 a1 = f2(0.f, 0.f), a2 = f2(0.f, 0.f);
            float a11 = 0.f;
#pragma unroll
            for (int d = 0; d <= 2 * kHalo; d++) {
                const float2 g2 = f2(args.g[d], args.g[d]);
                const float2 dd = __ffma2_rn(c, neg1, XY[ly + d][tx + kHalo]);
                const float2 m1 = H1[ly + d][tx];
                const float2 r1 = __ffma2_rn(dd, gsum2, m1);
                const float2 r2 = __ffma2_rn(dd, __fadd2_rn(m1, r1), H2[ly + d][tx]);
                const float r11 = H11[ly + d][tx] + fmaf(dd.y, m1.x, dd.x * r1.y);
                a1 = __ffma2_rn(g2, r1, a1);
                a2 = __ffma2_rn(g2, r2, a2);
                a11 = fmaf(args.g[d], r11, a11);
            }
            const float vx = a2.x - a1.x * a1.x, vy = a2.y - a1.y * a1.y, cxy = a11 - a1.x * a1.y;
            const float ux = c.x + a1.x, uy = c.y + a1.y;
            const float ssim = ((2.f * ux * uy + C1) * (2.f * cxy + C2)) /
                               ((ux * ux + uy * uy + C1) * (vx + vy + C2));
            const float q = ssim > 0.f ? ssim : 0.f;
            float wk = 0.f;
            if (x < w && y < h) {
                const float z = Zs[ly][tx];
                wk = well_exposed(z, args.we_k) * q * clip_taper(z);
                Ns[ly][tx] = fmaf(wk, z * s.inv_ratio, Ns[ly][tx]);
                Ds[ly][tx] += wk;
                if (q_out) q_out[(size_t)k * w * h + (size_t)y * w + x] = q;
            }
            Wk[ly][tx] = wk;
        }
        __syncthreads();
        if (c_ok) {
            const int lx = 2 * (tid % 16), ly = 2 * (tid / 16);
            const float wb =
                ((Wk[ly][lx] + Wk[ly][lx + 1]) + (Wk[ly + 1][lx] + Wk[ly + 1][lx + 1])) * 0.25f;
            cnu = fmaf(wb, (su - 128.f) * s.inv_ratio, cnu);
            cnv = fmaf(wb, (sv - 128.f) * s.inv_ratio, cnv);
            cden += wb;
        }
    }
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const int x = x0 + tx, y = y0 + ty0 + 8 * k;
        if (x < w && y < h) oy[(size_t)y * w + x] = Ns[ty0 + 8 * k][tx] / Ds[ty0 + 8 * k][tx];
    }
    if (c_ok) {
        const size_t o = (size_t)cy * cw + cx;
        ou[o] = cnu / cden;
        ov[o] = cnv / cden;
    }
}

}  // namespace

void launch_warp(const uint8_t* src_y, const uint8_t* src_u, const uint8_t* src_v, int w, int h,
                 const double* H, const float* fu, const float* fv, float* oy, float* ou,
                 float* ov, cudaStream_t s)
{
    const long long nb = (long long)((w + 1) / 2) * ((h + 1) / 2);
    const int grid = (int)((nb + 255) / 256);
    note_launch();
    k_warp<<<grid, 256, 0, s>>>(src_y, src_u, src_v, w, h, H, fu, fv, oy, ou, ov);
}

void launch_predictor_input(const uint8_t* ref_q, const uint8_t* src_q, int w, int h,
                            const double* H, void* out, cudaStream_t s)
{
    const long long n = (long long)w * h;
    long long g = (n + 255) / 256;
    if (g > 4096) g = 4096;
    note_launch();
    k_predictor_input<<<(int)g, 256, 0, s>>>(ref_q, src_q, w, h, H,
                                             static_cast<__nv_bfloat162*>(out));
}

void launch_merge(const uint8_t* ref_y, const uint8_t* ref_u, const uint8_t* ref_v, int w, int h,
                  int nsrc, const MergeSrcDev* srcs, double ssim_sigma, double we_sigma,
                  float* oy, float* ou, float* ov, float* q_out, cudaStream_t s)
{
    MergeArgs a;
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
    a.we_k = (float)(1.0 / (2.0 * we_sigma * we_sigma));
    dim3 grid((w + kTile - 1) / kTile, (h + kTile - 1) / kTile);
    note_launch();
    k_merge<<<grid, 256, 0, s>>>(ref_y, ref_u, ref_v, w, h, a, oy, ou, ov, q_out);
}

}  // namespace hdrreg
