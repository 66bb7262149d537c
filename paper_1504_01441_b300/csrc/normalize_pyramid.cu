// Rows a1-a2: exposure normalization (ratio or histogram equalization) and the
// 2x2 box pyramid of the matcher (Sec. 2.2, Sec. 2.6, Sec. 3).
//
// Both are byte-streaming kernels bound by HBM: 16-byte vector loads/stores,
// the 256-entry map staged in shared memory, grids sized to the SM count.
#include "hdrreg_internal.cuh"

namespace hdrreg {

__device__ __forceinline__ void build_lut(uint8_t* lut, LutSpec spec)
{
    for (int v = threadIdx.x; v < 256; v += blockDim.x) {
        if (spec.dev) {
            lut[v] = spec.dev[v];
        } else {
            const long long r = ((long long)v * spec.gn + spec.gd / 2) / spec.gd;
            lut[v] = (uint8_t)(r > 255 ? 255 : r);
        }
    }
}

__device__ __forceinline__ uint32_t map4(const uint8_t* lut, uint32_t x)
{
    return (uint32_t)lut[x & 255] | ((uint32_t)lut[(x >> 8) & 255] << 8) |
           ((uint32_t)lut[(x >> 16) & 255] << 16) | ((uint32_t)lut[x >> 24] << 24);
}

// out = lut(in) for two frames (blockIdx.y selects the frame)
__global__ void __launch_bounds__(256) k_lut2(const uint8_t* __restrict__ a,
                                              const uint8_t* __restrict__ b,
                                              uint8_t* __restrict__ an, uint8_t* __restrict__ bn,
                                              size_t n, LutSpec la, LutSpec lb, int vec)
{
    __shared__ uint8_t lut[256];
    const bool second = blockIdx.y == 1;
    const uint8_t* in = second ? b : a;
    uint8_t* out = second ? bn : an;
    build_lut(lut, second ? lb : la);
    __syncthreads();
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t done = 0;
    if (vec) {
        const size_t nv = n / 16;
        const uint4* iv = reinterpret_cast<const uint4*>(in);
        uint4* ov = reinterpret_cast<uint4*>(out);
        for (size_t i = tid; i < nv; i += stride) {
            uint4 x = iv[i];
            x.x = map4(lut, x.x);
            x.y = map4(lut, x.y);
            x.z = map4(lut, x.z);
            x.w = map4(lut, x.w);
            ov[i] = x;
        }
        done = nv * 16;
    }
    for (size_t i = done + tid; i < n; i += stride) out[i] = lut[in[i]];
}

static int grid_for(size_t work, int per_block)
{
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    size_t blocks = (work + per_block - 1) / per_block;
    size_t cap = (size_t)sms * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    return (int)blocks;
}

void launch_lut2(const uint8_t* a, const uint8_t* b, uint8_t* an, uint8_t* bn, size_t n,
                 LutSpec la, LutSpec lb, cudaStream_t s)
{
    const int vec = ((((uintptr_t)a | (uintptr_t)b | (uintptr_t)an | (uintptr_t)bn) & 15) == 0);
    dim3 grid(grid_for(n / 16 + 1, 256), 2);
    note_launch();
    k_lut2<<<grid, 256, 0, s>>>(a, b, an, bn, n, la, lb, vec);
}

// Per-frame 256-bin histograms (blockIdx.y = frame): 16 pixels per load where the frame
// allows it and a sub-histogram per warp in shared memory (fewer warps contend for a bin);
// the block's bins are added to
// hist[frame * 256 + v] (zeroed by the caller).
__global__ void __launch_bounds__(256) k_histograms(const uint8_t* __restrict__ a,
                                                    const uint8_t* __restrict__ b, size_t n,
                                                    uint32_t* __restrict__ hist)
{
    __shared__ uint32_t hs[8][256];
    const uint8_t* in = blockIdx.y ? b : a;
    const int warp = threadIdx.x >> 5;
    for (int v = threadIdx.x; v < 8 * 256; v += blockDim.x) hs[v >> 8][v & 255] = 0;
    __syncthreads();
    auto add = [&](uint32_t v, bool on) {
        if (on) atomicAdd(&hs[warp][v], 1u);
    };
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t first = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t done = 0;
    if (((uintptr_t)in & 15) == 0) {
        const size_t nv = n / 16;
        const uint4* in4 = reinterpret_cast<const uint4*>(in);
        const size_t rounds = (nv + stride - 1) / stride;  // the same for every lane of a warp
        for (size_t r = 0; r < rounds; r++) {
            const size_t i = first + r * stride;
            const bool ok = i < nv;
            const uint4 q = ok ? in4[i] : make_uint4(0, 0, 0, 0);
            const uint32_t wd[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int k = 0; k < 16; k++) add((wd[k >> 2] >> (8 * (k & 3))) & 255u, ok);
        }
        done = nv * 16;
    }
    const size_t rest = n - done;
    const size_t rounds = (rest + stride - 1) / stride;
    for (size_t r = 0; r < rounds; r++) {
        const size_t i = done + first + r * stride;
        const bool ok = i < n;
        add(ok ? in[i] : 0u, ok);
    }
    __syncthreads();
    for (int v = threadIdx.x; v < 256; v += blockDim.x) {
        uint32_t t = 0;
#pragma unroll
        for (int wv = 0; wv < 8; wv++) t += hs[wv][v];
        if (t) atomicAdd(&hist[blockIdx.y * 256 + v], t);
    }
}

__global__ void k_write_luts(LutSpec a, LutSpec b, uint8_t* __restrict__ luts)
{
    __shared__ uint8_t lut[256];
    build_lut(lut, blockIdx.x ? b : a);
    __syncthreads();
    luts[blockIdx.x * 256 + threadIdx.x] = lut[threadIdx.x];
}

void launch_write_luts(LutSpec a, LutSpec b, uint8_t* luts, cudaStream_t s)
{
    note_launch();
    k_write_luts<<<2, 256, 0, s>>>(a, b, luts);
}

void launch_histograms(const uint8_t* a, const uint8_t* b, size_t n, uint32_t* hist,
                       cudaStream_t s)
{
    dim3 grid(grid_for(n, 256 * 64), 2);
    note_launch();
    k_histograms<<<grid, 256, 0, s>>>(a, b, n, hist);
}

// Equalization maps of both frames: lut[v] = round((cdf[v]-cdf_min)*255/(N-cdf_min)),
// integer arithmetic, halves up; identity for a constant frame. One block of 256 threads
// per frame: thread v holds bin v; the CDF is a block-wide inclusive prefix sum, cdf_min
// the count of the first nonzero bin.
__global__ void __launch_bounds__(256) k_histeq_luts(const uint32_t* __restrict__ hist,
                                                     long long n, uint8_t* __restrict__ luts)
{
    __shared__ long long wsum[8];
    __shared__ int vmin;
    const int f = blockIdx.x, v = threadIdx.x, warp = v >> 5, lane = v & 31;
    const uint32_t hv = hist[f * 256 + v];
    if (v == 0) vmin = 256;
    long long inc = hv;
    for (int o = 1; o < 32; o <<= 1) {
        const long long u = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += u;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (hv) atomicMin(&vmin, v);
    long long pre = 0;
    for (int k = 0; k < warp; k++) pre += wsum[k];
    __syncthreads();
    const long long cdf = pre + inc;
    const long long cdf_min = vmin < 256 ? (long long)hist[f * 256 + vmin] : 0;
    const long long den = n - cdf_min;
    uint8_t out;
    if (den <= 0) {
        out = (uint8_t)v;
    } else {
        long long num = cdf - cdf_min;
        if (num < 0) num = 0;
        out = (uint8_t)((num * 255 + den / 2) / den);
    }
    luts[f * 256 + v] = out;
}

void launch_histeq_luts(const uint32_t* hist, size_t n, uint8_t* luts, cudaStream_t s)
{
    note_launch();
    k_histeq_luts<<<2, 256, 0, s>>>(hist, (long long)n, luts);
}

// Pyramid: one block per S x S tile of level 0 (S = max(64, 2^(levels-1))).
// Level l+1 pixel (x, y) = (a+b+c+d+2) >> 2 of its 2x2 block on level l; it
// exists iff x < w >> (l+1) and y < h >> (l+1), in which case its whole block
// exists on level l, so each tile computes its levels independently in
// shared memory. blockIdx.z selects the frame (two frames per launch).
struct PyrArgs {
    const uint8_t* in0[2];
    uint8_t* out0[2];                  // remapped level 0, or nullptr
    uint8_t* lv[2][kMaxLevels];        // levels 1..levels-1
    LutSpec lut[2];
    int w, h, levels, S;
};

__global__ void __launch_bounds__(256) k_pyramid(PyrArgs a)
{
    extern __shared__ __align__(16) uint8_t sm[];
    __shared__ uint8_t lut[256];
    const int f = blockIdx.z;
    build_lut(lut, a.lut[f]);
    __syncthreads();
    const int S = a.S;
    const int x0 = blockIdx.x * S, y0 = blockIdx.y * S;
    uint8_t* cur = sm;
    // level 0: S x S, zero outside the frame; 16 pixels per item, one 16-byte load and
    // store where the row segment lies inside the frame and the addresses are aligned
    const uint8_t* in = a.in0[f];
    uint8_t* out0 = a.out0[f];
    const bool vec = (a.w & 15) == 0 && ((uintptr_t)in & 15) == 0 &&
                     (out0 == nullptr || ((uintptr_t)out0 & 15) == 0);
    for (int i = threadIdx.x; i < S * S / 16; i += blockDim.x) {
        const int yy = i / (S / 16), xx = (i % (S / 16)) * 16;
        const int gy = y0 + yy, gx0 = x0 + xx;
        uint32_t wd[4];
        if (vec && gy < a.h && gx0 + 16 <= a.w) {
            const size_t o = (size_t)gy * a.w + gx0;
            const uint4 v = *reinterpret_cast<const uint4*>(in + o);
            const uint32_t src[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int q = 0; q < 4; q++) {
                uint32_t r = 0;
#pragma unroll
                for (int k = 0; k < 4; k++) r |= (uint32_t)lut[(src[q] >> (8 * k)) & 255u] << (8 * k);
                wd[q] = r;
            }
            if (out0) *reinterpret_cast<uint4*>(out0 + o) = make_uint4(wd[0], wd[1], wd[2], wd[3]);
        } else {
#pragma unroll
            for (int q = 0; q < 4; q++) {
                uint32_t r = 0;
                for (int k = 0; k < 4; k++) {
                    const int gx = gx0 + 4 * q + k;
                    uint32_t v = 0;
                    if (gx < a.w && gy < a.h) {
                        v = lut[in[(size_t)gy * a.w + gx]];
                        if (out0) out0[(size_t)gy * a.w + gx] = (uint8_t)v;
                    }
                    r |= v << (8 * k);
                }
                wd[q] = r;
            }
        }
        *reinterpret_cast<uint4*>(cur + yy * S + xx) = make_uint4(wd[0], wd[1], wd[2], wd[3]);
    }
    __syncthreads();
    int side = S;
    for (int l = 1; l < a.levels; l++) {
        const int ns = side / 2;
        uint8_t* nxt = cur + side * side;
        const int lw = a.w >> l, lh = a.h >> l;
        const int bx = (x0 >> l), by = (y0 >> l);
        uint8_t* lvo = a.lv[f][l];
        const bool vec4 = (lw & 3) == 0 && ((uintptr_t)lvo & 3) == 0 && (ns & 3) == 0;
        if (vec4) {  // four output pixels per item, one 4-byte store
            for (int i = threadIdx.x; i < ns * ns / 4; i += blockDim.x) {
                const int yy = i / (ns / 4), xx = (i % (ns / 4)) * 4;
                const uint8_t* r0 = cur + (2 * yy) * side + 2 * xx;
                const uint8_t* r1 = r0 + side;
                uint32_t word = 0;
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const int s = r0[2 * k] + r0[2 * k + 1] + r1[2 * k] + r1[2 * k + 1];
                    word |= (uint32_t)((s + 2) >> 2) << (8 * k);
                }
                *reinterpret_cast<uint32_t*>(nxt + yy * ns + xx) = word;
                const int gx = bx + xx, gy = by + yy;
                if (gy < lh) {
                    if (gx + 4 <= lw) {
                        *reinterpret_cast<uint32_t*>(lvo + (size_t)gy * lw + gx) = word;
                    } else {
                        for (int k = 0; k < 4 && gx + k < lw; k++)
                            lvo[(size_t)gy * lw + gx + k] = (uint8_t)(word >> (8 * k));
                    }
                }
            }
        } else {
            for (int i = threadIdx.x; i < ns * ns; i += blockDim.x) {
                const int yy = i / ns, xx = i % ns;
                const int s = cur[(2 * yy) * side + 2 * xx] + cur[(2 * yy) * side + 2 * xx + 1] +
                              cur[(2 * yy + 1) * side + 2 * xx] + cur[(2 * yy + 1) * side + 2 * xx + 1];
                const uint8_t v = (uint8_t)((s + 2) >> 2);
                nxt[i] = v;
                const int gx = bx + xx, gy = by + yy;
                if (gx < lw && gy < lh) lvo[(size_t)gy * lw + gx] = v;
            }
        }
        __syncthreads();
        cur = nxt;
        side = ns;
    }
}

void launch_pyramid2(const uint8_t* const in0[2], int w, int h, int levels, const LutSpec lut[2],
                     uint8_t* const out0[2], uint8_t* const* const lv[2], int nframes,
                     cudaStream_t s)
{
    PyrArgs a;
    a.w = w;
    a.h = h;
    a.levels = levels;
    a.S = 64;
    while (a.S < (1 << (levels - 1))) a.S *= 2;
    for (int f = 0; f < 2; f++) {
        const int g = f < nframes ? f : 0;
        a.in0[f] = in0[g];
        a.out0[f] = out0[g];
        a.lut[f] = lut[g];
        for (int l = 0; l < kMaxLevels; l++) a.lv[f][l] = (l < levels && l > 0) ? lv[g][l] : nullptr;
    }
    size_t smem = 0;
    for (int side = a.S, l = 0; l < levels; l++, side /= 2) smem += (size_t)side * side;
    dim3 grid((w + a.S - 1) / a.S, (h + a.S - 1) / a.S, nframes);
    ensure_smem((const void*)k_pyramid, smem);  // static + dynamic may pass 48 KB
    note_launch();
    k_pyramid<<<grid, 256, smem, s>>>(a);
}

void launch_pyramid(const uint8_t* in0, int w, int h, int levels, LutSpec lut, uint8_t* out0,
                    uint8_t* const* out_levels, cudaStream_t s)
{
    const uint8_t* ins[2] = {in0, in0};
    LutSpec luts[2] = {lut, lut};
    uint8_t* outs[2] = {out0, out0};
    uint8_t* const* lvs[2] = {out_levels, out_levels};
    launch_pyramid2(ins, w, h, levels, luts, outs, lvs, 1, s);
}

}  // namespace hdrreg
