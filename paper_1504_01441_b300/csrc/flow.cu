// Row a8: sparse-to-dense flow by the recursive domain-transform filter
// (Sec. 2.4, Eq. 5-6; Gastal and Oliveira 2011).
//
// Each pass is the first-order recurrence J[n] = x[n] + w[n] (J[n-1] - x[n])
// along every row (then back), or every column (then back), of the three planes
// P_u, P_v, N, with w[n] = a_i^(1 + (sigma_s/sigma_r) |g[n] - g[n-1]| / 255).
// The guide is 8-bit, so w takes 256 values per iteration: a table computed in
// binary64 and rounded once to FP32.
//
// A recurrence is an affine map per element; a pass is a chunked parallel scan:
// every thread runs its segment with a zero carry while recording the segment's
// map (A, B), the maps are scanned across threads, and a second sweep adds
// A_prefix * carry. Rows: one CTA per row (256 segments, warp-shuffle scan).
// Columns: one CTA per strip of SW (4, or 2 for tall frames) adjacent columns
// holding the whole strip in shared memory (SW x NSEG segments), sized so that
// two CTAs share an SM. Staging uses cp.async so all copies are in flight at once. Each pass therefore reads and writes the
// planes exactly once; the first row pass builds its input from the corner
// list (no dense zero planes are read) and the last column pass writes
// F = P~ / N~ directly.
#include <math.h>

#include "hdrreg_internal.cuh"

namespace hdrreg {

namespace {

constexpr int kNT = 256;
constexpr int kMaxDtIters = 8;

struct Aff {  // y -> A y + B, one A for the three planes
    float A, B0, B1, B2;
};

__device__ __forceinline__ Aff compose(const Aff& first, const Aff& second)
{
    Aff r;
    r.A = second.A * first.A;
    r.B0 = fmaf(second.A, first.B0, second.B0);
    r.B1 = fmaf(second.A, first.B1, second.B1);
    r.B2 = fmaf(second.A, first.B2, second.B2);
    return r;
}

__device__ __forceinline__ Aff shfl_up_aff(const Aff& a, int d)
{
    Aff r;
    r.A = __shfl_up_sync(0xffffffffu, a.A, d);
    r.B0 = __shfl_up_sync(0xffffffffu, a.B0, d);
    r.B1 = __shfl_up_sync(0xffffffffu, a.B1, d);
    r.B2 = __shfl_up_sync(0xffffffffu, a.B2, d);
    return r;
}

// Exclusive scan of the 256 per-thread maps in thread order (first = thread 0);
// returns the carry (B of the composed prefix applied to 0) for this thread.
__device__ __forceinline__ Aff block_exclusive_scan(Aff mine, Aff* wtot)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    Aff inc = mine;
    for (int d = 1; d < 32; d <<= 1) {
        const Aff o = shfl_up_aff(inc, d);
        if (lane >= d) inc = compose(o, inc);
    }
    Aff exc = shfl_up_aff(inc, 1);
    if (lane == 0) exc = Aff{1.f, 0.f, 0.f, 0.f};
    if (lane == 31) wtot[warp] = inc;
    __syncthreads();
    Aff pre{1.f, 0.f, 0.f, 0.f};
    for (int k = 0; k < warp; k++) pre = compose(pre, wtot[k]);
    __syncthreads();
    return compose(pre, exc);
}

__device__ __forceinline__ int absdiff(int a, int b) { return a > b ? a - b : b - a; }

// ------------------------------------------------------------------ row pass
template <bool kSparse>
__global__ void __launch_bounds__(kNT) k_dt_rows(float* __restrict__ P0, float* __restrict__ P1,
                                                 float* __restrict__ P2,
                                                 const uint8_t* __restrict__ guide, int w, int h,
                                                 int L, int gmode, DtLut lut_in, FlowCorners fc)
{
    extern __shared__ __align__(16) float sm[];
    __shared__ float lut[256];
    __shared__ Aff wtot[kNT / 32];
    const int Wp = kNT * L;
    float* s0 = sm;
    float* s1 = sm + Wp;
    float* s2 = sm + 2 * Wp;
    uint8_t* g = reinterpret_cast<uint8_t*>(sm + 3 * Wp);
    const int y = blockIdx.x, tid = threadIdx.x;
    lut[tid] = lut_in.w[tid];
    const size_t row = (size_t)y * w;
    // guide row: 16-byte, 4-byte or byte copies depending on alignment (gmode 2/1/0)
    if (gmode == 2) {
        for (int i = tid; i < w / 16; i += kNT) cp_async16(g + 16 * i, guide + row + 16 * i);
    } else if (gmode == 1) {
        for (int i = tid; i < w / 4; i += kNT) cp_async4(g + 4 * i, guide + row + 4 * i);
    } else {
        for (int x = tid; x < w; x += kNT) g[x] = guide[row + x];
    }
    if (kSparse) {
        for (int x = tid; x < w; x += kNT) {
            s0[x] = 0.f;
            s1[x] = 0.f;
            s2[x] = 0.f;
        }
        __syncthreads();
        const int ty = y / fc.tile;
        if (ty < fc.nty) {
            for (int tx = tid; tx < fc.ntx; tx += kNT) {
                const int t = ty * fc.ntx + tx;
                if (!((fc.mask[t >> 5] >> (t & 31)) & 1u)) continue;
                if (fc.corner_xy[2 * t + 1] != y) continue;
                const int cx = fc.corner_xy[2 * t];
                double bx = (double)cx, by = (double)y;
                if (!fc.full) {
                    double xs, ys;
                    if (!project_px(fc.H, cx, y, w, h, xs, ys)) continue;
                    bx = xs;
                    by = ys;
                }
                s0[cx] = (float)((double)fc.match_xy[2 * t] - bx);
                s1[cx] = (float)((double)fc.match_xy[2 * t + 1] - by);
                s2[cx] = 1.f;
            }
        }
    } else if ((w & 3) == 0) {
        for (int i = tid; i < w / 4; i += kNT) {
            cp_async16(s0 + 4 * i, P0 + row + 4 * i);
            cp_async16(s1 + 4 * i, P1 + row + 4 * i);
            cp_async16(s2 + 4 * i, P2 + row + 4 * i);
        }
    } else {
        for (int x = tid; x < w; x += kNT) {
            cp_async4(s0 + x, P0 + row + x);
            cp_async4(s1 + x, P1 + row + x);
            cp_async4(s2 + x, P2 + row + x);
        }
    }
    cp_async_wait_all();
    __syncthreads();

    const int x0 = tid * L, x1 = min(x0 + L, w);
    // forward, zero carry
    Aff m{1.f, 0.f, 0.f, 0.f};
    {
        float y0 = 0.f, y1 = 0.f, y2 = 0.f, A = 1.f;
        for (int x = x0; x < x1; x++) {
            const float a0 = s0[x], a1 = s1[x], a2 = s2[x];
            if (x == 0) {
                y0 = a0; y1 = a1; y2 = a2; A = 0.f;
            } else {
                const float wt = lut[absdiff(g[x], g[x - 1])];
                y0 = fmaf(wt, y0 - a0, a0);
                y1 = fmaf(wt, y1 - a1, a1);
                y2 = fmaf(wt, y2 - a2, a2);
                A *= wt;
            }
            s0[x] = y0; s1[x] = y1; s2[x] = y2;
        }
        m = Aff{A, y0, y1, y2};
    }
    Aff c = block_exclusive_scan(m, wtot);
    {
        float pre = 1.f;
        for (int x = x0; x < x1; x++) {
            pre = (x == 0) ? 0.f : pre * lut[absdiff(g[x], g[x - 1])];
            s0[x] = fmaf(pre, c.B0, s0[x]);
            s1[x] = fmaf(pre, c.B1, s1[x]);
            s2[x] = fmaf(pre, c.B2, s2[x]);
        }
    }
    __syncthreads();
    // backward, zero carry from the right; scanned in reverse thread order
    {
        float k0 = 0.f, k1 = 0.f, k2 = 0.f, A = 1.f;
        for (int x = x1 - 1; x >= x0; x--) {
            const float a0 = s0[x], a1 = s1[x], a2 = s2[x];
            if (x == w - 1) {
                k0 = a0; k1 = a1; k2 = a2; A = 0.f;
            } else {
                const float wt = lut[absdiff(g[x + 1], g[x])];
                k0 = fmaf(wt, k0 - a0, a0);
                k1 = fmaf(wt, k1 - a1, a1);
                k2 = fmaf(wt, k2 - a2, a2);
                A *= wt;
            }
            s0[x] = k0; s1[x] = k1; s2[x] = k2;
        }
        m = Aff{A, k0, k1, k2};
    }
    // thread r of the reversed order holds segment kNT-1-r
    __shared__ Aff agg[kNT];
    agg[tid] = m;
    __syncthreads();
    const Aff mine_rev = agg[kNT - 1 - tid];
    __syncthreads();
    const Aff crev = block_exclusive_scan(mine_rev, wtot);
    agg[kNT - 1 - tid] = crev;
    __syncthreads();
    c = agg[tid];
    {
        float suf = 1.f;
        for (int x = x1 - 1; x >= x0; x--) {
            suf = (x == w - 1) ? 0.f : suf * lut[absdiff(g[x + 1], g[x])];
            s0[x] = fmaf(suf, c.B0, s0[x]);
            s1[x] = fmaf(suf, c.B1, s1[x]);
            s2[x] = fmaf(suf, c.B2, s2[x]);
        }
    }
    __syncthreads();
    if ((w & 3) == 0) {
        float4* a = reinterpret_cast<float4*>(P0 + row);
        float4* b = reinterpret_cast<float4*>(P1 + row);
        float4* cc = reinterpret_cast<float4*>(P2 + row);
        for (int i = tid; i < w / 4; i += kNT) {
            a[i] = reinterpret_cast<const float4*>(s0)[i];
            b[i] = reinterpret_cast<const float4*>(s1)[i];
            cc[i] = reinterpret_cast<const float4*>(s2)[i];
        }
    } else {
        for (int x = tid; x < w; x += kNT) {
            P0[row + x] = s0[x];
            P1[row + x] = s1[x];
            P2[row + x] = s2[x];
        }
    }
}

// --------------------------------------------------------------- column pass
template <int SW>
__global__ void __launch_bounds__(kNT) k_dt_cols(float* __restrict__ P0, float* __restrict__ P1,
                                                 float* __restrict__ P2,
                                                 const uint8_t* __restrict__ guide, int w, int h,
                                                 int L, int vec, DtLut lut_in, int final_pass,
                                                 float flow_eps, float* __restrict__ Fu,
                                                 float* __restrict__ Fv, int fpitch)
{
    constexpr int NSEG = kNT / SW;
    extern __shared__ __align__(16) float sm[];
    __shared__ float lut[256];
    __shared__ Aff agg[NSEG][SW];
    const int Hp = NSEG * L;  // padded rows
    float* s0 = sm;
    float* s1 = sm + (size_t)Hp * SW;
    float* s2 = sm + (size_t)2 * Hp * SW;
    uint8_t* g = reinterpret_cast<uint8_t*>(sm + (size_t)3 * Hp * SW);
    const int tid = threadIdx.x;
    const int xs0 = blockIdx.x * SW;
    const int ncols = min(SW, w - xs0);
    lut[tid] = lut_in.w[tid];
    // stage the strip: SW floats per row and plane, SW guide bytes per row
    if (ncols == SW && vec) {
        for (int r = tid; r < h; r += kNT) {
            const size_t off = (size_t)r * w + xs0;
            if (SW == 4) {
                cp_async16(s0 + r * SW, P0 + off);
                cp_async16(s1 + r * SW, P1 + off);
                cp_async16(s2 + r * SW, P2 + off);
                cp_async4(g + r * SW, guide + off);
            } else {
                cp_async8(s0 + r * SW, P0 + off);
                cp_async8(s1 + r * SW, P1 + off);
                cp_async8(s2 + r * SW, P2 + off);
                g[r * SW] = guide[off];
                g[r * SW + 1] = guide[off + 1];
            }
        }
    } else {
        for (int i = tid; i < h * SW; i += kNT) {
            const int r = i / SW, cc = i % SW;
            if (cc < ncols) {
                const size_t off = (size_t)r * w + xs0 + cc;
                cp_async4(s0 + r * SW + cc, P0 + off);
                cp_async4(s1 + r * SW + cc, P1 + off);
                cp_async4(s2 + r * SW + cc, P2 + off);
            }
            g[r * SW + cc] = cc < ncols ? guide[(size_t)r * w + xs0 + cc] : 0;
        }
    }
    cp_async_wait_all();
    __syncthreads();

    const int c = tid % SW, s = tid / SW;
    const bool col_ok = c < ncols;
    const int r0 = s * L, r1 = min(r0 + L, h);
    // forward, zero carry
    {
        float y0 = 0.f, y1 = 0.f, y2 = 0.f, A = 1.f;
        if (col_ok)
            for (int r = r0; r < r1; r++) {
                const int o = r * SW + c;
                const float a0 = s0[o], a1 = s1[o], a2 = s2[o];
                if (r == 0) {
                    y0 = a0; y1 = a1; y2 = a2; A = 0.f;
                } else {
                    const float wt = lut[absdiff(g[o], g[o - SW])];
                    y0 = fmaf(wt, y0 - a0, a0);
                    y1 = fmaf(wt, y1 - a1, a1);
                    y2 = fmaf(wt, y2 - a2, a2);
                    A *= wt;
                }
                s0[o] = y0; s1[o] = y1; s2[o] = y2;
            }
        agg[s][c] = Aff{A, y0, y1, y2};
    }
    __syncthreads();
    if (tid < SW) {  // per column: sequential exclusive scan over the segments
        Aff run{1.f, 0.f, 0.f, 0.f};
        for (int k = 0; k < NSEG; k++) {
            const Aff a = agg[k][tid];
            agg[k][tid] = run;
            run = compose(run, a);
        }
    }
    __syncthreads();
    {
        const Aff cin = agg[s][c];
        float pre = 1.f;
        if (col_ok)
            for (int r = r0; r < r1; r++) {
                const int o = r * SW + c;
                pre = (r == 0) ? 0.f : pre * lut[absdiff(g[o], g[o - SW])];
                s0[o] = fmaf(pre, cin.B0, s0[o]);
                s1[o] = fmaf(pre, cin.B1, s1[o]);
                s2[o] = fmaf(pre, cin.B2, s2[o]);
            }
    }
    __syncthreads();
    // backward, zero carry from below
    {
        float k0 = 0.f, k1 = 0.f, k2 = 0.f, A = 1.f;
        if (col_ok)
            for (int r = r1 - 1; r >= r0; r--) {
                const int o = r * SW + c;
                const float a0 = s0[o], a1 = s1[o], a2 = s2[o];
                if (r == h - 1) {
                    k0 = a0; k1 = a1; k2 = a2; A = 0.f;
                } else {
                    const float wt = lut[absdiff(g[o + SW], g[o])];
                    k0 = fmaf(wt, k0 - a0, a0);
                    k1 = fmaf(wt, k1 - a1, a1);
                    k2 = fmaf(wt, k2 - a2, a2);
                    A *= wt;
                }
                s0[o] = k0; s1[o] = k1; s2[o] = k2;
            }
        agg[s][c] = Aff{A, k0, k1, k2};
    }
    __syncthreads();
    if (tid < SW) {  // reverse exclusive scan (from the last segment up)
        Aff run{1.f, 0.f, 0.f, 0.f};
        for (int k = NSEG - 1; k >= 0; k--) {
            const Aff a = agg[k][tid];
            agg[k][tid] = run;
            run = compose(run, a);
        }
    }
    __syncthreads();
    {
        const Aff cin = agg[s][c];
        float suf = 1.f;
        if (col_ok)
            for (int r = r1 - 1; r >= r0; r--) {
                const int o = r * SW + c;
                suf = (r == h - 1) ? 0.f : suf * lut[absdiff(g[o + SW], g[o])];
                s0[o] = fmaf(suf, cin.B0, s0[o]);
                s1[o] = fmaf(suf, cin.B1, s1[o]);
                s2[o] = fmaf(suf, cin.B2, s2[o]);
            }
    }
    __syncthreads();
    // store
    if (final_pass && ncols == SW && vec && SW == 4) {
        for (int r = tid; r < h; r += kNT) {
            const float4 a = *reinterpret_cast<const float4*>(s0 + r * SW);
            const float4 b = *reinterpret_cast<const float4*>(s1 + r * SW);
            const float4 n = *reinterpret_cast<const float4*>(s2 + r * SW);
            float4 u, v;
            u.x = n.x >= flow_eps ? a.x / n.x : 0.f;
            u.y = n.y >= flow_eps ? a.y / n.y : 0.f;
            u.z = n.z >= flow_eps ? a.z / n.z : 0.f;
            u.w = n.w >= flow_eps ? a.w / n.w : 0.f;
            v.x = n.x >= flow_eps ? b.x / n.x : 0.f;
            v.y = n.y >= flow_eps ? b.y / n.y : 0.f;
            v.z = n.z >= flow_eps ? b.z / n.z : 0.f;
            v.w = n.w >= flow_eps ? b.w / n.w : 0.f;
            const size_t off = (size_t)r * fpitch + xs0;
            *reinterpret_cast<float4*>(Fu + off) = u;
            *reinterpret_cast<float4*>(Fv + off) = v;
        }
    } else if (final_pass) {
        for (int i = tid; i < h * SW; i += kNT) {
            const int r = i / SW, cc = i % SW;
            if (cc < ncols) {
                const float n = s2[r * SW + cc];
                const bool ok = n >= flow_eps;
                const size_t off = (size_t)r * fpitch + xs0 + cc;
                Fu[off] = ok ? s0[r * SW + cc] / n : 0.f;
                Fv[off] = ok ? s1[r * SW + cc] / n : 0.f;
            }
        }
    } else if (ncols == SW && vec && SW == 4) {
        for (int r = tid; r < h; r += kNT) {
            const size_t off = (size_t)r * w + xs0;
            *reinterpret_cast<float4*>(P0 + off) = *reinterpret_cast<const float4*>(s0 + r * SW);
            *reinterpret_cast<float4*>(P1 + off) = *reinterpret_cast<const float4*>(s1 + r * SW);
            *reinterpret_cast<float4*>(P2 + off) = *reinterpret_cast<const float4*>(s2 + r * SW);
        }
    } else {
        for (int i = tid; i < h * SW; i += kNT) {
            const int r = i / SW, cc = i % SW;
            if (cc < ncols) {
                const size_t off = (size_t)r * w + xs0 + cc;
                P0[off] = s0[r * SW + cc];
                P1[off] = s1[r * SW + cc];
                P2[off] = s2[r * SW + cc];
            }
        }
    }
}

int odd_up(int v) { return (v & 1) ? v : v + 1; }

// Two CTAs per SM need <= ~110 KB of dynamic shared memory each; one CTA per SM
// can take up to 220 KB (the static part of the column kernel is ~5 KB).
constexpr size_t kSmemTwoPerSm = 110 * 1024;
constexpr size_t kSmemBudget = 220 * 1024;

size_t col_smem(int h, int sw)
{
    const int nseg = kNT / sw;
    const int L = odd_up((h + nseg - 1) / nseg);
    const size_t hp = (size_t)nseg * L;
    return hp * sw * 12 + align_up(hp * sw, 16);
}

int pick_sw(int h)
{
    for (int sw : {4, 2})
        if (col_smem(h, sw) <= kSmemTwoPerSm) return sw;
    for (int sw : {4, 2})
        if (col_smem(h, sw) <= kSmemBudget) return sw;
    return 0;
}

size_t row_smem(int w)
{
    const int L = odd_up((w + kNT - 1) / kNT);
    const size_t wp = (size_t)kNT * L;
    return wp * 12 + align_up(wp, 16);
}

template <int SW>
void launch_cols(float* P0, float* P1, float* P2, const uint8_t* guide, int w, int h,
                 const DtLut& lut, int final_pass, float eps, float* Fu, float* Fv, int fpitch,
                 cudaStream_t s)
{
    constexpr int NSEG = kNT / SW;
    const int L = odd_up((h + NSEG - 1) / NSEG);
    const size_t smem = col_smem(h, SW);
    ensure_smem((const void*)k_dt_cols<SW>, smem);
    const int grid = (w + SW - 1) / SW;
    // vector staging needs every strip row start aligned: planes (workspace) and the
    // caller's guide / flow planes
    const uintptr_t al = (uintptr_t)guide | (uintptr_t)Fu | (uintptr_t)Fv;
    const int vec = (w % SW == 0) && (w % 4 == 0) && (fpitch % 4 == 0) && (al % 4 == 0) &&
                    (((uintptr_t)Fu | (uintptr_t)Fv) % 16 == 0);
    note_launch();
    k_dt_cols<SW><<<grid, kNT, smem, s>>>(P0, P1, P2, guide, w, h, L, vec, lut, final_pass, eps,
                                          Fu, Fv, fpitch);
}

}  // namespace

DtLut make_dt_lut(double sigma_s, double sigma_r, int iters, int i)
{
    const double sig = sigma_s * sqrt(3.0) * pow(2.0, (double)(iters - 1 - i)) /
                       sqrt(pow(4.0, (double)iters) - 1.0);
    const double a = exp(-sqrt(2.0) / sig);
    DtLut t;
    for (int v = 0; v < 256; v++) {
        const double d = 1.0 + (sigma_s / sigma_r) * (double)v / 255.0;
        t.w[v] = (float)pow(a, d);
    }
    return t;
}

int flow_supported(int w, int h)
{
    return w >= 1 && h >= 1 && row_smem(w) <= kSmemBudget && pick_sw(h) != 0;
}

int flow_pitch(int w) { return (w + 15) / 16 * 16; }

// Three FP32 planes at the padded pitch, the error word, the fast path's tile maps and
// corner records, and a copy of the guide at the padded pitch (for widths whose rows
// are not 16-byte aligned).
size_t flow_ws_bytes(int w, int h)
{
    const size_t pp = (size_t)flow_pitch(w);
    return 3 * align_up(pp * h * 4, 256) + 256 + flow_fast_extra_bytes(w, h) +
           align_up(pp * h, 256);
}

namespace {
__global__ void k_copy_rows(const uint8_t* __restrict__ in, int w, int h, uint8_t* __restrict__ out,
                            int pitch)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x < pitch) out[(size_t)y * pitch + x] = x < w ? in[(size_t)y * w + x] : 0;
}
}  // namespace

int* flow_error_word(void* ws, int w, int h)
{
    const size_t plane = align_up((size_t)flow_pitch(w) * h * 4, 256);
    return reinterpret_cast<int*>(static_cast<uint8_t*>(ws) + 3 * plane);
}

void launch_flow(const uint8_t* guide, int w, int h, const FlowCorners& fc, double sigma_s,
                 double sigma_r, int iters, double flow_eps, float* flow_u, float* flow_v,
                 int fpitch, void* ws, cudaStream_t s)
{
    const int pp = flow_pitch(w);
    const size_t plane = align_up((size_t)pp * h * 4, 256);
    float* P0 = static_cast<float*>(ws);
    float* P1 = reinterpret_cast<float*>(static_cast<uint8_t*>(ws) + plane);
    float* P2 = reinterpret_cast<float*>(static_cast<uint8_t*>(ws) + 2 * plane);
    int* err = flow_error_word(ws, w, h);
    uint8_t* extra = static_cast<uint8_t*>(ws) + 3 * plane + 256;
    uint8_t* gcopy = extra + flow_fast_extra_bytes(w, h);
    const bool out_ok = fpitch % 4 == 0 && ((uintptr_t)flow_u % 16) == 0 &&
                        ((uintptr_t)flow_v % 16) == 0;
    if (iters <= kMaxDtIters && out_ok && flow_fast_supported(w, h)) {
        // the guide at a 16-byte-aligned pitch: the caller's rows, or a padded copy
        const uint8_t* g = guide;
        int gp = w;
        if ((w % 16) != 0 || ((uintptr_t)guide % 16) != 0) {
            note_launch();
            k_copy_rows<<<dim3((pp + 255) / 256, h), 256, 0, s>>>(guide, w, h, gcopy, pp);
            g = gcopy;
            gp = pp;
        }
        DtLut luts[kMaxDtIters];
        for (int i = 0; i < iters; i++) luts[i] = make_dt_lut(sigma_s, sigma_r, iters, i);
        if (launch_flow_fast(g, gp, w, h, fc, luts, iters, flow_eps, flow_u, flow_v, fpitch, P0, P1,
                             P2, pp, err, extra, s))
            return;
    }
    cudaMemsetAsync(err, 0, sizeof(int), s);  // the basic path has no waits that could set it
    const int Lr = odd_up((w + kNT - 1) / kNT);
    const size_t rs = row_smem(w);
    ensure_smem((const void*)k_dt_rows<true>, rs);
    ensure_smem((const void*)k_dt_rows<false>, rs);
    const int sw = pick_sw(h);
    const int gmode = ((uintptr_t)guide % 16 == 0 && w % 16 == 0) ? 2
                      : (((uintptr_t)guide % 4 == 0 && w % 4 == 0) ? 1 : 0);
    for (int i = 0; i < iters; i++) {
        const DtLut lut = make_dt_lut(sigma_s, sigma_r, iters, i);
        note_launch();
        if (i == 0)
            k_dt_rows<true><<<h, kNT, rs, s>>>(P0, P1, P2, guide, w, h, Lr, gmode, lut, fc);
        else
            k_dt_rows<false><<<h, kNT, rs, s>>>(P0, P1, P2, guide, w, h, Lr, gmode, lut, fc);
        const int fin = i == iters - 1;
        if (sw == 4)
            launch_cols<4>(P0, P1, P2, guide, w, h, lut, fin, (float)flow_eps, flow_u, flow_v,
                           fpitch, s);
        else
            launch_cols<2>(P0, P1, P2, guide, w, h, lut, fin, (float)flow_eps, flow_u, flow_v,
                           fpitch, s);
    }
}

}  // namespace hdrreg
