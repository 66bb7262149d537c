// Row a8, fast path: the domain-transform passes with register-resident
// segments and TMA staging (Sec. 2.4; Gastal and Oliveira 2011).
//
// Both passes run the same chunked scan as the basic kernels in flow.cu, but
// every thread keeps its whole segment of the three planes (P_u, P_v, N) and
// the segment's link weights in registers, so the four sweeps (forward local,
// forward carry, backward local, backward carry) are pure FMA chains.
//  * Row pass: persistent CTAs walk the rows with two buffers; rows are staged
//    with 1D bulk copies (cp.async.bulk, mbarrier completion) and written back
//    the same way; the first pass builds its planes from the corner list.
//  * Column pass: tiles of 32 columns x 64 rows in three phases (tile maps,
//    per-column carry chain, tile apply); tiles move with 2D tensor copies
//    (cp.async.bulk.tensor, 32 x 64 boxes of 128-byte rows).
// Link weights: w_link(r) = a_i^(1 + (sigma_s/sigma_r)|g_r - g_{r-1}|/255) from the
// 256-entry table, and 0 across the frame ends, so J[0] = x[0] and K[n-1] = J[n-1]
// without branches. Every wait on a barrier is bounded; a timeout sets the
// error word and the kernel drains its copies and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "hdrreg_internal.cuh"

namespace hdrreg {

namespace {

constexpr int kRowNT = 256;
constexpr uint32_t kWaitIters = 1u << 22;

struct Aff {  // y -> A y + B, shared A for the three planes
    float A, B0, B1, B2;
};

__device__ __forceinline__ Aff compose(const Aff& first, const Aff& second)
{
    return Aff{second.A * first.A, fmaf(second.A, first.B0, second.B0),
               fmaf(second.A, first.B1, second.B1), fmaf(second.A, first.B2, second.B2)};
}

template <bool kUp>
__device__ __forceinline__ Aff shfl_aff(const Aff& a, int d)
{
    if (kUp)
        return Aff{__shfl_up_sync(0xffffffffu, a.A, d), __shfl_up_sync(0xffffffffu, a.B0, d),
                   __shfl_up_sync(0xffffffffu, a.B1, d), __shfl_up_sync(0xffffffffu, a.B2, d)};
    return Aff{__shfl_down_sync(0xffffffffu, a.A, d), __shfl_down_sync(0xffffffffu, a.B0, d),
               __shfl_down_sync(0xffffffffu, a.B1, d), __shfl_down_sync(0xffffffffu, a.B2, d)};
}

__device__ __forceinline__ int absdiff(int a, int b) { return (int)__sad(a, b, 0u); }

// ---------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(su32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait: false after kWaitIters polls (about a second at most)
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity)
{
    for (uint32_t i = 0; i < kWaitIters; i++) {
        if (mbar_try(bar, parity)) return true;
        if (i > 16) __nanosleep(64);
    }
    return false;
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(su32(dst)),
        "l"(src), "r"(bytes), "r"(su32(bar))
        : "memory");
}

__device__ __forceinline__ void bulk_store(void* dst, const void* src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
                 "r"(su32(src)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, "
        "{%2, %3}], [%4];" ::"r"(su32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(su32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, int x, int y, const void* src)
{
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     map),
                 "r"(x), "r"(y), "r"(su32(src))
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// ------------------------------------------------ register-resident sweeps
// v[k][i]: element i of the thread's segment in plane k; wl[i]: weight of the link
// into element i (from i-1); wl[L]: link from the segment's last element to the
// next segment's first. The local sweeps start from a zero carry and return the
// segment's affine map; the carry sweeps add prefix (suffix) products times the
// scanned carry.
template <int LM>
__device__ __forceinline__ Aff sweep_fwd(float (&v)[3][LM], const float (&wl)[LM + 1], int L)
{
    float y0 = 0.f, y1 = 0.f, y2 = 0.f, A = 1.f;
#pragma unroll
    for (int i = 0; i < LM; i++) {
        if (i < L) {
            const float wt = wl[i];
            y0 = fmaf(wt, y0 - v[0][i], v[0][i]);
            y1 = fmaf(wt, y1 - v[1][i], v[1][i]);
            y2 = fmaf(wt, y2 - v[2][i], v[2][i]);
            A *= wt;
            v[0][i] = y0;
            v[1][i] = y1;
            v[2][i] = y2;
        }
    }
    return Aff{A, y0, y1, y2};
}

template <int LM>
__device__ __forceinline__ void carry_fwd(float (&v)[3][LM], const float (&wl)[LM + 1], int L,
                                          const Aff& c)
{
    float P = 1.f;
#pragma unroll
    for (int i = 0; i < LM; i++) {
        if (i < L) {
            P *= wl[i];
            v[0][i] = fmaf(P, c.B0, v[0][i]);
            v[1][i] = fmaf(P, c.B1, v[1][i]);
            v[2][i] = fmaf(P, c.B2, v[2][i]);
        }
    }
}

template <int LM>
__device__ __forceinline__ Aff sweep_bwd(float (&v)[3][LM], const float (&wl)[LM + 1], int L)
{
    float k0 = 0.f, k1 = 0.f, k2 = 0.f, A = 1.f;
#pragma unroll
    for (int i = LM - 1; i >= 0; i--) {
        if (i < L) {
            const float wt = (i == L - 1) ? wl[LM] : wl[i + 1];
            k0 = fmaf(wt, k0 - v[0][i], v[0][i]);
            k1 = fmaf(wt, k1 - v[1][i], v[1][i]);
            k2 = fmaf(wt, k2 - v[2][i], v[2][i]);
            A *= wt;
            v[0][i] = k0;
            v[1][i] = k1;
            v[2][i] = k2;
        }
    }
    return Aff{A, k0, k1, k2};
}

template <int LM>
__device__ __forceinline__ void carry_bwd(float (&v)[3][LM], const float (&wl)[LM + 1], int L,
                                          const Aff& c)
{
    float S = 1.f;
#pragma unroll
    for (int i = LM - 1; i >= 0; i--) {
        if (i < L) {
            S *= (i == L - 1) ? wl[LM] : wl[i + 1];
            v[0][i] = fmaf(S, c.B0, v[0][i]);
            v[1][i] = fmaf(S, c.B1, v[1][i]);
            v[2][i] = fmaf(S, c.B2, v[2][i]);
        }
    }
}

// Exclusive scan over segments ordered by lane (stride `st` lanes within a warp),
// then by warp; kUp = forward order, otherwise reverse order. `tot` holds one map
// per (warp, column). Returns the composed map of all earlier segments.
template <bool kUp, int kWarps, int kCols>
__device__ __forceinline__ Aff seg_scan(Aff mine, Aff (*tot)[kCols], int col)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int st = kCols;            // lanes between consecutive segments of one column
    constexpr int nseg = 32 / kCols;     // segments per warp
    const int sl = lane / kCols;
    Aff inc = mine;
#pragma unroll
    for (int d = 1; d < nseg; d <<= 1) {
        const Aff o = shfl_aff<kUp>(inc, d * st);
        if (kUp ? (sl >= d) : (sl + d < nseg)) inc = compose(o, inc);
    }
    Aff exc = shfl_aff<kUp>(inc, st);
    if (kUp ? (sl == 0) : (sl == nseg - 1)) exc = Aff{1.f, 0.f, 0.f, 0.f};
    if (kUp ? (sl == nseg - 1) : (sl == 0)) tot[warp][col] = inc;
    __syncthreads();
    // unrolled and predicated: the warps' maps are all loaded before the chain
    Aff pre{1.f, 0.f, 0.f, 0.f};
    if (kUp) {
#pragma unroll
        for (int k = 0; k < kWarps - 1; k++)
            if (k < warp) pre = compose(pre, tot[k][col]);
    } else {
#pragma unroll
        for (int k = kWarps - 1; k > 0; k--)
            if (k > warp) pre = compose(pre, tot[k][col]);
    }
    __syncthreads();
    return compose(pre, exc);
}

// ------------------------------------------------------ corner records
// One record per level-0 tile for the first row pass: {x, y, residual u, residual v}
// of its kept corner (y = -1 without one). The residual is q - H(p) (q - p when the
// full displacement is propagated), evaluated in binary64 and rounded to FP32 once.
// Also zeroes the flow's error word (it is the first launch of the fast path).
__global__ void k_flow_corner_records(FlowCorners fc, int w, int h, int4* __restrict__ rec,
                                      int* __restrict__ err)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) *err = 0;
    const int n = fc.ntx * fc.nty;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        int4 r = make_int4(0, -1, 0, 0);
        if ((fc.mask[t >> 5] >> (t & 31)) & 1u) {
            const int cx = fc.corner_xy[2 * t], cy = fc.corner_xy[2 * t + 1];
            double bx = (double)cx, by = (double)cy;
            bool ok = true;
            if (!fc.full) ok = project_px(fc.H, cx, cy, w, h, bx, by);
            if (ok)
                r = make_int4(cx, cy, __float_as_int((float)((double)fc.match_xy[2 * t] - bx)),
                              __float_as_int((float)((double)fc.match_xy[2 * t + 1] - by)));
        }
        rec[t] = r;
    }
}

// ---------------------------------------------------------------- row pass
// Persistent, double-buffered row pass: each CTA walks
// rows y = blockIdx.x + k * gridDim.x; while row k computes, row k+1 is loading
// into the other buffer and row k-1 is storing.
template <int LM, bool kSparse>
__global__ void __launch_bounds__(kRowNT, LM <= 17 ? 3 : 1) k_dt_rows_pipe(float* __restrict__ P0,
                                                         float* __restrict__ P1,
                                                         float* __restrict__ P2,
                                                         const uint8_t* __restrict__ guide,
                                                         int w, int h, int ppitch, int gpitch,
                                                         DtLut lut_in, FlowCorners fc,
                                                         const int4* __restrict__ rec, int* err)
{
    extern __shared__ __align__(128) float sm[];
    __shared__ float lut[256];
    __shared__ Aff tot[kRowNT / 32][1];
    __shared__ __align__(8) uint64_t bar[2];
    constexpr int Wp = kRowNT * LM;          // floats per plane buffer
    constexpr int kBuf = 3 * Wp + Wp / 4;    // floats per buffer (3 planes + guide bytes)
    const int tid = threadIdx.x;
    for (int i = tid; i < 256; i += blockDim.x) lut[i] = lut_in.w[i];
    if (tid == 0) {
        mbar_init(&bar[0]);
        mbar_init(&bar[1]);
    }
    __syncthreads();
    // whole padded rows (pitches are multiples of 16 bytes); columns >= w are never used
    const uint32_t bytes = (kSparse ? 0u : 3u * (uint32_t)ppitch * 4u) + (uint32_t)gpitch;
    auto issue = [&](int y, int b) {
        if (tid == 0) {
            float* B = sm + b * kBuf;
            const size_t row = (size_t)y * ppitch;
            fence_async_smem();  // earlier reads of the buffer come before the copy's writes
            mbar_expect(&bar[b], bytes);
            if (!kSparse) {
                bulk_load(B, P0 + row, ppitch * 4, &bar[b]);
                bulk_load(B + Wp, P1 + row, ppitch * 4, &bar[b]);
                bulk_load(B + 2 * Wp, P2 + row, ppitch * 4, &bar[b]);
            }
            bulk_load(B + 3 * Wp, guide + (size_t)y * gpitch, gpitch, &bar[b]);
        }
    };
    uint32_t ph0 = 0, ph1 = 0;
    int y = blockIdx.x;
    if (y < h) issue(y, 0);
    // first pass: this thread's corner record (tile column tid) of the current row's tile
    // row, loaded one row ahead
    auto rec_of = [&](int yy) {
        const int ty = yy / fc.tile;
        return (kSparse && yy < h && ty < fc.nty && tid < fc.ntx) ? rec[ty * fc.ntx + tid]
                                                                  : make_int4(0, -1, 0, 0);
    };
    int4 rc = rec_of(y);
    for (int k = 0; y < h; y += gridDim.x, k++) {
        const int b = k & 1;
        const int yn = y + gridDim.x;
        const int4 rc_next = rec_of(yn);
        if (yn < h) {
            if (tid == 0) bulk_wait_read();  // the store of row k-1 has left buffer 1-b
            issue(yn, 1 - b);
        }
        const bool ok = __syncthreads_and(mbar_wait(&bar[b], b ? ph1 : ph0));
        if (b) ph1 ^= 1u; else ph0 ^= 1u;
        if (!ok) {
            if (tid == 0) {
                atomicExch(err, 1);
                mbar_wait(&bar[1 - b], b ? ph0 : ph1);
                bulk_wait_read();
            }
            return;
        }
        float* s0 = sm + b * kBuf;
        float* s1 = s0 + Wp;
        float* s2 = s0 + 2 * Wp;
        const uint8_t* g = reinterpret_cast<const uint8_t*>(s0 + 3 * Wp);
        const int x0 = tid * LM;
        bool empty = false;  // a row without corners filters to zeros: nothing to compute
        if (kSparse) {  // the planes of the first pass: residuals at this row's corners, else 0
#pragma unroll
            for (int i = 0; i < LM; i++) {
                s0[x0 + i] = 0.f;
                s1[x0 + i] = 0.f;
                s2[x0 + i] = 0.f;
            }
            __syncthreads();
            const int ty = y / fc.tile;
            int mine = 0;
            if (ty < fc.nty) {
                for (int tx = tid; tx < fc.ntx; tx += kRowNT) {
                    const int4 c = tx == tid ? rc : rec[ty * fc.ntx + tx];
                    if (c.y != y) continue;
                    s0[c.x] = __int_as_float(c.z);
                    s1[c.x] = __int_as_float(c.w);
                    s2[c.x] = 1.f;
                    mine = 1;
                }
            }
            empty = !__syncthreads_or(mine);
        }
        if (!empty) {
        float v[3][LM];
        float wl[LM + 1];
        // warps whose segments and their links all lie inside the row skip the frame tests
        const int wp = tid >> 5;
        if (wp > 0 && (32 * wp + 32) * LM < w) {
#pragma unroll
            for (int i = 0; i < LM; i++) {
                const int x = x0 + i;
                v[0][i] = s0[x];
                v[1][i] = s1[x];
                v[2][i] = s2[x];
                wl[i] = lut[absdiff(g[x], g[x - 1])];
            }
            wl[LM] = lut[absdiff(g[x0 + LM], g[x0 + LM - 1])];
        } else {
#pragma unroll
            for (int i = 0; i < LM; i++) {
                const int x = x0 + i;
                const bool in = x < w;
                v[0][i] = in ? s0[x] : 0.f;
                v[1][i] = in ? s1[x] : 0.f;
                v[2][i] = in ? s2[x] : 0.f;
                wl[i] = (in && x > 0) ? lut[absdiff(g[x], g[x - 1])] : 0.f;
            }
            const int x = x0 + LM;
            wl[LM] = (x < w) ? lut[absdiff(g[x], g[x - 1])] : 0.f;
        }
        Aff m = sweep_fwd<LM>(v, wl, LM);
        Aff c = seg_scan<true, kRowNT / 32, 1>(m, tot, 0);
        carry_fwd<LM>(v, wl, LM, c);
        m = sweep_bwd<LM>(v, wl, LM);
        c = seg_scan<false, kRowNT / 32, 1>(m, tot, 0);
        carry_bwd<LM>(v, wl, LM, c);
#pragma unroll
        for (int i = 0; i < LM; i++) {
            const int x = x0 + i;
            if (x < w) {
                s0[x] = v[0][i];
                s1[x] = v[1][i];
                s2[x] = v[2][i];
            }
        }
        }  // !empty
        fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            const size_t row = (size_t)y * ppitch;
            bulk_store(P0 + row, s0, ppitch * 4);
            bulk_store(P1 + row, s1, ppitch * 4);
            bulk_store(P2 + row, s2, ppitch * 4);
            bulk_commit();
        }
        rc = rc_next;
    }
    if (tid == 0) bulk_wait_read();
}

// ------------------------------------------------------------- column pass
// Three phases over tiles of 32 columns x 64 rows (one lane per column, eight
// 8-row segments = eight warps per tile):
//  A) per tile, the forward map (J_bottom = A_f c + B_f) and the backward value
//     at the tile's top row as a function of both carries,
//     K_top = K0 + Q c + S c' (c: forward carry entering at the top, c': backward
//     carry entering at the bottom; Q because the backward pass is linear in J =
//     J0 + P c): each segment's own map, folded over the tile's segments;
//  B) per column, the carries down and up its tiles (one warp per column, one CTA
//     per 32-column strip);
//  C) every tile recomputes its sweeps with the exact carries and stores.
// Tiles never wait on one another; phase C re-reads the tile (partly from L2). The
// maps and carries are stored [tile][value][column], so phases A and C move them as
// whole 128-byte lines.
constexpr int kTW = 32;
constexpr int kTSeg = 8;
constexpr int kTLS = 8;
constexpr int kTR = kTSeg * kTLS;  // 64 rows per tile
constexpr int kTNT = kTSeg * 32;   // 256 threads
constexpr int kAgg = 9;            // per (tile, column): A_f, B_f[3], K0[3], Q, S
constexpr int kCar = 6;            // per (tile, column): c[3], c'[3]

struct ColMaps {
    CUtensorMap in[3];   // planes, FP32 {w, h}, box {32, 64}
    CUtensorMap out[3];  // planes, or the flow planes (out[0], out[1]) for the final pass
    CUtensorMap guide;   // guide, u8 {w, h}, box {32, 66}: the tile plus a row above and below
};

constexpr int kGRows = kTR + 2;
constexpr int kTileBuf = (3 * kTR * kTW * 4 + kGRows * kTW + 1023) / 1024 * 1024;  // bytes

// One 8-row segment of a column tile in registers: rows r0 + sg*8 + i of column
// `lane`; plane k of the tile at P + k*kTR*kTW (rows of kTW floats); G row j is global
// row r0 - 1 + j. kInterior: every row of the tile and the row after it lie inside the
// frame (0 < r0 and r0 + kTR < h), so no element needs the frame tests.
template <bool kInterior>
__device__ __forceinline__ void tile_seg_load(const float* P, const uint8_t* G, const float* lut,
                                              int sg, int lane, int r0, int h,
                                              float (&v)[3][kTLS], float (&wl)[kTLS + 1])
{
#pragma unroll
    for (int i = 0; i < kTLS; i++) {
        const int rr = sg * kTLS + i, r = r0 + rr;
        const bool in = kInterior || r < h;
        v[0][i] = in ? P[(0 * kTR + rr) * kTW + lane] : 0.f;
        v[1][i] = in ? P[(1 * kTR + rr) * kTW + lane] : 0.f;
        v[2][i] = in ? P[(2 * kTR + rr) * kTW + lane] : 0.f;
        const float l = lut[absdiff(G[(rr + 1) * kTW + lane], G[rr * kTW + lane])];
        wl[i] = (kInterior || (r > 0 && r < h)) ? l : 0.f;
    }
    const int rr = sg * kTLS + kTLS, r = r0 + rr;
    const float l = lut[absdiff(G[(rr + 1) * kTW + lane], G[rr * kTW + lane])];
    wl[kTLS] = (kInterior || r < h) ? l : 0.f;
}

// Nine values of a row range of one column, as functions of the carries entering it:
// forward J_bottom = A c + B (c: J of the row above the range); backward K_top = K0 + Q c +
// S c' (c': K of the row below). fold(u, d) joins a range u with the range d below it:
// A = Ad Au, B = Ad Bu + Bd, K0 = K0u + Su (K0d + Qd Bu), Q = Qu + Su Qd Au, S = Su Sd.
struct Map9 {
    float A, B[3], K0[3], Q, S;
};

__device__ __forceinline__ Map9 fold(const Map9& u, const Map9& d)
{
    Map9 r;
    r.A = d.A * u.A;
#pragma unroll
    for (int p = 0; p < 3; p++) {
        r.B[p] = fmaf(d.A, u.B[p], d.B[p]);
        r.K0[p] = fmaf(u.S, fmaf(d.Q, u.B[p], d.K0[p]), u.K0[p]);
    }
    r.Q = fmaf(u.S * d.Q, u.A, u.Q);
    r.S = u.S * d.S;
    return r;
}

// Phase A on one tile (all threads): each 8-row segment's own Map9 (both sweeps from
// zero carries, with the derivative of the backward sweep in the forward carry carried
// along); the first segment's warp folds the eight, top to bottom, into the tile's nine
// values of column `lane`, out[k * ostride] in Map9 order. seg ([9][kTSeg][kTW] floats)
// is free again on return.
__device__ __forceinline__ void tile_maps(float (&v)[3][kTLS], const float (&wl)[kTLS + 1],
                                          float* seg, int sg, int lane, bool colok, float* out,
                                          size_t ostride)
{
    float y0 = 0.f, y1 = 0.f, y2 = 0.f, A = 1.f;
    float pv[kTLS];  // d J / d c: products of the links from the segment's top
#pragma unroll
    for (int i = 0; i < kTLS; i++) {
        const float wt = wl[i];
        y0 = fmaf(wt, y0 - v[0][i], v[0][i]);
        y1 = fmaf(wt, y1 - v[1][i], v[1][i]);
        y2 = fmaf(wt, y2 - v[2][i], v[2][i]);
        A *= wt;
        pv[i] = A;
        v[0][i] = y0;
        v[1][i] = y1;
        v[2][i] = y2;
    }
    float k0 = 0.f, k1 = 0.f, k2 = 0.f, k3 = 0.f, S = 1.f;
#pragma unroll
    for (int i = kTLS - 1; i >= 0; i--) {
        const float wt = wl[i + 1];
        k0 = fmaf(wt, k0 - v[0][i], v[0][i]);
        k1 = fmaf(wt, k1 - v[1][i], v[1][i]);
        k2 = fmaf(wt, k2 - v[2][i], v[2][i]);
        k3 = fmaf(wt, k3 - pv[i], pv[i]);
        S *= wt;
    }
    const float mv[9] = {A, y0, y1, y2, k0, k1, k2, k3, S};
#pragma unroll
    for (int k = 0; k < 9; k++) seg[(k * kTSeg + sg) * kTW + lane] = mv[k];
    __syncthreads();
    if (sg == 0 && colok) {
        auto at = [&](int q) {
            const float* p = seg + q * kTW + lane;
            return Map9{p[0], {p[kTSeg * kTW], p[2 * kTSeg * kTW], p[3 * kTSeg * kTW]},
                        {p[4 * kTSeg * kTW], p[5 * kTSeg * kTW], p[6 * kTSeg * kTW]},
                        p[7 * kTSeg * kTW], p[8 * kTSeg * kTW]};
        };
        Map9 m = at(0);
#pragma unroll
        for (int q = 1; q < kTSeg; q++) m = fold(m, at(q));
        out[0 * ostride] = m.A;
        out[1 * ostride] = m.B[0];
        out[2 * ostride] = m.B[1];
        out[3 * ostride] = m.B[2];
        out[4 * ostride] = m.K0[0];
        out[5 * ostride] = m.K0[1];
        out[6 * ostride] = m.K0[2];
        out[7 * ostride] = m.Q;
        out[8 * ostride] = m.S;
    }
    __syncthreads();  // seg is reused by the next tile
}

// Phase C on one tile (all threads): the sweeps again from the exact carries
// cr = {c[3] entering at the top, c'[3] entering at the bottom}; the results go to the
// output planes P in shared memory, once the store that last read them has drained (the
// flow u, v in planes 0 and 1 on the final pass: the sums over N, which is at least
// flow_eps = 1e-20 there, so the fast quotient is within 2 ulp).
__device__ __forceinline__ void tile_apply(float (&v)[3][kTLS], const float (&wl)[kTLS + 1],
                                           Aff (*agg)[kTW], int sg, int lane, const float (&cr)[6],
                                           float* P, int final_pass, float flow_eps)
{
    Aff m = sweep_fwd<kTLS>(v, wl, kTLS);
    agg[sg][lane] = m;
    __syncthreads();
    Aff pre = Aff{0.f, cr[0], cr[1], cr[2]};  // zero carries outside the image
#pragma unroll
    for (int q = 0; q < kTSeg - 1; q++) {
        if (q < sg) {
            pre = compose(pre, agg[q][lane]);
        }
    }
    carry_fwd<kTLS>(v, wl, kTLS, pre);
    __syncthreads();
    m = sweep_bwd<kTLS>(v, wl, kTLS);
    agg[sg][lane] = m;
    if (threadIdx.x == 0) bulk_wait_read();  // the output buffer's previous store has left it
    __syncthreads();
    Aff suf = Aff{0.f, cr[3], cr[4], cr[5]};
#pragma unroll
    for (int q = kTSeg - 1; q > 0; q--) {
        if (q > sg) {
            suf = compose(suf, agg[q][lane]);
        }
    }
    carry_bwd<kTLS>(v, wl, kTLS, suf);
#pragma unroll
    for (int i = 0; i < kTLS; i++) {
        const int rr = sg * kTLS + i;
        if (final_pass) {
            const bool okn = v[2][i] >= flow_eps;
            P[(0 * kTR + rr) * kTW + lane] = okn ? __fdividef(v[0][i], v[2][i]) : 0.f;
            P[(1 * kTR + rr) * kTW + lane] = okn ? __fdividef(v[1][i], v[2][i]) : 0.f;
        } else {
            P[(0 * kTR + rr) * kTW + lane] = v[0][i];
            P[(1 * kTR + rr) * kTW + lane] = v[1][i];
            P[(2 * kTR + rr) * kTW + lane] = v[2][i];
        }
    }
}

// Dynamic shared memory of the tile passes, bytes. Phase A: the tile (planes + guide rows,
// 1 KB-rounded), the link table, the segment maps, the barrier. Phase C, packed so that
// four CTAs fit an SM: the tile, the output planes 128-byte aligned after its bytes, the
// link table, the composition records, the barrier, the item's six carry lines.
constexpr int kTileOut = (3 * kTR * kTW * 4 + kGRows * kTW + 127) / 128 * 128;
template <bool kApply>
constexpr int kTileLut = kApply ? kTileOut + 3 * kTR * kTW * 4 : kTileBuf;
template <bool kApply>
constexpr int kTileBar = kTileLut<kApply> + 256 * 4 + kTSeg * kTW * (kApply ? 4 : kAgg) * 4;
template <bool kApply>
constexpr int kTileCar = kTileBar<kApply> + 16;  // phase C: the item's six carry lines
template <bool kApply>
constexpr int kTileSmem = kApply ? kTileCar<true> + kCar * kTW * 4 : kTileBar<false> + 8;

// Persistent tile pass over items i = tile * ntx + strip. An item's tile lands in the
// input buffer; once every thread holds its segment in registers, the next item's copy is
// issued into the same buffer, so the copy overlaps the item's arithmetic.
// kApply = false: phase A (tile maps to agg_out). kApply = true: phase C (apply the
// carries); the results go out through a second buffer, whose previous store has had the
// item's arithmetic to drain before the buffer is written again.
template <bool kApply>
__global__ void __launch_bounds__(kTNT) k_dt_tiles(const __grid_constant__ ColMaps maps, int w,
                                                   int h, int ntx, int ntile, DtLut lut_in,
                                                   float* __restrict__ agg_out,
                                                   const float* __restrict__ car, int final_pass,
                                                   float flow_eps, int* err)
{
    // all in the dynamic block (kTileSmem bytes, laid out above): the segment maps are
    // [9][kTSeg][kTW] floats in phase A and Aff [kTSeg][kTW] in phase C
    extern __shared__ __align__(1024) uint8_t smt[];
    float* lut = reinterpret_cast<float*>(smt + kTileLut<kApply>);
    float* segbuf = lut + 256;
    Aff (*agg)[kTW] = reinterpret_cast<Aff (*)[kTW]>(segbuf);
    uint64_t& bar = *reinterpret_cast<uint64_t*>(smt + kTileBar<kApply>);
    const int tid = threadIdx.x, lane = tid & 31, sg = tid >> 5;
    for (int i = tid; i < 256; i += blockDim.x) lut[i] = lut_in.w[i];
    if (tid == 0) mbar_init(&bar);
    __syncthreads();
    float* P = reinterpret_cast<float*>(smt);
    const uint8_t* G = smt + 3 * kTR * kTW * 4;
    float* Q = reinterpret_cast<float*>(smt + kTileOut);
    const int nitems = ntx * ntile;
    auto issue = [&](int item) {
        if (tid == 0) {
            const int x0 = (item % ntx) * kTW, r0 = (item / ntx) * kTR;
            // the threads' reads of the buffer (ordered before this by a barrier) come
            // before the copy's writes into it
            fence_async_smem();
            mbar_expect(&bar, 3u * kTR * kTW * 4u + kGRows * kTW + (kApply ? kCar * kTW * 4u : 0u));
            for (int k = 0; k < 3; k++) tma_load_2d(P + k * kTR * kTW, &maps.in[k], x0, r0, &bar);
            tma_load_2d(smt + 3 * kTR * kTW * 4, &maps.guide, x0, r0 - 1, &bar);
            if (kApply) {  // car[tile][q][x]: the item's six 128-byte lines, with the tile
                const size_t wp = (size_t)ntx * kTW;
                const float* c0 = car + (size_t)(item / ntx) * kCar * wp + x0;
                for (int q = 0; q < kCar; q++)
                    bulk_load(smt + kTileCar<kApply> + q * kTW * 4, c0 + (size_t)q * wp, kTW * 4, &bar);
            }
        }
    };
    uint32_t ph = 0;
    int item = blockIdx.x;
    if (item < nitems) issue(item);
    for (; item < nitems; item += gridDim.x) {
        const bool ok = __syncthreads_and(mbar_wait(&bar, ph));
        ph ^= 1u;
        if (!ok) {
            if (tid == 0) {
                atomicExch(err, 1);
                mbar_wait(&bar, ph ^ 1u);  // no copy may land after the CTA has left
                bulk_wait_read();
            }
            return;
        }
        const int x0 = (item % ntx) * kTW, tile = item / ntx, r0 = tile * kTR;
        // phase C: this item's six carries (written by the chain kernel), arrived with the
        // tile; read before the barrier that frees the buffers for the next item's copies
        float cr[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (kApply) {
            const float* cs = reinterpret_cast<const float*>(smt + kTileCar<kApply>);
#pragma unroll
            for (int q = 0; q < 6; q++) cr[q] = cs[q * kTW + lane];
        }
        float v[3][kTLS], wl[kTLS + 1];
        if (r0 > 0 && r0 + kTR < h)
            tile_seg_load<true>(P, G, lut, sg, lane, r0, h, v, wl);
        else
            tile_seg_load<false>(P, G, lut, sg, lane, r0, h, v, wl);
        __syncthreads();  // every thread holds its segment: the input buffer is free
        if (item + (int)gridDim.x < nitems) issue(item + gridDim.x);
        if (!kApply) {
            // agg[tile][k][x]: one 128-byte line per warp and value
            const size_t wp = (size_t)ntx * kTW;
            tile_maps(v, wl, segbuf, sg, lane, true,
                      agg_out + (size_t)tile * kAgg * wp + x0 + lane, wp);
        } else {
            tile_apply(v, wl, agg, sg, lane, cr, Q, final_pass, flow_eps);
            fence_async_smem();
            __syncthreads();  // also: agg reads of this item are done
            if (tid == 0) {
                const int np = final_pass ? 2 : 3;
                for (int q = 0; q < np; q++) tma_store_2d(&maps.out[q], x0, r0, Q + q * kTR * kTW);
                bulk_commit();
            }
        }
    }
    if (kApply && tid == 0) bulk_wait_read();
}

// The carry chain of one column, one warp, lane = tile (32 tiles per round, carried across
// rounds): forward carries by an exclusive shuffle scan of the maps (A_f, B_f), then the
// backward carries by a reverse exclusive scan of (S, K0 + Q c). ag(k, t) reads value k of
// tile t's map, ca(k, t) is carry k of tile t (c[3], then c'[3]). Columns of at most 32
// tiles (frames up to 2,048 rows) take one round from registers.
template <typename AG, typename CA>
__device__ __forceinline__ void column_chain(int ntile, int lane, AG ag, CA ca)
{
    const Aff id{1.f, 0.f, 0.f, 0.f};
    if (ntile <= 32) {
        const int t = lane;
        const bool in = t < ntile;
        float a[kAgg];
#pragma unroll
        for (int k = 0; k < kAgg; k++) a[k] = in ? ag(k, t) : 0.f;
        Aff inc = in ? Aff{a[0], a[1], a[2], a[3]} : id;
        for (int d = 1; d < 32; d <<= 1) {
            const Aff q = shfl_aff<true>(inc, d);
            if (lane >= d) inc = compose(q, inc);
        }
        Aff exc = shfl_aff<true>(inc, 1);
        if (lane == 0) exc = id;
        const Aff c = compose(id, exc);
        inc = in ? Aff{a[8], fmaf(a[7], c.B0, a[4]), fmaf(a[7], c.B1, a[5]), fmaf(a[7], c.B2, a[6])}
                 : id;
        for (int d = 1; d < 32; d <<= 1) {
            const Aff q = shfl_aff<false>(inc, d);
            if (lane + d < 32) inc = compose(q, inc);
        }
        exc = shfl_aff<false>(inc, 1);
        if (lane == 31) exc = id;
        const Aff cb = compose(id, exc);
        if (in) {
            ca(0, t) = c.B0;
            ca(1, t) = c.B1;
            ca(2, t) = c.B2;
            ca(3, t) = cb.B0;
            ca(4, t) = cb.B1;
            ca(5, t) = cb.B2;
        }
        return;
    }
    Aff run = id;  // maps of the tiles before this round
    for (int t0 = 0; t0 < ntile; t0 += 32) {
        const int t = t0 + lane;
        const Aff m = t < ntile ? Aff{ag(0, t), ag(1, t), ag(2, t), ag(3, t)} : id;
        Aff inc = m;
        for (int d = 1; d < 32; d <<= 1) {
            const Aff q = shfl_aff<true>(inc, d);
            if (lane >= d) inc = compose(q, inc);
        }
        Aff exc = shfl_aff<true>(inc, 1);
        if (lane == 0) exc = id;
        const Aff c = compose(run, exc);
        if (t < ntile) {
            ca(0, t) = c.B0;
            ca(1, t) = c.B1;
            ca(2, t) = c.B2;
        }
        run = compose(run, Aff{__shfl_sync(0xffffffffu, inc.A, 31), __shfl_sync(0xffffffffu, inc.B0, 31),
                               __shfl_sync(0xffffffffu, inc.B1, 31), __shfl_sync(0xffffffffu, inc.B2, 31)});
    }
    run = id;  // maps of the tiles after this round, from the bottom
    for (int rd = (ntile + 31) / 32 - 1; rd >= 0; rd--) {
        const int t = rd * 32 + lane;
        Aff m = id;
        if (t < ntile) {
            const float Q = ag(7, t);
            m = Aff{ag(8, t), fmaf(Q, ca(0, t), ag(4, t)), fmaf(Q, ca(1, t), ag(5, t)),
                    fmaf(Q, ca(2, t), ag(6, t))};
        }
        Aff inc = m;
        for (int d = 1; d < 32; d <<= 1) {
            const Aff q = shfl_aff<false>(inc, d);
            if (lane + d < 32) inc = compose(q, inc);
        }
        Aff exc = shfl_aff<false>(inc, 1);
        if (lane == 31) exc = id;
        const Aff c = compose(run, exc);
        if (t < ntile) {
            ca(3, t) = c.B0;
            ca(4, t) = c.B1;
            ca(5, t) = c.B2;
        }
        run = compose(run, Aff{__shfl_sync(0xffffffffu, inc.A, 0), __shfl_sync(0xffffffffu, inc.B0, 0),
                               __shfl_sync(0xffffffffu, inc.B1, 0), __shfl_sync(0xffffffffu, inc.B2, 0)});
    }
}

// The maps and carries live as agg[t][k][x] and car[t][k][x], so that the tile passes move
// them as whole 128-byte lines. One CTA of eight warps per eight columns: the columns' maps
// come in as 32-byte sectors into shared memory ([k][t][9], padded against bank conflicts),
// each warp chains one column there, and the carries leave the same way.
constexpr int kChainCols = 8;
constexpr int kChainPad = kChainCols + 1;
constexpr size_t kChainSmemMax = 48 * 1024;  // columns of up to 91 tiles (5,800 rows)

size_t chain_smem(int ntile) { return (size_t)(kAgg + kCar) * ntile * kChainPad * 4; }

constexpr int kChainNT = 32 * kChainCols;

__global__ void __launch_bounds__(kChainNT) k_dt_cols_chain(const float* __restrict__ agg, int w,
                                                           int ntile, float* __restrict__ car)
{
    extern __shared__ float cs[];
    float* M = cs;                                   // M[(k * ntile + t) * kChainPad + c]
    float* C = cs + (size_t)kAgg * ntile * kChainPad;  // C[(k * ntile + t) * kChainPad + c]
    const size_t wp = (size_t)((w + kTW - 1) / kTW * kTW);
    const int x0 = blockIdx.x * kChainCols, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int e = threadIdx.x; e < ntile * kAgg * kChainCols; e += kChainNT) {
        const int r = e / kChainCols, c = e - r * kChainCols, t = r / kAgg, k = r - t * kAgg;
        M[(k * ntile + t) * kChainPad + c] = __ldg(agg + ((size_t)t * kAgg + k) * wp + x0 + c);
    }
    __syncthreads();
    {
        const int c = warp;
        column_chain(ntile, lane,
                     [&](int k, int t) { return M[(k * ntile + t) * kChainPad + c]; },
                     [&](int k, int t) -> float& { return C[(k * ntile + t) * kChainPad + c]; });
    }
    __syncthreads();
    for (int e = threadIdx.x; e < ntile * kCar * kChainCols; e += kChainNT) {
        const int r = e / kChainCols, c = e - r * kChainCols, t = r / kCar, k = r - t * kCar;
        car[((size_t)t * kCar + k) * wp + x0 + c] = C[(k * ntile + t) * kChainPad + c];
    }
}

// The same chain for columns too tall for the strip's maps to fit shared memory: one
// warp per column, each lane reading its own tile's values from global memory.
__global__ void __launch_bounds__(256) k_dt_cols_chain_tall(const float* __restrict__ agg, int w,
                                                           int ntile, float* __restrict__ car)
{
    const size_t wp = (size_t)((w + kTW - 1) / kTW * kTW);
    const int x = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (x >= (int)wp) return;
    column_chain(ntile, lane,
                 [&](int k, int t) { return __ldg(agg + ((size_t)t * kAgg + k) * wp + x); },
                 [&](int k, int t) -> float& { return car[((size_t)t * kCar + k) * wp + x]; });
}

// ------------------------------------------------------------- host side
PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// 2D tensor map over a w x h plane (row pitch `pitch` elements) with 32 x `rows` boxes
// (4-byte FP32 or 1-byte u8 elements)
bool make_map(CUtensorMap* m, const void* base, int w, int h, int esize, int rows, int pitch)
{
    auto fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)w, (cuuint64_t)h};
    const cuuint64_t strides[1] = {(cuuint64_t)pitch * esize};
    const cuuint32_t box[2] = {(cuuint32_t)kTW, (cuuint32_t)rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUtensorMapDataType t =
        esize == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT8;
    return fn(m, t, 2, const_cast<void*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

int odd_up(int v) { return (v & 1) ? v : v + 1; }


// row segment length: the smem plane length kRowNT*L must keep 16-byte alignment
int row_L(int w)
{
    int L = odd_up((w + kRowNT - 1) / kRowNT);
    return L;
}

size_t row_fast_smem(int w)
{
    const size_t Wp = (size_t)kRowNT * row_L(w);
    return Wp * 12 + align_up(Wp, 16);
}

constexpr size_t kFastBudget = 225 * 1024;

int sm_count()
{
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

void launch_cols_tiles(const ColMaps& maps, int w, int h, const DtLut& lut, int final_pass,
                       float eps, float* agg, float* car, int* err, cudaStream_t s)
{
    // phase A holds one tile; phase C one tile and one tile's output planes
    const size_t smem_a = (size_t)kTileSmem<false>, smem_c = (size_t)kTileSmem<true>;
    ensure_smem((const void*)k_dt_tiles<false>, smem_a);
    ensure_smem((const void*)k_dt_tiles<true>, smem_c);
    const int ntx = (w + kTW - 1) / kTW, ntile = (h + kTR - 1) / kTR;
    const int nitems = ntx * ntile;
    // persistent grids of the resident CTAs, at most four per SM in both phases: five
    // phase-A CTAs (at 48 registers) made the flow replayed alone faster (171 against
    // 174 us) but the batch of many stacks on concurrent lanes slower
    auto grid_of = [&](const void* fn, size_t smem, int most) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kTNT, smem) != cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
        if (per_sm > most) per_sm = most;
        const int cap = per_sm * sm_count();
        return nitems < cap ? nitems : cap;
    };
    note_launch();
    k_dt_tiles<false><<<grid_of((const void*)k_dt_tiles<false>, smem_a, 4), kTNT, smem_a, s>>>(
        maps, w, h, ntx, ntile, lut, agg, car, 0, eps, err);
    note_launch();
    const size_t cs = chain_smem(ntile);
    if (cs <= kChainSmemMax) {
        ensure_smem((const void*)k_dt_cols_chain, cs);
        k_dt_cols_chain<<<ntx * (kTW / kChainCols), kChainNT, cs, s>>>(agg, w, ntile, car);
    } else {
        k_dt_cols_chain_tall<<<(ntx * kTW + 7) / 8, 256, 0, s>>>(agg, w, ntile, car);
    }
    note_launch();
    k_dt_tiles<true><<<grid_of((const void*)k_dt_tiles<true>, smem_c, 4), kTNT, smem_c, s>>>(
        maps, w, h, ntx, ntile, lut, agg, car, final_pass, eps, err);
}

template <int LM>
void launch_rows_pipe(int first, float* P0, float* P1, float* P2, const uint8_t* guide, int w,
                      int h, int ppitch, int gpitch, const DtLut& lut, const FlowCorners& fc,
                      const int4* rec, int* err, cudaStream_t s)
{
    const size_t smem = 2 * ((size_t)3 * kRowNT * LM * 4 + (size_t)kRowNT * LM);
    const int per_sm = (int)((225 * 1024) / (smem + 2048));
    const int grid = h < per_sm * sm_count() ? h : per_sm * sm_count();
    note_launch();
    if (first) {
        ensure_smem((const void*)k_dt_rows_pipe<LM, true>, smem);
        k_dt_rows_pipe<LM, true><<<grid, kRowNT, smem, s>>>(P0, P1, P2, guide, w, h, ppitch,
                                                             gpitch, lut, fc, rec, err);
    } else {
        ensure_smem((const void*)k_dt_rows_pipe<LM, false>, smem);
        k_dt_rows_pipe<LM, false><<<grid, kRowNT, smem, s>>>(P0, P1, P2, guide, w, h, ppitch,
                                                              gpitch, lut, fc, rec, err);
    }
}

}  // namespace

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() { return encode_fn(); }

// Sizes the fast path handles (the caller provides 16-byte-aligned bases and pitches: the
// guide's pitch a multiple of 16, the planes' and the flow planes' multiples of 4).
bool flow_fast_supported(int w, int h)
{
    if (w < 32 || h < 2) return false;
    if (row_L(w) > 23 || 2 * row_fast_smem(w) > kFastBudget) return false;
    return encode_fn() != nullptr;
}

// The six passes of the flow on the fast path; `ws` holds the three planes and,
// after them, the error word.
// Records of the first row pass: at most one per 8 x 8 level-0 tile (tiles are >= 8 px).
size_t corner_rec_bytes(int w, int h) { return align_up((size_t)(w / 8 + 1) * (h / 8 + 1) * 16, 256); }

size_t flow_fast_extra_bytes(int w, int h)
{
    const size_t ntile = (size_t)((h + kTR - 1) / kTR);
    const size_t wp = (size_t)((w + kTW - 1) / kTW) * kTW;
    return align_up((size_t)kAgg * ntile * wp * 4, 256) + align_up((size_t)kCar * ntile * wp * 4, 256) +
           corner_rec_bytes(w, h);
}

bool launch_flow_fast(const uint8_t* guide, int gpitch, int w, int h, const FlowCorners& fc,
                      const DtLut* luts, int iters, double flow_eps, float* flow_u, float* flow_v,
                      int fpitch, float* P0, float* P1, float* P2, int ppitch, int* err,
                      void* extra, cudaStream_t s)
{
    if (gpitch % 16 != 0 || ppitch % 4 != 0 || fpitch % 4 != 0 || gpitch < w || ppitch < w ||
        fpitch < w)
        return false;
    const size_t ntile = (size_t)((h + kTR - 1) / kTR);
    const size_t wp = (size_t)((w + kTW - 1) / kTW) * kTW;
    float* agg = static_cast<float*>(extra);
    float* car = reinterpret_cast<float*>(static_cast<uint8_t*>(extra) +
                                          align_up((size_t)kAgg * ntile * wp * 4, 256));
    int4* rec = reinterpret_cast<int4*>(static_cast<uint8_t*>(extra) +
                                        align_up((size_t)kAgg * ntile * wp * 4, 256) +
                                        align_up((size_t)kCar * ntile * wp * 4, 256));
    {
        const int n = fc.ntx * fc.nty;
        if ((size_t)n * 16 > corner_rec_bytes(w, h)) return false;
        note_launch();
        k_flow_corner_records<<<n > 0 ? (n + 255) / 256 : 1, 256, 0, s>>>(fc, w, h, rec, err);
    }
    ColMaps mid, fin;
    if (!make_map(&mid.in[0], P0, w, h, 4, kTR, ppitch) || !make_map(&mid.in[1], P1, w, h, 4, kTR, ppitch) ||
        !make_map(&mid.in[2], P2, w, h, 4, kTR, ppitch) ||
        !make_map(&mid.guide, guide, w, h, 1, kGRows, gpitch))
        return false;
    mid.out[0] = mid.in[0];
    mid.out[1] = mid.in[1];
    mid.out[2] = mid.in[2];
    fin = mid;
    if (!make_map(&fin.out[0], flow_u, w, h, 4, kTR, fpitch) ||
        !make_map(&fin.out[1], flow_v, w, h, 4, kTR, fpitch))
        return false;
    const int Lr = row_L(w);
    for (int i = 0; i < iters; i++) {
        const DtLut& lut = luts[i];
        const int first = i == 0;
        switch (Lr) {
            case 1: launch_rows_pipe<1>(first, P0, P1, P2, guide, w, h, ppitch, gpitch, lut, fc, rec, err, s); break;
            case 3: launch_rows_pipe<3>(first, P0, P1, P2, guide, w, h, ppitch, gpitch, lut, fc, rec, err, s); break;
            case 5: launch_rows_pipe<5>(first, P0, P1, P2, guide, w, h, ppitch, gpitch, lut, fc, rec, err, s); break;
            case 7: launch_rows_pipe<7>(first, P0, P1, P2, guide, w, h, ppitch, gpitch, lut, fc, rec, err, s); break;
            case 9: launch_rows_pipe<9>(first, P0, P1, P2, guide, w, h, ppitch, gpitch, lut, fc, rec, err, s); break;
            case 11: launch_rows_pipe<11>(first, P0, P1, P2, guide, w, h, ppitch, gpitch, lut, fc, rec, err, s); break;
            case 13: launch_rows_pipe<13>(first, P0, P1, P2, guide, w, h, ppitch, gpitch, lut, fc, rec, err, s); break;
            case 15: launch_rows_pipe<15>(first, P0, P1, P2, guide, w, h, ppitch, gpitch, lut, fc, rec, err, s); break;
            case 17: launch_rows_pipe<17>(first, P0, P1, P2, guide, w, h, ppitch, gpitch, lut, fc, rec, err, s); break;
            case 19: launch_rows_pipe<19>(first, P0, P1, P2, guide, w, h, ppitch, gpitch, lut, fc, rec, err, s); break;
            case 21: launch_rows_pipe<21>(first, P0, P1, P2, guide, w, h, ppitch, gpitch, lut, fc, rec, err, s); break;
            default: launch_rows_pipe<23>(first, P0, P1, P2, guide, w, h, ppitch, gpitch, lut, fc, rec, err, s); break;
        }
        launch_cols_tiles((i == iters - 1) ? fin : mid, w, h, lut, i == iters - 1, (float)flow_eps,
                          agg, car, err, s);
    }
    return true;
}

}  // namespace hdrreg
