// Rows a3-a5: per-tile corner pick (Eq. 1-2), search initialization by the
// coarser level's homography (Eq. 3) and the integer SSD patch search (Sec. 2.2).
//
// One CTA per tile. The reference region around the tile (candidate grid plus
// quadrants / patch) and the source search window are staged in shared memory
// with aligned 4-byte loads and funnel shifts (byte gathers with clamp-to-edge
// only for blocks that touch the border). Quadrant sums come from an integral
// image of the region (Sec. 2.2 notes they come cheaply from integral images),
// built one row, then one column, per thread. The search centre is evaluated in
// FP32 with a certified interval and in binary64 only when that interval
// straddles a rounding boundary. The SSD is computed as sum a^2 + sum b_d^2 -
// 2 sum a b_d in 32-bit unsigned integers (exact: a 31x31 patch sums to < 2^26): the
// patch energy once, the window energies from sliding box sums, and the cross term
// of four pixels as one unsigned __dp4a; the window words of four neighbouring
// offsets are funnel shifts by 0, 8, 16, 24 bits of the same two aligned words, so a
// thread takes four offsets per load. A tile's CTA is a chain of short dependent
// phases (staging, integral image, corner pick, centre, window, SSD, argmin), so the
// kernel is bounded for eight resident CTAs per SM (32 registers; the few spills cost
// less than the latency they hide). Costs
// and argmins are exact integers; the argmin key (cost << 16 | row-major index of
// d) is reduced with warp shuffles.
#include "hdrreg_internal.cuh"

namespace hdrreg {

namespace {

// Threads per tile CTA: a template parameter (64, 128 or 256, chosen per workload by
// search_threads); every loop below strides by it, and the results do not depend on it.

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

__device__ __forceinline__ uint64_t warp_max_u64(uint64_t v)
{
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t u = __shfl_xor_sync(kFull, v, o);
        v = u > v ? u : v;
    }
    return v;
}

__device__ __forceinline__ uint64_t warp_min_u64(uint64_t v)
{
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t u = __shfl_xor_sync(kFull, v, o);
        v = u < v ? u : v;
    }
    return v;
}

// Stage the rows x cols block with top-left pixel (x0, y0) of a w x h plane into
// shared-memory rows of pw <= 32 words (4 pw >= cols; the bytes past cols are
// don't-care). Pixels outside the plane clamp to the edge. A warp covers
// floor(32 / pw) rows per step. Blocks inside the plane of a 4-byte aligned buffer
// read two aligned words per output word (the last read stays inside the buffer by
// the explicit bound below).
template <int NWARPS>
__device__ __forceinline__ void stage_block(const uint8_t* __restrict__ img, int w, int h, int x0,
                                            int y0, int cols, int rows, uint32_t* dst, int pw)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int rpw = 32 / pw, sub = lane / pw, j = lane - sub * pw;
    if (sub >= rpw) return;
    const bool fast = ((uintptr_t)img & 3u) == 0 && x0 >= 0 && y0 >= 0 && x0 + cols <= w &&
                      y0 + rows <= h &&
                      (size_t)(y0 + rows - 1) * w + x0 + 4 * (size_t)pw + 4 <= (size_t)w * h;
    for (int r = warp * rpw + sub; r < rows; r += NWARPS * rpw) {
        uint32_t word;
        if (fast) {
            const size_t off = (size_t)(y0 + r) * w + x0 + 4 * j;
            const uint32_t* q = reinterpret_cast<const uint32_t*>(img + (off & ~(size_t)3));
            word = __funnelshift_r(__ldg(q), __ldg(q + 1), 8u * (unsigned)(off & 3));
        } else {
            const uint8_t* row = img + (size_t)clampi(y0 + r, 0, h - 1) * w;
            word = 0;
#pragma unroll
            for (int b = 0; b < 4; b++)
                word |= (uint32_t)__ldg(row + clampi(x0 + 4 * j + b, 0, w - 1)) << (8 * b);
        }
        dst[r * pw + j] = word;
    }
}

}  // namespace

// shared-memory layout sizes (host and device agree through this helper)
struct SearchSmem {
    int E, RS, RPW, IS, WS, WW, P, PWc;
    size_t off_region, off_ii, off_win, off_patch, off_ssd, off_hs, total;
    __host__ __device__ SearchSmem(const SearchGeom& g)
    {
        E = g.grid_half * g.step + (g.quad > g.patch_half ? g.quad : g.patch_half);
        RS = 2 * E + 1;                        // reference region side
        RPW = (RS + 3) / 4;                    // words per region row
        IS = RS + 1;                           // integral image side
        P = 2 * g.patch_half + 1;              // patch side
        PWc = (P + 3) / 4;                     // words per patch row (last one partial)
        WS = 2 * g.radius + P;                 // search window side
        WW = (2 * g.radius) / 4 + PWc + 1;     // words per window row (funnel reads one past)
        size_t o = 0;
        off_region = o;
        o += (size_t)RS * RPW * 4;
        off_ii = o;
        o += (size_t)IS * IS * 4;
        off_win = o;
        o += (size_t)WS * WW * 4;
        off_patch = o;
        o += (size_t)P * PWc * 4;
        off_ssd = o;
        o += (size_t)(2 * g.radius + 1) * (2 * g.radius + 1) * 4;
        off_hs = o;                            // row box sums of squares, WS x (2R+1)
        o += (size_t)WS * (2 * g.radius + 1) * 4;
        total = o;
    }
};

template <int NT>
__global__ void __launch_bounds__(NT, 2048 / NT) k_local_search(
    const uint8_t* __restrict__ ref, const uint8_t* __restrict__ src, const double* __restrict__ H,
    SearchGeom g, int32_t* __restrict__ corner_xy, int32_t* __restrict__ match_xy,
    uint32_t* __restrict__ cost_out, uint8_t* __restrict__ valid_out,
    uint32_t* __restrict__ mask_zero, PredSearch ps)
{
    constexpr int kWarps = NT / 32;
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ uint64_t red[kWarps];
    __shared__ float hs[18];  // (float)H, |(float)H|
    __shared__ int s_corner[2], s_center[2];

    const SearchSmem L(g);
    uint32_t* region = reinterpret_cast<uint32_t*>(smem + L.off_region);
    const uint8_t* rb = smem + L.off_region;
    int32_t* ii = reinterpret_cast<int32_t*>(smem + L.off_ii);
    uint32_t* win = reinterpret_cast<uint32_t*>(smem + L.off_win);
    uint32_t* patch = reinterpret_cast<uint32_t*>(smem + L.off_patch);
    uint32_t* ssd = reinterpret_cast<uint32_t*>(smem + L.off_ssd);
    uint32_t* hsq = reinterpret_cast<uint32_t*>(smem + L.off_hs);
    __shared__ uint32_t s_a2;

    const int t = blockIdx.x;
    const int tx = t % g.ntx, ty = t / g.ntx;
    const int cx = tx * g.tile + g.tile / 2, cy = ty * g.tile + g.tile / 2;
    const int ox = cx - L.E, oy = cy - L.E;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int RSP = 4 * L.RPW, IS = L.IS;

    if (mask_zero && tid == 0 && (t & 31) == 0) mask_zero[t >> 5] = 0u;
    if (tid < 9) {
        const float f = (float)H[tid];
        hs[tid] = f;
        hs[9 + tid] = fabsf(f);
    }
    // ---- stage the reference region (clamp-to-edge) and its integral image
    stage_block<kWarps>(ref, g.w, g.h, ox, oy, L.RS, L.RS, region, L.RPW);
    __syncthreads();
    for (int r = tid; r < IS; r += NT) {  // row prefix sums, one row per thread (row 0 and column 0 zero)
        int32_t* out = ii + r * IS;
        out[0] = 0;
        int run = 0;
        if (r == 0) {
            for (int x = 1; x < IS; x++) out[x] = 0;
        } else {
            const uint32_t* row = region + (r - 1) * L.RPW;
            for (int j = 0; j < L.RPW; j++) {
                const uint32_t wv = row[j];
#pragma unroll
                for (int b = 0; b < 4; b++) {
                    const int x = 4 * j + b + 1;
                    if (x < IS) {
                        run += (int)((wv >> (8 * b)) & 255u);
                        out[x] = run;
                    }
                }
            }
        }
    }
    __syncthreads();
    for (int c = tid; c < IS; c += NT) {  // column prefix sums, one column per thread
        int run = 0;
        for (int r = 1; r < IS; r++) {
            run += ii[r * IS + c];
            ii[r * IS + c] = run;
        }
    }
    __syncthreads();

    // ---- corner pick: max cornerness among candidates passing Eq. 2;
    //      ties -> lowest row-major candidate index
    const int K = g.grid_half, side = 2 * K + 1, q = g.quad;
    uint64_t best = 0;
    for (int c = tid; c < side * side; c += NT) {
        const int j = c / side - K, i = c % side - K;
        const int rx = L.E + g.step * i, ry = L.E + g.step * j;
        auto box = [&](int x0, int y0) {
            return ii[(y0 + q) * IS + (x0 + q)] - ii[y0 * IS + (x0 + q)] - ii[(y0 + q) * IS + x0] +
                   ii[y0 * IS + x0];
        };
        const int S0 = box(rx - q, ry - q), S1 = box(rx, ry - q), S2 = box(rx, ry),
                  S3 = box(rx - q, ry);
        const int d0 = abs(S1 - S0), d1 = abs(S2 - S1), d2 = abs(S3 - S2), d3 = abs(S0 - S3);
        const int m = min(min(d0, d1), min(d2, d3));
        if ((long long)m > g.corner_thr) {
            const uint64_t key = ((uint64_t)(d0 + d1 + d2 + d3) << 20) | (uint64_t)(0xFFFFF - c);
            best = key > best ? key : best;
        }
    }
    best = warp_max_u64(best);
    if (lane == 0) red[warp] = best;
    __syncthreads();
    if (warp == 0) {
        uint64_t v = lane < kWarps ? red[lane] : 0;
        v = warp_max_u64(v);
        if (lane == 0) {
            if (v == 0) {
                s_corner[0] = -1;
            } else {
                const int c = 0xFFFFF - (int)(v & 0xFFFFF);
                const int px = cx + g.step * (c % side - K), py = cy + g.step * (c / side - K);
                s_corner[0] = px;
                s_corner[1] = py;
                int sx, sy;
                if (!search_center_f32(hs, hs + 9, px, py, g.w, g.h, sx, sy))
                    search_center(H, px, py, g.w, g.h, sx, sy);
                s_center[0] = sx;
                s_center[1] = sy;
            }
        }
    }
    __syncthreads();
    if (s_corner[0] < 0) {
        if (tid == 0) {
            corner_xy[2 * t] = cx;
            corner_xy[2 * t + 1] = cy;
            match_xy[2 * t] = cx;
            match_xy[2 * t + 1] = cy;
            cost_out[t] = 0xFFFFFFFFu;
            valid_out[t] = 0;
            if (ps.fell_back) ps.fell_back[t] = 0;
        }
        return;
    }
    const int px = s_corner[0], py = s_corner[1];
    const int sx = s_center[0], sy = s_center[1];
    const int R = g.radius, hp = g.patch_half, P = L.P, PWc = L.PWc;

    // ---- the reference patch as words (byte 0 = column px - hp)
    const int prx = px - ox - hp, pry = py - oy - hp;  // patch origin inside the region
    {
        const int rpw = 32 / PWc, sub = lane / PWc, j = lane - sub * PWc;
        if (sub < rpw) {
            for (int v = warp * rpw + sub; v < P; v += kWarps * rpw) {
                const uint8_t* rr = rb + (pry + v) * RSP + prx + 4 * j;
                uint32_t word = 0;
#pragma unroll
                for (int b = 0; b < 4; b++)
                    if (4 * j + b < P) word |= (uint32_t)rr[b] << (8 * b);
                patch[v * PWc + j] = word;
            }
        }
    }
    __syncthreads();
    if (warp == 0) {  // sum of squares of the patch (its words are zero past column P)
        uint32_t a2 = 0;
        for (int i = lane; i < P * PWc; i += 32) a2 = __dp4a(patch[i], patch[i], a2);
        for (int o = 16; o > 0; o >>= 1) a2 += __shfl_xor_sync(kFull, a2, o);
        if (lane == 0) s_a2 = a2;
    }
    // Pass 1 of the learned search: offsets [-r, r]^2 around the rounded prediction; the
    // plain search (and the fallback) is one pass over [-R, R]^2 around the centre.
    bool learned = ps.pred != nullptr;
    int ccx = sx, ccy = sy, RR = R;
    if (learned) {
        const float* pp = ps.pred + 2 * ((size_t)ty * ps.pred_ld + tx);
        ccx = sx + (int)floorf(pp[0] + 0.5f);
        ccy = sy + (int)floorf(pp[1] + 0.5f);
        RR = ps.refine;
    }
    for (;;) {
        // ---- stage the source window (byte 0 of a row = column ccx - RR - hp)
        const int side_d = 2 * RR + 1, nd = side_d * side_d, nq = (side_d + 3) >> 2;
        const int ws = 2 * RR + P;
        stage_block<kWarps>(src, g.w, g.h, ccx - RR - hp, ccy - RR - hp, ws, ws, win, L.WW);
        __syncthreads();
        // ---- sum of squares of every window position: SSD(d) = sum a^2 + sum b_d^2 -
        //      2 sum a b_d, exact in 32-bit unsigned arithmetic (every term < 2^32).
        //      Row box sums (one window row per thread, sliding over dx), then column
        //      box sums (one dx per thread, sliding over dy) start ssd at a^2 + b_d^2.
        for (int row = tid; row < ws; row += NT) {
            const uint32_t* wr = win + row * L.WW;
            auto sq = [&](int c) {
                const uint32_t b = (wr[c >> 2] >> (8 * (c & 3))) & 255u;
                return b * b;
            };
            uint32_t run = 0;
            for (int c = 0; c < P; c++) run += sq(c);
            hsq[row * side_d] = run;
            for (int dx = 1; dx < side_d; dx++) {
                run += sq(dx + P - 1) - sq(dx - 1);
                hsq[row * side_d + dx] = run;
            }
        }
        __syncthreads();
        for (int dx = tid; dx < side_d; dx += NT) {
            uint32_t run = 0;
            for (int r = 0; r < P; r++) run += hsq[r * side_d + dx];
            const uint32_t a2 = s_a2;
            ssd[dx] = a2 + run;
            for (int dy = 1; dy < side_d; dy++) {
                run += hsq[(dy + P - 1) * side_d + dx] - hsq[(dy - 1) * side_d + dx];
                ssd[dy * side_d + dx] = a2 + run;
            }
        }
        __syncthreads();

        // ---- SSD over d in [-RR, RR]^2, exact unsigned integers. A thread takes four
        //      horizontal offsets 4q..4q+3 of one row dy of offsets (the same two window
        //      words, shifted by 0, 8, 16, 24 bits) over a quarter of the patch rows; the
        //      partial sums meet in shared memory.
        {
            constexpr int kSplit = 4;
            const int rows_per = (P + kSplit - 1) / kSplit;
            for (int item = tid; item < side_d * nq * kSplit; item += NT) {
                const int part = item % kSplit, rest = item / kSplit;
                const int dq = rest % nq, dy = rest / nq;
                const int v0 = part * rows_per, v1 = min(P, v0 + rows_per);
                uint32_t acc0 = 0, acc1 = 0, acc2 = 0, acc3 = 0;
                for (int v = v0; v < v1; v++) {
                    const uint32_t* pr = patch + v * PWc;
                    const uint32_t* wr = win + (dy + v) * L.WW + dq;
                    uint32_t cur = wr[0];
#pragma unroll 8
                    for (int j = 0; j < PWc; j++) {  // cross terms sum a b_d
                        const uint32_t nxt = wr[j + 1], pv = pr[j];
                        acc0 = __dp4a(pv, cur, acc0);
                        acc1 = __dp4a(pv, __funnelshift_r(cur, nxt, 8), acc1);
                        acc2 = __dp4a(pv, __funnelshift_r(cur, nxt, 16), acc2);
                        acc3 = __dp4a(pv, __funnelshift_r(cur, nxt, 24), acc3);
                        cur = nxt;
                    }
                }
                // ssd -= 2 sum a b_d (modulo 2^32; the final value is the exact SSD)
                const int dx0 = 4 * dq, base = dy * side_d + dx0;
                atomicAdd(&ssd[base], 0u - 2u * acc0);
                if (dx0 + 1 < side_d) atomicAdd(&ssd[base + 1], 0u - 2u * acc1);
                if (dx0 + 2 < side_d) atomicAdd(&ssd[base + 2], 0u - 2u * acc2);
                if (dx0 + 3 < side_d) atomicAdd(&ssd[base + 3], 0u - 2u * acc3);
            }
        }
        __syncthreads();
        uint64_t bestk = ~0ull;
        for (int di = tid; di < nd; di += NT) {
            const uint64_t key = ((uint64_t)ssd[di] << 16) | (uint64_t)di;
            bestk = key < bestk ? key : bestk;
        }
        bestk = warp_min_u64(bestk);
        if (lane == 0) red[warp] = bestk;
        __syncthreads();
        uint64_t v = lane < kWarps ? red[lane] : ~0ull;
        v = warp_min_u64(v);  // every warp holds the CTA minimum
        const uint32_t best_cost = (uint32_t)(v >> 16);
        if (!learned || best_cost <= ps.fallback_cost) {
            if (tid == 0) {
                const int di = (int)(v & 0xFFFF);
                const int dy = di / side_d - RR, dx = di % side_d - RR;
                corner_xy[2 * t] = px;
                corner_xy[2 * t + 1] = py;
                match_xy[2 * t] = ccx + dx;
                match_xy[2 * t + 1] = ccy + dy;
                cost_out[t] = best_cost;
                valid_out[t] = 1;
                if (ps.fell_back) ps.fell_back[t] = learned ? 0 : (ps.pred ? 1 : 0);
            }
            return;
        }
        // the prediction was not good enough: the full search around the centre
        learned = false;
        ccx = sx;
        ccy = sy;
        RR = R;
        __syncthreads();  // every thread is done with win, ssd and red
    }
}

void launch_local_search(const uint8_t* ref, const uint8_t* src, const double* H,
                         const SearchGeom& g, int32_t* corner_xy, int32_t* match_xy,
                         uint32_t* cost, uint8_t* valid, cudaStream_t s, uint32_t* mask_zero,
                         const PredSearch* pred)
{
    const int n = g.ntx * g.nty;
    if (n <= 0) return;
    const SearchSmem L(g);
    const PredSearch ps = pred ? *pred : PredSearch{nullptr, 0, 0, 0u, nullptr};
    note_launch();
    auto go = [&](auto kern, int nt) {
        ensure_smem((const void*)kern, L.total);  // static + dynamic may pass 48 KB
        kern<<<n, nt, L.total, s>>>(ref, src, H, g, corner_xy, match_xy, cost, valid, mask_zero,
                                    ps);
    };
    if (g.threads == 64)
        go(k_local_search<64>, 64);
    else if (g.threads == 128)
        go(k_local_search<128>, 128);
    else
        go(k_local_search<256>, 256);
}

// Training label of every tile: match - search centre (Eq. 3), 0 without a corner.
__global__ void k_tile_labels(const int32_t* __restrict__ corner_xy,
                              const int32_t* __restrict__ match_xy,
                              const uint8_t* __restrict__ valid, int n, int w, int h,
                              const double* __restrict__ H, float* __restrict__ label)
{
    __shared__ float hs[18];
    if (threadIdx.x < 9) {
        const float f = (float)H[threadIdx.x];
        hs[threadIdx.x] = f;
        hs[9 + threadIdx.x] = fabsf(f);
    }
    __syncthreads();
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        float lx = 0.f, ly = 0.f;
        if (valid[t]) {
            const int px = corner_xy[2 * t], py = corner_xy[2 * t + 1];
            int cx, cy;
            if (!search_center_f32(hs, hs + 9, px, py, w, h, cx, cy)) search_center(H, px, py, w, h, cx, cy);
            lx = (float)(match_xy[2 * t] - cx);
            ly = (float)(match_xy[2 * t + 1] - cy);
        }
        label[2 * t] = lx;
        label[2 * t + 1] = ly;
    }
}

void launch_tile_labels(const int32_t* corner_xy, const int32_t* match_xy, const uint8_t* valid,
                        int n, int w, int h, const double* H, float* label, cudaStream_t s)
{
    if (n <= 0) return;
    note_launch();
    k_tile_labels<<<(n + 255) / 256, 256, 0, s>>>(corner_xy, match_xy, valid, n, w, h, H, label);
}

// Training crops: crop b covers tiles (tx0 .. tx0 + ct - 1, ty0 .. ty0 + ct - 1), i.e. the
// quarter-resolution pixels [8 tx0, 8 (tx0 + ct)) x [8 ty0, 8 (ty0 + ct)), seen through the
// symmetry origins[4b + 2] (bit 0: mirror x, bit 1: mirror y, bit 2: transpose, applied to
// the crop in that order): pixels and tiles move accordingly and each displacement label
// (dx, dy) becomes (+-dx, +-dy), swapped by the transpose. A label whose component reaches
// the search radius (|d| >= bound) marks its tile invalid (the plain search hit its border).
__device__ __forceinline__ void crop_src(int i, int j, int n, int sym, int& si, int& sj)
{
    // output (i, j) -> source (si, sj) inside an n x n crop
    int a = i, b = j;
    if (sym & 4) {
        const int t = a;
        a = b;
        b = t;
    }
    if (sym & 2) a = n - 1 - a;
    if (sym & 1) b = n - 1 - b;
    si = a;
    sj = b;
}

__global__ void k_predictor_crops(const uint32_t* __restrict__ x_full, int wq, int hq,
                                  const float* __restrict__ label_full,
                                  const uint8_t* __restrict__ valid_full, int ntx, int nty,
                                  const int32_t* __restrict__ origins, int ct, float bound,
                                  uint32_t* __restrict__ x_out, float* __restrict__ label_out,
                                  uint8_t* __restrict__ valid_out)
{
    const int b = blockIdx.y;
    const int tx0 = origins[4 * b], ty0 = origins[4 * b + 1], sym = origins[4 * b + 2] & 7;
    const int side = 8 * ct;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < side * side; i += gridDim.x * blockDim.x) {
        int sy, sx;
        crop_src(i / side, i % side, side, sym, sy, sx);
        const int gy = min(max(8 * ty0 + sy, 0), hq - 1), gx = min(max(8 * tx0 + sx, 0), wq - 1);
        x_out[(size_t)b * side * side + i] = x_full[(size_t)gy * wq + gx];
    }
    if (blockIdx.x == 0) {
        for (int i = threadIdx.x; i < ct * ct; i += blockDim.x) {
            int si, sj;
            crop_src(i / ct, i % ct, ct, sym, si, sj);
            const int ty = ty0 + si, tx = tx0 + sj;
            const bool in = tx >= 0 && tx < ntx && ty >= 0 && ty < nty;
            const size_t t = in ? (size_t)ty * ntx + tx : 0;
            float dx = in ? label_full[2 * t] : 0.f, dy = in ? label_full[2 * t + 1] : 0.f;
            bool ok = in && valid_full[t] && fabsf(dx) < bound && fabsf(dy) < bound;
            if (sym & 4) {  // undo in reverse order: the displacement of the output frame
                const float tmp = dx;
                dx = dy;
                dy = tmp;
            }
            // mirror of the source axes, expressed in output axes after the transpose
            const bool mx = (sym & 4) ? (sym & 2) : (sym & 1);
            const bool my = (sym & 4) ? (sym & 1) : (sym & 2);
            if (mx) dx = -dx;
            if (my) dy = -dy;
            label_out[((size_t)b * ct * ct + i) * 2] = ok ? dx : 0.f;
            label_out[((size_t)b * ct * ct + i) * 2 + 1] = ok ? dy : 0.f;
            valid_out[(size_t)b * ct * ct + i] = ok ? 1 : 0;
        }
    }
}

void launch_predictor_crops(const void* x_full, int wq, int hq, const float* label_full,
                            const uint8_t* valid_full, int ntx, int nty, const int32_t* origins,
                            int n, int ct, float bound, void* x_out, float* label_out,
                            uint8_t* valid_out, cudaStream_t s)
{
    if (n <= 0) return;
    note_launch();
    k_predictor_crops<<<dim3(16, n), 256, 0, s>>>(static_cast<const uint32_t*>(x_full), wq, hq,
                                                   label_full, valid_full, ntx, nty, origins, ct,
                                                   bound, static_cast<uint32_t*>(x_out), label_out,
                                                   valid_out);
}

}  // namespace hdrreg
