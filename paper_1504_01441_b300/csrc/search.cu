// Rows a3-a5: per-tile corner pick (Eq. 1-2), search initialization by the
// coarser level's homography (Eq. 3) and the integer SSD patch search (Sec. 2.2).
//
// One CTA per tile. The reference region around the tile (candidate grid plus
// quadrants / patch) is staged once in shared memory with an integral image
// (Sec. 2.2 notes quadrant means come cheaply from integral images); the
// source search window is staged as four byte-shifted word copies so every
// thread reads aligned 32-bit words for any horizontal offset. The SSD of four
// pixels is one __vabsdiffu4 + one unsigned __dp4a (exact: |a-b|^2 <= 65025,
// a 21x21 patch sums to < 2^25). Costs and argmins are exact integers; the
// argmin key (cost << 16 | row-major index of d) is reduced with warp shuffles.
#include "hdrreg_internal.cuh"

namespace hdrreg {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

__device__ __forceinline__ uint64_t warp_max_u64(uint64_t v)
{
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t u = __shfl_xor_sync(0xffffffffu, v, o);
        v = u > v ? u : v;
    }
    return v;
}

__device__ __forceinline__ uint64_t warp_min_u64(uint64_t v)
{
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t u = __shfl_xor_sync(0xffffffffu, v, o);
        v = u < v ? u : v;
    }
    return v;
}

}  // namespace

// shared-memory layout sizes (host and device agree through this helper)
struct SearchSmem {
    int E, RS, WS, WW, P, PW;
    size_t off_region, off_ii, off_win, off_patch, total;
    __host__ __device__ SearchSmem(const SearchGeom& g)
    {
        E = g.grid_half * g.step + (g.quad > g.patch_half ? g.quad : g.patch_half);
        RS = 2 * E + 1;                       // reference region side
        WS = 2 * (g.radius + g.patch_half) + 1;  // search window side
        WW = (WS + 3) / 4 + 1;                 // words per window row (per shifted copy)
        P = 2 * g.patch_half + 1;
        PW = P / 4;                            // full words per patch row
        size_t o = 0;
        off_region = o;
        o += (size_t)RS * RS;
        o = (o + 15) & ~(size_t)15;
        off_ii = o;
        o += (size_t)(RS + 1) * (RS + 1) * 4;
        off_win = o;
        o += (size_t)4 * WS * WW * 4;
        off_patch = o;
        o += (size_t)P * (PW > 0 ? PW : 1) * 4;
        total = o;
    }
};

__global__ void __launch_bounds__(kThreads) k_local_search(
    const uint8_t* __restrict__ ref, const uint8_t* __restrict__ src, const double* __restrict__ H,
    SearchGeom g, int32_t* __restrict__ corner_xy, int32_t* __restrict__ match_xy,
    uint32_t* __restrict__ cost_out, uint8_t* __restrict__ valid_out)
{
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ uint64_t red[kThreads / 32];
    __shared__ int s_corner[2], s_center[2];

    const SearchSmem L(g);
    uint8_t* region = smem + L.off_region;
    int32_t* ii = reinterpret_cast<int32_t*>(smem + L.off_ii);
    uint32_t* win = reinterpret_cast<uint32_t*>(smem + L.off_win);
    uint32_t* patch = reinterpret_cast<uint32_t*>(smem + L.off_patch);

    const int t = blockIdx.x;
    const int tx = t % g.ntx, ty = t / g.ntx;
    const int cx = tx * g.tile + g.tile / 2, cy = ty * g.tile + g.tile / 2;
    const int ox = cx - L.E, oy = cy - L.E;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // ---- stage the reference region (clamp-to-edge) and its integral image
    for (int i = tid; i < L.RS * L.RS; i += kThreads) {
        const int yy = i / L.RS, xx = i % L.RS;
        region[i] = ref[(size_t)clampi(oy + yy, 0, g.h - 1) * g.w + clampi(ox + xx, 0, g.w - 1)];
    }
    __syncthreads();
    const int IS = L.RS + 1;
    for (int r = tid; r <= L.RS; r += kThreads) {   // row prefix sums (row 0 = zeros)
        int run = 0;
        ii[r * IS] = 0;
        for (int x = 1; x <= L.RS; x++) {
            if (r > 0) run += region[(r - 1) * L.RS + (x - 1)];
            ii[r * IS + x] = run;
        }
    }
    __syncthreads();
    for (int c = tid; c <= L.RS; c += kThreads) {   // column prefix sums
        int run = 0;
        for (int r = 0; r <= L.RS; r++) {
            run += ii[r * IS + c];
            ii[r * IS + c] = run;
        }
    }
    __syncthreads();

    // ---- corner pick: max cornerness among candidates passing Eq. 2;
    //      ties -> lowest row-major candidate index
    const int K = g.grid_half, side = 2 * K + 1, q = g.quad;
    uint64_t best = 0;
    for (int c = tid; c < side * side; c += kThreads) {
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
        uint64_t v = lane < kThreads / 32 ? red[lane] : 0;
        v = warp_max_u64(v);
        if (lane == 0) {
            if (v == 0) {
                s_corner[0] = -1;
            } else {
                const int c = 0xFFFFF - (int)(v & 0xFFFFF);
                s_corner[0] = cx + g.step * (c % side - K);
                s_corner[1] = cy + g.step * (c / side - K);
                int sx, sy;
                search_center(H, s_corner[0], s_corner[1], g.w, g.h, sx, sy);
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
        }
        return;
    }
    const int px = s_corner[0], py = s_corner[1];
    const int sx = s_center[0], sy = s_center[1];
    const int R = g.radius, hp = g.patch_half;

    // ---- stage the source window as 4 byte-shifted word copies, and the patch words
    const int wx0 = sx - R - hp, wy0 = sy - R - hp;
    for (int i = tid; i < 4 * L.WS * L.WW; i += kThreads) {
        const int k = i / (L.WS * L.WW), rem = i % (L.WS * L.WW);
        const int r = rem / L.WW, j = rem % L.WW;
        const int gy = clampi(wy0 + r, 0, g.h - 1);
        const uint8_t* row = src + (size_t)gy * g.w;
        uint32_t word = 0;
        for (int b = 0; b < 4; b++) {
            const int col = 4 * j + k + b;
            const uint32_t v = col < L.WS ? row[clampi(wx0 + col, 0, g.w - 1)] : 0u;
            word |= v << (8 * b);
        }
        win[i] = word;
    }
    const int prx = px - ox - hp, pry = py - oy - hp;  // patch origin inside the region
    for (int i = tid; i < L.P * L.PW; i += kThreads) {
        const int v = i / L.PW, j = i % L.PW;
        const uint8_t* rr = region + (pry + v) * L.RS + prx + 4 * j;
        patch[i] = (uint32_t)rr[0] | ((uint32_t)rr[1] << 8) | ((uint32_t)rr[2] << 16) |
                   ((uint32_t)rr[3] << 24);
    }
    __syncthreads();

    // ---- SSD over d in [-R, R]^2, exact unsigned integers
    const int nd = (2 * R + 1) * (2 * R + 1);
    uint64_t bestk = ~0ull;
    for (int di = tid; di < nd; di += kThreads) {
        const int dy = di / (2 * R + 1), dx = di % (2 * R + 1);  // offsets from window origin
        uint32_t acc = 0;
        for (int v = 0; v < L.P; v++) {
            const uint32_t* prow = patch + v * L.PW;
            int o = dx;  // byte offset of this row's segment inside the window row
            const uint32_t* wrow = win + ((o & 3) * L.WS + (dy + v)) * L.WW + (o >> 2);
            for (int j = 0; j < L.PW; j++) {
                const uint32_t d = __vabsdiffu4(prow[j], wrow[j]);
                acc = __dp4a(d, d, acc);
            }
            const uint8_t* prb = region + (pry + v) * L.RS + prx;
            for (int u = 4 * L.PW; u < L.P; u++) {
                const int col = dx + u;
                const uint32_t wv = (win[((col & 3) * L.WS + (dy + v)) * L.WW + (col >> 2)]) & 255u;
                const int e = (int)prb[u] - (int)wv;
                acc += (uint32_t)(e * e);
            }
        }
        const uint64_t key = ((uint64_t)acc << 16) | (uint64_t)di;
        bestk = key < bestk ? key : bestk;
    }
    bestk = warp_min_u64(bestk);
    if (lane == 0) red[warp] = bestk;
    __syncthreads();
    if (warp == 0) {
        uint64_t v = lane < kThreads / 32 ? red[lane] : ~0ull;
        v = warp_min_u64(v);
        if (lane == 0) {
            const int di = (int)(v & 0xFFFF);
            const int dy = di / (2 * R + 1) - R, dx = di % (2 * R + 1) - R;
            corner_xy[2 * t] = px;
            corner_xy[2 * t + 1] = py;
            match_xy[2 * t] = sx + dx;
            match_xy[2 * t + 1] = sy + dy;
            cost_out[t] = (uint32_t)(v >> 16);
            valid_out[t] = 1;
        }
    }
}

void launch_local_search(const uint8_t* ref, const uint8_t* src, const double* H,
                         const SearchGeom& g, int32_t* corner_xy, int32_t* match_xy,
                         uint32_t* cost, uint8_t* valid, cudaStream_t s)
{
    const int n = g.ntx * g.nty;
    if (n <= 0) return;
    const SearchSmem L(g);
    if (L.total > 48 * 1024)
        ensure_smem((const void*)k_local_search, L.total);
    note_launch();
    k_local_search<<<n, kThreads, L.total, s>>>(ref, src, H, g, corner_xy, match_xy, cost, valid);
}

}  // namespace hdrreg
