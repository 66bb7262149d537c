// Rows a6-a7: the union-of-inliers weeding filter (Sec. 2.3, Eq. 4) and the
// least-squares level homography (Sec. 2.2).
//
// Weeding: every warp draws the samples of four iterations from the
// counter-based stream (so iterations are independent and the union over any
// split of the iteration range equals one run, Sec. 2.3), builds their 4-point
// DLT systems from exact integer-derived entries and solves all four at once
// (solve8_rows: one row per lane, eight lanes per system). The matches are then
// tested with an FP32 filter whose forward error bound certifies the decision,
// falling back to the division-free binary64 predicate only where the interval
// straddles the threshold. Masks are therefore bit-identical to the binary64
// definition while the binary64 pipe (a small fraction of the FP32 rate on this
// part, and paid per warp instruction) runs a few dozen instructions per
// iteration.
//
// Two weeding kernels share that code:
//  * k_weed_level (the fused path): a CTA of 16 warps takes four iterations. It
//    stages the level's matches in shared memory in tile order, with a bitmap of
//    valid tiles and its prefix counts (the i-th valid match is found by a binary
//    search); one warp solves the four systems while the others stage, then four
//    warps test each iteration's matches, and masks are ORed word by word. The CTA
//    that finishes last also computes the level homography (exact integer normal
//    equations, solve8_rows).
//  * k_weed_compact + k_weed_iters (hdrreg_weed, hdrreg_weed_static, and levels
//    too large for shared memory): an order-preserving compaction into a
//    workspace, then one warp per four iterations over the compacted FP32
//    coordinates.
#include "hdrreg_internal.cuh"

namespace hdrreg {

constexpr int kWeedWarps = 4;  // workspace path: warps per CTA, four iterations each
constexpr int kWeedThreads = 32 * kWeedWarps;
// Fused path: warps per CTA (four iterations per CTA). The CTA's time is set by the
// binary64 chains of warp 0 (the four hypotheses) and of the last CTA (the fit); four
// warps keep the register and thread footprint small for the kernels of other lanes.
// Two CTA shapes: four warps for small levels (the chains set the time; a small footprint
// leaves the SMs to the other lanes), sixteen from kWideLevel tiles up (staging the matches
// and testing them against eight hypotheses is then real work).
constexpr int kHypWarps = 2;               // warps drawing and solving hypotheses, 4 each
constexpr int kIterPerCta = 4 * kHypWarps;  // weeding iterations per CTA
constexpr int kNarrowWarps = 4, kWideWarps = 16, kWideLevel = 2048;
constexpr int kFitSums = 23;

__device__ __forceinline__ int ilog2_pow2(int s) { return 31 - __clz(s); }

// ------------------------------------------------------------ inlier test
// FP32 filter with a forward error bound (u = 2^-24): the values X, Y, D of the
// predicate, computed from FP32-rounded H and exact FP32 coordinates, are within
// 4u * (|h0 x| + |h1 y| + |h2|) of the exact ones; the residual interval follows.
// Decisions whose interval does not straddle the threshold equal the exact
// predicate and hence the binary64 one; the rest are evaluated in binary64.
struct InlierGeom {  // per-level constants, computed on the host
    double S, eps2x;  // 2^lg, 2 eps (exact)
    float Sf, cth;    // S; ((2 eps) / S)^2 rounded to FP32
};

struct InlierTest {
    double Hr[9];
    float hf[9], ha[9];

    __device__ __forceinline__ void init(const double* x)
    {
#pragma unroll
        for (int k = 0; k < 8; k++) Hr[k] = x[k];
        Hr[8] = 1.0;
#pragma unroll
        for (int k = 0; k < 9; k++) {
            hf[k] = (float)Hr[k];
            ha[k] = fabsf(hf[k]);
        }
    }

    // c = (x~, y~, x_qc / S, y_qc / S), all exact in FP32
    __device__ __forceinline__ bool operator()(const float4 c, const InlierGeom& G) const
    {
        const float kB = 4.0f * 5.9604645e-8f;
        const float u1 = 1.01f * 5.9604645e-8f;
        const float lo_f = 1.0f - 6.0f * 5.9604645e-8f, hi_f = 1.0f + 6.0f * 5.9604645e-8f;
        const float ax = fabsf(c.x), ay = fabsf(c.y);
        const float X = fmaf(hf[0], c.x, fmaf(hf[1], c.y, hf[2]));
        const float Y = fmaf(hf[3], c.x, fmaf(hf[4], c.y, hf[5]));
        const float D = fmaf(hf[6], c.x, fmaf(hf[7], c.y, hf[8]));
        const float BX = kB * fmaf(ha[0], ax, fmaf(ha[1], ay, ha[2]));
        const float BY = kB * fmaf(ha[3], ax, fmaf(ha[4], ay, ha[5]));
        const float BD = kB * fmaf(ha[6], ax, fmaf(ha[7], ay, ha[8]));
        const float ex = fmaf(-c.z, D, X), ey = fmaf(-c.w, D, Y);
        const float Ex = fmaf(fabsf(c.z), BD, BX) + u1 * fabsf(ex);
        const float Ey = fmaf(fabsf(c.w), BD, BY) + u1 * fabsf(ey);
        const float hx = fabsf(ex) + Ex, hy = fabsf(ey) + Ey;
        const float lx = fmaxf(fabsf(ex) - Ex, 0.f), ly = fmaxf(fabsf(ey) - Ey, 0.f);
        const float Lhi = fmaf(hx, hx, hy * hy) * hi_f;
        const float Llo = fmaf(lx, lx, ly * ly) * lo_f;
        const float Dlo = D - BD, Dhi = fabsf(D) + BD;
        if (Dlo > 0.f && Lhi < G.cth * (Dlo * Dlo) * lo_f) return true;
        if ((D + BD <= 0.f) || Llo > G.cth * (Dhi * Dhi) * hi_f) return false;
        return is_inlier(Hr, (double)c.x, (double)c.y, (double)(c.z * G.Sf),
                         (double)(c.w * G.Sf), G.S, G.eps2x);
    }
};

InlierGeom make_inlier_geom(int w, double eps)
{
    InlierGeom G;
    const int s = pow2_scale(w);
    G.S = (double)s;
    G.Sf = (float)s;
    G.eps2x = 2.0 * eps;
    const double t = (2.0 * eps) / G.S;
    G.cth = (float)(t * t);
    return G;
}

__device__ __forceinline__ float4 tilde4(int cx, int cy, int qx, int qy, int w, int h, float invS)
{
    return make_float4((float)(2 * cx - (w - 1)) * invS, (float)(2 * cy - (h - 1)) * invS,
                       (float)(2 * qx - (w - 1)) * invS, (float)(2 * qy - (h - 1)) * invS);
}

__device__ __forceinline__ int weed_delta(int nv, int delta_min, int delta_div)
{
    const int d = (nv + delta_div - 1) / delta_div;
    return d < delta_min ? delta_min : d;
}

// Warp-collective: the homographies of iterations it_base + g (g = 0..3, those
// below it1) through their four sampled matches; coord_of(j) gives the FP32
// coordinates of the j-th valid match (j < nv). Lanes 8g..8g+7 receive iteration
// g's solution in x; bit g of the result is set if it has one (drawn and not
// singular). Requires nv >= 4.
template <class CoordOf>
__device__ __forceinline__ unsigned weed_hypotheses4(uint64_t seed, long long it_base,
                                                     long long it1, int nv, float Sf, int lg,
                                                     CoordOf coord_of, double (&x)[8])
{
    const int lane = threadIdx.x & 31, g = lane >> 3, r = lane & 7;
    unsigned ok = 0;
    int mine = 0;  // pick r/2 of iteration g
#pragma unroll
    for (int i = 0; i < 4; i++) {
        int pick = 0;
        const bool has = it_base + i < it1 && weed_sample_warp(seed, it_base + i, nv, pick);
        const int pk = __shfl_sync(kFull, pick, r >> 1);  // lane k < 4 holds pick k
        if (g == i) mine = pk;
        if (has) ok |= 1u << i;
    }
    const float4 c = coord_of(mine);
    double a[9];
    dlt4_row(r, (int)(c.x * Sf), (int)(c.y * Sf), (int)(c.z * Sf), (int)(c.w * Sf), lg, a);
    const int bad = solve8_rows(a, x, 1e-12);
    const unsigned bb = __ballot_sync(kFull, bad);
#pragma unroll
    for (int i = 0; i < 4; i++)
        if ((bb >> (8 * i)) & 0xFFu) ok &= ~(1u << i);
    return ok;
}

// --------------------------------------------------------------- level fit
// The 44 distinct entries of A^T A and A^T b of the DLT rows
//   a1 = [x, y, 1, 0, 0, 0, -x u, -y u], b1 = u ;  a2 = [0, 0, 0, x, y, 1, -x v, -y v], b2 = v
// in centred integer coordinates (x = 2 p_x - (w-1), u = 2 q_x - (w-1), ...)
// reduce to 23 distinct sums, accumulated exactly. With |x|, |y| < 2^14 and |u|,
// |v| < 2^14 + R, the 18 sums without u^2 + v^2 have terms below 2^42.01 and stay
// in int64 for up to 2^20 matches; the 5 with it (terms below 2^57.01) are summed in
// int64 over at most 32 matches per thread, then in __int128.
constexpr int kFitSmall = 18, kFitBig = 5;
__constant__ unsigned char c_small_idx[kFitSmall] = {0, 1, 2,  3,  4,  5,  6,  7,  8,
                                                      9, 10, 11, 12, 13, 14, 15, 19, 20};
__constant__ unsigned char c_big_idx[kFitBig] = {16, 17, 18, 21, 22};

struct FitAcc {
    long long s[kFitSmall];  // 0..15, 19, 20
    long long p[kFitBig];    // partial 16, 17, 18, 21, 22
    __int128 b[kFitBig];

    __device__ __forceinline__ void zero()
    {
#pragma unroll
        for (int k = 0; k < kFitSmall; k++) s[k] = 0;
#pragma unroll
        for (int k = 0; k < kFitBig; k++) {
            p[k] = 0;
            b[k] = 0;
        }
    }
    __device__ __forceinline__ void flush()
    {
#pragma unroll
        for (int k = 0; k < kFitBig; k++) {
            b[k] += (__int128)p[k];
            p[k] = 0;
        }
    }
    __device__ __forceinline__ void add(int x, int y, int u, int v)
    {
        const int x2 = x * x, xy = x * y, y2 = y * y, r2 = u * u + v * v;
        s[0] += x2;
        s[1] += xy;
        s[2] += x;
        s[3] += y2;
        s[4] += y;
        s[5] += 1;
        s[6] += (long long)x2 * u;
        s[7] += (long long)xy * u;
        s[8] += (long long)y2 * u;
        s[9] += (long long)x * u;
        s[10] += (long long)y * u;
        s[11] += (long long)x2 * v;
        s[12] += (long long)xy * v;
        s[13] += (long long)y2 * v;
        s[14] += (long long)x * v;
        s[15] += (long long)y * v;
        s[16] += u;
        s[17] += v;
        p[0] += (long long)x2 * r2;
        p[1] += (long long)xy * r2;
        p[2] += (long long)y2 * r2;
        p[3] += (long long)x * r2;
        p[4] += (long long)y * r2;
    }
};

template <int kWarps>
struct FitShared {
    long long ps[kWarps][kFitSmall];
    __int128 pb[kWarps][kFitBig];
    __int128 S[kFitSums];
    int cnt[kWarps];
    int total;
};

// Block-wide exact sums over the tiles whose mask bit is set; fetch(t, x, y, u, v)
// returns tile t's centred integers. Ends with a __syncthreads(); sh.S / sh.total
// are then valid in every thread.
template <int kThreads, class Fetch>
__device__ void fit_accumulate(int n, const uint32_t* mask, Fetch fetch,
                               FitShared<kThreads / 32>& sh)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    FitAcc acc;
    acc.zero();
    int cnt = 0, since = 0;
    for (int t = tid; t < n; t += kThreads) {
        if (!((__ldcg(mask + (t >> 5)) >> (t & 31)) & 1u)) continue;
        int x, y, u, v;
        fetch(t, x, y, u, v);
        acc.add(x, y, u, v);
        cnt++;
        if (++since == 32) {
            acc.flush();
            since = 0;
        }
    }
    acc.flush();
    for (int o = 16; o > 0; o >>= 1) {
        cnt += __shfl_xor_sync(kFull, cnt, o);
#pragma unroll
        for (int k = 0; k < kFitSmall; k++) acc.s[k] += __shfl_xor_sync(kFull, acc.s[k], o);
#pragma unroll
        for (int k = 0; k < kFitBig; k++) {
            const unsigned long long lo = (unsigned long long)acc.b[k];
            const long long hi = (long long)(acc.b[k] >> 64);
            const unsigned long long lo2 = __shfl_xor_sync(kFull, lo, o);
            const long long hi2 = __shfl_xor_sync(kFull, hi, o);
            acc.b[k] += ((__int128)hi2 << 64) | (__int128)lo2;
        }
    }
    if (lane == 0) {
        sh.cnt[warp] = cnt;
#pragma unroll
        for (int k = 0; k < kFitSmall; k++) sh.ps[warp][k] = acc.s[k];
#pragma unroll
        for (int k = 0; k < kFitBig; k++) sh.pb[warp][k] = acc.b[k];
    }
    __syncthreads();
    if (tid < kFitSmall) {
        long long s = 0;
        for (int wv = 0; wv < kThreads / 32; wv++) s += sh.ps[wv][tid];
        sh.S[c_small_idx[tid]] = (__int128)s;
    } else if (tid < kFitSmall + kFitBig) {
        __int128 s = 0;
        for (int wv = 0; wv < kThreads / 32; wv++) s += sh.pb[wv][tid - kFitSmall];
        sh.S[c_big_idx[tid - kFitSmall]] = s;
    } else if (tid == kFitSmall + kFitBig) {
        int tot = 0;
        for (int wv = 0; wv < kThreads / 32; wv++) tot += sh.cnt[wv];
        sh.total = tot;
    }
    __syncthreads();
}

// Normal-equation entry (row r, column c; c = 8 is the right-hand side) as
// +-(index of its sum + 1), 0 for a structural zero.
__constant__ signed char c_fit_code[8][9] = {
    {1, 2, 3, 0, 0, 0, -7, -8, 10},           {2, 4, 5, 0, 0, 0, -8, -9, 11},
    {3, 5, 6, 0, 0, 0, -10, -11, 20},         {0, 0, 0, 1, 2, 3, -12, -13, 15},
    {0, 0, 0, 2, 4, 5, -13, -14, 16},         {0, 0, 0, 3, 5, 6, -15, -16, 21},
    {-7, -8, -10, -12, -13, -15, 17, 18, -22}, {-8, -9, -11, -13, -14, -16, 18, 19, -23}};

// Entry of the S-scaled system: the sum (negated where the code says so) converted
// to binary64 as (double)(s >> 32) * 2^32 + (double)(s mod 2^32) -- one rounding --
// and scaled exactly by 2^-scale_exp.
__device__ __forceinline__ double fit_entry(const __int128* S, int code, int scale_exp)
{
    if (code == 0) return 0.0;
    const __int128 v = code > 0 ? S[code - 1] : -S[-code - 1];
    double d;
    if (i128_rn_scaled(v, scale_exp, d)) return d;
    const long long hi = (long long)(v >> 32);
    const unsigned long long lo = (unsigned long long)(v & (__int128)0xFFFFFFFFu);
    return dmul(dadd(dmul(__ll2double_rn(hi), 4294967296.0), __ull2double_rn(lo)),
                exact_scaled(1, scale_exp));
}

// Warp-collective (lanes 0..7 carry the system): scale the sums into the S-scaled
// system, solve it, write H^l in the normalized coordinates of Eq. 3 (or keep H_prev:
// status 1 = fewer than 4 matches, 2 = singular).
__device__ void fit_solve_warp(const __int128* S, int total, int w, const double* H_prev,
                               double* H_out, int32_t* status)
{
    const int lane = threadIdx.x & 31, r = lane & 7;
    const int s2 = pow2_scale(w), lg = ilog2_pow2(s2);
    int st = 0;
    double x[8];
    if (total < 4) {
        st = 1;
    } else {
        const int e[8] = {1, 1, 0, 1, 1, 0, 2, 2};
        double a[9];
#pragma unroll
        for (int c = 0; c < 8; c++) a[c] = fit_entry(S, c_fit_code[r][c], lg * (e[r] + e[c]));
        a[8] = fit_entry(S, c_fit_code[r][8], lg * (e[r] + 1));
        if (solve8_rows(a, x, 1e-12)) st = 2;
        st = __shfl_sync(kFull, st, 0);
    }
    if (lane != 0) return;
    if (st == 0) {
        const double Sd = (double)s2, W = (double)w;
        const double WS = ddiv(W, Sd);  // exact
        H_out[0] = x[0];
        H_out[1] = x[1];
        H_out[2] = ddiv(dmul(x[2], Sd), W);
        H_out[3] = x[3];
        H_out[4] = x[4];
        H_out[5] = ddiv(dmul(x[5], Sd), W);
        H_out[6] = dmul(x[6], WS);
        H_out[7] = dmul(x[7], WS);
        H_out[8] = 1.0;
    } else {
        for (int k = 0; k < 9; k++) H_out[k] = H_prev[k];
    }
    if (status) *status = st;
}

// ====================================================== fused level kernel
size_t weed_level_smem_bytes(int n)
{
    const size_t nn = n > 0 ? (size_t)n : 0, nw = (nn + 31) / 32;
    return align_up(nn * 16, 16) + nw * 4 * (2 + kIterPerCta) + 16;
}

bool weed_level_fits(int n) { return weed_level_smem_bytes(n) <= kWeedLevelSmemMax; }

template <int NW>
__global__ void __launch_bounds__(32 * NW, 1) k_weed_level(WeedLevelArgs a, InlierGeom G)
{
    constexpr int kLevelWarps = NW, kLevelThreads = 32 * NW;
    static_assert(kHypWarps < kLevelWarps, "some warps stage the coordinates");
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ FitShared<kLevelWarps> fsh;
    __shared__ double s_h[kIterPerCta][8];
    __shared__ int wsum[kLevelWarps];
    __shared__ int s_cnt[kIterPerCta];
    __shared__ unsigned s_ok;
    __shared__ int last_s;
    const int n = a.n, nw = (n + 31) >> 5;
    float4* crd = reinterpret_cast<float4*>(smem);                        // [n] tile order
    uint32_t* vbits = reinterpret_cast<uint32_t*>(smem + align_up((size_t)n * 16, 16));
    int* vpref = reinterpret_cast<int*>(vbits + nw);                      // [nw + 1]
    uint32_t* bw = reinterpret_cast<uint32_t*>(vpref + nw + 1);           // [kIterPerCta][nw]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int lg = ilog2_pow2(pow2_scale(a.w));
    const float invS = 1.0f / G.Sf;  // exact

    // ---- valid bits and their prefix counts (all warps)
    for (int wi = warp; wi < nw; wi += kLevelWarps) {
        const int t = 32 * wi + lane;
        const unsigned b = __ballot_sync(kFull, t < n && a.valid[t] != 0);
        if (lane == 0) vbits[wi] = b;
    }
    if (tid < kIterPerCta) s_cnt[tid] = 0;
    if (tid == 0) s_ok = 0;
    __syncthreads();
    {
        const int per = (nw + kLevelThreads - 1) / kLevelThreads;
        const int b0 = min(nw, tid * per), b1 = min(nw, b0 + per);
        int sum = 0;
        for (int i = b0; i < b1; i++) sum += __popc(vbits[i]);
        int incl = sum;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        int run = incl - sum;
        for (int k = 0; k < warp; k++) run += wsum[k];
        for (int i = b0; i < b1; i++) {
            vpref[i] = run;
            run += __popc(vbits[i]);
        }
        if (tid == kLevelThreads - 1) vpref[nw] = run;
    }
    __syncthreads();
    const int nv = vpref[nw];
    const long long it_base = (long long)a.it0 + (long long)kIterPerCta * blockIdx.x;

    // ---- warps 0 .. kHypWarps-1: four hypotheses each (coordinates of the picks read
    //      from global); the other warps stage the coordinates of every valid match
    if (warp < kHypWarps) {
        unsigned ok = 0;
        if (nv >= 4) {
            double x[8];
            ok = weed_hypotheses4(
                a.seed, it_base + 4 * warp, a.it1, nv, G.Sf, lg,
                [&](int j) {
                    int lo = 0, hi = nw;  // vpref[lo] <= j < vpref[hi]
                    while (hi - lo > 1) {
                        const int mid = (lo + hi) >> 1;
                        if (vpref[mid] <= j) lo = mid;
                        else hi = mid;
                    }
                    const int t = 32 * lo + (int)__fns(vbits[lo], 0, j - vpref[lo] + 1);
                    return tilde4(a.corner_xy[2 * t], a.corner_xy[2 * t + 1], a.match_xy[2 * t],
                                  a.match_xy[2 * t + 1], a.w, a.h, invS);
                },
                x);
            if ((lane & 7) == 0)
                for (int k = 0; k < 8; k++) s_h[4 * warp + (lane >> 3)][k] = x[k];
        }
        if (lane == 0 && ok) atomicOr(&s_ok, ok << (4 * warp));
    } else {
        constexpr int kStage = kLevelThreads - 32 * kHypWarps;  // staging threads
        for (int t0 = tid - 32 * kHypWarps; t0 < n; t0 += 4 * kStage) {
            int v[4], c0[4], c1[4], m0[4], m1[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int t = t0 + u * kStage;
                const bool in = t < n;
                v[u] = in ? a.valid[t] : 0;
                c0[u] = in ? a.corner_xy[2 * t] : 0;
                c1[u] = in ? a.corner_xy[2 * t + 1] : 0;
                m0[u] = in ? a.match_xy[2 * t] : 0;
                m1[u] = in ? a.match_xy[2 * t + 1] : 0;
            }
#pragma unroll
            for (int u = 0; u < 4; u++)
                if (v[u]) crd[t0 + u * kStage] = tilde4(c0[u], c1[u], m0[u], m1[u], a.w, a.h, invS);
        }
    }
    __syncthreads();

    // ---- the iterations' inlier tests: iteration i on warps i mod kLevelWarps (each
    //      over all words) when there are at least as many iterations as warps, else
    //      kLevelWarps / kIterPerCta warps per iteration over equal shares of the words
    const unsigned ok = s_ok;
    {
        constexpr int kParts = kLevelWarps > kIterPerCta ? kLevelWarps / kIterPerCta : 1;
        constexpr int kStep = kLevelWarps > kIterPerCta ? kIterPerCta : kLevelWarps;
        static_assert(kLevelWarps <= kIterPerCta || kLevelWarps % kIterPerCta == 0,
                      "whole warps per iteration");
        const int part = kLevelWarps > kIterPerCta ? warp / kIterPerCta : 0;
        for (int i = warp % kStep; i < kIterPerCta; i += kStep) {
            if (!((ok >> i) & 1u)) continue;
            InlierTest T;
            T.init(s_h[i]);
            const int per = (nw + kParts - 1) / kParts;
            const int w0 = part * per, w1 = min(nw, w0 + per);
            uint32_t* mine = bw + i * nw;
            int cnt = 0;
            for (int wi = w0; wi < w1; wi++) {
                const uint32_t vb = vbits[wi];
                bool in = false;
                if ((vb >> lane) & 1u) in = T(crd[32 * wi + lane], G);
                const unsigned b = __ballot_sync(kFull, in);
                cnt += __popc(b);
                if (lane == 0) mine[wi] = b;
            }
            if (lane == 0) atomicAdd(&s_cnt[i], cnt);
        }
    }
    __syncthreads();
    {
        const int delta = weed_delta(nv, a.delta_min, a.delta_div);
        unsigned acc = 0;
        for (int i = 0; i < kIterPerCta; i++)
            if (((ok >> i) & 1u) && s_cnt[i] > delta) acc |= 1u << i;
        if (acc) {
            for (int wi = tid; wi < nw; wi += kLevelThreads) {
                uint32_t m = 0;
                for (int i = 0; i < kIterPerCta; i++)
                    if ((acc >> i) & 1u) m |= bw[i * nw + wi];
                if (m) atomicOr(&a.mask[wi], m);
            }
        }
    }

    // ---- the last CTA to finish fits the level homography over the final mask
    if (!a.done) return;
    __threadfence();
    __syncthreads();
    if (tid == 0) last_s = atomicAdd(a.done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last_s) return;
    __threadfence();
    const float Sf = G.Sf;
    fit_accumulate<kLevelThreads>(
        n, a.mask,
        [&](int t, int& x, int& y, int& u, int& v) {
            const float4 c = crd[t];
            x = (int)(c.x * Sf);
            y = (int)(c.y * Sf);
            u = (int)(c.z * Sf);
            v = (int)(c.w * Sf);
        },
        fsh);
    if (warp == 0) fit_solve_warp(fsh.S, fsh.total, a.w, a.H_prev, a.H_out, a.status);
    if (tid == 0) *a.done = 0u;  // ready for the next launch
}

void launch_weed_level(const WeedLevelArgs& a, cudaStream_t s)
{
    const int iters = a.it1 > a.it0 ? a.it1 - a.it0 : 0;
    int blocks = (iters + kIterPerCta - 1) / kIterPerCta;
    if (blocks < 1) blocks = 1;  // the fit still runs
    const size_t smem = weed_level_smem_bytes(a.n);
    note_launch();
    if (a.n >= kWideLevel) {
        ensure_smem((const void*)k_weed_level<kWideWarps>, smem);  // static + dynamic may pass 48 KB
        k_weed_level<kWideWarps><<<blocks, 32 * kWideWarps, smem, s>>>(a, make_inlier_geom(a.w, a.eps));
    } else {
        ensure_smem((const void*)k_weed_level<kNarrowWarps>, smem);
        k_weed_level<kNarrowWarps><<<blocks, 32 * kNarrowWarps, smem, s>>>(a, make_inlier_geom(a.w, a.eps));
    }
}

// ================================================== workspace weeding path
size_t weed_ws_bytes(int n)
{
    const size_t nn = n > 0 ? (size_t)n : 1;
    return align_up(nn * 4, 256) + 256 + align_up(nn * 16, 256);
}

WeedWs weed_ws_carve(void* base, int n)
{
    const size_t nn = n > 0 ? (size_t)n : 1;
    uint8_t* p = static_cast<uint8_t*>(base);
    WeedWs w;
    w.list = reinterpret_cast<int32_t*>(p);
    p += align_up(nn * 4, 256);
    w.count = reinterpret_cast<int32_t*>(p);
    p += 256;
    w.coords32 = reinterpret_cast<float4*>(p);
    return w;
}

// Order-preserving compaction of valid tiles and their FP32 coordinates.
__global__ void __launch_bounds__(1024) k_weed_compact(const int32_t* __restrict__ corner_xy,
                                                       const int32_t* __restrict__ match_xy,
                                                       const uint8_t* __restrict__ valid, int n,
                                                       int w, int h, WeedWs ws)
{
    __shared__ int warp_cnt[32];
    __shared__ int base_s;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) base_s = 0;
    __syncthreads();
    const float invS = 1.0f / (float)pow2_scale(w);  // exact
    for (int start = 0; start < n; start += 1024) {
        const int t = start + tid;
        const bool f = t < n && valid[t];
        const unsigned bal = __ballot_sync(kFull, f);
        if (lane == 0) warp_cnt[warp] = __popc(bal);
        __syncthreads();
        int off = base_s;
        for (int k = 0; k < warp; k++) off += warp_cnt[k];
        off += __popc(bal & ((1u << lane) - 1u));
        if (f) {
            ws.list[off] = t;
            ws.coords32[off] = tilde4(corner_xy[2 * t], corner_xy[2 * t + 1], match_xy[2 * t],
                                      match_xy[2 * t + 1], w, h, invS);
        }
        __syncthreads();
        if (tid == 0) {
            int tot = 0;
            for (int k = 0; k < 32; k++) tot += warp_cnt[k];
            base_s += tot;
        }
        __syncthreads();
    }
    if (tid == 0) *ws.count = base_s;
}

__global__ void __launch_bounds__(kWeedThreads) k_weed_iters(int n, int w, int delta_min,
                                                             int delta_div, uint64_t seed,
                                                             int it0, int it1,
                                                             uint32_t* __restrict__ mask,
                                                             WeedWs ws, InlierGeom G)
{
    extern __shared__ uint32_t bal_words[];  // [kWeedWarps][ceil(n/32)]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long it_base = (long long)it0 + 4LL * ((long long)blockIdx.x * kWeedWarps + warp);
    const int nv = *ws.count;
    if (it_base >= it1 || nv < 4) return;
    const int lg = ilog2_pow2(pow2_scale(w));
    double x[8];
    const unsigned ok = weed_hypotheses4(seed, it_base, it1, nv, G.Sf, lg,
                                         [&](int j) { return ws.coords32[j]; }, x);
    const int nw = (nv + 31) / 32;
    const int delta = weed_delta(nv, delta_min, delta_div);
    uint32_t* bw = bal_words + warp * ((n + 31) / 32);
    for (int i = 0; i < 4; i++) {
        double hx[8];
#pragma unroll
        for (int k = 0; k < 8; k++) hx[k] = __shfl_sync(kFull, x[k], 8 * i);
        if (!((ok >> i) & 1u)) continue;
        InlierTest T;
        T.init(hx);
        int cnt = 0;
        for (int j = 0; j < nw; j++) {
            const int k = 32 * j + lane;
            const bool in = k < nv && T(ws.coords32[k], G);
            const unsigned b = __ballot_sync(kFull, in);
            cnt += __popc(b);
            if (lane == 0) bw[j] = b;
        }
        __syncwarp();
        if (cnt > delta) {
            for (int j = lane; j < nw; j += 32) {
                uint32_t b = bw[j];
                while (b) {
                    const int bit = __ffs(b) - 1;
                    b &= b - 1;
                    const int t = ws.list[32 * j + bit];
                    atomicOr(&mask[t >> 5], 1u << (t & 31));
                }
            }
        }
        __syncwarp();
    }
}

void launch_weed(const int32_t* corner_xy, const int32_t* match_xy, const uint8_t* valid, int n,
                 int w, int h, double eps, int delta_min, int delta_div, uint64_t seed, int it0,
                 int it1, uint32_t* mask, const WeedWs& ws, cudaStream_t s)
{
    if (n <= 0) return;
    note_launch();
    k_weed_compact<<<1, 1024, 0, s>>>(corner_xy, match_xy, valid, n, w, h, ws);
    if (it1 <= it0) return;
    const int iters = it1 - it0;
    const int warps = (iters + 3) / 4;
    const int blocks = (warps + kWeedWarps - 1) / kWeedWarps;
    const size_t smem = (size_t)kWeedWarps * ((n + 31) / 32) * 4;
    ensure_smem((const void*)k_weed_iters, smem);  // static + dynamic may pass 48 KB
    note_launch();
    k_weed_iters<<<blocks, kWeedThreads, smem, s>>>(n, w, delta_min, delta_div, seed, it0, it1,
                                                    mask, ws, make_inlier_geom(w, eps));
}

// ============================================================ standalone fit
constexpr int kFitThreads = 256;

__global__ void __launch_bounds__(kFitThreads) k_fit(const int32_t* __restrict__ corner_xy,
                                                     const int32_t* __restrict__ match_xy,
                                                     const uint32_t* __restrict__ mask, int n,
                                                     int w, int h, const double* H_prev,
                                                     double* H_out, int32_t* status)
{
    __shared__ FitShared<kFitThreads / 32> sh;
    fit_accumulate<kFitThreads>(
        n, mask,
        [&](int t, int& x, int& y, int& u, int& v) {
            x = 2 * __ldg(corner_xy + 2 * t) - (w - 1);
            y = 2 * __ldg(corner_xy + 2 * t + 1) - (h - 1);
            u = 2 * __ldg(match_xy + 2 * t) - (w - 1);
            v = 2 * __ldg(match_xy + 2 * t + 1) - (h - 1);
        },
        sh);
    if (threadIdx.x < 32) fit_solve_warp(sh.S, sh.total, w, H_prev, H_out, status);
}

void launch_fit(const int32_t* corner_xy, const int32_t* match_xy, const uint32_t* mask, int n,
                int w, int h, const double* H_prev, double* H_out, int32_t* status,
                cudaStream_t s)
{
    note_launch();
    k_fit<<<1, kFitThreads, 0, s>>>(corner_xy, match_xy, mask, n, w, h, H_prev, H_out, status);
}

// H <- identity; the completion counters of the fused level kernels <- 0.
__global__ void k_set_identity(double* H, unsigned* counters, int ncounters)
{
    if (threadIdx.x < 9) H[threadIdx.x] = (threadIdx.x % 4 == 0) ? 1.0 : 0.0;
    if (counters && (int)threadIdx.x < ncounters) counters[threadIdx.x] = 0u;
}

void launch_set_identity(double* H, cudaStream_t s, unsigned* counters, int ncounters)
{
    note_launch();
    k_set_identity<<<1, 32, 0, s>>>(H, counters, ncounters);
}

}  // namespace hdrreg
