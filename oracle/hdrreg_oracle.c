/*
 * hdrreg_oracle.c -- CPU reference of the registration + merge path.
 *
 * TEST INFRASTRUCTURE ONLY (see hdrreg_oracle.h). Plain loops, FP64 and
 * int64/__int128, evaluated in the written order. The loops over independent
 * rows, columns, tiles and weeding iterations carry OpenMP pragmas: the serial
 * build ignores them, the OpenMP build (liboracle_omp.so) runs them on all
 * cores. Every output element is computed by the same operations in the same
 * order either way, and the weeding union is order-free, so both builds give
 * the same bits. Each function names the
 * passage of the paper (section / equation) it restates, plus the reading
 * taken where the paper is silent.
 */
#include "hdrreg_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

static int pix(const uint8_t* img, int w, int h, int x, int y)
{
    /* every read clamps to the nearest edge pixel (reading of the paper's silence on borders) */
    return img[(long)clampi(y, 0, h - 1) * w + clampi(x, 0, w - 1)];
}

/* ===================================================================== a1 */
/*
 * Exposure normalization by the known exposure ratio r = num/den = t_src/t_ref.
 * The paper equalizes histograms (Sec. 3); with known ratios the frames are put
 * in one domain by brightening the darker frame by g = max(r, 1/r) and clipping
 * at 255, which keeps both frames integral. Rounding: nearest, halves up.
 */
void orc_normalize_ratio(const uint8_t* ref, const uint8_t* src, long n, int num, int den,
                         uint8_t* ref_n, uint8_t* src_n)
{
    int ref_darker = num >= den;
    long gn = ref_darker ? num : den;
    long gd = ref_darker ? den : num;
    for (long i = 0; i < n; i++) {
        if (ref_darker) {
            long v = ((long)ref[i] * gn + gd / 2) / gd;
            ref_n[i] = (uint8_t)(v > 255 ? 255 : v);
            src_n[i] = src[i];
        } else {
            long v = ((long)src[i] * gn + gd / 2) / gd;
            src_n[i] = (uint8_t)(v > 255 ? 255 : v);
            ref_n[i] = ref[i];
        }
    }
}

/*
 * Histogram equalization of one frame (Sec. 3: all inputs are equalized to
 * attenuate brightness differences): lut[v] = round((cdf[v]-cdf_min)*255 /
 * (N-cdf_min)), integer arithmetic, halves up; a constant frame maps to itself.
 */
void orc_histeq_lut(const uint8_t* img, long n, uint8_t lut[256])
{
    long hist[256];
    memset(hist, 0, sizeof(hist));
    for (long i = 0; i < n; i++) hist[img[i]]++;
    long cdf[256];
    long run = 0;
    for (int v = 0; v < 256; v++) { run += hist[v]; cdf[v] = run; }
    long cdf_min = 0;
    for (int v = 0; v < 256; v++) if (hist[v] > 0) { cdf_min = cdf[v]; break; }
    long den = n - cdf_min;
    for (int v = 0; v < 256; v++) {
        if (den <= 0) { lut[v] = (uint8_t)v; continue; }
        long num = cdf[v] - cdf_min;
        if (num < 0) num = 0;
        lut[v] = (uint8_t)((num * 255 + den / 2) / den);
    }
}

void orc_apply_lut(const uint8_t* img, long n, const uint8_t lut[256], uint8_t* out)
{
    for (long i = 0; i < n; i++) out[i] = lut[img[i]];
}

/* ===================================================================== a2 */
/*
 * Number of pyramid levels (Sec. 2.6): up to levels_max, and a level is kept
 * only while both of its sides are at least min_size pixels.
 */
int orc_num_levels(int w, int h, int levels_max, int min_size)
{
    int L = 1;
    while (L < levels_max) {
        int lw = w >> L, lh = h >> L;
        if (lw < min_size || lh < min_size) break;
        L++;
    }
    return L;
}

/* 2x2 box reduction, rounded to nearest (halves up); an odd last row/column is dropped. */
void orc_downsample(const uint8_t* in, int w, int h, uint8_t* out)
{
    int ow = w / 2, oh = h / 2;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < oh; y++)
        for (int x = 0; x < ow; x++) {
            int s = in[(long)(2 * y) * w + 2 * x] + in[(long)(2 * y) * w + 2 * x + 1] +
                    in[(long)(2 * y + 1) * w + 2 * x] + in[(long)(2 * y + 1) * w + 2 * x + 1];
            out[(long)y * ow + x] = (uint8_t)((s + 2) >> 2);
        }
}

/* ===================================================================== a3 */
static long box_sum(const uint8_t* img, int w, int h, int x0, int y0, int q)
{
    long s = 0;
    for (int y = y0; y < y0 + q; y++)
        for (int x = x0; x < x0 + q; x++) s += pix(img, w, h, x, y);
    return s;
}

/*
 * Cornerness, Eq. 1, and the minimum-activity value of Eq. 2 at pixel (x, y).
 * The four q x q quadrants share the corner (x, y): TL = [x-q, x-1] x [y-q, y-1],
 * TR = [x, x+q-1] x [y-q, y-1], BR = [x, x+q-1] x [y, y+q-1], BL = [x-q, x-1] x [y, y+q-1],
 * taken in that cyclic order so that successive quadrants are contiguous; the
 * index mod(j+1, 4) of Eq. 1 is read as the cyclic successor. Sums replace
 * means (same ordering; the threshold is scaled by q^2). Writes the four sums,
 * C(p) and min_j |S_{j+1} - S_j|; returns 0.
 */
int orc_cornerness(const uint8_t* img, int w, int h, int x, int y, int q, long sums_out[4],
                   long* c_out, long* minact_out)
{
    long S[4];
    S[0] = box_sum(img, w, h, x - q, y - q, q);
    S[1] = box_sum(img, w, h, x, y - q, q);
    S[2] = box_sum(img, w, h, x, y, q);
    S[3] = box_sum(img, w, h, x - q, y, q);
    long c = 0, m = -1;
    for (int j = 0; j < 4; j++) {
        long d = S[(j + 1) % 4] - S[j];
        if (d < 0) d = -d;
        c += d;
        if (m < 0 || d < m) m = d;
    }
    if (sums_out) for (int j = 0; j < 4; j++) sums_out[j] = S[j];
    if (c_out) *c_out = c;
    if (minact_out) *minact_out = m;
    return 0;
}

/*
 * Per-tile corner pick (Sec. 2.2): full tiles only; candidates on a regular
 * grid c + s*(i, j), s = max(1, T/16) (Sec. 2.6), i, j in [-K, K], around the
 * tile centre c = (tx*T + T/2, ty*T + T/2); keep the candidate of highest
 * cornerness among those passing Eq. 2 (min activity > T_c * q^2); ties go to
 * the first candidate in row-major order (offset j outer, i inner). A tile with
 * no passing candidate has no corner (Sec. 2.2, flat tiles).
 * Returns the number of tiles.
 */
int orc_pick_corners(const uint8_t* img, int w, int h, const orc_params* p,
                     int32_t* corner_xy, uint8_t* valid, int64_t* score)
{
    int T = p->tile, K = p->grid_half, q = p->quad;
    int s = T / 16 > 1 ? T / 16 : 1;
    int ntx = w / T, nty = h / T;
    long thr = (long)p->corner_thresh * q * q;
#pragma omp parallel for collapse(2) schedule(dynamic, 8)
    for (int ty = 0; ty < nty; ty++)
        for (int tx = 0; tx < ntx; tx++) {
            int t = ty * ntx + tx;
            int cx = tx * T + T / 2, cy = ty * T + T / 2;
            long best = -1;
            int bx = 0, by = 0;
            for (int j = -K; j <= K; j++)
                for (int i = -K; i <= K; i++) {
                    int x = cx + s * i, y = cy + s * j;
                    long c, m;
                    orc_cornerness(img, w, h, x, y, q, NULL, &c, &m);
                    if (m > thr && c > best) { best = c; bx = x; by = y; }
                }
            valid[t] = best >= 0;
            corner_xy[2 * t] = best >= 0 ? bx : cx;
            corner_xy[2 * t + 1] = best >= 0 ? by : cy;
            if (score) score[t] = best;
        }
    return ntx * nty;
}

/* ===================================================================== a4 */
/*
 * Apply H (reference -> source, normalized coordinates of Sec. 2.2, Eq. 3) to
 * the integer pixel (x, y) of a w x h level and return the source position in
 * pixels of that level. Every operation is one IEEE binary64 rounding in the
 * written order. Returns 1 if the projective denominator is positive.
 */
int orc_project(const double H[9], int x, int y, int w, int h, double* xs, double* ys)
{
    double W = (double)w;
    double xn = (double)(2 * x - (w - 1)) / W;
    double yn = (double)(2 * y - (h - 1)) / W;
    double X = (H[0] * xn + H[1] * yn) + H[2];
    double Y = (H[3] * xn + H[4] * yn) + H[5];
    double D = (H[6] * xn + H[7] * yn) + H[8];
    double xsn = X / D;
    double ysn = Y / D;
    *xs = (xsn * W + (double)(w - 1)) * 0.5;
    *ys = (ysn * W + (double)(h - 1)) * 0.5;
    return D > 0.0;
}

/*
 * Search centre of Eq. 3: x_src = H^{l+1} x_ref, rounded to the nearest pixel
 * (floor(x + 0.5)) and clamped into the level; an unusable projection
 * (denominator <= 0 or not finite) falls back to the corner itself.
 */
void orc_search_center(const double H[9], int x, int y, int w, int h, int32_t* cx, int32_t* cy)
{
    double xs, ys;
    int ok = orc_project(H, x, y, w, h, &xs, &ys);
    if (!ok || !isfinite(xs) || !isfinite(ys)) { *cx = x; *cy = y; return; }
    double tx = floor(xs + 0.5), ty = floor(ys + 0.5);
    tx = fmin(fmax(tx, 0.0), (double)(w - 1));
    ty = fmin(fmax(ty, 0.0), (double)(h - 1));
    *cx = (int32_t)tx;
    *cy = (int32_t)ty;
}

/* ===================================================================== a5 */
/*
 * SSD patch search (Sec. 2.2): for each tile with a corner p, compare the
 * (2h+1)^2 patch of ref_n around p with the patch of src_n around c + d for
 * every d in [-R, R]^2, c the search centre of Eq. 3. Integer costs; the
 * minimum is taken over the key (cost, row-major index of d) so ties go to the
 * lowest (dy, then dx). Reads clamp to the edge.
 */
void orc_search(const uint8_t* ref_n, const uint8_t* src_n, int w, int h, const double H[9],
                const orc_params* p, int ntiles, const int32_t* corner_xy, const uint8_t* valid,
                int32_t* center_xy, int32_t* match_xy, uint32_t* cost)
{
    int R = p->radius, hp = p->patch_half;
#pragma omp parallel for schedule(dynamic, 4)
    for (int t = 0; t < ntiles; t++) {
        int px = corner_xy[2 * t], py = corner_xy[2 * t + 1];
        int32_t cx = px, cy = py;
        if (valid[t]) orc_search_center(H, px, py, w, h, &cx, &cy);
        center_xy[2 * t] = cx;
        center_xy[2 * t + 1] = cy;
        if (!valid[t]) {
            match_xy[2 * t] = cx;
            match_xy[2 * t + 1] = cy;
            cost[t] = 0xFFFFFFFFu;
            continue;
        }
        uint64_t best = UINT64_MAX;
        int bdx = 0, bdy = 0;
        for (int dy = -R; dy <= R; dy++)
            for (int dx = -R; dx <= R; dx++) {
                uint64_t c = 0;
                for (int v = -hp; v <= hp; v++)
                    for (int u = -hp; u <= hp; u++) {
                        long e = (long)pix(ref_n, w, h, px + u, py + v) -
                                 (long)pix(src_n, w, h, cx + dx + u, cy + dy + v);
                        c += (uint64_t)(e * e);
                    }
                uint64_t idx = (uint64_t)((dy + R) * (2 * R + 1) + (dx + R));
                uint64_t key = (c << 16) | idx;
                if (key < best) { best = key; bdx = dx; bdy = dy; }
            }
        match_xy[2 * t] = cx + bdx;
        match_xy[2 * t + 1] = cy + bdy;
        cost[t] = (uint32_t)(best >> 16);
    }
}

/* ==================================================================== a-L */
/*
 * Learned-path pieces (the paper has none; they replace the level-0 search of
 * Sec. 2.2 by a prediction). Network input at quarter resolution (level q of
 * the pyramid, w x h): channel 0 = (ref - 127.5) / 127.5, channel 1 = the source
 * level sampled bilinearly at H(p) (the coarser homography, Eq. 3, reference ->
 * source), or at p itself when the projection is unusable, scaled the same way.
 */
void orc_predictor_input(const uint8_t* ref_q, const uint8_t* src_q, int w, int h,
                         const double H[9], double* x_out)
{
    for (int y = 0; y < h; y++)
        for (int x = 0; x < w; x++) {
            long i = (long)y * w + x;
            double xs, ys;
            int ok = orc_project(H, x, y, w, h, &xs, &ys);
            if (!ok || !isfinite(xs) || !isfinite(ys)) { xs = x; ys = y; }
            x_out[2 * i] = ((double)ref_q[i] - 127.5) / 127.5;
            x_out[2 * i + 1] = (orc_bilinear(src_q, w, h, xs, ys) - 127.5) / 127.5;
        }
}

/*
 * Training label of a tile: its level-0 match minus its search centre (Eq. 3 with
 * the level-1 homography), i.e. the displacement the plain search found; (0, 0)
 * for tiles without a corner.
 */
void orc_tile_labels(const int32_t* corner_xy, const int32_t* match_xy, const uint8_t* valid,
                     int n, int w, int h, const double H[9], float* label)
{
    for (int t = 0; t < n; t++) {
        label[2 * t] = label[2 * t + 1] = 0.f;
        if (!valid[t]) continue;
        int32_t cx, cy;
        orc_search_center(H, corner_xy[2 * t], corner_xy[2 * t + 1], w, h, &cx, &cy);
        label[2 * t] = (float)(match_xy[2 * t] - cx);
        label[2 * t + 1] = (float)(match_xy[2 * t + 1] - cy);
    }
}

/*
 * Search with a prediction: for a tile with a corner p and search centre c, the
 * predicted displacement d (FP32) is rounded to floor(d + 0.5) (in FP32), giving
 * q = c + round(d); the SSD is evaluated at q + e for every e in [-r, r]^2
 * (r = refine; r = 0 is the single SSD at q) and the least key (cost, row-major
 * index of e) is taken as in orc_search. If that cost is at most `fallback_cost`
 * it is the match, otherwise the tile falls back to the full search of
 * orc_search (fell_back = 1). Tiles without a corner are as in orc_search.
 */
void orc_search_predicted(const uint8_t* ref_n, const uint8_t* src_n, int w, int h,
                          const double H[9], const orc_params* p, int ntiles,
                          const int32_t* corner_xy, const uint8_t* valid, const float* pred,
                          int refine, uint32_t fallback_cost, int32_t* match_xy, uint32_t* cost,
                          uint8_t* fell_back)
{
    int hp = p->patch_half;
    for (int t = 0; t < ntiles; t++) {
        int32_t ctr[2];
        fell_back[t] = 0;
        if (!valid[t]) {
            orc_search(ref_n, src_n, w, h, H, p, 1, corner_xy + 2 * t, valid + t, ctr,
                       match_xy + 2 * t, cost + t);
            continue;
        }
        int px = corner_xy[2 * t], py = corner_xy[2 * t + 1];
        int32_t cx, cy;
        orc_search_center(H, px, py, w, h, &cx, &cy);
        float fx = pred[2 * t] + 0.5f, fy = pred[2 * t + 1] + 0.5f;
        int qx = cx + (int)floorf(fx), qy = cy + (int)floorf(fy);
        uint64_t best = UINT64_MAX;
        int bex = 0, bey = 0;
        for (int ey = -refine; ey <= refine; ey++)
            for (int ex = -refine; ex <= refine; ex++) {
                uint64_t c = 0;
                for (int v = -hp; v <= hp; v++)
                    for (int u = -hp; u <= hp; u++) {
                        long e = (long)pix(ref_n, w, h, px + u, py + v) -
                                 (long)pix(src_n, w, h, qx + ex + u, qy + ey + v);
                        c += (uint64_t)(e * e);
                    }
                uint64_t idx = (uint64_t)((ey + refine) * (2 * refine + 1) + (ex + refine));
                uint64_t key = (c << 16) | idx;
                if (key < best) { best = key; bex = ex; bey = ey; }
            }
        if ((best >> 16) <= fallback_cost) {
            match_xy[2 * t] = qx + bex;
            match_xy[2 * t + 1] = qy + bey;
            cost[t] = (uint32_t)(best >> 16);
        } else {
            fell_back[t] = 1;
            orc_search(ref_n, src_n, w, h, H, p, 1, corner_xy + 2 * t, valid + t, ctr,
                       match_xy + 2 * t, cost + t);
        }
    }
}

/* ===================================================================== a6 */
/*
 * SplitMix64 (Steele, Lea and Flood, 2014) used as a counter-based generator:
 * the k-th value of stream `seed` is the mix of seed + (k+1) * golden gamma.
 */
uint64_t orc_splitmix64_at(uint64_t seed, uint64_t k)
{
    uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/*
 * The 4 distinct samples of iteration `iter` (Sec. 2.3): draws k = 16*iter + t,
 * t = 0..15, index = (high 32 bits of the draw * nv) >> 32, duplicates
 * rejected. Returns 1 if four distinct indices were found.
 */
int orc_weed_sample(uint64_t seed, long iter, int nv, int pick[4])
{
    int np = 0;
    for (int t = 0; t < 16 && np < 4; t++) {
        uint64_t z = orc_splitmix64_at(seed, (uint64_t)iter * 16u + (uint64_t)t);
        uint64_t r = z >> 32;
        int j = (int)((r * (uint64_t)nv) >> 32);
        int dup = 0;
        for (int k = 0; k < np; k++) if (pick[k] == j) dup = 1;
        if (!dup) pick[np++] = j;
    }
    return np == 4;
}

/*
 * Solve the 8x8 system A x = b by Gaussian elimination with partial pivoting
 * (pivot = first row of largest |a_ik|): each pivot is inverted once, the
 * elimination factors are a_ik * (1 / a_kk). Back substitution runs by
 * columns: x_k = b_k * (1 / a_kk) once every column to its right has been
 * removed from b_k, then the term a_ik x_k is subtracted from every row i
 * above it, so each b_i loses its terms in decreasing column order. Every
 * operation is rounded in the written order. Returns 0 on success, 1 if a pivot
 * magnitude is below tol.
 */
int orc_solve8(const double A_in[64], const double b_in[8], double x[8], double tol)
{
    double A[8][8], b[8], inv[8];
    for (int i = 0; i < 8; i++) {
        for (int j = 0; j < 8; j++) A[i][j] = A_in[i * 8 + j];
        b[i] = b_in[i];
    }
    for (int k = 0; k < 8; k++) {
        int piv = k;
        double best = fabs(A[k][k]);
        for (int i = k + 1; i < 8; i++)
            if (fabs(A[i][k]) > best) { best = fabs(A[i][k]); piv = i; }
        if (!(best >= tol)) return 1;
        if (piv != k) {
            for (int j = 0; j < 8; j++) { double t = A[k][j]; A[k][j] = A[piv][j]; A[piv][j] = t; }
            double t = b[k]; b[k] = b[piv]; b[piv] = t;
        }
        inv[k] = 1.0 / A[k][k];
        for (int i = k + 1; i < 8; i++) {
            double f = A[i][k] * inv[k];
            for (int j = k + 1; j < 8; j++) A[i][j] = A[i][j] - f * A[k][j];
            b[i] = b[i] - f * b[k];
        }
    }
    for (int k = 7; k >= 0; k--) {
        x[k] = b[k] * inv[k];
        for (int i = 0; i < k; i++) b[i] = b[i] - A[i][k] * x[k];
    }
    return 0;
}

/*
 * Coordinates in which the weeding and level-fit systems are solved: the
 * centred integers x_c = 2x - (w-1), y_c = 2y - (h-1) divided by S, the smallest
 * power of two >= w. The division is exact, so these are the same numbers on
 * every machine; x_n = x_c / w of Eq. 3 is (S / w) times them.
 */
int orc_pow2_scale(int w)
{
    int s = 1;
    while (s < w) s <<= 1;
    return s;
}

static double tilde(int v, int extent, double S) { return (double)(2 * v - (extent - 1)) / S; }

/*
 * Inlier test of the weeding filter: the match q of corner p is an inlier of
 * the homography Ht (written in the S-scaled coordinates above) if it maps p
 * within eps pixels of q (Sec. 2.3). With the source pixel x_s =
 * (S X/D + (w-1)) / 2 this is (X S - x_qc D)^2 + (Y S - y_qc D)^2 <= (2 eps D)^2
 * for D > 0, where (X, Y, D) = Ht (x~, y~, 1) and x_qc = 2 q_x - (w-1), y_qc =
 * 2 q_y - (h-1): the same predicate multiplied through by (2D)^2, evaluated
 * without division in the written order.
 */
int orc_is_inlier(const double Ht[9], int px, int py, int qx, int qy, int w, int h, double eps)
{
    double S = (double)orc_pow2_scale(w);
    double x = tilde(px, w, S);
    double y = tilde(py, h, S);
    double X = (Ht[0] * x + Ht[1] * y) + Ht[2];
    double Y = (Ht[3] * x + Ht[4] * y) + Ht[5];
    double D = (Ht[6] * x + Ht[7] * y) + Ht[8];
    double qxc = (double)(2 * qx - (w - 1));
    double qyc = (double)(2 * qy - (h - 1));
    double ex = X * S - qxc * D;
    double ey = Y * S - qyc * D;
    double lhs = ex * ex + ey * ey;
    double t = (2.0 * eps) * D;
    return D > 0.0 && lhs <= t * t;
}

/*
 * Weeding filter of Sec. 2.3, Eq. 4, iterations [iter_begin, iter_end): for
 * each iteration sample 4 distinct valid matches, fit the homography H^i
 * through them exactly (8x8 DLT in the S-scaled coordinates of orc_pow2_scale,
 * h22 = 1; skipped if singular), collect the inliers I^i = matches whose projection lands within
 * eps pixels of their match (orc_is_inlier), and if |I^i| > delta set M |= I^i. Inliers are
 * not removed from the pool. mask_bits (bit t = tile t) is OR-ed into, so that
 * runs over disjoint iteration ranges compose by union (Sec. 2.3, last
 * paragraph). delta = max(delta_min, ceil(n_valid / delta_div)).
 */
void orc_weed(const int32_t* corner_xy, const int32_t* match_xy, const uint8_t* valid, int n,
              int w, int h, const orc_params* p, uint64_t seed, int iter_begin, int iter_end,
              uint32_t* mask_bits, int32_t* accepted_out)
{
    int* V = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
    int nv = 0;
    for (int t = 0; t < n; t++) if (valid[t]) V[nv++] = t;
    int accepted = 0;
    if (nv >= 4) {
        int delta = (nv + p->weed_delta_div - 1) / p->weed_delta_div;
        if (delta < p->weed_delta_min) delta = p->weed_delta_min;
        double S = (double)orc_pow2_scale(w);
        /* the iterations are independent and M is their union (order-free), so they may
         * run in any order: one inlier buffer per thread, the union by atomic OR */
#pragma omp parallel
        {
        uint8_t* inl = (uint8_t*)malloc((size_t)(n > 0 ? n : 1));
#pragma omp for reduction(+ : accepted) schedule(dynamic, 8)
        for (int it = iter_begin; it < iter_end; it++) {
            int pick[4];
            if (!orc_weed_sample(seed, it, nv, pick)) continue;
            double A[64], b[8], hv[8];
            memset(A, 0, sizeof(A));
            for (int k = 0; k < 4; k++) {
                int t = V[pick[k]];
                double x = tilde(corner_xy[2 * t], w, S), y = tilde(corner_xy[2 * t + 1], h, S);
                double u = tilde(match_xy[2 * t], w, S), v = tilde(match_xy[2 * t + 1], h, S);
                double* r1 = &A[(2 * k) * 8];
                double* r2 = &A[(2 * k + 1) * 8];
                r1[0] = x; r1[1] = y; r1[2] = 1.0; r1[6] = -(x * u); r1[7] = -(y * u);
                r2[3] = x; r2[4] = y; r2[5] = 1.0; r2[6] = -(x * v); r2[7] = -(y * v);
                b[2 * k] = u;
                b[2 * k + 1] = v;
            }
            if (orc_solve8(A, b, hv, 1e-12)) continue;
            double H[9] = {hv[0], hv[1], hv[2], hv[3], hv[4], hv[5], hv[6], hv[7], 1.0};
            int cnt = 0;
            for (int k = 0; k < nv; k++) {
                int t = V[k];
                inl[k] = orc_is_inlier(H, corner_xy[2 * t], corner_xy[2 * t + 1],
                                       match_xy[2 * t], match_xy[2 * t + 1], w, h, p->weed_eps);
                cnt += inl[k];
            }
            if (cnt > delta) {
                accepted++;
                for (int k = 0; k < nv; k++)
                    if (inl[k]) {
#pragma omp atomic
                        mask_bits[V[k] >> 5] |= 1u << (V[k] & 31);
                    }
            }
        }
        free(inl);
        }
    }
    if (accepted_out) *accepted_out = accepted;
    free(V);
}

/* ===================================================================== a7 */
static double i128_to_double(__int128 s)
{
    /* defined conversion: (double)(s >> 32) * 2^32 + (double)(s mod 2^32), one rounding */
    int64_t hi = (int64_t)(s >> 32);
    uint64_t lo = (uint64_t)(s & (__int128)0xFFFFFFFFu);
    return (double)hi * 4294967296.0 + (double)lo;
}

/*
 * Homography H^l of one pyramid level (Sec. 2.2: computed from the level's
 * corners and matches; used to initialize the next finer level): linear least
 * squares (DLT with h22 = 1) over the weeded set M. The normal equations are
 * accumulated exactly in integers over the centred coordinates x_c = 2x - (w-1),
 * each entry is converted once to binary64 and scaled exactly by the power of
 * S (orc_pow2_scale) that the S-scaled coordinates put on its row and column,
 * and the 8x8 system is solved as in orc_solve8. The solution Ht is returned in
 * the normalized coordinates of Eq. 3 (x_n = (S/w) x~): h2 = (t2 S) / w,
 * h5 = (t5 S) / w, h6 = t6 (w / S), h7 = t7 (w / S), the rest unchanged. Fewer than
 * 4 matches or a singular system keep H_prev. Returns 0 (fitted), 1 (too few
 * matches) or 2 (singular).
 */
int orc_fit_homography(const int32_t* corner_xy, const int32_t* match_xy,
                       const uint32_t* mask_bits, int n, int w, int h,
                       const double H_prev[9], double H_out[9])
{
    __int128 Sm[8][8], Rv[8];
    memset(Sm, 0, sizeof(Sm));
    memset(Rv, 0, sizeof(Rv));
    long cnt = 0;
    for (int t = 0; t < n; t++) {
        if (!((mask_bits[t >> 5] >> (t & 31)) & 1u)) continue;
        int64_t x = 2 * (int64_t)corner_xy[2 * t] - (w - 1);
        int64_t y = 2 * (int64_t)corner_xy[2 * t + 1] - (h - 1);
        int64_t u = 2 * (int64_t)match_xy[2 * t] - (w - 1);
        int64_t v = 2 * (int64_t)match_xy[2 * t + 1] - (h - 1);
        int64_t a1[8] = {x, y, 1, 0, 0, 0, -x * u, -y * u};
        int64_t a2[8] = {0, 0, 0, x, y, 1, -x * v, -y * v};
        for (int j = 0; j < 8; j++) {
            for (int k = 0; k < 8; k++)
                Sm[j][k] += (__int128)a1[j] * a1[k] + (__int128)a2[j] * a2[k];
            Rv[j] += (__int128)a1[j] * u + (__int128)a2[j] * v;
        }
        cnt++;
    }
    if (cnt < 4) { memcpy(H_out, H_prev, sizeof(double) * 9); return 1; }
    /* S-scaled row: a~[j] = a_c[j] / S^e[j], b~ = b_c / S (exact power-of-two scaling) */
    static const int e[8] = {1, 1, 0, 1, 1, 0, 2, 2};
    int s = orc_pow2_scale(w), lg = 0;
    while ((1 << lg) < s) lg++;
    double A[64], b[8], hv[8];
    for (int j = 0; j < 8; j++) {
        for (int k = 0; k < 8; k++) A[j * 8 + k] = ldexp(i128_to_double(Sm[j][k]), -lg * (e[j] + e[k]));
        b[j] = ldexp(i128_to_double(Rv[j]), -lg * (e[j] + 1));
    }
    if (orc_solve8(A, b, hv, 1e-12)) { memcpy(H_out, H_prev, sizeof(double) * 9); return 2; }
    double S = (double)s, W = (double)w;
    double WS = W / S; /* exact */
    H_out[0] = hv[0];
    H_out[1] = hv[1];
    H_out[2] = (hv[2] * S) / W;
    H_out[3] = hv[3];
    H_out[4] = hv[4];
    H_out[5] = (hv[5] * S) / W;
    H_out[6] = hv[6] * WS;
    H_out[7] = hv[7] * WS;
    H_out[8] = 1.0;
    return 0;
}

/* Same least-squares DLT from real-valued normalized correspondences (used by the pins). */
int orc_fit_homography_real(const double* p_xy, const double* q_xy, int n, double H_out[9])
{
    double A[64], b[8], hv[8];
    memset(A, 0, sizeof(A));
    memset(b, 0, sizeof(b));
    for (int i = 0; i < n; i++) {
        double x = p_xy[2 * i], y = p_xy[2 * i + 1], u = q_xy[2 * i], v = q_xy[2 * i + 1];
        double a1[8] = {x, y, 1.0, 0.0, 0.0, 0.0, -x * u, -y * u};
        double a2[8] = {0.0, 0.0, 0.0, x, y, 1.0, -x * v, -y * v};
        for (int j = 0; j < 8; j++) {
            for (int k = 0; k < 8; k++) A[j * 8 + k] += a1[j] * a1[k] + a2[j] * a2[k];
            b[j] += a1[j] * u + a2[j] * v;
        }
    }
    if (orc_solve8(A, b, hv, 1e-300)) return 1;
    for (int k = 0; k < 8; k++) H_out[k] = hv[k];
    H_out[8] = 1.0;
    return 0;
}

/* ============================================================ a2..a7 loop */
/*
 * The pyramid matcher of Sec. 2.2-2.3: build the levels, then from the
 * coarsest level (H = identity) to level 0: corners on the level (recomputed,
 * not upsampled), search around H^{l+1} x, weed with the level's stream
 * (seed + l), fit H^l. Level-0 corners / matches / costs / validity / mask are
 * returned with H^0. level_stats (optional, 4 ints per level from the finest):
 * tiles, valid, weeded, fit status.
 */
int orc_match(const uint8_t* ref_n, const uint8_t* src_n, int w, int h, const orc_params* p,
              double H0_out[9], int32_t* corner_xy, int32_t* match_xy, uint32_t* cost,
              uint8_t* valid, uint32_t* mask_bits, int32_t* level_stats)
{
    int L = orc_num_levels(w, h, p->levels_max, p->min_level_size);
    const uint8_t* rl[8];
    const uint8_t* sl[8];
    int lw[8], lh[8];
    rl[0] = ref_n; sl[0] = src_n; lw[0] = w; lh[0] = h;
    for (int l = 1; l < L; l++) {
        lw[l] = lw[l - 1] / 2;
        lh[l] = lh[l - 1] / 2;
        uint8_t* r = (uint8_t*)malloc((size_t)lw[l] * lh[l]);
        uint8_t* s = (uint8_t*)malloc((size_t)lw[l] * lh[l]);
        orc_downsample(rl[l - 1], lw[l - 1], lh[l - 1], r);
        orc_downsample(sl[l - 1], lw[l - 1], lh[l - 1], s);
        rl[l] = r; sl[l] = s;
    }
    double H[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    for (int l = L - 1; l >= 0; l--) {
        int nt = (lw[l] / p->tile) * (lh[l] / p->tile);
        int32_t* cxy = (int32_t*)malloc(sizeof(int32_t) * 2 * (nt > 0 ? nt : 1));
        int32_t* ctr = (int32_t*)malloc(sizeof(int32_t) * 2 * (nt > 0 ? nt : 1));
        int32_t* mxy = (int32_t*)malloc(sizeof(int32_t) * 2 * (nt > 0 ? nt : 1));
        uint32_t* cst = (uint32_t*)malloc(sizeof(uint32_t) * (nt > 0 ? nt : 1));
        uint8_t* vld = (uint8_t*)malloc((size_t)(nt > 0 ? nt : 1));
        uint32_t* msk = (uint32_t*)calloc((size_t)(nt / 32 + 1), sizeof(uint32_t));
        orc_pick_corners(rl[l], lw[l], lh[l], p, cxy, vld, NULL);
        orc_search(rl[l], sl[l], lw[l], lh[l], H, p, nt, cxy, vld, ctr, mxy, cst);
        orc_weed(cxy, mxy, vld, nt, lw[l], lh[l], p, p->weed_seed + (uint64_t)l, 0,
                 p->weed_iters, msk, NULL);
        double Hn[9];
        int st = orc_fit_homography(cxy, mxy, msk, nt, lw[l], lh[l], H, Hn);
        memcpy(H, Hn, sizeof(H));
        if (level_stats) {
            int nvld = 0, nm = 0;
            for (int t = 0; t < nt; t++) {
                nvld += vld[t];
                nm += (msk[t >> 5] >> (t & 31)) & 1u;
            }
            level_stats[4 * l + 0] = nt;
            level_stats[4 * l + 1] = nvld;
            level_stats[4 * l + 2] = nm;
            level_stats[4 * l + 3] = st;
        }
        if (l == 0) {
            memcpy(corner_xy, cxy, sizeof(int32_t) * 2 * nt);
            memcpy(match_xy, mxy, sizeof(int32_t) * 2 * nt);
            memcpy(cost, cst, sizeof(uint32_t) * nt);
            memcpy(valid, vld, (size_t)nt);
            memcpy(mask_bits, msk, sizeof(uint32_t) * (nt / 32 + 1));
        }
        free(cxy); free(ctr); free(mxy); free(cst); free(vld); free(msk);
    }
    for (int l = 1; l < L; l++) { free((void*)rl[l]); free((void*)sl[l]); }
    memcpy(H0_out, H, sizeof(H));
    return L;
}

/* ===================================================================== a8 */
/*
 * Per-iteration parameters of the recursive-filter domain transform (Gastal
 * and Oliveira 2011, the filter named in Sec. 2.4): iteration i = 0..N-1 uses
 * sigma_i = sigma_s * sqrt(3) * 2^(N-1-i) / sqrt(4^N - 1) and feedback
 * a_i = exp(-sqrt(2) / sigma_i).
 */
void orc_dt_sigma(double sigma_s, int iters, int i, double* sigma_i, double* a_i)
{
    double s = sigma_s * sqrt(3.0) * pow(2.0, (double)(iters - 1 - i)) /
               sqrt(pow(4.0, (double)iters) - 1.0);
    *sigma_i = s;
    *a_i = exp(-sqrt(2.0) / s);
}

/*
 * Edge-aware (cross-bilateral) recursive domain-transform filter of nplanes
 * planes guided by the 8-bit image `guide` (Sec. 2.4). Per iteration: every
 * row forward then backward, then every column forward then backward, with
 * J[n] = (1 - a^d) J[n] + a^d J[n-1] and d = 1 + (sigma_s / sigma_r) *
 * |g[n] - g[n-1]| / 255 the domain-transform distance between neighbours.
 */
void orc_dt_filter(double** P, int np, const uint8_t* g, int w, int h, double sigma_s,
                   double sigma_r, int iters)
{
    double ratio = sigma_s / sigma_r;
    for (int it = 0; it < iters; it++) {
        double sig, a;
        orc_dt_sigma(sigma_s, iters, it, &sig, &a);
#pragma omp parallel for schedule(static)
        for (int y = 0; y < h; y++) {
            const uint8_t* gr = g + (long)y * w;
            for (int x = 1; x < w; x++) {
                double d = 1.0 + ratio * fabs((double)gr[x] - (double)gr[x - 1]) / 255.0;
                double wt = pow(a, d);
                for (int k = 0; k < np; k++) {
                    double* r = P[k] + (long)y * w;
                    r[x] = (1.0 - wt) * r[x] + wt * r[x - 1];
                }
            }
            for (int x = w - 2; x >= 0; x--) {
                double d = 1.0 + ratio * fabs((double)gr[x + 1] - (double)gr[x]) / 255.0;
                double wt = pow(a, d);
                for (int k = 0; k < np; k++) {
                    double* r = P[k] + (long)y * w;
                    r[x] = (1.0 - wt) * r[x] + wt * r[x + 1];
                }
            }
        }
#pragma omp parallel for schedule(static)
        for (int x = 0; x < w; x++) {
            for (int y = 1; y < h; y++) {
                double d = 1.0 + ratio * fabs((double)g[(long)y * w + x] -
                                              (double)g[(long)(y - 1) * w + x]) / 255.0;
                double wt = pow(a, d);
                for (int k = 0; k < np; k++) {
                    double* c = P[k] + x;
                    c[(long)y * w] = (1.0 - wt) * c[(long)y * w] + wt * c[(long)(y - 1) * w];
                }
            }
            for (int y = h - 2; y >= 0; y--) {
                double d = 1.0 + ratio * fabs((double)g[(long)(y + 1) * w + x] -
                                              (double)g[(long)y * w + x]) / 255.0;
                double wt = pow(a, d);
                for (int k = 0; k < np; k++) {
                    double* c = P[k] + x;
                    c[(long)y * w] = (1.0 - wt) * c[(long)y * w] + wt * c[(long)(y + 1) * w];
                }
            }
        }
    }
}

/*
 * Sparse-to-dense flow (Sec. 2.4, Eq. 5-6): P_u, P_v hold the flow at the
 * weeded corners and 0 elsewhere, N is 1 at those corners; all three are
 * filtered with the reference-guided domain transform and F = P~ / N~
 * (F = 0 where N~ < flow_eps). The propagated flow is the residual of the
 * match to the level-0 homography, q - H0(p), so the dense map is H0 + F
 * (propagate_full = 1 propagates the whole displacement q - p instead).
 */
void orc_flow(const uint8_t* guide, int w, int h, int n, const int32_t* corner_xy,
              const int32_t* match_xy, const uint32_t* mask_bits, const double H0[9],
              const orc_params* p, double* flow_u, double* flow_v, double* n_tilde)
{
    long np = (long)w * h;
    double* Pu = (double*)calloc((size_t)np, sizeof(double));
    double* Pv = (double*)calloc((size_t)np, sizeof(double));
    double* N = (double*)calloc((size_t)np, sizeof(double));
    for (int t = 0; t < n; t++) {
        if (!((mask_bits[t >> 5] >> (t & 31)) & 1u)) continue;
        int x = corner_xy[2 * t], y = corner_xy[2 * t + 1];
        double bx = (double)x, by = (double)y;
        if (!p->propagate_full) {
            double xs, ys;
            if (!orc_project(H0, x, y, w, h, &xs, &ys)) continue;
            bx = xs; by = ys;
        }
        long i = (long)y * w + x;
        Pu[i] = (double)match_xy[2 * t] - bx;
        Pv[i] = (double)match_xy[2 * t + 1] - by;
        N[i] = 1.0;
    }
    double* planes[3] = {Pu, Pv, N};
    orc_dt_filter(planes, 3, guide, w, h, p->sigma_s, p->sigma_r, p->dt_iters);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < np; i++) {
        if (N[i] >= p->flow_eps) {
            flow_u[i] = Pu[i] / N[i];
            flow_v[i] = Pv[i] / N[i];
        } else {
            flow_u[i] = 0.0;
            flow_v[i] = 0.0;
        }
        if (n_tilde) n_tilde[i] = N[i];
    }
    free(Pu); free(Pv); free(N);
}

/* ===================================================================== a9 */
/*
 * Bilinear sample with clamp-to-edge taps, written as two nested lerps
 * (a + f (b - a)) so that four equal taps return that value exactly.
 */
double orc_bilinear(const uint8_t* img, int w, int h, double x, double y)
{
    double x0 = floor(x), y0 = floor(y);
    double fx = x - x0, fy = y - y0;
    int ix = (int)x0, iy = (int)y0;
    double a = pix(img, w, h, ix, iy), b = pix(img, w, h, ix + 1, iy);
    double c = pix(img, w, h, ix, iy + 1), d = pix(img, w, h, ix + 1, iy + 1);
    double top = a + fx * (b - a);
    double bot = c + fx * (d - c);
    return top + fy * (bot - top);
}

/*
 * Does the bilinear sample at (x, y) draw on a clipped pixel? The frames are
 * 8-bit (Sec. 2.1), so a pixel at 0 or 255 recorded only a bound on its
 * irradiance, and any sample that gives such a pixel a nonzero weight inherits
 * that bound. The taps with nonzero weight are the one at (floor x, floor y),
 * always; its right neighbour when the x fraction is above zero; the tap below
 * when the y fraction is above zero; and the diagonal one when both are.
 * Returns 1 when one of them holds 0 or 255, else 0 (clamp-to-edge taps).
 */
int orc_bilinear_clipped(const uint8_t* img, int w, int h, double x, double y)
{
    double x0 = floor(x), y0 = floor(y);
    int ix = (int)x0, iy = (int)y0;
    int right = x - x0 > 0.0, below = y - y0 > 0.0;
    int t[4], nt = 0;
    t[nt++] = pix(img, w, h, ix, iy);
    if (right) t[nt++] = pix(img, w, h, ix + 1, iy);
    if (below) t[nt++] = pix(img, w, h, ix, iy + 1);
    if (right && below) t[nt++] = pix(img, w, h, ix + 1, iy + 1);
    for (int k = 0; k < nt; k++)
        if (t[k] == 0 || t[k] == 255) return 1;
    return 0;
}

/*
 * Warp the source to the reference (Sec. 2.4): reference pixel p samples the
 * source at M(p) = H0(p) + F(p) (bilinear, clamp-to-edge). Chroma (half
 * resolution, optional) samples at (Mbar(q) - 0.5) / 2, Mbar the mean of the
 * four luma positions of the 2x2 block of chroma pixel q. Optionally clip_y[p]
 * = orc_bilinear_clipped at M(p): whether the luma sample draws on a pixel at
 * 0 or 255.
 */
void orc_warp(const uint8_t* src_y, const uint8_t* src_u, const uint8_t* src_v, int w, int h,
              const double H0[9], const double* flow_u, const double* flow_v,
              double* out_y, double* out_u, double* out_v, uint8_t* clip_y)
{
    long np = (long)w * h;
    double* mx = (double*)malloc(sizeof(double) * (size_t)np);
    double* my = (double*)malloc(sizeof(double) * (size_t)np);
#pragma omp parallel for schedule(static)
    for (int y = 0; y < h; y++)
        for (int x = 0; x < w; x++) {
            long i = (long)y * w + x;
            double xs, ys;
            if (!orc_project(H0, x, y, w, h, &xs, &ys)) { xs = x; ys = y; }
            mx[i] = xs + flow_u[i];
            my[i] = ys + flow_v[i];
            out_y[i] = orc_bilinear(src_y, w, h, mx[i], my[i]);
            if (clip_y) clip_y[i] = (uint8_t)orc_bilinear_clipped(src_y, w, h, mx[i], my[i]);
        }
    if (src_u && src_v && out_u && out_v) {
        int cw = w / 2, ch = h / 2;
#pragma omp parallel for schedule(static)
        for (int j = 0; j < ch; j++)
            for (int i = 0; i < cw; i++) {
                long a = (long)(2 * j) * w + 2 * i, b = a + w;
                double bx = ((mx[a] + mx[a + 1]) + (mx[b] + mx[b + 1])) * 0.25;
                double by = ((my[a] + my[a + 1]) + (my[b] + my[b + 1])) * 0.25;
                double cx = (bx - 0.5) * 0.5, cy = (by - 0.5) * 0.5;
                out_u[(long)j * cw + i] = orc_bilinear(src_u, cw, ch, cx, cy);
                out_v[(long)j * cw + i] = orc_bilinear(src_v, cw, ch, cx, cy);
            }
    }
    free(mx);
    free(my);
}

/* ==================================================================== a10 */
/*
 * SSIM map (Wang et al. 2004; the fourth fusion weight of Sec. 2.5): Gaussian
 * window of the given sigma truncated at `radius` and normalized to sum 1,
 * clamp-to-edge, K1 = 0.01, K2 = 0.03, L = 255; local moments in the centred
 * (two-pass) form.
 */
void orc_ssim(const double* X, const double* Y, int w, int h, double sigma, int radius,
              double* out)
{
    int n = 2 * radius + 1;
    double* g = (double*)malloc(sizeof(double) * (size_t)(n * n));
    double gs = 0.0;
    for (int j = -radius; j <= radius; j++)
        for (int i = -radius; i <= radius; i++) {
            double v = exp(-(double)(i * i + j * j) / (2.0 * sigma * sigma));
            g[(j + radius) * n + (i + radius)] = v;
            gs += v;
        }
    for (int k = 0; k < n * n; k++) g[k] /= gs;
    double C1 = (0.01 * 255.0) * (0.01 * 255.0);
    double C2 = (0.03 * 255.0) * (0.03 * 255.0);
#pragma omp parallel for schedule(static)
    for (int y = 0; y < h; y++)
        for (int x = 0; x < w; x++) {
            double mx = 0.0, my = 0.0;
            for (int j = -radius; j <= radius; j++)
                for (int i = -radius; i <= radius; i++) {
                    long o = (long)clampi(y + j, 0, h - 1) * w + clampi(x + i, 0, w - 1);
                    double gw = g[(j + radius) * n + (i + radius)];
                    mx += gw * X[o];
                    my += gw * Y[o];
                }
            double vx = 0.0, vy = 0.0, cxy = 0.0;
            for (int j = -radius; j <= radius; j++)
                for (int i = -radius; i <= radius; i++) {
                    long o = (long)clampi(y + j, 0, h - 1) * w + clampi(x + i, 0, w - 1);
                    double gw = g[(j + radius) * n + (i + radius)];
                    double ex = X[o] - mx, ey = Y[o] - my;
                    vx += gw * ex * ex;
                    vy += gw * ey * ey;
                    cxy += gw * ex * ey;
                }
            out[(long)y * w + x] = ((2.0 * mx * my + C1) * (2.0 * cxy + C2)) /
                                   ((mx * mx + my * my + C1) * (vx + vy + C2));
        }
    free(g);
}

/*
 * Ghost / consistency mask Q = max(0, SSIM(ref_n, N_s(warped))) (Sec. 2.5):
 * the warped source is put in the normalized domain of the registration with
 * the same map as its frame: ratio mode min(255, gain * z); histogram mode the
 * frame's LUT, linearly interpolated between integer levels.
 */
void orc_ghost_mask(const uint8_t* ref_n, const double* warped_y, int w, int h, int mode,
                    double gain, const uint8_t* src_lut, double sigma, int radius, double* q)
{
    long np = (long)w * h;
    double* X = (double*)calloc((size_t)np, sizeof(double));
    double* Y = (double*)calloc((size_t)np, sizeof(double));
#pragma omp parallel for schedule(static)
    for (long i = 0; i < np; i++) {
        X[i] = (double)ref_n[i];
        double z = warped_y[i];
        if (mode == 0) {
            double v = gain * z;
            Y[i] = v < 255.0 ? v : 255.0;
        } else {
            double f0 = floor(z);
            int i0 = (int)f0;
            if (i0 >= 255) Y[i] = src_lut[255];
            else {
                if (i0 < 0) { i0 = 0; f0 = 0.0; }
                double f = z - f0;
                Y[i] = (double)src_lut[i0] + f * ((double)src_lut[i0 + 1] - (double)src_lut[i0]);
            }
        }
    }
    orc_ssim(X, Y, w, h, sigma, radius, q);
    for (long i = 0; i < np; i++) if (!(q[i] > 0.0)) q[i] = 0.0;
    free(X);
    free(Y);
}

/* ==================================================================== a11 */
/* Well-exposedness weight of exposure fusion (Mertens et al. 2007), z in DN. */
double orc_well_exposedness(double z, double sigma)
{
    double t = z / 255.0 - 0.5;
    return exp(-(t * t) / (2.0 * sigma * sigma));
}

/*
 * Weighted irradiance merge (Sec. 2.5 weights; Sec. 3.1 irradiance map):
 * E(p) = sum_k w_k Z_k / r_k / sum_k w_k with r_ref = 1, w_ref = WE(Z_ref) and
 * for every warped source w_k = WE(Z_k) * Q_k, or 0 where the sample is clipped:
 * a clipped sample measured only a bound on the irradiance, so it carries none.
 * clip[k][p] says whether source k's sample at p draws on a pixel at 0 or 255
 * (orc_bilinear_clipped, written by orc_warp); without it (clip or clip[k]
 * NULL) a sample is clipped when Z_k <= 0 or Z_k >= 255, the same test for a
 * sample that sits on one pixel. Chroma U-128, V-128 is merged with the mean of
 * the four luma weights of its 2x2 block and the same 1/r_k.
 */
void orc_merge(int w, int h, const uint8_t* ref_y, const uint8_t* ref_u, const uint8_t* ref_v,
               int nsrc, const double* const* wy, const double* const* wu,
               const double* const* wv, const double* const* q,
               const uint8_t* const* clip, const double* ratio, double we_sigma,
               double* out_y, double* out_u, double* out_v)
{
    long np = (long)w * h;
    double* wts = (double*)malloc(sizeof(double) * (size_t)np * (size_t)(nsrc + 1));
#pragma omp parallel for schedule(static)
    for (long i = 0; i < np; i++) {
        double z0 = (double)ref_y[i];
        double w0 = orc_well_exposedness(z0, we_sigma);
        double num = w0 * z0, den = w0;
        wts[i] = w0;
        for (int k = 0; k < nsrc; k++) {
            double z = wy[k][i];
            int clipped = (clip && clip[k]) ? clip[k][i] != 0 : (z <= 0.0 || z >= 255.0);
            double wk = clipped ? 0.0 : orc_well_exposedness(z, we_sigma) * q[k][i];
            wts[(long)(k + 1) * np + i] = wk;
            num += wk * (z / ratio[k]);
            den += wk;
        }
        out_y[i] = num / den;
    }
    if (ref_u && ref_v && out_u && out_v) {
        int cw = w / 2, ch = h / 2;
#pragma omp parallel for schedule(static)
        for (int j = 0; j < ch; j++)
            for (int i = 0; i < cw; i++) {
                long a = (long)(2 * j) * w + 2 * i, b = a + w, c = (long)j * cw + i;
                double nu = 0.0, nv = 0.0, den = 0.0;
                for (int k = 0; k <= nsrc; k++) {
                    const double* W = wts + (long)k * np;
                    double wk = ((W[a] + W[a + 1]) + (W[b] + W[b + 1])) * 0.25;
                    double u, v, r;
                    if (k == 0) { u = (double)ref_u[c]; v = (double)ref_v[c]; r = 1.0; }
                    else { u = wu[k - 1][c]; v = wv[k - 1][c]; r = ratio[k - 1]; }
                    nu += wk * ((u - 128.0) / r);
                    nv += wk * ((v - 128.0) / r);
                    den += wk;
                }
                out_u[c] = nu / den;
                out_v[c] = nv / den;
            }
    }
    free(wts);
}

/* =========================================================== whole path */
/*
 * One exposure stack: the reference frame plus nsrc sources, each registered
 * to the reference independently (n-1 runs, Sec. 2), then merged. Per source:
 * normalize (a1), pyramid matcher (a2-a7), sparse-to-dense flow guided by the
 * normalized reference (a8), warp (a9), ghost mask (a10); then the merge
 * (a11). Optional per-source outputs: H0 (9 doubles each), warped luma, flow,
 * mask and clip flags of the warped luma. Returns 0.
 */
int orc_register_merge(int w, int h, const uint8_t* ref_y, const uint8_t* ref_u,
                       const uint8_t* ref_v, int nsrc, const uint8_t* const* src_y,
                       const uint8_t* const* src_u, const uint8_t* const* src_v,
                       const int32_t* ratio_num, const int32_t* ratio_den,
                       const orc_params* p, double* out_y, double* out_u, double* out_v,
                       double* H0_out, double* const* warped_y_out,
                       double* const* flow_u_out, double* const* flow_v_out,
                       double* const* q_out, uint8_t* const* clip_out)
{
    long np = (long)w * h;
    long nc = (long)(w / 2) * (h / 2);
    int chroma = ref_u && ref_v && out_u && out_v;
    double* wy[8] = {0}; double* wu[8] = {0}; double* wv[8] = {0}; double* qq[8] = {0};
    uint8_t* cl[8] = {0};
    if (nsrc < 1 || nsrc > 8) return 1;
    double ratio[8] = {0};
    int ntmax = (w / p->tile) * (h / p->tile) + 1;
    uint8_t* ref_n = (uint8_t*)malloc((size_t)np);
    uint8_t* src_n = (uint8_t*)malloc((size_t)np);
    int32_t* cxy = (int32_t*)malloc(sizeof(int32_t) * 2 * ntmax);
    int32_t* mxy = (int32_t*)malloc(sizeof(int32_t) * 2 * ntmax);
    uint32_t* cst = (uint32_t*)malloc(sizeof(uint32_t) * ntmax);
    uint8_t* vld = (uint8_t*)malloc((size_t)ntmax);
    uint32_t* msk = (uint32_t*)malloc(sizeof(uint32_t) * (ntmax / 32 + 1));
    double* fu = (double*)malloc(sizeof(double) * np);
    double* fv = (double*)malloc(sizeof(double) * np);
    for (int k = 0; k < nsrc; k++) {
        int num = ratio_num[k], den = ratio_den[k];
        ratio[k] = (double)num / (double)den;
        uint8_t lut_s[256];
        double gain = 1.0;
        if (p->norm_mode == 0) {
            orc_normalize_ratio(ref_y, src_y[k], np, num, den, ref_n, src_n);
            if (num < den) gain = (double)den / (double)num;
        } else {
            uint8_t lut_r[256];
            orc_histeq_lut(ref_y, np, lut_r);
            orc_histeq_lut(src_y[k], np, lut_s);
            orc_apply_lut(ref_y, np, lut_r, ref_n);
            orc_apply_lut(src_y[k], np, lut_s, src_n);
        }
        double H0[9];
        orc_match(ref_n, src_n, w, h, p, H0, cxy, mxy, cst, vld, msk, NULL);
        int nt = (w / p->tile) * (h / p->tile);
        orc_flow(ref_n, w, h, nt, cxy, mxy, msk, H0, p, fu, fv, NULL);
        double Hw[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
        const double* Huse = p->propagate_full ? Hw : H0;
        wy[k] = (double*)malloc(sizeof(double) * np);
        wu[k] = chroma ? (double*)malloc(sizeof(double) * nc) : NULL;
        wv[k] = chroma ? (double*)malloc(sizeof(double) * nc) : NULL;
        qq[k] = (double*)malloc(sizeof(double) * np);
        cl[k] = (uint8_t*)malloc((size_t)np);
        orc_warp(src_y[k], chroma ? src_u[k] : NULL, chroma ? src_v[k] : NULL, w, h, Huse, fu,
                 fv, wy[k], wu[k], wv[k], cl[k]);
        orc_ghost_mask(ref_n, wy[k], w, h, p->norm_mode, gain, lut_s, p->ssim_sigma,
                       p->ssim_radius, qq[k]);
        if (H0_out) memcpy(H0_out + 9 * k, H0, sizeof(H0));
        if (warped_y_out && warped_y_out[k]) memcpy(warped_y_out[k], wy[k], sizeof(double) * np);
        if (flow_u_out && flow_u_out[k]) memcpy(flow_u_out[k], fu, sizeof(double) * np);
        if (flow_v_out && flow_v_out[k]) memcpy(flow_v_out[k], fv, sizeof(double) * np);
        if (q_out && q_out[k]) memcpy(q_out[k], qq[k], sizeof(double) * np);
        if (clip_out && clip_out[k]) memcpy(clip_out[k], cl[k], (size_t)np);
    }
    orc_merge(w, h, ref_y, chroma ? ref_u : NULL, chroma ? ref_v : NULL, nsrc,
              (const double* const*)wy, (const double* const*)wu, (const double* const*)wv,
              (const double* const*)qq, (const uint8_t* const*)cl, ratio, p->we_sigma, out_y,
              chroma ? out_u : NULL,
              chroma ? out_v : NULL);
    for (int k = 0; k < nsrc; k++) {
        free(wy[k]); free(wu[k]); free(wv[k]); free(qq[k]); free(cl[k]);
    }
    free(ref_n); free(src_n); free(cxy); free(mxy); free(cst); free(vld); free(msk);
    free(fu); free(fv);
    return 0;
}

/* Threads an OpenMP region of this build would use (1 in the serial build). */
#ifdef _OPENMP
#include <omp.h>
int orc_max_threads(void) { return omp_get_max_threads(); }
#else
int orc_max_threads(void) { return 1; }
#endif
