/*
 * hdrreg_oracle.h -- plain, slow CPU reference ("oracle") of the locally
 * non-rigid HDR registration + merge path of Gallo et al., "Locally Non-rigid
 * Registration for Mobile HDR Photography" (arXiv 1504.01441).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may include, link or
 * call this code: only the test-suite, the smoke check and the CPU-baseline leg
 * of the benchmark do. It shares no source with the CUDA library.
 *
 * Arithmetic: integer steps in int64 / __int128, everything else in IEEE
 * binary64 evaluated in the written order (compiled with -ffp-contract=off,
 * no fast-math). Plain loops; the OpenMP build runs the independent ones on
 * all cores with the same per-element arithmetic (bit-identical results).
 *
 * Conventions: images are row-major, tightly packed; pixel centres sit at
 * integer coordinates; "normalized" coordinates are those of Sec. 2.2 (Eq. 3):
 * x_n = (2x - (w-1)) / w, y_n = (2y - (h-1)) / w, so x_n is in [-1, 1] and y_n
 * in [-h/w, h/w] with the origin at the image centre.
 * A homography is double[9], row-major, H[8] == 1, mapping reference ->
 * source in normalized coordinates.
 */
#ifndef HDRREG_ORACLE_H
#define HDRREG_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_params {
    int tile;             /* T: tile side (pixels of the current level)              */
    int radius;           /* R: SSD search radius                                    */
    int patch_half;       /* patch is (2*patch_half+1)^2, 10 -> 21x21 (Sec. 2.6)     */
    int levels_max;       /* up to 5 pyramid levels (Sec. 2.6)                       */
    int min_level_size;   /* a level is kept only if both sides >= 100 (Sec. 2.6)    */
    int grid_half;        /* K: candidates c + s*(i,j), i,j in [-K, K]               */
    int quad;             /* q: quadrant side for Eq. 1-2                            */
    int corner_thresh;    /* T of Eq. 2 as a mean difference in DN                   */
    int weed_iters;       /* total iterations of the Eq. 4 filter                    */
    int weed_delta_min;   /* delta = max(delta_min, ceil(n_valid / delta_div))      */
    int weed_delta_div;
    int norm_mode;        /* 0 = exposure ratio, 1 = histogram equalization          */
    int dt_iters;         /* domain-transform iterations                             */
    int ssim_radius;      /* Gaussian window radius of SSIM                          */
    int propagate_full;   /* 0: propagate q - H0(p) (dense map H0 + F); 1: q - p     */
    int pad_;
    double weed_eps;      /* inlier distance in pixels of the level                  */
    double sigma_s;       /* domain-transform spatial sigma (Sec. 2.6: 400)          */
    double sigma_r;       /* domain-transform range sigma, on a [0,1] intensity scale */
    double ssim_sigma;    /* Gaussian window sigma of SSIM                           */
    double we_sigma;      /* well-exposedness sigma of the merge weights             */
    double flow_eps;      /* F = 0 where the filtered normalization map < flow_eps   */
    uint64_t weed_seed;
} orc_params;

/* ---- a1: exposure normalization ---------------------------------------- */
void orc_normalize_ratio(const uint8_t* ref, const uint8_t* src, long n, int num, int den,
                         uint8_t* ref_n, uint8_t* src_n);
void orc_histeq_lut(const uint8_t* img, long n, uint8_t lut[256]);
void orc_apply_lut(const uint8_t* img, long n, const uint8_t lut[256], uint8_t* out);

/* ---- a2: pyramid --------------------------------------------------------- */
int  orc_num_levels(int w, int h, int levels_max, int min_size);
void orc_downsample(const uint8_t* in, int w, int h, uint8_t* out);

/* ---- a3: corners (Eq. 1-2) ------------------------------------------------ */
int  orc_cornerness(const uint8_t* img, int w, int h, int x, int y, int q, long sums_out[4],
                    long* c_out, long* minact_out);
int  orc_pick_corners(const uint8_t* img, int w, int h, const orc_params* p,
                      int32_t* corner_xy, uint8_t* valid, int64_t* score);

/* ---- a4: search initialization (Eq. 3) ----------------------------------- */
int  orc_project(const double H[9], int x, int y, int w, int h, double* xs, double* ys);
void orc_search_center(const double H[9], int x, int y, int w, int h, int32_t* cx, int32_t* cy);

/* ---- a5: SSD search ------------------------------------------------------ */
void orc_search(const uint8_t* ref_n, const uint8_t* src_n, int w, int h, const double H[9],
                const orc_params* p, int ntiles, const int32_t* corner_xy, const uint8_t* valid,
                int32_t* center_xy, int32_t* match_xy, uint32_t* cost);

/* ---- a6: weeding (Eq. 4) ------------------------------------------------- */
uint64_t orc_splitmix64_at(uint64_t seed, uint64_t k);
int  orc_weed_sample(uint64_t seed, long iter, int nv, int pick[4]);
void orc_predictor_input(const uint8_t* ref_q, const uint8_t* src_q, int w, int h,
                         const double H[9], double* x_out);
void orc_tile_labels(const int32_t* corner_xy, const int32_t* match_xy, const uint8_t* valid,
                     int n, int w, int h, const double H[9], float* label);
void orc_search_predicted(const uint8_t* ref_n, const uint8_t* src_n, int w, int h,
                          const double H[9], const orc_params* p, int ntiles,
                          const int32_t* corner_xy, const uint8_t* valid, const float* pred,
                          int refine, uint32_t fallback_cost, int32_t* match_xy, uint32_t* cost,
                          uint8_t* fell_back);
int  orc_solve8(const double A[64], const double b[8], double x[8], double tol);
int  orc_pow2_scale(int w);
int  orc_is_inlier(const double Ht[9], int px, int py, int qx, int qy, int w, int h, double eps);
void orc_weed(const int32_t* corner_xy, const int32_t* match_xy, const uint8_t* valid, int n,
              int w, int h, const orc_params* p, uint64_t seed, int iter_begin, int iter_end,
              uint32_t* mask_bits, int32_t* accepted_out);

/* ---- a7: least-squares homography over the weeded set -------------------- */
int  orc_fit_homography(const int32_t* corner_xy, const int32_t* match_xy,
                        const uint32_t* mask_bits, int n, int w, int h,
                        const double H_prev[9], double H_out[9]);
int  orc_fit_homography_real(const double* p_xy, const double* q_xy, int n, double H_out[9]);

/* ---- pyramid matcher: a2..a7 over all levels ------------------------------ */
int  orc_match(const uint8_t* ref_n, const uint8_t* src_n, int w, int h, const orc_params* p,
               double H0_out[9], int32_t* corner_xy, int32_t* match_xy, uint32_t* cost,
               uint8_t* valid, uint32_t* mask_bits, int32_t* level_stats);

/* ---- a8: sparse-to-dense flow (Eq. 5-6, domain transform) ---------------- */
void orc_dt_sigma(double sigma_s, int iters, int i, double* sigma_i, double* a_i);
void orc_dt_filter(double** planes, int nplanes, const uint8_t* guide, int w, int h,
                   double sigma_s, double sigma_r, int iters);
void orc_flow(const uint8_t* guide, int w, int h, int n, const int32_t* corner_xy,
              const int32_t* match_xy, const uint32_t* mask_bits, const double H0[9],
              const orc_params* p, double* flow_u, double* flow_v, double* n_tilde);

/* ---- a9: warp ------------------------------------------------------------ */
double orc_bilinear(const uint8_t* img, int w, int h, double x, double y);
int  orc_bilinear_clipped(const uint8_t* img, int w, int h, double x, double y);
void orc_warp(const uint8_t* src_y, const uint8_t* src_u, const uint8_t* src_v, int w, int h,
              const double H0[9], const double* flow_u, const double* flow_v,
              double* out_y, double* out_u, double* out_v, uint8_t* clip_y);

/* ---- a10: SSIM ghost mask -------------------------------------------------- */
void orc_ssim(const double* x, const double* y, int w, int h, double sigma, int radius,
              double* out);
void orc_ghost_mask(const uint8_t* ref_n, const double* warped_y, int w, int h, int mode,
                    double gain, const uint8_t* src_lut, double sigma, int radius, double* q);

/* ---- a11: weighted irradiance merge --------------------------------------- */
double orc_well_exposedness(double z, double sigma);
void orc_merge(int w, int h, const uint8_t* ref_y, const uint8_t* ref_u, const uint8_t* ref_v,
               int nsrc, const double* const* wy, const double* const* wu,
               const double* const* wv, const double* const* q,
               const uint8_t* const* clip, const double* ratio, double we_sigma,
               double* out_y, double* out_u, double* out_v);

int  orc_max_threads(void);

/* ---- whole path for one stack (n-1 registrations, Sec. 2) ----------------- */
int  orc_register_merge(int w, int h, const uint8_t* ref_y, const uint8_t* ref_u,
                        const uint8_t* ref_v, int nsrc, const uint8_t* const* src_y,
                        const uint8_t* const* src_u, const uint8_t* const* src_v,
                        const int32_t* ratio_num, const int32_t* ratio_den,
                        const orc_params* p, double* out_y, double* out_u, double* out_v,
                        double* H0_out, double* const* warped_y_out,
                        double* const* flow_u_out, double* const* flow_v_out,
                        double* const* q_out, uint8_t* const* clip_out);

#ifdef __cplusplus
}
#endif
#endif
