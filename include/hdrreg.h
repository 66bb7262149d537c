/*
 * hdrreg.h -- C ABI of the B300 (sm_103a) library for locally non-rigid HDR
 * registration and merging of exposure stacks, after Gallo, Troccoli, Hu,
 * Pulli and Kautz, "Locally Non-rigid Registration for Mobile HDR
 * Photography" (arXiv 1504.01441).
 *
 * The source frame of a stack is brought to the reference frame's exposure,
 * matched to the reference on a pyramid (per-tile corners and an SSD search
 * around a per-level homography, Sec. 2.2), its matches weeded (Sec. 2.3),
 * the sparse displacements spread into a dense flow by an edge-aware filter
 * (Sec. 2.4), the source resampled onto the reference, and the frames merged
 * into an irradiance map weighted by well-exposedness and an SSIM
 * consistency mask (Sec. 2.5, Sec. 3.1).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every image / array pointer is a DEVICE pointer owned by the caller,
 *    unless the parameter says "host". Planes are row-major and tightly
 *    packed: luma is w x h bytes, YUV420 chroma (U, V) is (w/2) x (h/2).
 *  - Pixel centres are at integer coordinates. "Normalized" coordinates are
 *    those of Sec. 2.2 (Eq. 3): x_n = (2x - (w-1)) / w, y_n = (2y - (h-1)) / w.
 *    A homography is double[9] in device memory, row-major, H[8] = 1, mapping
 *    reference -> source in normalized coordinates.
 *  - Step calls never allocate. They are asynchronous on `stream` (a
 *    cudaStream_t; NULL = legacy default stream), never synchronize the host,
 *    and can be captured into a CUDA graph. Scratch memory, where needed, is
 *    passed in as `workspace` of at least the size the matching *_workspace_size
 *    call returns (256-byte aligned). hdrreg_weed_static, which takes no
 *    workspace, is described on its own where it is declared.
 *  - Arguments are validated on the host before anything is launched; an
 *    invalid argument returns HDRREG_E_INVALID_ARG and launches nothing. A
 *    launch failure returns HDRREG_E_CUDA. hdrreg_last_error() returns a
 *    thread-local text for the last failure of the calling thread.
 *  - Conditions found on the device (a level with too few matches, a singular
 *    fit) do not fail the call; they are written to the optional device
 *    status words / diagnostics named below.
 */
#ifndef HDRREG_H
#define HDRREG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HDRREG_ABI_VERSION 1

typedef enum hdrreg_status {
    HDRREG_OK = 0,
    HDRREG_E_INVALID_ARG = 1,
    HDRREG_E_CUDA = 2,
    HDRREG_E_DEGENERATE = 3,
    HDRREG_E_TIMEOUT = 4,
    HDRREG_E_UNSUPPORTED = 5,
    HDRREG_E_WORKSPACE = 6
} hdrreg_status;

/* Exposure normalization modes (row a1). */
#define HDRREG_NORM_RATIO 0   /* brighten the darker frame by the known ratio, clip at 255 */
#define HDRREG_NORM_HISTEQ 1  /* equalize each frame's histogram (Sec. 3)                  */

/*
 * Method parameters. hdrreg_params_default() fills the paper's values where
 * the paper gives them (Sec. 2.6: 21x21 patches, search radius 10, up to 5
 * levels, levels >= 100 px, candidate grid spacing T/16, sigma_s = 400; the
 * frames' histograms equalized before matching, Sec. 3) and this library's
 * readings of its silences elsewhere, among them that the flow carries the residual
 * to the level-0 homography (dense map H0 + F). hdrreg_params_paper() is the same
 * with the paper's literal propagation (the corners' whole displacement q - p is
 * spread, Sec. 2.4; the homography is then used only to seed the matcher).
 */
typedef struct hdrreg_params {
    int tile;             /* T: tile side in pixels of the level, 8..128, even          */
    int radius;           /* R: SSD search radius, 1..15                                */
    int patch_half;       /* SSD patch is (2*patch_half+1)^2; 1..15                     */
    int levels_max;       /* maximum pyramid levels, 1..8                               */
    int min_level_size;   /* a level is kept only if both sides >= this                 */
    int grid_half;        /* K: corner candidates c + s*(i,j), i,j in [-K,K], 0..8      */
    int quad;             /* q: quadrant side of the cornerness measure, 1..32          */
    int corner_thresh;    /* T of Eq. 2 as a mean difference in DN (sum thr T*q*q)      */
    int weed_iters;       /* iterations of the Eq. 4 filter per level, 0..65536         */
    int weed_delta_min;   /* delta = max(delta_min, ceil(n_valid / delta_div))         */
    int weed_delta_div;
    int norm_mode;        /* HDRREG_NORM_RATIO or HDRREG_NORM_HISTEQ                    */
    int dt_iters;         /* domain-transform iterations, 1..8                          */
    int ssim_radius;      /* SSIM Gaussian window radius; must be 5                     */
    int propagate_full;   /* 0: flow = residual to H0 (dense map H0+F); 1: q - p (H ignored) */
    int output_mode;      /* fused call's output: 0 the irradiance merge (a11); 1 the
                             error-tolerant exposure fusion of Sec. 2.5 (contrast x
                             well-exposedness x SSIM, hdrreg_fuse); 2 the same without the
                             contrast factor                                           */
    double weed_eps;      /* inlier distance, pixels of the level                       */
    double sigma_s;       /* domain-transform spatial sigma                             */
    double sigma_r;       /* domain-transform range sigma, on a [0,1] intensity scale   */
    double ssim_sigma;    /* SSIM Gaussian window sigma                                 */
    double we_sigma;      /* well-exposedness sigma                                     */
    double flow_eps;      /* F = 0 where the filtered normalization map is below this   */
    uint64_t weed_seed;   /* stream of the counter-based sampler (level l uses seed+l)  */
    const float* predictor; /* learned level-0 search (row a-L): device parameters of the
                               displacement network, or NULL for the plain SSD search   */
    uint32_t fallback_cost; /* learned search: a tile whose least SSD around the
                               predicted match exceeds this falls back to the full search */
    int32_t predictor_refine; /* learned search: offsets [-r, r]^2 around the rounded
                               prediction are tried before the fallback test, 0..radius */
    int32_t search_threads; /* threads per tile CTA of the SSD search (one CTA per tile):
                               0 (= 128), 64, 128 or 256; a launch shape only, the
                               results do not depend on it                              */
} hdrreg_params;

/* A YUV420 (or luma-only: u = v = NULL) 8-bit frame, device pointers. */
typedef struct hdrreg_frame {
    const uint8_t* y;
    const uint8_t* u;
    const uint8_t* v;
} hdrreg_frame;

/* FP32 output planes (device). u, v may be NULL for luma-only stacks. */
typedef struct hdrreg_planes_f32 {
    float* y;
    float* u;
    float* v;
} hdrreg_planes_f32;

/* One warped source as the merge consumes it (row a10-a11). */
typedef struct hdrreg_merge_src {
    const float* y;          /* warped source luma, w x h                                  */
    const float* u;          /* warped source chroma, (w/2) x (h/2), or NULL               */
    const float* v;
    const uint8_t* ref_n;    /* reference normalized for this source's registration        */
    const uint8_t* src_lut;  /* HISTEQ only: the source frame's 256-entry LUT (device)     */
    int ratio_num;           /* exposure ratio t_src / t_ref = num / den, both > 0          */
    int ratio_den;
    const uint8_t* clip;     /* w x h, nonzero where the warped luma sample draws on a source
                                pixel at 0 or 255 (hdrreg_warp's clip_out), or NULL: then a
                                sample is clipped when its value is <= 0 or >= 255          */
} hdrreg_merge_src;

/* Per-source diagnostics written on the device by hdrreg_register_merge. */
typedef struct hdrreg_diag {
    double H0[9];            /* level-0 homography                                          */
    int32_t levels;          /* pyramid levels used                                         */
    int32_t tiles;           /* level-0 tiles                                               */
    int32_t valid;           /* level-0 tiles with a corner                                 */
    int32_t kept;            /* level-0 matches kept by the weeding                         */
    int32_t fit_status;      /* bit l set: level l kept the coarser homography              */
    int32_t fallbacks;       /* learned search: level-0 tiles that fell back to the full
                                search; -1 on the plain path                                */
    int32_t flow_status;     /* 0; 1 if a bounded wait of the flow's pipelined passes ran out
                                (the kernel then stops early and the flow is not valid)     */
    int32_t reserved;
} hdrreg_diag;

/* ---------------------------------------------------------------- misc */
void hdrreg_params_default(hdrreg_params* p);
void hdrreg_params_paper(hdrreg_params* p);
const char* hdrreg_last_error(void);
const char* hdrreg_version(void);
/* Number of kernels this library has enqueued in this process (host counter,
 * incremented at every launch; a graph captured from library calls replays the
 * launches counted while it was captured). */
unsigned long long hdrreg_launch_count(void);
/* Number of pyramid levels for a w x h frame under p (host computation, Sec. 2.6). */
int hdrreg_num_levels(int w, int h, const hdrreg_params* p);
/* Check p; returns HDRREG_OK or HDRREG_E_INVALID_ARG (message in hdrreg_last_error). */
hdrreg_status hdrreg_validate_params(const hdrreg_params* p);

/* ------------------------------------------------------ a1: normalization
 * Bring both luma planes into one 8-bit domain (Sec. 2.1, Sec. 3). RATIO: the
 * exposure ratio r = ratio_num / ratio_den = t_src / t_ref is known; the darker
 * frame is multiplied by max(r, 1/r), rounded to nearest (halves up) and
 * clipped at 255; the other is copied. HISTEQ: each frame is mapped through its
 * own histogram-equalization LUT (ratio ignored). `luts` (optional, 512 bytes:
 * reference LUT then source LUT) receives the maps applied. Workspace:
 * hdrreg_normalize_workspace_size(mode) bytes (0 for RATIO).
 */
size_t hdrreg_normalize_workspace_size(int mode);
hdrreg_status hdrreg_normalize_exposure(const uint8_t* ref_y, const uint8_t* src_y, int w, int h,
                                        int mode, int ratio_num, int ratio_den, uint8_t* ref_n,
                                        uint8_t* src_n, uint8_t* luts, void* workspace,
                                        size_t ws_bytes, void* stream);

/* --------------------------------------------------------- a2: pyramid
 * Levels 1..levels-1 of a 2x2 box pyramid ((a+b+c+d+2)>>2, odd last row /
 * column dropped; Sec. 2.2, Sec. 2.6) of the w x h plane `level0`, written one
 * after the other into `pyr` (level l is (w>>l) x (h>>l) bytes).
 * hdrreg_pyramid_bytes gives the size of `pyr`.
 */
size_t hdrreg_pyramid_bytes(int w, int h, int levels);
hdrreg_status hdrreg_build_pyramid(const uint8_t* level0, int w, int h, int levels, uint8_t* pyr,
                                   void* stream);

/* ---------------------------------------------- a3-a5: local search (one level)
 * For every full tile (floor(w/T) x floor(h/T), row-major) of the normalized
 * reference: pick the corner of highest cornerness (Eq. 1) among the
 * candidate grid that passes the minimum-activity test (Eq. 2); project it by
 * H (Eq. 3, `H` = the coarser level's homography, device) to the rounded
 * search centre c; and find the integer displacement d in [-R, R]^2 of least
 * SSD between the (2h+1)^2 patches (ties: lowest row-major index of d).
 * Outputs per tile (device, n = tiles): corner_xy[2n] (tile centre if no
 * corner), match_xy[2n] = c + d, cost[n] (0xFFFFFFFF if no corner), valid[n].
 * Reads outside the level clamp to the edge.
 */
int hdrreg_num_tiles(int w, int h, int tile);
hdrreg_status hdrreg_local_search(const uint8_t* ref_n, const uint8_t* src_n, int w, int h,
                                  const double* H, const hdrreg_params* p, int32_t* corner_xy,
                                  int32_t* match_xy, uint32_t* cost, uint8_t* valid,
                                  void* stream);

/* ---------------------------------------------------------- a6: weeding
 * Iterations [iter_begin, iter_end) of the union-of-inliers filter of Eq. 4
 * (Sec. 2.3) over the n tiles' matches: each iteration draws 4 distinct valid
 * matches from the counter-based SplitMix64 stream `seed`, fits the
 * homography through them exactly, and if more than delta matches reproject
 * within eps pixels of their match, ORs those matches into mask_bits (bit t of
 * word t/32 = tile t; the caller zeroes it before the first range). Disjoint
 * ranges compose by union: running the ranges in any order equals one run
 * (Sec. 2.3). Workspace: hdrreg_weed_workspace_size(n).
 */
size_t hdrreg_weed_workspace_size(int n);
hdrreg_status hdrreg_weed(const int32_t* corner_xy, const int32_t* match_xy, const uint8_t* valid,
                          int n, int w, int h, const hdrreg_params* p, uint64_t seed,
                          int iter_begin, int iter_end, uint32_t* mask_bits, void* workspace,
                          size_t ws_bytes, void* stream);

/* ------------------------------------ a6 without caller-provided scratch
 * The paper has no counterpart: this is hdrreg_weed for callers that cannot
 * allocate device memory and therefore have no workspace to pass -- real-time
 * pipelines that allow no allocation after start-up, plugins whose host owns
 * all device memory, or code that runs where the CUDA allocator may not be
 * called. Same inputs, output and result as hdrreg_weed; it allocates nothing
 * and calls no allocating routine. As there, mask_bits is OR-ed into: the
 * caller zeroes it before the first iteration range.
 * Its scratch is a fixed array inside this library (about 160 KB on every GPU
 * that loads the library, kept until the process exits), so n must not exceed
 * HDRREG_WEED_STATIC_MAX_TILES (larger n returns HDRREG_E_INVALID_ARG and
 * launches nothing). The first call on each device looks up the array's device
 * address with that device current; make that first call before any stream
 * capture. All calls share the array: calls whose kernels overlap on the GPU
 * (other streams or host threads on the same device) race and must be
 * serialized by the caller.
 */
#define HDRREG_WEED_STATIC_MAX_TILES 8192
hdrreg_status hdrreg_weed_static(const int32_t* corner_xy, const int32_t* match_xy,
                                 const uint8_t* valid, int n, int w, int h,
                                 const hdrreg_params* p, uint64_t seed, int iter_begin,
                                 int iter_end, uint32_t* mask_bits, void* stream);

/* ---------------------------------------------------------- a7: level fit
 * Least-squares homography (DLT, h22 = 1, normalized coordinates) over the
 * matches set in mask_bits (Sec. 2.2: H^l from the level's corners and
 * matches). Normal equations are accumulated exactly in integers. If fewer
 * than 4 matches are set or the system is singular, H_out = H_prev and the
 * optional device word *status is set to 1 (too few) or 2 (singular), else 0.
 * H_prev and H_out may alias.
 */
hdrreg_status hdrreg_fit_homography(const int32_t* corner_xy, const int32_t* match_xy,
                                    const uint32_t* mask_bits, int n, int w, int h,
                                    const double* H_prev, double* H_out, int32_t* status,
                                    void* stream);

/* ------------------------------------- a6 + a7 of one level in one launch
 * The weeding of hdrreg_weed over iterations [iter_begin, iter_end) followed
 * by the level fit of hdrreg_fit_homography over the weeded set, as one
 * kernel: every CTA stages the level's matches in shared memory and the CTA
 * that finishes last solves the fit. Results are bit-identical to
 * hdrreg_weed + hdrreg_fit_homography. mask_bits (ceil(n/32) words, device)
 * is zeroed by the call and receives the weeded set; H_out and *status
 * (optional) as in hdrreg_fit_homography; H_prev and H_out may alias.
 * `counter` is one device word that must be zero before the first call and
 * that every call leaves zero; calls that may run concurrently need distinct
 * counters. Needs hdrreg_weed_fit_supported(n) (the staged matches fit in
 * shared memory, about 12,000 tiles), else HDRREG_E_UNSUPPORTED.
 */
int hdrreg_weed_fit_supported(int n);
hdrreg_status hdrreg_weed_fit(const int32_t* corner_xy, const int32_t* match_xy,
                              const uint8_t* valid, int n, int w, int h,
                              const hdrreg_params* p, uint64_t seed, int iter_begin,
                              int iter_end, uint32_t* mask_bits, const double* H_prev,
                              double* H_out, int32_t* status, uint32_t* counter, void* stream);

/* -------------------------------------------------- a8: sparse-to-dense flow
 * Dense flow from the weeded matches (Sec. 2.4, Eq. 5-6): the maps P_u, P_v
 * hold the residual q - H(p) of every kept match at its corner p (or q - p
 * when p->propagate_full), N holds 1 there; all three are filtered by the
 * recursive domain transform guided by `guide_n` (the normalized reference),
 * and flow = P~ / N~ (0 where N~ < flow_eps). Outputs flow_u, flow_v: w x h
 * FP32. Workspace: hdrreg_flow_workspace_size(w, h).
 */
size_t hdrreg_flow_workspace_size(int w, int h);
hdrreg_status hdrreg_flow_upsample(const uint8_t* guide_n, int w, int h, const int32_t* corner_xy,
                                   const int32_t* match_xy, const uint32_t* mask_bits, int n,
                                   const double* H, const hdrreg_params* p, float* flow_u,
                                   float* flow_v, void* workspace, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------- a9: warp
 * Resample the source onto the reference grid: reference pixel p reads the
 * source at H(p) + flow(p), bilinear with clamp-to-edge taps. Chroma (when
 * src->u, src->v and out->u, out->v are all set; w, h even) samples at
 * (Mbar - 0.5) / 2 with Mbar the mean of the four luma positions of its 2x2
 * block. Outputs FP32 planes. clip_out (optional, device, w x h bytes): 1 where
 * the luma sample draws on a source pixel at 0 or 255 -- a tap with a nonzero
 * bilinear weight: the one at (floor x, floor y) always, its right neighbour
 * when the x fraction is above 0, the row below when the y fraction is above 0
 * -- else 0. The merge gives such a sample no weight (Sec. 2.1: 8-bit frames,
 * so a clipped pixel measured only a bound on its irradiance).
 */
hdrreg_status hdrreg_warp(const hdrreg_frame* src, int w, int h, const double* H,
                          const float* flow_u, const float* flow_v, const hdrreg_planes_f32* out,
                          uint8_t* clip_out, void* stream);

/* ------------------------------------------------ a10-a11: ghost mask + merge
 * Irradiance merge of the reference with nsrc warped sources (host array of
 * descriptors): E = sum_k w_k Z_k / r_k / sum_k w_k with r_ref = 1,
 * w_ref = WE(Z_ref), w_k = WE(Z_k) * max(0, SSIM(ref_n_k, N_k(Z_k))) for a
 * sample that draws on no clipped pixel and w_k = 0 for one that does (the
 * source's clip plane; clipped samples carry no irradiance). WE is the
 * well-exposedness weight of exposure
 * fusion; SSIM uses a Gaussian window (ssim_sigma, radius 5) with clamp-to-edge;
 * N_k maps the warped source into the registration's normalized domain (RATIO:
 * min(255, g z) with g the gain its frame received; HISTEQ: its LUT,
 * interpolated). Chroma: U-128, V-128 merged with the mean luma weight of each
 * 2x2 block. out->y (w x h) and, for YUV420, out->u, out->v ((w/2) x (h/2))
 * are FP32. q_out (optional): nsrc consecutive w x h FP32 masks.
 */
hdrreg_status hdrreg_merge(const hdrreg_frame* ref, int w, int h, int nsrc,
                           const hdrreg_merge_src* srcs, const hdrreg_params* p,
                           const hdrreg_planes_f32* out, float* q_out, void* stream);

/* ------------------------------------------------ a1-a11 fused, one stack
 * The whole path for one stack: each of the nsrc sources (host array) is
 * registered to the reference independently (Sec. 2: n-1 runs) -- a1..a9 --
 * then all are merged (a10-a11). ratio_num / ratio_den (host arrays) give
 * t_src / t_ref per source. Everything stays on the device; diag (optional,
 * device, nsrc entries) receives per-source diagnostics. Workspace:
 * hdrreg_register_merge_workspace_size(w, h, nsrc, p).
 */
size_t hdrreg_register_merge_workspace_size(int w, int h, int nsrc, const hdrreg_params* p);
hdrreg_status hdrreg_register_merge(const hdrreg_frame* ref, int w, int h, int nsrc,
                                    const hdrreg_frame* srcs, const int* ratio_num,
                                    const int* ratio_den, const hdrreg_params* p,
                                    void* workspace, size_t ws_bytes,
                                    const hdrreg_planes_f32* out, hdrreg_diag* diag,
                                    void* stream);

/* --------------------------------------- a-L: tensor-core bf16 product
 * The paper has no counterpart (it has no learned component): the dense
 * contraction under every convolution of the learned displacement predictor.
 * C[M x N] (FP32, row stride ldc) = A[M x K] * B[N x K]^T, A and B bfloat16 with K
 * contiguous (row strides lda, ldb elements), accumulated in FP32 on the tensor
 * cores. A and B must be 16-byte aligned with lda, ldb multiples of 8; M, N, K >= 1.
 * status (device int32, zero on entry) is set to 1 if the kernel gave up waiting
 * for its own copies (nothing then is written to C). HDRREG_E_UNSUPPORTED if the
 * alignment rules are not met or the driver has no tensor-map support.
 */
hdrreg_status hdrreg_gemm_bf16(const void* A, int lda, const void* B, int ldb, int M, int N,
                               int K, float* C, int ldc, int32_t* status, void* stream);

/* ----------------------------------- a-L: the learned displacement predictor
 * The paper has no counterpart (its level-0 displacements come from the SSD search
 * of Sec. 2.2). A convolutional network reads the normalized reference and the
 * source pre-warped by the level-1 homography at quarter resolution, x [n][h][w][2]
 * (bfloat16 bits, NHWC), and outputs one displacement per 32x32 full-resolution
 * tile, out [n][ho][wo][2] FP32 (ho, wo from hdrreg_cnn_out_dims: three stride-2
 * steps, ceil). A fixed feature stage gives per pixel a, b and -(a(p) - b(p + o))^2
 * for o in [-2, 2]^2 (a local SSD cost volume, 27 channels); then 3x3 convolutions
 * 27-16, 16-16, 16-32 (stride 2), 32-32, 32-48 (stride 2), 48-48, 48-64 (stride 2),
 * 64-64, each with bias and ReLU, then a 1x1 head 64-2. theta: HDRREG_CNN_PARAMS FP32 values, per layer W[cout][ky][kx][cin]
 * then b[cout]. Activations are stored in bfloat16, products accumulate in FP32 on
 * the tensor cores. hdrreg_cnn_backward uses the activations the preceding
 * hdrreg_cnn_forward left in the same workspace (same n, h, w, x, theta): loss (a
 * device float) = sum over valid cells |out - label|^2 / max(n_valid, 1), grad
 * (HDRREG_CNN_PARAMS floats) = its gradient. hdrreg_cnn_adam applies one Adam step
 * (beta1 0.9, beta2 0.999, eps 1e-8, bias correction at step >= 1) in place.
 * status: device int32, zero on entry, set to 1 if a tensor-core kernel gave up
 * waiting for its copies. Workspace: hdrreg_cnn_workspace_size(n, h, w).
 */
#define HDRREG_CNN_PARAMS 119538
size_t hdrreg_cnn_workspace_size(int n, int h, int w);
int hdrreg_cnn_out_dims(int h, int w, int* ho, int* wo);
hdrreg_status hdrreg_cnn_forward(const float* theta, const uint16_t* x, int n, int h, int w,
                                 float* out, void* workspace, size_t ws_bytes, int32_t* status,
                                 void* stream);
hdrreg_status hdrreg_cnn_backward(const float* theta, const uint16_t* x, int n, int h, int w,
                                  const float* out, const float* label, const uint8_t* valid,
                                  float* grad, float* loss, void* workspace, size_t ws_bytes,
                                  int32_t* status, void* stream);
hdrreg_status hdrreg_cnn_adam(float* theta, float* m, float* v, const float* grad, int step,
                              float lr, void* stream);
/* Inference form of hdrreg_cnn_forward: the same network on the same inputs, computed
 * without the stored intermediates a backward pass needs. The 3x3 convolutions are
 * implicit GEMMs on the tensor cores (inputs gathered per tap into shared memory, no
 * im2col matrix in memory) with the parameters rounded to bfloat16 as they are staged;
 * the 1x1 head sums in FP32. Results equal hdrreg_cnn_forward's up to the order of the
 * FP32 sums. x must be 4-byte aligned and the workspace 256-byte aligned; the library
 * allocates nothing. Workspace: hdrreg_cnn_infer_workspace_size(n, h, w) (0 for a bad
 * batch). The fused call runs this form for its learned level-0 search.
 */
size_t hdrreg_cnn_infer_workspace_size(int n, int h, int w);
hdrreg_status hdrreg_cnn_infer(const float* theta, const uint16_t* x, int n, int h, int w,
                               float* out, void* workspace, size_t ws_bytes, int32_t* status,
                               void* stream);
/* Where a workspace of batch (n, h, w) keeps what the last hdrreg_cnn_forward stored:
 * layer -1 = the feature stage (bfloat16 [n*h*w][27]), layers 0..7 = the post-ReLU
 * outputs (bfloat16 [rows][cols]). Writes the device address (inside the workspace,
 * valid until the next call that uses it) and the shape; the head (layer 8) stores no
 * bfloat16 output (its FP32 result is `out`): HDRREG_E_INVALID_ARG. */
hdrreg_status hdrreg_cnn_activation(const void* workspace, int n, int h, int w, int layer,
                                    const uint16_t** ptr, int* rows, int* cols);

/* ------------------------------------------- a-L: the learned level-0 search
 * The paper has no counterpart. hdrreg_predictor_input: the network input at
 * quarter resolution (pyramid level 2, w x h): x[y][x] = ((ref - 127.5) / 127.5,
 * (s - 127.5) / 127.5) as bfloat16 pairs, s the source level sampled bilinearly
 * (clamp to edge) at H(p) (H = the level-1 homography, Eq. 3), or at p where the
 * projection's denominator is not positive. hdrreg_tile_labels: per tile the
 * displacement match - centre (FP32 integers; 0 without a corner), the centre
 * being the rounded projection of the corner by H (Eq. 3): the training label.
 * hdrreg_predictor_crops: gathers n training crops of crop_tiles x crop_tiles
 * tiles (8 x 8 quarter-resolution pixels each) from the full input, labels and
 * validity; origins (device int32, 4 per crop) = tile origin x, y inside the tile
 * grid, a symmetry (bit 0 mirror x, bit 1 mirror y, bit 2 transpose; pixels, tiles
 * and label components follow it) and an unused word. A label is valid where the
 * tile has a corner and both components are below label_bound in magnitude (use
 * the search radius: a displacement on the border of the search is not a
 * measurement). hdrreg_local_search_predicted:
 * hdrreg_local_search where a tile with a corner first searches the offsets
 * [-refine, refine]^2 around its centre plus floor(pred + 0.5) (pred: FP32 pairs,
 * pred_rows x pred_ld cells covering the tile grid, cell (ty, tx)); if the least SSD
 * there is at most fallback_cost that is the match, else the tile runs the full
 * search (fell_back[t] = 1). refine = 0 checks the single predicted match. All pointers are device pointers. The fused calls use
 * the learned search when params.predictor is set, the tile is 32 and the pyramid has
 * at least three levels (the network reads level 2); otherwise the plain search.
 */
hdrreg_status hdrreg_predictor_input(const uint8_t* ref_q, const uint8_t* src_q, int w, int h,
                                     const double* H, uint16_t* x_out, void* stream);
hdrreg_status hdrreg_tile_labels(const int32_t* corner_xy, const int32_t* match_xy,
                                 const uint8_t* valid, int n, int w, int h, const double* H,
                                 float* label, void* stream);
hdrreg_status hdrreg_predictor_crops(const uint16_t* x_full, int wq, int hq, const float* label_full,
                                     const uint8_t* valid_full, int ntx, int nty,
                                     const int32_t* origins, int n, int crop_tiles,
                                     float label_bound, uint16_t* x_out, float* label_out,
                                     uint8_t* valid_out, void* stream);
hdrreg_status hdrreg_local_search_predicted(const uint8_t* ref_n, const uint8_t* src_n, int w,
                                            int h, const double* H, const hdrreg_params* p,
                                            const float* pred, int pred_rows, int pred_ld,
                                            int refine, uint32_t fallback_cost,
                                            int32_t* corner_xy, int32_t* match_xy,
                                            uint32_t* cost, uint8_t* valid, uint8_t* fell_back,
                                            void* stream);

/* ------------------------------------- a1-a11 fused, a batch of stacks
 * The paper has no counterpart (it registers one burst at a time): many stacks of
 * one shape run through the fused path of hdrreg_register_merge, stack i on lane
 * i % lanes. Lanes are streams owned by this library, forked from `stream` and
 * joined back into it, so that the latency-bound matching of one stack overlaps
 * the bandwidth-bound flow and merge of others; everything completes before later
 * work on `stream`, and the call can be captured into a CUDA graph. Results are
 * identical to one hdrreg_register_merge per stack. The first batched call on a
 * device (with lanes > 1 and count > 1) creates its lane streams: make it before
 * any stream capture. Calls from several host threads are serialized inside.
 * stacks (host array of `count`) and the arrays it points to are read during the
 * call only. Workspace: hdrreg_register_merge_batch_workspace_size(w, h, nsrc,
 * lanes, p) (one fused workspace per lane).
 */
#define HDRREG_MAX_LANES 16
typedef struct hdrreg_stack {
    const hdrreg_frame* ref;  /* reference frame */
    const hdrreg_frame* srcs; /* nsrc source frames */
    const int* ratio_num;     /* nsrc exposure ratios t_src / t_ref = num / den */
    const int* ratio_den;
    hdrreg_planes_f32 out;    /* merged planes (FP32, device) */
    hdrreg_diag* diag;        /* optional, device, nsrc entries */
} hdrreg_stack;
size_t hdrreg_register_merge_batch_workspace_size(int w, int h, int nsrc, int lanes,
                                                  const hdrreg_params* p);
hdrreg_status hdrreg_register_merge_batch(const hdrreg_stack* stacks, int count, int w, int h,
                                          int nsrc, int lanes, const hdrreg_params* p,
                                          void* workspace, size_t ws_bytes, void* stream);

/* ---------------------------------- f1: error-tolerant exposure fusion (Sec. 2.5)
 * The paper's output image: the exposure fusion of Mertens et al. (2007) over the
 * reference and the warped sources, with each source's SSIM map as a fourth weight
 * (colour saturation has no luma counterpart and is left out). Per luma pixel and frame:
 * W = C * WE(Z) * Q + 1e-12 (C omitted when use_contrast = 0), C = |4 I - its 4
 * neighbours| of I = Z / 255 (edges replicated), WE(z) = exp(-(z/255 - 0.5)^2 /
 * (2 we_sigma^2)), Q = the source's SSIM map (1 for the reference), normalized over the
 * frames. The images (Z / 255; chroma (c - 128) / 255 with the 2x2 means of the luma
 * weights) are blended in Laplacian pyramids weighted by the Gaussian pyramids of the
 * weights (Burt and Adelson: [1 4 6 4 1] / 16 with clamped coordinates, floor(log2
 * min(w, h)) levels) and collapsed. out: 255 x the result (FP32; chroma as signed
 * offsets, like the merge's). ref: u8 planes; srcs: warped FP32 planes (0..255) and the
 * SSIM map (FP32 w x h, as hdrreg_merge writes it). All device pointers; the library
 * allocates nothing. Workspace: hdrreg_fuse_workspace_size(w, h, nsrc, chroma).
 */
typedef struct hdrreg_fuse_src {
    const float* y;
    const float* u;
    const float* v;
    const float* q;
} hdrreg_fuse_src;
size_t hdrreg_fuse_workspace_size(int w, int h, int nsrc, int chroma);
hdrreg_status hdrreg_fuse(const hdrreg_frame* ref, int w, int h, int nsrc,
                          const hdrreg_fuse_src* srcs, int use_contrast, double we_sigma,
                          hdrreg_planes_f32* out, void* workspace, size_t ws_bytes, void* stream);

/* ------------------------- a1-a11 fused, a batch of stacks in host memory
 * The paper has no counterpart. hdrreg_register_merge_batch for stacks whose planes
 * (ref/srcs frames), merged outputs (out) and optional diagnostics (diag) are HOST
 * pointers. On every lane the library copies one stack's input planes into that lane's
 * part of the workspace, runs the fused path and copies the FP32 planes (and the
 * diagnostics) back, all on the lane's stream, so copies of one lane overlap the
 * kernels of the others. The call returns once everything is enqueued: the host
 * buffers must stay valid and untouched until `stream` has passed the call (synchronize
 * it). Page-locked host buffers are needed for the copies to run asynchronously.
 * Workspace (device): hdrreg_register_merge_host_workspace_size(w, h, nsrc, lanes, p),
 * 0 for bad arguments. Results equal hdrreg_register_merge's bit for bit.
 */
size_t hdrreg_register_merge_host_workspace_size(int w, int h, int nsrc, int lanes,
                                                 const hdrreg_params* p);
hdrreg_status hdrreg_register_merge_host(const hdrreg_stack* stacks, int count, int w, int h,
                                         int nsrc, int lanes, const hdrreg_params* p,
                                         void* workspace, size_t ws_bytes, void* stream);

/* ------------------------- a1-a11 fused, a batch of stacks of different shapes
 * The paper has no counterpart. Like hdrreg_register_merge_batch, but every stack
 * carries its own size, source count and parameters (e.g. the tile and radius an
 * autotuner picked for its size). Stacks are placed on `lanes` lanes longest first
 * (by w * h * nsrc), each on the lane with the least work so far; a lane runs its
 * stacks one after another in a workspace sized for its largest. Everything forks
 * from and joins back into `stream` (graph-capturable; the first call per device
 * creates the lane streams). Results are identical to one hdrreg_register_merge per
 * stack. Workspace: hdrreg_register_merge_multi_workspace_size(stacks, count, lanes).
 */
typedef struct hdrreg_stack_ex {
    hdrreg_stack s;            /* frames, ratios, output planes, optional diagnostics */
    int w, h, nsrc;            /* luma size and number of sources of this stack       */
    const hdrreg_params* p;    /* parameters of this stack (host)                    */
} hdrreg_stack_ex;
size_t hdrreg_register_merge_multi_workspace_size(const hdrreg_stack_ex* stacks, int count,
                                                  int lanes);
hdrreg_status hdrreg_register_merge_multi(const hdrreg_stack_ex* stacks, int count, int lanes,
                                          void* workspace, size_t ws_bytes, void* stream);

/* ------------------------- extension: the same batch, merges as one stage
 * The paper has no counterpart (it registers one stack at a time). As
 * hdrreg_register_merge_multi, with the stacks' registrations (a1-a9) on the lanes and
 * then, once every lane has joined `stream`, every stack's merge (a10-a11) in
 * persistent launches that take tiles of any stack (up to 48 stacks per launch) instead
 * of one merge per stack on its lane. Each stack's merge inputs (warped planes,
 * normalized reference, LUTs) stay in the workspace until then. Results are identical to
 * hdrreg_register_merge_multi. Stacks must ask for the irradiance merge (output_mode
 * 0); HDRREG_E_UNSUPPORTED otherwise. Workspace:
 * hdrreg_register_merge_staged_workspace_size(stacks, count, lanes).
 */
size_t hdrreg_register_merge_staged_workspace_size(const hdrreg_stack_ex* stacks, int count,
                                                   int lanes);
hdrreg_status hdrreg_register_merge_staged(const hdrreg_stack_ex* stacks, int count, int lanes,
                                           void* workspace, size_t ws_bytes, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* HDRREG_H */
