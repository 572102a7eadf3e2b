/*
 * tdpm.h -- C-ABI of the tensor-decomposed DPM scoring library (sm_103a / GB300).
 *
 * The library scores deformable part models (Sec. 2 of "Tensor-based approach to accelerate deformable part models"):
 *   step 1  correlate every root and part filter with every level of a HOG feature pyramid, either with the full
 *           h x w x 32 filter (Sec. 2, score equation) or with its CP decomposition (Sec. 4, I o T = sum_r ((I o a_r)
 *           o b_r) o c_r; joint mode shares a_r, b_r, c_r across the filters of one shape and recombines per filter);
 *   step 2  generalised distance transform with argmax of every part score map (Sec. 2, argmax equation);
 *   step 3  shift the transformed part maps to their anchors and add them to the root map (Sec. 2, score equation);
 *   step 4  keep the positions whose score reaches the threshold tau (Algorithm 1, steps 15-16).
 *
 * Conventions shared by every entry point
 *   - Status: 0 (TDPM_OK) or a negative TDPM_ERR_* code; no C++ exception or abort crosses the ABI. The message of the
 *     last failure on the calling thread is returned by tdpm_last_error().
 *   - Features: 32 channels per cell, NHWC FP32 ("[H][W][32]", cell (y, x) channel c at ((y*W)+x)*32+c).
 *   - Filters: [h][w][32] FP32, same cell/channel order. A filter is correlated at every valid placement: the score
 *     map of an h x w filter on an H x W level is (H-h+1) x (W-w+1); a level the filter does not fit is skipped.
 *   - Deformation: d[4] = coefficients of (dx, dx^2, dy, dy^2), displacement = part position - anchor, in part-level
 *     cells. d[1] and d[3] must be > 0.
 *   - Pyramid: level j >= lambda holds root positions; its parts are scored on level j - lambda (twice the
 *     resolution). Part i of a root placed at (y, x) is anchored at (2y + anchor_y, 2x + anchor_x). A root position is
 *     scored only when the root filter and every anchored part placement lie inside their maps.
 *   - Ties: the part position is the lexicographically smallest (row, column) among the maximisers.
 *   - Streams: a `void* stream` is a cudaStream_t (NULL = legacy default stream). Device pointers passed in must stay
 *     valid until the work enqueued on that stream has completed.
 *   - Thread safety: one internal mutex per context; calls on one context are serialised.
 */
#ifndef TDPM_H
#define TDPM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TDPM_FEAT_DIM 32
#define TDPM_MAX_PARTS 16

typedef int32_t tdpm_status;
#define TDPM_OK 0
#define TDPM_ERR_ARG (-1)      /* bad argument (NULL pointer, out-of-range value) */
#define TDPM_ERR_SHAPE (-2)    /* inconsistent sizes */
#define TDPM_ERR_OOM (-3)      /* device memory budget or cudaMalloc exhausted */
#define TDPM_ERR_CAPACITY (-4) /* caller buffer too small; the required count is still reported */
#define TDPM_ERR_TIMEOUT (-5)  /* a bounded wait expired */
#define TDPM_ERR_CUDA (-6)     /* CUDA runtime error */
#define TDPM_ERR_STATE (-7)    /* unknown id or call out of order */
#define TDPM_ERR_IO (-8)       /* file error or corrupt factor file */

/* correlation form, Sec. 2 (full filter) and Sec. 4 (CP-decomposed filter) */
#define TDPM_FORM_FULL 0
#define TDPM_FORM_DECOMPOSED 1

/* arithmetic of the correlation, FP32 accumulation always:
 *   FP32     FP32 operands on the FP32 ALUs;
 *   BF16     BF16 operands on the tensor cores (features and tensor-core factors rounded to BF16);
 *   FP8      E4M3 operands on the tensor cores (kind::f8f6f4) for the full correlation and the decomposed channel
 *            stage: features scaled by 448/0.2 (HOG cells are truncated at 0.2), each bank of filters (or of channel
 *            factors c_r) by 448 / its largest magnitude, rounded to nearest even; results rescaled in FP32. The
 *            separable passes and the joint recombination keep FP32 and BF16. Accuracy is reported, not guaranteed;
 *   BF16X3   split BF16 on the tensor cores: every operand x = hi + lo with hi = bf16(x), lo = bf16(x - hi), and each
 *            product is formed as hi*hi + hi*lo + lo*hi (relative error about 2^-16, three MMAs per product). */
#define TDPM_PREC_FP32 0
#define TDPM_PREC_BF16 1
#define TDPM_PREC_FP8 2
#define TDPM_PREC_BF16X3 3

/* decomposition mode: one CP per filter (Sec. 4, per-filter rank R) or one CP per stacked shape group with shared
 * factors a_r, b_r, c_r and per-filter weights Lambda[k][r] */
#define TDPM_DECOMP_PER_FILTER 0
#define TDPM_DECOMP_JOINT 1

typedef struct tdpm_ctx tdpm_ctx;

/* ---------------------------------------------------------------- model (Sec. 2: root f0, parts f_i, costs d_i) */
typedef struct {
    int32_t h, w;
    const float *data; /* host [h][w][32]; copied by tdpm_load_model */
} tdpm_filter;

typedef struct {
    tdpm_filter filter;
    int32_t anchor_y, anchor_x; /* part-level cells, relative to twice the root position */
    float deform[4];            /* coefficients of (dx, dx^2, dy, dy^2); deform[1], deform[3] > 0 */
} tdpm_part;

typedef struct {
    tdpm_filter root;
    float bias;
    int32_t n_parts; /* 0 .. TDPM_MAX_PARTS */
    const tdpm_part *parts;
} tdpm_component;

typedef struct {
    int32_t n_components; /* mixture components (Sec. 2), scored independently */
    const tdpm_component *components;
} tdpm_model_desc;

/* ---------------------------------------------------------------- feature pyramid (device memory, caller-owned) */
typedef struct {
    int32_t H, W;
    const float *data; /* device NHWC FP32 [H][W][32] */
} tdpm_level;

typedef struct {
    int32_t n_levels;
    int32_t lambda; /* levels per octave: root level j uses part level j - lambda */
    const tdpm_level *levels;
} tdpm_pyramid;

/* ---------------------------------------------------------------- detections (Algorithm 1 result set D) */
typedef struct {
    int32_t image;                  /* index of the pyramid in the batch (0 for tdpm_build_pyramid_scores) */
    int32_t model;                  /* id of the model that scored it */
    int32_t component, level, y, x; /* root placement (top-left cell) */
    float score;                    /* s = f0.phi(p0) + sum_i (f_i.phi(p_i) - d_i.psi(p_i, p0)) + bias */
    int32_t n_parts;
    int32_t part_y[TDPM_MAX_PARTS], part_x[TDPM_MAX_PARTS]; /* best part placements on level - lambda */
} tdpm_detection;

typedef struct {
    int32_t n_groups;       /* shape groups decomposed */
    int32_t total_rank;     /* sum over groups of the number of rank-1 terms */
    int32_t total_iters;    /* ALS cycles over all decompositions */
    double max_rel_error;   /* max over filters of ||f - CP(f)||_F / ||f||_F */
    double mean_rel_error;  /* mean of the same */
    double gain;            /* formula (1) over the whole model: full products / decomposed products */
} tdpm_decomp_report;

/* ================================================================================================= context */

/* Create a context on CUDA device `device`. mem_budget_bytes caps the device memory the context allocates for score
 * buffers (0 = no cap). The context owns every allocation it makes; tdpm_destroy frees them. */
tdpm_status tdpm_create(tdpm_ctx **out, int32_t device, size_t mem_budget_bytes);
void tdpm_destroy(tdpm_ctx *ctx);
/* Message of the last failed call made by this thread (empty if none). Valid until the thread's next call. */
const char *tdpm_last_error(void);
/* Library build string (compiler, architecture). */
const char *tdpm_version(void);

/* ================================================================================================= model */

/* Copy a model (Sec. 2) to the context: host filters are copied (caller keeps ownership) and uploaded. Filters are
 * numbered in model order: component 0 root, its parts, component 1 root, ... Filters with the same role (root or
 * part) and shape form one shape group. Errors: ERR_ARG (NULL, n_parts > TDPM_MAX_PARTS, deform[1] or deform[3] <= 0,
 * non-positive sizes). */
tdpm_status tdpm_load_model(tdpm_ctx *ctx, const tdpm_model_desc *desc, int32_t *model_id);

/* n_filters, n_groups of a loaded model. */
tdpm_status tdpm_model_info(tdpm_ctx *ctx, int32_t model_id, int32_t *n_filters, int32_t *n_groups);

/* Shape group g: role (0 root, 1 part), h, w, number of filters, current rank (0 = not decomposed); filter_ids gets
 * the model-order ids of its filters (capacity entries at most). */
tdpm_status tdpm_group_info(tdpm_ctx *ctx, int32_t model_id, int32_t group, int32_t *role, int32_t *h, int32_t *w,
                            int32_t *n_filters, int32_t *rank, int32_t *filter_ids, int32_t capacity);

/* CP-decompose the model's filters (Sec. 4): host FP64 alternating least squares, one exact least-squares solve per
 * factor per cycle, stopping after max_iters cycles or when the fit changes by at most tol * ||T||_F. mode
 * TDPM_DECOMP_PER_FILTER gives every filter `rank` terms (rank >= h*w uses the exact slice decomposition);
 * TDPM_DECOMP_JOINT gives every shape group `rank` shared terms. The factors are kept in FP64 and uploaded in FP32 and
 * BF16. Errors: ERR_ARG (rank <= 0, bad mode), ERR_STATE (unknown model). */
tdpm_status tdpm_decompose(tdpm_ctx *ctx, int32_t model_id, int32_t rank, int32_t mode, int32_t max_iters, double tol,
                           uint64_t seed, tdpm_decomp_report *report);

/* Rank detection (Sec. 4) with per-filter decomposition: for every filter f (h x w x 32), the smallest r in
 * [1, max_rank] with ||f - CP(f, r)||_F < e * (r (h + w + 32) / (h w 32))^2, CP(f, r) being the rank-r ALS
 * decomposition of tdpm_decompose (same iterations, tolerance and seed). r is searched upward from 1: the paper starts
 * a binary search, but the error of an ALS fit need not decrease with r, so only the scan finds the smallest r. A
 * filter that meets the test at no r <= max_rank keeps rank max_rank (the exact slice form, error 0, when max_rank >=
 * h*w). e: the criterion's constant, which the paper leaves open (> 0). ranks (optional): the chosen rank of every
 * filter, indexed by filter id (tdpm_model_info's n_filters entries). The factors replace any earlier decomposition;
 * the report is that of tdpm_decompose. Errors: ERR_ARG (e <= 0 or not finite, max_rank <= 0), ERR_STATE. */
tdpm_status tdpm_decompose_auto(tdpm_ctx *ctx, int32_t model_id, double e, int32_t max_rank, int32_t max_iters,
                                double tol, uint64_t seed, int32_t *ranks, tdpm_decomp_report *report);

/* Per-filter decomposition (Sec. 4) with a rank chosen for every filter, e.g. the (S, T) pairs of Sec. 5: rank S for
 * the root filters and T for the part filters. ranks: host array indexed by filter id (tdpm_model_info's n_filters
 * entries), each > 0; a rank >= h*w gives the exact slice form of that filter (error 0). Iterations, tolerance, seed
 * and report are those of tdpm_decompose; the factors replace any earlier decomposition.
 * Errors: ERR_ARG (NULL, a rank <= 0, max_iters <= 0), ERR_STATE (unknown model). */
tdpm_status tdpm_decompose_ranks(tdpm_ctx *ctx, int32_t model_id, const int32_t *ranks, int32_t max_iters, double tol,
                                 uint64_t seed, tdpm_decomp_report *report);

/* FP64 factors of shape group g: A [h][R], B [w][R], C [32][R], Lambda [n_filters][R] (row-major). Any output may be
 * NULL. Errors: ERR_STATE (not decomposed). */
tdpm_status tdpm_get_factors(tdpm_ctx *ctx, int32_t model_id, int32_t group, double *A, double *B, double *C,
                             double *Lambda);

/* Save / load the decomposition of a model (versioned binary file with FP64 factors and a checksum). Loading checks
 * that the shapes match the model. Errors: ERR_IO. */
tdpm_status tdpm_save_factors(tdpm_ctx *ctx, int32_t model_id, const char *path);
tdpm_status tdpm_load_factors(tdpm_ctx *ctx, int32_t model_id, const char *path);

/* ================================================================================================= scoring */

/* Steps 1-3 for every component and root level of one pyramid: correlation in `form` and `precision`, distance
 * transform of every part map, shift-and-sum into per-(component, level) score maps. Enqueued on `stream`; returns
 * before the GPU finishes. The score buffers live in the context until tdpm_release(scores_id).
 * Limit: a part filter's score map may be at most 800 cells wide and tall (the distance transform keeps a strip of
 * its x-pass result for every row in shared memory), i.e. part levels of images up to about 3,200 pixels on a side at
 * 4-pixel part cells; larger maps return ERR_ARG.
 * Errors: ERR_ARG, ERR_STATE (decomposed form before tdpm_decompose), ERR_OOM (budget). */
tdpm_status tdpm_build_pyramid_scores(tdpm_ctx *ctx, int32_t model_id, const tdpm_pyramid *pyr, int32_t form,
                                      int32_t precision, void *stream, int32_t *scores_id);

/* Steps 1-3 for a batch of pyramids (images of any sizes) in one scores set: every stage is one launch over all
 * levels of all images, and repeated batches of the same shapes replay one captured CUDA graph. Detections carry the
 * image index. Same errors as tdpm_build_pyramid_scores; ERR_ARG for n_images < 1. */
tdpm_status tdpm_build_batch_scores(tdpm_ctx *ctx, int32_t model_id, const tdpm_pyramid *pyrs, int32_t n_images,
                                    int32_t form, int32_t precision, void *stream, int32_t *scores_id);

/* tdpm_build_batch_scores for a subset of the model's components per image (not in the paper: a bank of class models
 * loaded as one model, each image scored for the classes it asks for). component_mask: host [n_images][components],
 * nonzero = score that component on that image; NULL = all. Step 1 (the correlation) still covers every filter of
 * the model, as one contraction; steps 2-4 run only for the selected components, and their results are those the
 * full batch gives. */
tdpm_status tdpm_build_batch_scores_subset(tdpm_ctx *ctx, int32_t model_id, const tdpm_pyramid *pyrs,
                                           int32_t n_images, const uint8_t *component_mask, int32_t form,
                                           int32_t precision, void *stream, int32_t *scores_id);

/* Step 4: every scored position with s >= tau, ordered by (image, component, level, y, x), copied to the host array
 * `out` (capacity records). Blocks until `stream` has finished. *n_out = number of detections, even when it exceeds
 * capacity (then ERR_CAPACITY and the first `capacity` records are written). Records of `out` past *n_out (within
 * capacity) may be overwritten: the count and a prefix of the records come back in one copy, sized from the previous
 * read-back of the same plan. */
tdpm_status tdpm_detect(tdpm_ctx *ctx, int32_t scores_id, float tau, tdpm_detection *out, size_t capacity,
                        size_t *n_out, void *stream);

/* tdpm_detect with one threshold per (image, component): tau is a host array [n_images][components] (a class model's
 * own threshold, a request's threshold). Same results and errors; ERR_ARG for a NaN threshold. */
tdpm_status tdpm_detect_thresholds(tdpm_ctx *ctx, int32_t scores_id, const float *tau, tdpm_detection *out,
                                   size_t capacity, size_t *n_out, void *stream);

/* Step 4 followed by greedy non-maximum suppression (not in the paper: the DPM convention), on the device. The
 * detections with s >= tau are grouped by (image, class), class = component_class[component] (n_components entries,
 * ids >= 0; NULL = one class). A detection's box is its component's root filter at its level: cells of
 * cell0 * 2^(level / lambda) image pixels (cell0 = the pixel size of a level-0 cell, e.g. 4 for sbin 8 with a 2x
 * first octave), box [x c, x c + w0 c) x [y c, y c + h0 c). Within a group the detections are taken by score (ties:
 * record order); each one not yet suppressed is kept and suppresses every later one whose box it covers by more than
 * `overlap` (in [0, 1]) of that later box's own area. Boxes and overlaps are FP64. The kept records are written to
 * `out` in the order of tdpm_detect; *n_out = their number (ERR_CAPACITY as tdpm_detect). */
tdpm_status tdpm_detect_nms(tdpm_ctx *ctx, int32_t scores_id, float tau, const int32_t *component_class,
                            double overlap, double cell0, tdpm_detection *out, size_t capacity, size_t *n_out,
                            void *stream);

/* ---------------------------------------------------------------- feature extraction block (Sec. 2): HOG pyramid */
/* The paper scores DPM v5's HOG features and notes that extracting them costs about a twentieth of the scoring
 * (Sec. 2). The library computes them on the device in that form (Felzenszwalb et al., PAMI 2010, Sec. 6), 32
 * channels per cell: per pixel the colour channel with the largest squared central-difference gradient and the nearest
 * of 18 oriented directions (both decided in FP32, products and sums rounded once), bilinear votes of the magnitude
 * into cells of sbin pixels (floor(n / sbin + 1/2) cells per side), four 2x2-block normalisations per cell
 * (1 / sqrt(block energy + 1e-4)), truncation at 0.2, and the projection to 18 contrast-sensitive, 9 -insensitive and
 * 4 texture channels plus a zero channel; the outermost ring of cells is dropped. The pyramid resamples the image by
 * area averaging at the lambda scales 2^(-i / lambda), then halves each octave into the next; levels 0..lambda-1 are
 * the first octave at sbin / 2 (the part levels), then the root levels at sbin while both sides keep at least
 * min_cells cells. */

/* Level count, level sizes (level_hw[2 j], level_hw[2 j + 1] = rows, columns; may be NULL) and the bytes of the FP32
 * NHWC output of an img_h x img_w image. sbin 4, 8 or 16; lambda 1..64. ERR_ARG for an image too small for one root
 * level; ERR_CAPACITY when level_hw is given and max_levels is below the level count. */
tdpm_status tdpm_hog_pyramid_shape(int32_t img_h, int32_t img_w, int32_t sbin, int32_t lambda, int32_t min_cells,
                                   int32_t *n_levels, int32_t *level_hw, int32_t max_levels, size_t *out_bytes);

/* The feature pyramid of a device 8-bit RGB image [img_h][img_w][3] into d_out (device, 16-byte aligned, at least
 * the bytes tdpm_hog_pyramid_shape gives; caller-owned): levels[j] (host array of max_levels) receives each level's
 * rows, columns and device pointer inside d_out, ready for tdpm_build_pyramid_scores. Asynchronous on `stream`; the
 * context's scratch is reused by its next HOG call (ordered by an event). A call repeating the previous one (same
 * sizes, parameters, image and output buffers) reuses its device tables, and from the third call on replays its
 * launches as one CUDA graph. ERR_ARG for sides outside [16, 16384], a bad sbin, lambda or min_cells, or a d_out
 * that is not 16-byte aligned; ERR_CAPACITY when out_bytes or max_levels is too small. */
tdpm_status tdpm_hog_pyramid(tdpm_ctx *ctx, const uint8_t *d_image, int32_t img_h, int32_t img_w, int32_t sbin,
                             int32_t lambda, int32_t min_cells, float *d_out, size_t out_bytes, tdpm_level *levels,
                             int32_t max_levels, int32_t *n_levels, void *stream);

/* The features of one device FP32 RGB image [h][w][3] at cell size sbin (2, 4, 8 or 16) into d_out ([*out_h][*out_w]
 * [32], 16-byte aligned). Synchronous. */
tdpm_status tdpm_hog_features(tdpm_ctx *ctx, const float *d_img, int32_t h, int32_t w, int32_t sbin, float *d_out,
                              size_t out_bytes, int32_t *out_h, int32_t *out_w, void *stream);

/* Area-averaging resample of a device FP32 image [h][w][3] by scale in (0, 1] into d_dst ([*out_h][*out_w][3],
 * floor(n scale + 1/2) per side). Asynchronous on `stream`. */
tdpm_status tdpm_resize(tdpm_ctx *ctx, const float *d_src, int32_t h, int32_t w, double scale, float *d_dst,
                        size_t dst_bytes, int32_t *out_h, int32_t *out_w, void *stream);

/* ---------------------------------------------------------------- convolution shortening (Sec. 4, Algorithm 1) */
/* A root hypothesis (a record's component, level, y, x) is pruned as soon as, for some filter of its component, the
 * partial sum of the filter's first q CP terms at the hypothesis falls below the filter's threshold t_q. Filters are
 * visited root first, then the parts in model order; the root is evaluated at (y, x) on the record's level, part i
 * at its anchor (2y + vy_i, 2x + vx_i) on the level lambda below. Term r of a filter at window phi is
 * lambda_r sum_{dy,dx,c} phi[dy][dx][c] a_r[dy] b_r[dx] c_r[c]; a filter's terms are taken in decreasing |lambda_r|
 * (ties by term index). Partial sums are FP32 from the FP32 levels and FP32 factors. The model must be decomposed per
 * filter (ERR_STATE otherwise), and `pyrs` must describe the very device levels the scores set was built from, still
 * alive and unchanged (ERR_ARG when the count, a size, lambda or a level pointer differs). */
typedef struct {
    int64_t candidates;      /* records tested (those with s >= tau) */
    int64_t pruned;          /* of them, pruned by a threshold */
    int64_t terms_evaluated; /* CP terms evaluated before each hypothesis's exit, summed */
    int64_t terms_total;     /* CP terms of every filter of every candidate's component (the work without exits) */
} tdpm_cascade_stats;

/* Every filter's partial sums at caller records (host array, e.g. from tdpm_detect), without exits: out is a host
 * array [n][max_slots][max_terms]; out[i][s][q] = the partial sum of the first q + 1 terms of slot s (0 = root, 1 + p
 * = part p) of record i's component; NaN beyond a filter's rank or slot count. ERR_CAPACITY when max_slots is below
 * 1 + the largest part count or max_terms below the largest per-filter rank; ERR_ARG for a record outside the scores
 * set or whose window leaves its level. */
tdpm_status tdpm_cascade_partials(tdpm_ctx *ctx, int32_t scores_id, const tdpm_pyramid *pyrs, int32_t n_images,
                                  const tdpm_detection *records, size_t n, float *out, int32_t max_slots,
                                  int32_t max_terms, void *stream);

/* Thresholds of Sec. 4 from positive examples: t[f][q] = min over the positives (host records of the scores set) of
 * filter f's partial sum of its first q + 1 terms, the tightest values that prune no positive. t is a host array
 * [n_filters][stride], stride >= the largest per-filter rank; filters of components with no positive, and entries
 * beyond a filter's rank, get -inf (never prune). */
tdpm_status tdpm_cascade_thresholds(tdpm_ctx *ctx, int32_t scores_id, const tdpm_pyramid *pyrs, int32_t n_images,
                                    const tdpm_detection *positives, size_t n, float *t, int32_t stride, void *stream);

/* Step 4 with convolution shortening: the detections with s >= tau that no threshold prunes (host thresholds
 * [n_filters][stride] as tdpm_cascade_thresholds writes them), in the order of tdpm_detect, evaluated on the device
 * one warp per hypothesis with an exit at the first partial sum below its threshold. *n_out and ERR_CAPACITY as
 * tdpm_detect; stats (may be NULL) receives the pruning counts. ERR_ARG for a NaN threshold or tau. */
tdpm_status tdpm_detect_cascade(tdpm_ctx *ctx, int32_t scores_id, const tdpm_pyramid *pyrs, int32_t n_images,
                                const float *t, int32_t stride, float tau, tdpm_detection *out, size_t capacity,
                                size_t *n_out, tdpm_cascade_stats *stats, void *stream);

/* Map kinds for tdpm_get_maps */
#define TDPM_MAP_FILTER_SCORE 0 /* index_a = filter id, index_b = level: correlation map [H-h+1][W-w+1] FP32 */
#define TDPM_MAP_FINAL_SCORE 1  /* index_a = component, index_b = root level: score map [Y][X] FP32 */
#define TDPM_MAP_PART_DT 2      /* index_a = part filter id, index_b = root level: transformed part map at the
                                   anchored positions [Y][X] FP32 */
#define TDPM_MAP_PART_ARG 3     /* same indices: argmax (part_y << 16) | part_x, int32 [Y][X] */

/* Device bytes tdpm_build_batch_scores would hold for this batch (the scores set's arena, rounded up to the size the
 * library allocates), without launching anything. Same argument rules; errors as tdpm_build_batch_scores. */
tdpm_status tdpm_scores_bytes(tdpm_ctx *ctx, int32_t model_id, const tdpm_pyramid *pyrs, int32_t n_images,
                              int32_t form, int32_t precision, size_t *bytes);

/* Copy one map of image `image` of a scores set to host memory (blocks on `stream`). rows/cols receive its size; a map
 * that was not computed (filter does not fit, empty domain) has 0 rows. Errors: ERR_CAPACITY (bytes too small),
 * ERR_STATE, ERR_ARG (image out of range). */
tdpm_status tdpm_get_maps(tdpm_ctx *ctx, int32_t scores_id, int32_t kind, int32_t image, int32_t index_a,
                          int32_t index_b, void *out_host, size_t capacity_bytes, int32_t *rows, int32_t *cols,
                          void *stream);

/* Free a scores set. */
tdpm_status tdpm_release(tdpm_ctx *ctx, int32_t scores_id);

/* ================================================================================================= stateless ops */

/* Generalised distance transform of one score map (Sec. 2 argmax equation), on device buffers:
 *   D[i][k] = max_{qy,qx} S[qy][qx] - d . (qx - px, (qx - px)^2, qy - py, (qy - py)^2),
 *   px = x_off + x_step*k (k < nx), py = y_off + y_step*i (i < ny), both inside the map;
 *   arg[i][k] = (qy << 16) | qx, the lexicographically smallest maximiser.
 * S: device [H][W] FP32 (1 <= H, W <= 800); D: device [ny][nx] FP32; arg: device [ny][nx] int32; scratch: device
 * buffer of at least tdpm_dt_scratch_bytes(H, nx) bytes (intermediate x-pass result), owned by the caller.
 * Errors: ERR_ARG (d[1] or d[3] <= 0, sampled positions outside the map, NULL pointers). */
size_t tdpm_dt_scratch_bytes(int32_t H, int32_t nx);
tdpm_status tdpm_dt(const float *S, int32_t H, int32_t W, const float d[4], int32_t x_off, int32_t x_step, int32_t nx,
                    int32_t y_off, int32_t y_step, int32_t ny, float *D, int32_t *arg, void *scratch, void *stream);

/* Allocation-free variant of tdpm_dt. The paper has no counterpart; this entry point exists for callers that must not
 * allocate device memory: applications whose device memory is owned entirely by another allocator (a framework's
 * caching allocator or a memory pool that has reserved the GPU, where a stray cudaMalloc can fail or fragment it),
 * and latency-critical loops that cannot afford the device-wide synchronisation cudaMalloc/cudaFree may imply.
 *   - Same arguments, layouts and results as tdpm_dt, without the scratch buffer: the job record and the x-pass
 *     intermediate live in a fixed 4 MiB device array inside the library, which every GPU that loads the library
 *     holds until the process exits. H * nx may not exceed tdpm_dt_noalloc_max_elements() (524,224): larger sizes
 *     return TDPM_ERR_ARG.
 *   - The job record reaches the array as a kernel argument, so the call copies nothing from host memory and does
 *     not wait for the stream.
 *   - The first call on a device looks up that array's device address (with the device current); make that first
 *     call before any stream capture starts.
 *   - Every call on a device shares the one array and overwrites it: calls whose work overlaps on the GPU (other
 *     streams, or other threads) race and corrupt each other's results. Serialise them, e.g. on one stream.
 *   - Calls no cudaMalloc, cudaFree or allocating library routine. */
size_t tdpm_dt_noalloc_max_elements(void);
tdpm_status tdpm_dt_noalloc(const float *S, int32_t H, int32_t W, const float d[4], int32_t x_off, int32_t x_step,
                            int32_t nx, int32_t y_off, int32_t y_step, int32_t ny, float *D, int32_t *arg,
                            void *stream);

/* Correlation of K filters of one shape with one feature level (step 1, Sec. 2), on device buffers:
 *   out[k][y][x] = sum_{dy<h,dx<w,c<32} filt[k][dy][dx][c] * feat[y+dy][x+dx][c], y < H-h+1, x < W-w+1.
 * feat: device NHWC FP32; filt: HOST [K][h][w][32] FP32 (uploaded per call); out: device [K][H-h+1][W-w+1] FP32.
 * precision FP32 runs the FP32 SIMT kernel, BF16 the tcgen05 tensor-core kernel on BF16-rounded operands. The
 * tensor-core precisions run the one-CTA-per-tile form, or the persistent form when the environment variable
 * TDPM_CORR_FORM is "persistent" (read at each call); both give the same results. */
tdpm_status tdpm_correlate(const float *feat, int32_t H, int32_t W, const float *filt_host, int32_t K, int32_t h,
                           int32_t w, int32_t precision, float *out, void *stream);

/* ================================================================================================= instrumentation */

/* Number of CUDA kernels this process has launched through the library (all contexts). */
uint64_t tdpm_kernel_launches(void);

/* When enabled, every stage the context enqueues is bracketed by CUDA events recorded on the stage's own stream, and
 * the device time is accumulated per stage name ("to_bf16", "corr_tc", "corr_f32", "zproj_tc", "zproj_f32", "sep",
 * "zsep_tc", "recomb_tc", "dt", "assemble", "detect"). While enabled, the shape groups' correlation chains run one after another
 * on the caller's stream instead of concurrently, so that each stage is timed alone. Disabled by default. */
tdpm_status tdpm_profile_enable(tdpm_ctx *ctx, int32_t enable);

/* Stage `index` of the accumulated profile (waits for the recorded events): its name (NUL-terminated, truncated to
 * name_cap), total device milliseconds and number of launches. *n_stages receives the number of stages; an index out
 * of range only sets *n_stages. */
tdpm_status tdpm_profile_read(tdpm_ctx *ctx, int32_t index, char *name, size_t name_cap, double *total_ms,
                              int64_t *launches, int32_t *n_stages);

/* Clear the accumulated profile. */
tdpm_status tdpm_profile_reset(tdpm_ctx *ctx);

/* Tile shapes picked by the context's autotuner (not in the paper). The first build of a new plan times the N tile
 * widths its tensor-core launches may use on the plan's own inputs and keeps the fastest per shape class; set the
 * environment variable TDPM_AUTOTUNE=0 before tdpm_create to use the untuned defaults. The candidates are every
 * balanced N tile width in two kernel forms: one CTA per tile, or persistent CTAs with two TMEM accumulators (the
 * epilogue of one tile overlapping the MMAs of the next). Entry `index`: its shape class ("kind:N:K blocks:
 * operands:M tiles", NUL-terminated, truncated to key_cap), the chosen width and form (1 = persistent); *n_entries
 * receives the number of entries (an index out of range only sets it). Entries of the fused decomposed kernel (keys
 * "zsep:16h+w:terms per group:operands:items") choose among its forms instead: *tile_n receives the form (0: one CTA
 * per item; 1: persistent, two feature stages; 2: persistent, two Z buffers; 3: both; 4: persistent, one of each)
 * and *persistent is 0. */
tdpm_status tdpm_autotune_read(tdpm_ctx *ctx, int32_t index, char *key, size_t key_cap, int32_t *tile_n,
                               int32_t *persistent, int32_t *n_entries);

/* Failure-detection self-test (not in the paper). Launches one kernel whose mbarrier wait can never complete: the
 * wait is the bounded one of every tensor-core kernel, so it gives up after its limit (about half a second), raises
 * the context's device error flag and the kernel exits. Returns ERR_TIMEOUT, the status any call reports after an
 * expired device wait, having cleared the flag: the context stays usable. ERR_STATE if the expiry was not reported.
 * No fault, trap or hang is involved. */
tdpm_status tdpm_selftest_bounded_wait(tdpm_ctx *ctx);

/* Kernel fusion of the decomposed form (Sec. 4) with per-filter factors and BF16 or split-BF16 operands. enable = 1
 * (the default; the environment variable TDPM_FUSE=0 before tdpm_create sets 0): the channel stage (Z_r = phi o c_r,
 * on the tensor cores) and the separable passes with the recombination run as ONE kernel per shape group, the
 * rank-1 maps Z_r staying in shared memory (stage name "zsep_tc" in the profile). Shapes with a compiled fused form:
 * 6x6, 5x11, 7x7, 11x5, each filter with at most 64 terms; other groups, joint factors, FP32 and FP8 run unfused.
 * enable = 0: two launches per group with Z_r in device memory ("zproj_tc", then "sep"). Both give bit-identical
 * score maps. Applies to score builds started afterwards (plans are cached per setting). */
tdpm_status tdpm_set_fusion(tdpm_ctx *ctx, int32_t enable);

/* ================================================================================ serving (continuous batching) */
/* Not in the paper: a request loop around the scoring path. A server thread owned by the context takes submitted
 * requests (an image pyramid already on the device plus the class models to score it with), groups the pending ones
 * that use the same (model, form, precision) into one multi-image batch (tdpm_build_batch_scores), and keeps up to
 * max_inflight batches on the device at once, each on its own stream: requests that arrive while others run are
 * launched as soon as a slot and the memory budget allow, and the detections of one batch are read back while the
 * next is already running. A batch's device footprint is its arena (every map and intermediate of its plan); the
 * batches in flight together stay within mem_budget_bytes. A request scored alone and in a mix gives the same
 * detections: every stage computes each image's positions with the same arithmetic whatever else is in the batch. */
#define TDPM_MAX_REQUEST_MODELS 64

typedef struct {
    int32_t max_batch_images; /* images in one batch (1..4096) */
    int32_t max_inflight;     /* batches on the device at once (1..4) */
    int32_t max_wait_us;      /* with nothing in flight, how long to wait for more requests before launching (>= 0) */
    size_t mem_budget_bytes;  /* device bytes the batches in flight may hold together (0 = no limit) */
} tdpm_server_config;

typedef struct {
    const tdpm_pyramid *pyramid; /* device levels (same rules as tdpm_build_pyramid_scores); the caller keeps them
                                    alive and unchanged until the request's result has been polled */
    const int32_t *model_ids;    /* the class models to score the image with: 1..TDPM_MAX_REQUEST_MODELS ids */
    int32_t n_models;
    int32_t form, precision;     /* as for tdpm_build_pyramid_scores */
    float tau;                   /* detection threshold (Algorithm 1, step 16) */
    const int32_t *components;   /* optional: only these components of each listed model (distinct ids); NULL = all */
    int32_t n_components;
} tdpm_request;

typedef struct {
    int32_t status;          /* TDPM_OK, or the error that ended one of the request's batches */
    int32_t batch_images;    /* images in the largest batch the request was scored in */
    uint64_t t_submit_ns;    /* steady clock: tdpm_submit accepted it */
    uint64_t t_start_ns;     /* its first batch was launched */
    uint64_t t_done_ns;      /* its last detections were read back */
    uint64_t n_detections;   /* detections over all of its models */
} tdpm_result_info;

/* Start the context's server thread. Errors: ERR_ARG (config out of range), ERR_STATE (already running). */
tdpm_status tdpm_server_start(tdpm_ctx *ctx, const tdpm_server_config *cfg);

/* Finish every submitted request, then stop and join the server thread (results stay pollable). No-op when not
 * running. tdpm_destroy calls it. */
tdpm_status tdpm_server_stop(tdpm_ctx *ctx);

/* Queue a request; *ticket identifies its result. The request is copied (the pyramid's level array and the model id
 * list may be reused at once; the device data they point to may not). Errors: ERR_ARG (invalid request),
 * ERR_STATE (server not running). A model id that is not loaded fails the request later, with ERR_STATE. */
tdpm_status tdpm_submit(tdpm_ctx *ctx, const tdpm_request *req, uint64_t *ticket);

/* Wait up to timeout_ms (< 0: no limit) for a request to finish. Returns ERR_TIMEOUT if it has not. When it has: the
 * detections of every model, ordered by (model as listed in the request, component, level, y, x), with image = 0 and
 * model = the model id, are copied to out (up to capacity records; *n_out = their number). The result is then
 * released, unless it did not fit (ERR_CAPACITY: poll again with a larger buffer). *info (optional) receives the
 * request's status and timestamps. A request that failed returns its error status, with *n_out = 0 (no records),
 * its info filled and the result released. Errors: ERR_STATE (unknown or already released ticket). */
tdpm_status tdpm_poll(tdpm_ctx *ctx, uint64_t ticket, int32_t timeout_ms, tdpm_detection *out, size_t capacity,
                      size_t *n_out, tdpm_result_info *info);

#ifdef __cplusplus
}
#endif

#endif /* TDPM_H */
