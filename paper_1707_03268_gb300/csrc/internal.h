// Internal declarations shared by the CUDA translation units of libtdpm (not part of the C-ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tdpm.h"

namespace tdpm {

constexpr int FD = TDPM_FEAT_DIM;  // channels per HOG cell
constexpr int MAXP = TDPM_MAX_PARTS;

// ------------------------------------------------------------------------------------------------ work-list jobs
// Every stage runs as ONE launch over all (level, map) jobs of a pyramid. A CTA (or a warp) finds its job by binary
// search of its linear index in the jobs' begin prefixes.

// Step 1, full form, FP32 SIMT: one (shape group, level) pair. Output maps are [K][Ho][Wo] contiguous per filter.
struct CorrJob {
    const float *feat;        // FP32 NHWC level
    float *out;               // [K][Ho][Wo]
    int H, W, Ho, Wo;
    int tiles_x, tiles_y;     // position tiles of this job
    int begin;                // first linear tile index of this job
};

// Step 1 on tensor cores (full form, or the channel stage of the decomposed form with a 1x1 tap): one (group,
// level) pair. The tensor map describes the level's BF16 planar copy [4][H*W][8].
struct alignas(128) TcJob {
    CUtensorMap tmap;         // BF16 (hi part) planar copy of the level
    CUtensorMap tmap_lo;      // lo part (split-BF16 precision only)
    float *out;               // [N][Ho][Wo] (channel stage: [R][H][W])
    int H, W, Ho, Wo;
    int begin;                // first M tile of this job (M tiles numbered across the jobs of a launch)
    int pad[3];
};

// Step 1, decomposed form, per-filter mode, channel stage and separable passes fused on the tensor cores: one
// (group, level) pair. The tensor maps describe the level's BF16 planar copy as [4][H][W][8] (box {8, 32, 4, 4}).
struct alignas(128) ZsJob {
    CUtensorMap tmap;         // hi part
    CUtensorMap tmap_lo;      // lo part (split-BF16 precision only)
    float *out;               // [K][Ho][Wo]
    int H, W, Ho, Wo;
    int pad[4];
};

// A spatial tile of the fused launch: its job, origin (first output column and row) and valid output rows.
struct ZsTile {
    int job, x0, y0, rows;
};

// A filter group of the fused launch: filters [k0, k1) of the shape group, whose terms [t0, t0 + n) (n <= nmax) are
// the N = n rounded up to 16 columns of one MMA.
struct ZsGroup {
    int k0, k1, t0, n;
};

// Step 1, decomposed form, stage Z on the FP32 SIMT path: Z[r][cell] = sum_c C[c][r] phi[cell][c].
struct ZJob {
    const float *feat;
    float *Z;                 // [R][H*W]
    int cells;                // H*W
    int begin;                // first linear tile index
};

// Step 1, decomposed form, separable passes + recombination (or, in the per-term mode, the per-term maps U_r).
struct SepJob {
    const float *Z;           // [R][H][W]
    float *out;               // [K][Ho][Wo]
    uint16_t *U, *U_lo;       // per-term mode: U_r as BF16 planar [Upad/8][Ho*Wo][8] (hi part, lo part or null)
    int H, W, Ho, Wo;
    int tiles_x, tiles_y;
    long long begin;          // first work item of this job
};

// FP32 NHWC level -> BF16 planar [4][cells][8].
struct ConvJob {
    const float *src;
    uint16_t *dst;            // bf16(x)
    uint16_t *dst_lo;         // bf16(x - bf16(x)), or null
    long long cells;
    long long begin;          // first (cell, chunk) item of this job
};

// Step 2: one part score map, transformed at sampled positions.
struct DtJob {
    const float *S;           // [H][W]
    int H, W;
    float lx, qx, ly, qy;     // d0 (dx), d1 (dx^2), d2 (dy), d3 (dy^2)
    int x_off, x_step, nx;    // sampled columns
    int y_off, y_step, ny;    // sampled rows
    float *V;                 // x-pass values  [H][nx]
    int32_t *IV;              // x-pass argmax  [H][nx]
    float *D;                 // result         [ny][nx]
    int32_t *A;               // (qy << 16) | qx [ny][nx]
    int xbegin;               // first CTA of this job in the x pass (ceil(H / dt_lines_per_cta()) CTAs per job)
    int ybegin;               // first CTA of this job in the y pass (ceil(nx / dt_lines_per_cta()) CTAs per job)
};

// Step 3: one (component, root level) pair.
struct AsmJob {
    const float *root;        // root score map, row stride root_W
    int root_W;
    int Y, X;                 // scored root positions
    float bias;
    int n_parts;
    int image, comp, level;   // level index within its image
    float *out;               // [Y][X]
    const float *D[MAXP];     // [Y][X] each
    const int32_t *A[MAXP];   // [Y][X] each
    long long begin;          // first linear position of this job
};

// --------------------------------------------------------------------------------------------------- launchers
// Every launcher adds the number of kernels it launched to the process-wide counter (tdpm_kernel_launches) and
// returns the launch error (cudaSuccess when the launch was accepted).
void note_launches(int n);
// While a thread captures a CUDA graph, its launches are counted here (they run at each replay) instead of now.
extern thread_local int *t_capture_launches;

// Raise a kernel's dynamic shared memory limit to the per-block maximum, once per device. Launches still request only
// what they use; a fixed limit keeps captured CUDA graphs valid whatever order their launches were recorded in.
// slot: a distinct number per kernel (0 .. kSmemSlots-1) under which the setting is remembered.
cudaError_t allow_max_dynamic_smem(const void *func, int slot);
constexpr int kMaxDynamicSmem = 232448;
constexpr int kSmemSlots = 48;

// K8: FP32 SIMT direct correlation. filt_t: [h*w*32][Kpad] (filter index fastest), Kpad a multiple of 64.
cudaError_t launch_corr_f32(const CorrJob *d_jobs, int n_jobs, int total_tiles, const float *filt_t, int K, int Kpad,
                            int h, int w, cudaStream_t s);
int corr_f32_tile_x();
int corr_f32_tile_y();
int corr_f32_tile_k();

// K1: tcgen05 BF16 implicit-GEMM correlation over m_tiles M tiles (the jobs' begin fields number them) and
// ceil(K / NT) N tiles of width NT (a multiple of 16, <= 256). filt_tc: [h*w*cb][4][ld][8] BF16 with ld >= the N tiles
// times NT (corr_tc_bank_rows). The input has 32*cb channels (cb = 1 for HOG features; cb = terms / 32 for the
// recombination of per-term maps). filt_tc_lo non-null selects split-BF16 operands (lo parts of the filters; the
// jobs' tmap_lo must describe the lo parts of the input). d_err: device flag raised when a bounded wait expires.
// fp8: E4M3 operands (bank [h*w*cb][2][ld][16] bytes, input tmap from encode_level_tmap_fp8, no lo parts); the
// results are multiplied by `scale` (the inverse of the operands' per-tensor scales).
// persistent: one CTA per SM slot walks many tiles, with two TMEM accumulators so that the epilogue of one tile
// overlaps the MMAs of the next; otherwise one CTA per tile. Both give the same results.
cudaError_t launch_corr_tc(const TcJob *d_jobs, int n_jobs, int m_tiles, const void *filt_tc, const void *filt_tc_lo,
                           int K, int ld, int NT, int h, int w, int cb, int *d_err, cudaStream_t s, bool fp8 = false,
                           float scale = 1.f, bool persistent = false);
int corr_tc_tile_m();
int corr_tc_n_tiles(int K, int NT);
int corr_tc_default_nt(int K, int taps);     // untuned N tile width for K filters over `taps` K blocks (h*w*cb)
int corr_tc_nt_candidates(int K, int *out);  // up to 4 widths a tuner may choose; returns their number
int corr_tc_bank_rows(int K);                // bank rows (ld) that fit every candidate width
constexpr int kTcPersistent = 1 << 16;       // tile configuration code: N tile width | kTcPersistent
// Tensor map of a BF16 planar array [chunks][cells][8] (chunks a multiple of 4), box {8, 144, 4}: a row segment.
bool encode_level_tmap(CUtensorMap *map, const uint16_t *planar, long long cells, int chunks = 4);
// Tensor map of an E4M3 planar level [2][cells][16] bytes, box {16, 144, 2}: a row segment.
bool encode_level_tmap_fp8(CUtensorMap *map, const uint8_t *planar, long long cells);

// Tensor map of a BF16 planar level [4][H][W][8] as a 4-D array, box {8, 32 columns, 4 rows, 4 chunks}.
bool encode_level_tmap_tiles(CUtensorMap *map, const uint16_t *planar, int H, int W, int box_w = 32, int box_h = 4);

// K2+K3+K4 fused (per-filter mode, BF16 or split-BF16 operands): the channel stage on the tensor cores and the
// separable passes with the recombination, over `tiles` spatial tiles (records d_tiles, each naming its job) times
// n_fg filter groups. cbank / cbank_lo: the channel-factor bank [1][4][ld][8] BF16 (hi, lo or null); every group
// needs t0 + n rounded up to 16 <= ld. nmax = 32 or 64 (zsep_nmax) bounds the terms of a group. Shapes: zsep_shape
// (the filter shapes of the separable warp form).
bool zsep_shape(int h, int w);
void zsep_tile(int h, int w, int *tile_cols, int *tile_rows);  // output columns and rows of one spatial tile
int zsep_nmax(int max_rank);                                     // 32, 64, or 0 when a filter has more terms
// form: ZSEP_TILE, one CTA per item; or a persistent form, one CTA per SM walking the items with a producer warp
// ahead of the compute warps (two TMEM accumulators), with one or two feature stages and one or two Z buffers
// (zsep_form_fits tells which fit). Every form reads the groups' packed factor records d_frec: per filter
// group, zsep_record_bytes bytes: a_r[0..h), b_r[0..w), lambda_r, zero-padded to zsep_factor_stride floats per term
// for nmax terms (zero beyond the group's terms), then the rank offsets of the group's filters minus t0 (nmax + 2
// ints). All forms give the same results.
enum ZsepForm { ZSEP_TILE = 0, ZSEP_PERSIST_S2 = 1, ZSEP_PERSIST_Z2 = 2, ZSEP_PERSIST_S2Z2 = 3, ZSEP_PERSIST_S1 = 4 };
cudaError_t launch_zsep_tc(const ZsJob *d_jobs, const ZsTile *d_tiles, int tiles, const ZsGroup *d_fg, int n_fg,
                           const void *cbank, const void *cbank_lo, int ld, const void *d_frec, int nmax, int h, int w,
                           int *d_err, cudaStream_t s, int form);
bool zsep_form_fits(int h, int w, bool split, int nmax, int form);
int zsep_record_bytes(int h, int w, int nmax);
int zsep_factor_stride(int h, int w);

// FP32 NHWC -> BF16 planar for many levels in one launch (total = sum of 4 * cells).
cudaError_t launch_to_bf16_planar(const ConvJob *d_jobs, int n_jobs, long long total, cudaStream_t s);
// FP32 NHWC -> E4M3 planar [2][cells][16] of x * scale (ConvJob.dst holds the bytes; total = sum of 2 * cells).
cudaError_t launch_to_fp8_planar(const ConvJob *d_jobs, int n_jobs, long long total, float scale, cudaStream_t s);
// Per-tensor scale of the FP8 features: HOG cells are truncated at 0.2, mapped to the largest E4M3 value 448.
constexpr float kFp8FeatureScale = 448.f / 0.2f;

// K2: Z projection, SIMT FP32. Ct: [R][32] FP32.
cudaError_t launch_zproj_simt(const ZJob *d_jobs, int n_jobs, int total_tiles, const float *Ct, int R, cudaStream_t s);
int zproj_simt_cells_per_tile();
int zproj_simt_r_chunk();

// K3+K4: separable passes along y (a_r) and x (b_r) + recombination. A: [h][R], B: [w][R].
//   SEP_PER_FILTER: lam[R] per-term weights, filter k owns terms [rank_off[k], rank_off[k+1]);
//   SEP_JOINT:      lam = Lambda [K][R], every filter sums all R terms;
//   SEP_TERMS:      no recombination: U_r for r < K (= Upad, a multiple of 8) written as BF16 planar (zero for r >= R).
enum SepMode { SEP_PER_FILTER = 0, SEP_JOINT = 1, SEP_TERMS = 2 };
cudaError_t launch_sep(const SepJob *d_jobs, int n_jobs, long long total_items, const float *A, const float *B,
                       const float *lam, const int *rank_off, int K, int R, int h, int w, int mode, cudaStream_t s);
// Work items of one level job of launch_sep (K filters, or Upad terms in SEP_TERMS mode): sets the job's tiles_x and
// tiles_y; the jobs' begin fields are the running sums of these counts.
long long sep_job_items(int mode, int h, int w, int Ho, int Wo, int K, int *tiles_x, int *tiles_y);

// K5/K6: distance transform passes (x_ctas / y_ctas: the CTA totals the jobs' xbegin / ybegin count; sides <= 800).
// K2+K3+K4 with the CP terms on the MMA's M dimension (zsept_tc.cu), per-filter decomposition of 6x6 or 7x7 filters:
// items = n_tiles spatial tiles (ZsTile: 16 x 16 cells of Z, 17 - w output columns, 17 - h output rows) x n_tg term
// groups (consecutive filters, at most zsept_terms() terms); d_grec: n_tg records of zsept_record_bytes() bytes
// (factors [16][128] floats: lambda a_r, b_r per term lane; then nf, k0, lane ranges); d_group_t0: first term of each
// group in the channel bank (whose rows must extend zsept_terms() rows past it). The jobs' tensor maps use a
// {8, 16, 16, 4} box.
bool zsept_shape(int h, int w);
int zsept_tile_side();
int zsept_terms();
int zsept_record_bytes();
int zsept_factor_stride();
cudaError_t launch_zsept_tc(const ZsJob *d_jobs, const ZsTile *d_tiles, int n_tiles, int n_tg, const void *d_grec,
                            const int *d_group_t0, const void *cbank, const void *cbank_lo, int ld, int h, int w,
                            int *d_err, cudaStream_t s);

cudaError_t launch_dt(const DtJob *d_jobs, int n_jobs, int x_ctas, int y_ctas, int max_W, int max_H, cudaStream_t s);
int dt_lines_per_cta();
// K5+K6 fused: one CTA per (job, strip of dt_strip_columns() sampled columns), the jobs' xbegin counting those CTAs;
// V and IV stay in shared memory (the jobs' V / IV are not used). Results identical to launch_dt.
// d_cta_jobs: the job of each CTA (null: found by a search of the jobs' xbegin).
cudaError_t launch_dt_fused(const DtJob *d_jobs, int n_jobs, const int *d_cta_jobs, int ctas, int max_W, int max_H,
                            cudaStream_t s);
int dt_strip_columns();
int dt_job_strips(int nx);  // strips (CTAs) of a job with nx sampled columns
// Largest side (rows or columns) of a part score map the distance transform accepts.
constexpr int kDtMaxSide = 800;

// K7: assembly (shift and sum), then detection count / scan / write.
cudaError_t launch_assemble(const AsmJob *d_jobs, int n_jobs, long long total, cudaStream_t s);
// count per block + exclusive scan (total to *d_total), then the ordered write of the first `capacity` records
// d_job_tau: null (every job uses tau) or one threshold per assembly job
cudaError_t launch_detect_count(const AsmJob *d_jobs, int n_jobs, long long total, float tau, const float *d_job_tau,
                                int *d_block_counts, int *d_block_offsets, int n_blocks, long long *d_total,
                                cudaStream_t s);
cudaError_t launch_detect_write(const AsmJob *d_jobs, int n_jobs, long long total, float tau, const float *d_job_tau,
                                const int *d_block_offsets, int n_blocks, tdpm_detection *d_out, long long capacity,
                                int model, cudaStream_t s);
int detect_positions_per_block();

// Greedy NMS per (image, class) of n detection records on the device (see nms.cu for the convention). d_cls: the
// class of each component (null: one class); d_root_h / d_root_w: root filter size per component; d_cell: cell size
// in image pixels per (image, level) [n_images][max_levels]. The kept records go to d_out in their original order
// and their number to *d_n_out. d_scratch: at least nms_scratch_bytes(n, n_images * n_classes) bytes.
size_t nms_scratch_bytes(long long n, int n_groups);
cudaError_t launch_nms(const tdpm_detection *d_rec, long long n, const int32_t *d_cls, int n_classes, int n_images,
                       const int32_t *d_root_h, const int32_t *d_root_w, const double *d_cell, int max_levels,
                       double overlap, void *d_scratch, size_t scratch_bytes, tdpm_detection *d_out,
                       long long *d_n_out, cudaStream_t s);

// Convolution shortening (Sec. 4, Algorithm 1) over detection records. Per (component, filter slot) one CascFilter:
// slot 0 the root, slot 1 + i part i. A term r of the filter is lam[r] * sum phi a_r b_r c_r over its window.
struct CascFilter {
    const float *A, *B, *Ct, *lam;  // the filter's shape group: A [h][R], B [w][R], Ct [R][32], lam [R] (FP32)
    const int *order;               // the filter's terms in visiting order (nterms entries, indices into R)
    const float *thr;               // threshold of each visiting position (nterms entries)
    int R, nterms, h, w, vy, vx, part;
};
struct CascLevel {
    const float *data;  // FP32 NHWC level of the caller's pyramid (null: absent)
    int H, W;
};
struct CascArgs {
    const tdpm_detection *rec = nullptr;
    long long n = 0;
    const CascFilter *filt = nullptr;
    const int *comp_first = nullptr, *comp_count = nullptr;  // per component: first slot in filt, slot count
    const CascLevel *levels = nullptr;                       // [n_images][max_levels]
    int max_levels = 0;
    const int *img_lam = nullptr;                            // per image: levels per octave
    bool apply_thr = false;                                  // exit at the first partial sum below its threshold
    float *partials = nullptr;                               // [n][max_slots][max_terms] evaluated partial sums, or null
    int max_slots = 0, max_terms = 0;
    uint8_t *alive = nullptr;                                // [n]: 1 = not pruned, or null
    unsigned long long *stats = nullptr;  // [4] (zeroed by the caller): terms evaluated, terms of all filters, pruned,
                                          // windows out of range (never read)
};
cudaError_t launch_cascade(const CascArgs &args, cudaStream_t s);

// Feature extraction block: HOG pyramid (hog.cu).
struct HogTap {
    int i0, n, w;  // first input index, number of taps, offset of their weights in the weight table
};
struct HogResizeJob {
    const void *src;  // [h][w][3], uint8 (octave 0) or FP32
    int h, w;
    float *dst;       // [ho][wo][3] FP32
    int ho, wo;
    const HogTap *ytaps, *xtaps;  // one per output row / column
    const float *weights;
};
struct HogImage {
    const float *img;  // [h][w][3]
    int h, w;
    float *mag;        // [h][w] gradient magnitude (0 on the border ring)
    uint8_t *bin;      // [h][w] orientation bin 0..17
};
struct HogLevelJob {
    const float *mag;
    const uint8_t *bin;
    int h, w;          // the image the level is computed from
    int sbin, cy, cx;  // cell size and cells per column / row (including the border ring)
    float *hist;       // [cy][cx][18] scratch
    float *energy;     // [cy][cx] scratch: sum_{o<9} (h_o + h_{o+9})^2 per cell
    float *out;        // [cy - 2][cx - 2][32] FP32 features
};
// blocks of the cell kernel for one level (2 sbin threads per cell)
int hog_hist_blocks(int cy, int cx, int sbin);
cudaError_t hog_set_orientations(const float *ux, const float *uy);
cudaError_t launch_hog_resize(const HogResizeJob *d_jobs, int n_jobs, long long max_pixels, bool from_u8,
                              cudaStream_t s);
cudaError_t launch_hog_grad(const HogImage *d_imgs, int n_imgs, long long max_pixels, cudaStream_t s);
cudaError_t launch_hog_levels(const HogLevelJob *d_jobs, int n_jobs, long long max_hist_blocks, long long max_out_cells,
                              cudaStream_t s);

// Ordered compaction: the records whose flag is nonzero go to d_out in record order, their number to *d_n_out.
// d_scratch: at least compact_scratch_bytes(n) bytes.
size_t compact_scratch_bytes(long long n);
cudaError_t launch_compact_records(const tdpm_detection *d_rec, const uint8_t *d_flags, long long n, void *d_scratch,
                                   size_t scratch_bytes, tdpm_detection *d_out, long long *d_n_out, cudaStream_t s);

// Failure-detection self-test: one kernel whose bounded mbarrier wait expires (nothing arrives); it raises *d_err.
cudaError_t launch_bounded_wait_probe(int *d_err, cudaStream_t s);

}  // namespace tdpm
