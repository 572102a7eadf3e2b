// Internal declarations shared by the CUDA translation units of libtdpm (not part of the C-ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tdpm.h"

namespace tdpm {

constexpr int FD = TDPM_FEAT_DIM;  // channels per HOG cell
constexpr int MAXP = TDPM_MAX_PARTS;

// ------------------------------------------------------------------------------------------------ work-list jobs
// Every stage runs as ONE launch over all (level, map) jobs of a pyramid. A CTA (or a warp) finds its job by binary
// search of its linear index in the jobs' begin prefixes.

// Step 1, full form: one (shape group, level) pair. Output maps are [K][Ho][Wo] contiguous per filter.
struct CorrJob {
    const float *feat;        // FP32 NHWC level
    const uint16_t *feat_bf;  // BF16 copy of the level: NHWC (SIMT paths) or tensor-core layout (tcgen05 paths)
    float *out;               // [K][Ho][Wo]
    int H, W, Ho, Wo;
    int tiles_x, tiles_y;     // position tiles of this job
    int begin;                // first linear tile index of this job
};

// Step 1, decomposed form, stage Z: per-cell projections Z[r][cell] = sum_c C[c][r] phi[cell][c].
struct ZJob {
    const float *feat;
    const uint16_t *feat_bf;
    float *Z;                 // [R][H*W]
    int cells;                // H*W
    int begin;                // first linear tile index
};

// Step 1, decomposed form, stage U+S: separable passes of Z and recombination into filter maps.
struct SepJob {
    const float *Z;           // [R][H][W]
    float *out;               // [K][Ho][Wo]
    int H, W, Ho, Wo;
    int tiles_x, tiles_y;
    int begin;
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
    int xbegin;               // first warp of this job in the x pass (warps of 32 rows)
    int ybegin;               // first warp of this job in the y pass (warps of 32 sampled columns)
};

// Step 3: one (component, root level) pair.
struct AsmJob {
    const float *root;        // root score map, row stride root_W
    int root_W;
    int Y, X;                 // scored root positions
    float bias;
    int n_parts;
    int comp, level;
    float *out;               // [Y][X]
    const float *D[MAXP];     // [Y][X] each
    const int32_t *A[MAXP];   // [Y][X] each
    long long begin;          // first linear position of this job
};

// --------------------------------------------------------------------------------------------------- launchers
// Every launcher adds the number of kernels it launched to the process-wide counter (tdpm_kernel_launches).
void note_launches(int n);

// All launchers enqueue on `s` and return the launch error (cudaSuccess when the launch was accepted).

// K8: FP32 SIMT direct correlation. filt_t: [h*w*32][Kpad] (filter index fastest), Kpad a multiple of 64.
cudaError_t launch_corr_f32(const CorrJob *d_jobs, int n_jobs, int total_tiles, const float *filt_t, int K, int Kpad,
                            int h, int w, cudaStream_t s);
int corr_f32_tile_x();
int corr_f32_tile_y();
int corr_f32_tile_k();

// K1: tcgen05 BF16 implicit-GEMM correlation. feat_bf in the tensor-core layout written by convert_levels_tc.
cudaError_t launch_corr_tc(const CorrJob *d_jobs, int n_jobs, int total_tiles, const uint16_t *filt_tc, int K, int Npad,
                           int h, int w, cudaStream_t s);
int corr_tc_tile_m();
int corr_tc_n_tile(int K);

// Conversions: FP32 NHWC -> BF16 NHWC (n elements), and FP32 NHWC -> BF16 tensor-core layout [4][H][W][8].
cudaError_t launch_to_bf16(const float *src, uint16_t *dst, long long n, cudaStream_t s);
cudaError_t launch_to_bf16_planar(const float *src, uint16_t *dst, int H, int W, cudaStream_t s);

// K2: Z projection, SIMT. Ct: [R][32] FP32 (BF16 precision: already rounded to BF16 values).
cudaError_t launch_zproj_simt(const ZJob *d_jobs, int n_jobs, int total_tiles, const float *Ct, int R, bool bf16_feat,
                              cudaStream_t s);
int zproj_simt_cells_per_tile();
int zproj_simt_r_chunk();

// K3+K4: separable passes + recombination, SIMT. A: [h][R], B: [w][R]; lam: per-rank weights (per-filter mode,
// rank range [rank_off[k], rank_off[k+1])) or dense Lambda [K][R] (joint mode).
cudaError_t launch_sep_simt(const SepJob *d_jobs, int n_jobs, int total_tiles, const float *A, const float *B,
                            const float *lam, const int *rank_off, int K, int R, int h, int w, bool joint,
                            cudaStream_t s);
int sep_tile_x();
int sep_tile_y();
int sep_filters_per_cta(bool joint);

// K5/K6: distance transform passes.
cudaError_t launch_dt(const DtJob *d_jobs, int n_jobs, int x_warps, int y_warps, int max_W, int max_H, cudaStream_t s);

// K7: assembly (shift and sum), then detection count / scan / write.
cudaError_t launch_assemble(const AsmJob *d_jobs, int n_jobs, long long total, cudaStream_t s);
cudaError_t launch_detect(const AsmJob *d_jobs, int n_jobs, long long total, float tau, int *d_block_counts,
                          int *d_block_offsets, int n_blocks, tdpm_detection *d_out, long long capacity,
                          long long *d_total, cudaStream_t s);
int detect_positions_per_block();

}  // namespace tdpm
