// Step 1 on the 5th-generation tensor cores (tcgen05, sm_103a): BF16 operands, FP32 accumulation in TMEM.
//
// One kernel serves three contractions of the path:
//   * full correlation (Sec. 2 score equation): S[k][y][x] = sum_{dy,dx,c} F_k[dy][dx][c] phi[y+dy][x+dx][c], an
//     implicit GEMM with M = positions, N = filters, K = taps x 32 channels, walked tap by tap;
//   * the channel stage of the decomposed form (Sec. 4, correlation with c_r): Z[r][cell] = sum_c C[c][r] phi[cell][c],
//     the same kernel with a single 1x1 tap and N = rank-1 terms;
//   * the recombination of the jointly decomposed form: S[k][pos] = sum_r Lambda[k][r] U_r[pos], a 1x1 tap over
//     cb blocks of 32 "channels" (the terms r), N = filters.
//
// Positions are flattened over the full level width (p = y*W + x, so a 128-row M tile is one contiguous run of cells
// and rows with x >= W-w+1 are computed and dropped). Features are stored as BF16 in a channel-chunk-planar layout
// [4][H*W][8] (16 bytes per cell per chunk). The taps of one filter row read the same cells shifted by dx, so one TMA
// box {8 ch, 144 cells, 4 chunks} at cell p0 + dy*W serves up to 17 of them: it lands in shared memory as the
// no-swizzle K-major canonical layout (core matrix = 8 cells x 16 bytes; 8-row groups 128 bytes apart, K chunks 2304
// bytes apart), and the A operand of tap dx is that segment with its descriptor's start moved by 16 dx bytes. Filter
// taps are stored [tap][4][N][8] and each tap's N-tile slice is fetched with four 1-D bulk copies into the same layout
// for B. A segments and B slices have rings of their own. One thread issues the copies, one
// issues the MMAs, and all four warps drain TMEM (32x32b loads) and store coalesced rows of the output maps.
// Every mbarrier wait is bounded: on expiry the kernel raises the context's error flag and carries on to a clean exit.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>

#include "internal.h"
#include "tc_ptx.h"

namespace tdpm {
namespace {

constexpr int TC_M = 128;
constexpr int TC_MS = 144;                        // cells of an A row segment: an M tile and up to 16 cells right of it
constexpr int TC_DXS = TC_MS - TC_M + 1;          // filter width one segment serves (17, above the widest filter: 16)
constexpr uint32_t A_SEG_PLANE = TC_MS * 16;      // one 16-byte K chunk of a segment

template <class Job>
__device__ __forceinline__ int find_job(const Job *jobs, int n, int idx)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].begin <= idx) lo = mid; else hi = mid - 1;
    }
    return lo;
}


// A tile is one (M tile, N tile) pair; M tiles are numbered across the jobs (a job's begin is its first M tile), so
// the job tables do not depend on the N tiling.
struct TileRef {
    const TcJob *J;
    int p0, n0;
};

__device__ __forceinline__ TileRef tile_ref(const TcJob *jobs, int n_jobs, int tile, int n_tiles_n, int NT)
{
    const int nt = tile % n_tiles_n, mg = tile / n_tiles_n;
    const TcJob *J = jobs + find_job(jobs, n_jobs, mg);
    return TileRef{J, (mg - J->begin) * TC_M, nt * NT};
}

// Persistent: each CTA walks the tiles blockIdx.x, blockIdx.x + gridDim.x, ... with three roles.
//   warp 0 lane 0  producer: per filter row (and channel block) of every tile, one TMA box of the input (a row
//                  segment of 144 cells x 32 channels, which serves up to 17 taps) into a ring of sa_n slots, and per
//                  tap its N-tile slice of the bank (1-D bulk copies) into a ring of sb_n slots; both rings run on
//                  across tile boundaries;
//   warp 1 lane 0  MMA issuer: the tile's taps into one of two TMEM accumulators (tiles alternate), then a commit that
//                  hands the accumulator to the epilogue;
//   warps 2..      epilogue (TC_EPI warps): drain the accumulator with 32x32b loads (warp w reads TMEM lanes
//                  32 (w % 4) .. +31; the TC_EPI / 4 warps of one quadrant split its columns in 16-column chunks)
//                  and store rows of the output maps, then hand the accumulator back; it overlaps the next tile's
//                  MMAs.
// filt: [h*w*cb][CHUNKS][ld][16 bytes] (tap-major, then channel block); NT = N tile width (multiple of 16, <= 256);
// the input has 32*cb channels in CHUNKS*cb planar 16-byte chunks.
// SPLIT: operands come as hi and lo BF16 parts (filt_lo, the job's tmap_lo) and every K step issues three MMAs,
// hi*hi + hi*lo + lo*hi, into the same FP32 accumulator.
// FP8: E4M3 operands, 32 channels = 32 bytes = two 16-byte chunks per tap ([2][cells][16] planar input, bank
// [taps][2][ld][16]); one kind::f8f6f4 MMA (K = 32) per tap; the epilogue multiplies by `scale` (the inverse of the
// product of the two per-tensor scales).
constexpr int TC_EPI = 16;                      // epilogue warps (a multiple of 4)
constexpr int TC_THREADS_P = 64 + 32 * TC_EPI;

template <bool SPLIT, bool FP8>
__global__ void __launch_bounds__(TC_THREADS_P, 1) corr_tc_persistent_kernel(const TcJob *__restrict__ jobs, int n_jobs,
                                                                  int total_tiles, const uint8_t *__restrict__ filt,
                                                                  const uint8_t *__restrict__ filt_lo, int K, int ld,
                                                                  int NT, int n_tiles_n, int h, int w, int cb,
                                                                  uint32_t acc_cols, int sa_n, int sb_n, float scale,
                                                                  int *err)
{
    static_assert(!(SPLIT && FP8), "split operands are BF16");
    extern __shared__ __align__(1024) uint8_t sm[];
    constexpr uint32_t NPART = SPLIT ? 2 : 1;
    constexpr int CHUNKS = FP8 ? 2 : 4;                              // 16-byte K chunks per tap
    constexpr uint32_t A_SEG_BYTES = A_SEG_PLANE * CHUNKS;            // one row segment of one channel block
    const uint32_t b_part_bytes = (uint32_t)NT * 16 * CHUNKS;
    const uint32_t a_stage_bytes = NPART * A_SEG_BYTES, b_stage_bytes = NPART * b_part_bytes;
    uint8_t *a_smem = sm;
    uint8_t *b_smem = sm + sa_n * a_stage_bytes;
    uint64_t *bars = reinterpret_cast<uint64_t *>(b_smem + sb_n * b_stage_bytes);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * sa_n + 2 * sb_n + 4);
    const uint32_t afull0 = smem_u32(bars), aempty0 = smem_u32(bars + sa_n);
    const uint32_t bfull0 = smem_u32(bars + 2 * sa_n), bempty0 = smem_u32(bars + 2 * sa_n + sb_n);
    const uint32_t acc_full0 = smem_u32(bars + 2 * sa_n + 2 * sb_n), acc_empty0 = acc_full0 + 16;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < sa_n; ++s) {
            mbar_init(afull0 + 8 * s, 1);
            mbar_init(aempty0 + 8 * s, 1);
        }
        for (int s = 0; s < sb_n; ++s) {
            mbar_init(bfull0 + 8 * s, 1);
            mbar_init(bempty0 + 8 * s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(acc_full0 + 8 * b, 1);
            mbar_init(acc_empty0 + 8 * b, 32 * TC_EPI);  // every epilogue thread arrives
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(2 * acc_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // producer: per filter row dy and channel block one TMA box of TC_MS cells (the row segment) into the A ring,
        // then each tap's N-tile slice of the bank into the B ring; both rings run on across tiles
        int ga = 0, gb = 0;
        for (int tile = blockIdx.x; tile < total_tiles; tile += gridDim.x) {
            const TileRef T = tile_ref(jobs, n_jobs, tile, n_tiles_n, NT);
            const int W = T.J->W;
            for (int dy = 0; dy < h; ++dy)
                for (int blk = 0; blk < cb; ++blk, ++ga) {
                    const int sa = ga % sa_n;
                    if (ga >= sa_n) mbar_wait(aempty0 + 8 * sa, ((ga / sa_n) - 1) & 1, err);
                    const uint32_t afull = afull0 + 8 * sa;
                    mbar_expect_tx(afull, a_stage_bytes);
                    const uint32_t adst = smem_u32(a_smem + sa * a_stage_bytes);
                    const int cell = T.p0 + dy * W;
                    tma_load_3d(adst, &T.J->tmap, 0, cell, CHUNKS * blk, afull);
                    if (SPLIT) tma_load_3d(adst + A_SEG_BYTES, &T.J->tmap_lo, 0, cell, CHUNKS * blk, afull);
                    for (int dx = 0; dx < w; ++dx, ++gb) {
                        const int sb = gb % sb_n;
                        if (gb >= sb_n) mbar_wait(bempty0 + 8 * sb, ((gb / sb_n) - 1) & 1, err);
                        const uint32_t bfull = bfull0 + 8 * sb;
                        mbar_expect_tx(bfull, b_stage_bytes);
                        const int t = (dy * w + dx) * cb + blk;
                        const uint32_t bdst = smem_u32(b_smem + sb * b_stage_bytes);
                        for (int kc = 0; kc < CHUNKS; ++kc) {
                            const size_t off = (((size_t)t * CHUNKS + kc) * ld + T.n0) * 16;  // bytes
                            bulk_load(bdst + kc * NT * 16, filt + off, (uint32_t)NT * 16, bfull);
                            if (SPLIT)
                                bulk_load(bdst + b_part_bytes + kc * NT * 16, filt_lo + off, (uint32_t)NT * 16,
                                          bfull);
                        }
                    }
                }
        }
        // the last fill of every slot has landed before the CTA can exit (immediate unless a wait gave up)
        for (int k = ga - sa_n < 0 ? 0 : ga - sa_n; k < ga; ++k) mbar_drain(afull0 + 8 * (k % sa_n), (k / sa_n) & 1);
        for (int k = gb - sb_n < 0 ? 0 : gb - sb_n; k < gb; ++k) mbar_drain(bfull0 + 8 * (k % sb_n), (k / sb_n) & 1);
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: tap dx of a segment is its A operand shifted by dx cells (16 bytes per cell in every K chunk);
        // BF16, two K=16 steps per tap (channel chunks {0,1} and {2,3}); FP8, one K=32 step
        const uint32_t idesc = FP8 ? instr_desc_e4m3(TC_M, NT) : instr_desc(TC_M, NT);
        int ga = 0, gb = 0, li = 0;
        for (int tile = blockIdx.x; tile < total_tiles; tile += gridDim.x, ++li) {
            const int b = li & 1;
            if (li >= 2) mbar_wait(acc_empty0 + 8 * b, ((li >> 1) - 1) & 1, err);  // epilogue done with it
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t acc = tmem + (uint32_t)b * acc_cols;
            uint32_t accum = 0;  // the tile's first MMA overwrites the accumulator
            for (int dy = 0; dy < h; ++dy)
                for (int blk = 0; blk < cb; ++blk, ++ga) {
                    const int sa = ga % sa_n;
                    mbar_wait(afull0 + 8 * sa, (ga / sa_n) & 1, err);
                    const uint32_t a_seg = smem_u32(a_smem + sa * a_stage_bytes);
                    for (int dx = 0; dx < w; ++dx, ++gb) {
                        const int sb = gb % sb_n;
                        mbar_wait(bfull0 + 8 * sb, (gb / sb_n) & 1, err);
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const uint32_t a_base = a_seg + (uint32_t)dx * 16;
                        const uint32_t b_base = smem_u32(b_smem + sb * b_stage_bytes);
                        if (FP8) {
                            const uint64_t ad = smem_desc(a_base, A_SEG_PLANE, 128);
                            const uint64_t bd = smem_desc(b_base, (uint32_t)NT * 16, 128);
                            mma_e4m3(acc, ad, bd, idesc, accum);
                            accum = 1;
                        } else {
#pragma unroll
                            for (int ks = 0; ks < 2; ++ks) {
                                const uint64_t ad = smem_desc(a_base + ks * 2 * A_SEG_PLANE, A_SEG_PLANE, 128);
                                const uint64_t bd = smem_desc(b_base + ks * 2 * NT * 16, (uint32_t)NT * 16, 128);
                                mma_bf16(acc, ad, bd, idesc, accum);
                                accum = 1;
                                if (SPLIT) {
                                    const uint64_t ad_lo = smem_desc(a_base + A_SEG_BYTES + ks * 2 * A_SEG_PLANE,
                                                                     A_SEG_PLANE, 128);
                                    const uint64_t bd_lo = smem_desc(b_base + b_part_bytes + ks * 2 * NT * 16,
                                                                     (uint32_t)NT * 16, 128);
                                    mma_bf16(acc, ad, bd_lo, idesc, 1u);
                                    mma_bf16(acc, ad_lo, bd, idesc, 1u);
                                }
                            }
                        }
                        mma_commit(bempty0 + 8 * sb);  // the B slot is free once these MMAs have read it
                    }
                    mma_commit(aempty0 + 8 * sa);  // and the segment once its last tap's MMAs have
                }
            mma_commit(acc_full0 + 8 * b);  // the accumulator is complete once every MMA has finished
        }
    } else if (warp >= 2) {
        // epilogue: TMEM lane m of the accumulator holds position p0 + m; columns are the N tile's filters
        const int q = warp & 3;              // the TMEM lane quadrant this warp may read
        const int cg = (warp - 2) >> 2;      // its share of the columns: chunks cg, cg + TC_EPI/4, ...
        constexpr int NCG = TC_EPI / 4;
        int li = 0;
        for (int tile = blockIdx.x; tile < total_tiles; tile += gridDim.x, ++li) {
            const int b = li & 1;
            mbar_wait(acc_full0 + 8 * b, (li >> 1) & 1, err);
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const TileRef T = tile_ref(jobs, n_jobs, tile, n_tiles_n, NT);
            const int W = T.J->W, Ho = T.J->Ho, Wo = T.J->Wo;
            const int p = T.p0 + q * 32 + lane;
            const int y = p / W, x = p - y * W;
            const bool valid = (y < Ho) && (x < Wo);
            float *out = T.J->out + (size_t)y * Wo + x;
            const size_t plane = (size_t)Ho * Wo;
            for (int c0 = 16 * cg; c0 < NT; c0 += 16 * NCG) {
                uint32_t r[16];
                tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)b * acc_cols + (uint32_t)c0, r);
                if (valid) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int k = T.n0 + c0 + j;
                        if (k < K) out[(size_t)k * plane] = FP8 ? __uint_as_float(r[j]) * scale : __uint_as_float(r[j]);
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(acc_empty0 + 8 * b);
        }
    }
    __syncwarp();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * acc_cols)
                     : "memory");
}

constexpr int TC_THREADS = 128;

// Tile form: one CTA per (M tile, N tile), M tiles numbered across the jobs (a job's begin is its first M tile), so the job
// tables do not depend on the N tiling; filt: [h*w*cb][4][ld][8] BF16 (tap-major, then channel block, ld rows per
// plane); NT = N tile width (multiple of 16, <= 256); the input has 32*cb channels in 4*cb planar chunks.
// SPLIT: operands come as hi and lo BF16 parts (filt_lo, the job's tmap_lo) and every K step issues three MMAs,
// hi*hi + hi*lo + lo*hi, into the same FP32 accumulator.
// FP8: E4M3 operands, 32 channels = 32 bytes = two 16-byte chunks per tap ([2][cells][16] planar input, bank
// [taps][2][ld][16]); one kind::f8f6f4 MMA (K = 32) per tap; the epilogue multiplies by `scale` (the inverse of the
// product of the two per-tensor scales).
template <bool SPLIT, bool FP8>
__global__ void __launch_bounds__(TC_THREADS, 1) corr_tc_tile_kernel(const TcJob *__restrict__ jobs, int n_jobs,
                                                                const uint8_t *__restrict__ filt,
                                                                const uint8_t *__restrict__ filt_lo, int K, int ld,
                                                                int NT, int n_tiles_n, int h, int w, int cb,
                                                                uint32_t tmem_cols, int sa_n, int sb_n, float scale,
                                                                int *err)
{
    static_assert(!(SPLIT && FP8), "split operands are BF16");
    extern __shared__ __align__(1024) uint8_t sm[];
    constexpr uint32_t NPART = SPLIT ? 2 : 1;
    constexpr int CHUNKS = FP8 ? 2 : 4;                              // 16-byte K chunks per tap
    constexpr uint32_t A_SEG_BYTES = A_SEG_PLANE * CHUNKS;            // one row segment of one channel block
    const uint32_t b_part_bytes = (uint32_t)NT * 16 * CHUNKS;
    const uint32_t a_stage_bytes = NPART * A_SEG_BYTES, b_stage_bytes = NPART * b_part_bytes;
    uint8_t *a_smem = sm;
    uint8_t *b_smem = sm + sa_n * a_stage_bytes;
    uint64_t *bars = reinterpret_cast<uint64_t *>(b_smem + sb_n * b_stage_bytes);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * sa_n + 2 * sb_n + 1);
    const uint32_t afull0 = smem_u32(bars), aempty0 = smem_u32(bars + sa_n);
    const uint32_t bfull0 = smem_u32(bars + 2 * sa_n), bempty0 = smem_u32(bars + 2 * sa_n + sb_n);
    const uint32_t done = smem_u32(bars + 2 * sa_n + 2 * sb_n);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nt = blockIdx.x % n_tiles_n, mg = blockIdx.x / n_tiles_n;
    const int ji = find_job(jobs, n_jobs, mg);
    const TcJob *J = jobs + ji;
    const int mt = mg - J->begin;
    const int p0 = mt * TC_M, n0 = nt * NT;
    const int W = J->W, Ho = J->Ho, Wo = J->Wo;

    if (threadIdx.x == 0) {
        for (int s = 0; s < sa_n; ++s) {
            mbar_init(afull0 + 8 * s, 1);
            mbar_init(aempty0 + 8 * s, 1);
        }
        for (int s = 0; s < sb_n; ++s) {
            mbar_init(bfull0 + 8 * s, 1);
            mbar_init(bempty0 + 8 * s, 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // producer: one A row segment (TC_MS cells) per filter row and channel block, and each tap's N-tile slice of
        // the bank
        int ga = 0, gb = 0;
        for (int dy = 0; dy < h; ++dy)
            for (int blk = 0; blk < cb; ++blk, ++ga) {
                const int sa = ga % sa_n;
                if (ga >= sa_n) mbar_wait(aempty0 + 8 * sa, ((ga / sa_n) - 1) & 1, err);
                const uint32_t afull = afull0 + 8 * sa;
                mbar_expect_tx(afull, a_stage_bytes);
                const uint32_t adst = smem_u32(a_smem + sa * a_stage_bytes);
                const int cell = p0 + dy * W;
                tma_load_3d(adst, &J->tmap, 0, cell, CHUNKS * blk, afull);
                if (SPLIT) tma_load_3d(adst + A_SEG_BYTES, &J->tmap_lo, 0, cell, CHUNKS * blk, afull);
                for (int dx = 0; dx < w; ++dx, ++gb) {
                    const int sb = gb % sb_n;
                    if (gb >= sb_n) mbar_wait(bempty0 + 8 * sb, ((gb / sb_n) - 1) & 1, err);
                    const uint32_t bfull = bfull0 + 8 * sb;
                    mbar_expect_tx(bfull, b_stage_bytes);
                    const int t = (dy * w + dx) * cb + blk;
                    const uint32_t bdst = smem_u32(b_smem + sb * b_stage_bytes);
                    for (int kc = 0; kc < CHUNKS; ++kc) {
                        const size_t off = (((size_t)t * CHUNKS + kc) * ld + n0) * 16;  // bytes
                        bulk_load(bdst + kc * NT * 16, filt + off, (uint32_t)NT * 16, bfull);
                        if (SPLIT)
                            bulk_load(bdst + b_part_bytes + kc * NT * 16, filt_lo + off, (uint32_t)NT * 16, bfull);
                    }
                }
            }
        // the last fill of every slot has landed before the CTA can exit (immediate unless a wait gave up)
        for (int k = ga - sa_n < 0 ? 0 : ga - sa_n; k < ga; ++k) mbar_drain(afull0 + 8 * (k % sa_n), (k / sa_n) & 1);
        for (int k = gb - sb_n < 0 ? 0 : gb - sb_n; k < gb; ++k) mbar_drain(bfull0 + 8 * (k % sb_n), (k / sb_n) & 1);
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: tap dx of a segment is its A operand shifted by dx cells; BF16, two K=16 steps per tap (channel
        // chunks {0,1} and {2,3}); FP8, one K=32 step
        const uint32_t idesc = FP8 ? instr_desc_e4m3(TC_M, NT) : instr_desc(TC_M, NT);
        int ga = 0, gb = 0;
        uint32_t accum = 0;  // the first MMA overwrites the accumulator
        for (int dy = 0; dy < h; ++dy)
            for (int blk = 0; blk < cb; ++blk, ++ga) {
                const int sa = ga % sa_n;
                mbar_wait(afull0 + 8 * sa, (ga / sa_n) & 1, err);
                const uint32_t a_seg = smem_u32(a_smem + sa * a_stage_bytes);
                for (int dx = 0; dx < w; ++dx, ++gb) {
                    const int sb = gb % sb_n;
                    mbar_wait(bfull0 + 8 * sb, (gb / sb_n) & 1, err);
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t a_base = a_seg + (uint32_t)dx * 16;
                    const uint32_t b_base = smem_u32(b_smem + sb * b_stage_bytes);
                    if (FP8) {
                        const uint64_t ad = smem_desc(a_base, A_SEG_PLANE, 128);
                        const uint64_t bd = smem_desc(b_base, (uint32_t)NT * 16, 128);
                        mma_e4m3(tmem, ad, bd, idesc, accum);
                        accum = 1;
                    } else {
#pragma unroll
                        for (int ks = 0; ks < 2; ++ks) {
                            const uint64_t ad = smem_desc(a_base + ks * 2 * A_SEG_PLANE, A_SEG_PLANE, 128);
                            const uint64_t bd = smem_desc(b_base + ks * 2 * NT * 16, (uint32_t)NT * 16, 128);
                            mma_bf16(tmem, ad, bd, idesc, accum);
                            accum = 1;
                            if (SPLIT) {
                                const uint64_t ad_lo =
                                    smem_desc(a_base + A_SEG_BYTES + ks * 2 * A_SEG_PLANE, A_SEG_PLANE, 128);
                                const uint64_t bd_lo =
                                    smem_desc(b_base + b_part_bytes + ks * 2 * NT * 16, (uint32_t)NT * 16, 128);
                                mma_bf16(tmem, ad, bd_lo, idesc, 1u);
                                mma_bf16(tmem, ad_lo, bd, idesc, 1u);
                            }
                        }
                    }
                    mma_commit(bempty0 + 8 * sb);
                }
                mma_commit(aempty0 + 8 * sa);
            }
        mma_commit(done);
    }
    __syncwarp();

    // epilogue: TMEM lane m holds position p0 + m; columns are the N tile's filters
    mbar_wait(done, 0, err);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int p = p0 + warp * 32 + lane;
    const int y = p / W, x = p - y * W;
    const bool valid = (y < Ho) && (x < Wo);
    float *out = J->out + (size_t)y * Wo + x;
    const size_t plane = (size_t)Ho * Wo;
    for (int c0 = 0; c0 < NT; c0 += 16) {
        uint32_t r[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
        if (valid) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int k = n0 + c0 + j;
                if (k < K) out[(size_t)k * plane] = FP8 ? __uint_as_float(r[j]) * scale : __uint_as_float(r[j]);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
}

// FP32 NHWC [cells][32] -> BF16 [4][cells][8] for many levels: one thread per (cell, chunk) item
__global__ void to_bf16_planar_kernel(const ConvJob *__restrict__ jobs, int n_jobs, long long total)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    int lo = 0, hi = n_jobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].begin <= i) lo = mid; else hi = mid - 1;
    }
    const ConvJob &J = jobs[lo];
    const long long item = i - J.begin;
    const long long cell = item >> 2;
    const int kc = (int)(item & 3);
    const float4 a = __ldg(reinterpret_cast<const float4 *>(J.src + cell * FD + kc * 8));
    const float4 b = __ldg(reinterpret_cast<const float4 *>(J.src + cell * FD + kc * 8 + 4));
    const float v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    uint32_t wv[4], wl[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const __nv_bfloat16 e0 = __float2bfloat16_rn(v[2 * j]), e1 = __float2bfloat16_rn(v[2 * j + 1]);
        wv[j] = (uint32_t)__bfloat16_as_ushort(e0) | ((uint32_t)__bfloat16_as_ushort(e1) << 16);
        // residuals (exact in FP32) rounded to BF16: the lo part of the split operand
        const __nv_bfloat16 r0 = __float2bfloat16_rn(v[2 * j] - __bfloat162float(e0));
        const __nv_bfloat16 r1 = __float2bfloat16_rn(v[2 * j + 1] - __bfloat162float(e1));
        wl[j] = (uint32_t)__bfloat16_as_ushort(r0) | ((uint32_t)__bfloat16_as_ushort(r1) << 16);
    }
    const size_t o = ((size_t)kc * J.cells + cell) * 8;
    *reinterpret_cast<uint4 *>(J.dst + o) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
    if (J.dst_lo) *reinterpret_cast<uint4 *>(J.dst_lo + o) = make_uint4(wl[0], wl[1], wl[2], wl[3]);
}

// FP32 NHWC [cells][32] -> E4M3 [2][cells][16] (x * scale, rounded to nearest even, saturated at +-448): one
// thread per (cell, 16-channel chunk) item
__global__ void to_fp8_planar_kernel(const ConvJob *__restrict__ jobs, int n_jobs, long long total, float scale)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    int lo = 0, hi = n_jobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].begin <= i) lo = mid; else hi = mid - 1;
    }
    const ConvJob &J = jobs[lo];
    const long long item = i - J.begin;
    const long long cell = item >> 1;
    const int kc = (int)(item & 1);
    const float4 *src = reinterpret_cast<const float4 *>(J.src + cell * FD + kc * 16);
    uint32_t w[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float4 v = __ldg(src + j);
        const uint32_t a = __nv_cvt_float2_to_fp8x2(make_float2(v.x * scale, v.y * scale), __NV_SATFINITE, __NV_E4M3);
        const uint32_t b = __nv_cvt_float2_to_fp8x2(make_float2(v.z * scale, v.w * scale), __NV_SATFINITE, __NV_E4M3);
        w[j] = a | (b << 16);
    }
    uint8_t *dst = reinterpret_cast<uint8_t *>(J.dst) + ((size_t)kc * J.cells + cell) * 16;
    *reinterpret_cast<uint4 *>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
}

}  // namespace

int corr_tc_tile_m() { return TC_M; }

// N tiling. A width cap mx gives the balanced tiling: n = ceil(K / mx) tiles of NT = ceil(K / n) rounded up to 16.
int corr_tc_balanced_nt(int K, int mx)
{
    const int n = (K + mx - 1) / mx;
    const int nt = (K + n - 1) / n;
    return (nt + 15) / 16 * 16;
}

int corr_tc_n_tiles(int K, int NT) { return (K + NT - 1) / NT; }

// Default without tuning: caps of 256 for multi-tap correlations (more MMA work per staged byte) and 128 for a single
// tap (the channel stage, bound by its output writes, gains from more CTAs per SM; TMEM holds 512 columns).
int corr_tc_default_nt(int K, int taps) { return corr_tc_balanced_nt(K, taps > 1 ? 256 : 128); }

// The widths a tuner may choose from: the balanced tilings under caps 256, 128, 64 and 32 (duplicates dropped).
int corr_tc_nt_candidates(int K, int *out)
{
    int n = 0;
    for (int mx : {256, 128, 64, 32}) {
        const int nt = corr_tc_balanced_nt(K, mx);
        bool dup = false;
        for (int i = 0; i < n; ++i) dup |= out[i] == nt;
        if (!dup) out[n++] = nt;
    }
    return n;
}

// Rows a bank of K filters is padded to (zero rows beyond K): enough for every candidate tiling.
int corr_tc_bank_rows(int K)
{
    int c[4];
    const int n = corr_tc_nt_candidates(K, c);
    int rows = (K + 15) / 16 * 16;
    for (int i = 0; i < n; ++i) rows = std::max(rows, corr_tc_n_tiles(K, c[i]) * c[i]);
    return rows;
}

// Shared memory of a dense launch: sa A row segments and sb B slices, their full / empty barriers, four more barriers
// and the TMEM address.
size_t corr_tc_smem_bytes(int NT, bool split, bool fp8, int sa, int sb)
{
    const size_t parts = split ? 2 : 1, tap_bytes = fp8 ? 32 : 64;  // bytes of one row (cell or filter) of one tap
    return parts * tap_bytes * ((size_t)sa * TC_MS + (size_t)sb * NT) + 8 * (2 * (size_t)sa + 2 * (size_t)sb + 4) + 16;
}

// Ring depths within a shared-memory budget: two A segments when one segment serves several taps (one per tap
// otherwise, so both rings advance together), and as many B slices as fit, 2..maxb.
void corr_tc_rings(int NT, bool split, bool fp8, int w, size_t budget, int maxb, int *sa, int *sb)
{
    const size_t seg = corr_tc_smem_bytes(NT, split, fp8, 1, 0) - corr_tc_smem_bytes(NT, split, fp8, 0, 0);
    const size_t slice = corr_tc_smem_bytes(NT, split, fp8, 0, 1) - corr_tc_smem_bytes(NT, split, fp8, 0, 0);
    if (w > 1) {
        *sa = 2;
        const size_t base = corr_tc_smem_bytes(NT, split, fp8, 2, 0);
        *sb = budget > base ? (int)std::min<size_t>((size_t)maxb, (budget - base) / slice) : 2;
    } else {
        *sb = (int)std::min<size_t>((size_t)maxb, budget / (seg + slice + 32));
        *sa = *sb;
    }
    *sb = std::max(2, *sb);
    *sa = std::max(2, *sa);
}

namespace {
int sm_count()
{
    static int n[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    if (!n[dev]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 1;
        n[dev] = v;
    }
    return n[dev];
}
}  // namespace

cudaError_t launch_corr_tc(const TcJob *d_jobs, int n_jobs, int m_tiles, const void *filt_tc, const void *filt_tc_lo,
                           int K, int ld, int NT, int h, int w, int cb, int *d_err, cudaStream_t s, bool fp8,
                           float scale, bool persistent)
{
    if (m_tiles <= 0 || K <= 0) return cudaSuccess;
    if (cb < 1) return cudaErrorInvalidValue;
    const bool split = filt_tc_lo != nullptr;
    if (split && fp8) return cudaErrorInvalidValue;
    const int n_tiles_n = corr_tc_n_tiles(K, NT);
    // every N tile's bulk copies stay inside the bank's ld rows
    if (NT % 16 != 0 || NT < 16 || NT > 256 || n_tiles_n * NT > ld) return cudaErrorInvalidValue;
    if (w > TC_DXS) return cudaErrorInvalidValue;  // one row segment serves every tap of a filter row
    if ((long long)m_tiles * n_tiles_n > 0x7fffffffll) return cudaErrorInvalidValue;
    const int total_tiles = m_tiles * n_tiles_n;
    const uint8_t *fb = static_cast<const uint8_t *>(filt_tc), *fl = static_cast<const uint8_t *>(filt_tc_lo);
    if (!persistent) {
        // tile form: one CTA per tile, at most 512 / cols CTAs per SM (TMEM), enforced through the shared memory
        // request
        const int taps = h * w * cb;
        uint32_t cols = 32;
        while (cols < (uint32_t)NT) cols <<= 1;
        const int max_ctas = 512 / (int)cols;
        // rings within the share of shared memory of one of the CTAs that fit in TMEM (at least 48 KB)
        const size_t budget = std::max<size_t>((size_t)kMaxDynamicSmem / (size_t)max_ctas - 1024, 49152);
        int sa = 2, sb = 2;
        corr_tc_rings(NT, split, fp8, w, budget, std::max(2, std::min(8, taps)), &sa, &sb);
        size_t smem = corr_tc_smem_bytes(NT, split, fp8, sa, sb);
        const size_t floor_bytes = 233472 / (size_t)(max_ctas + 1);
        if (smem < floor_bytes) smem = floor_bytes;
        if (smem > (size_t)kMaxDynamicSmem) return cudaErrorInvalidValue;
        const void *fn = split ? reinterpret_cast<const void *>(corr_tc_tile_kernel<true, false>)
                         : fp8 ? reinterpret_cast<const void *>(corr_tc_tile_kernel<false, true>)
                               : reinterpret_cast<const void *>(corr_tc_tile_kernel<false, false>);
        cudaError_t e = allow_max_dynamic_smem(fn, split ? 2 : fp8 ? 3 : 0);
        if (e != cudaSuccess) return e;
        note_launches(1);
        if (split)
            corr_tc_tile_kernel<true, false><<<total_tiles, TC_THREADS, smem, s>>>(
                d_jobs, n_jobs, fb, fl, K, ld, NT, n_tiles_n, h, w, cb, cols, sa, sb, 1.f, d_err);
        else if (fp8)
            corr_tc_tile_kernel<false, true><<<total_tiles, TC_THREADS, smem, s>>>(
                d_jobs, n_jobs, fb, nullptr, K, ld, NT, n_tiles_n, h, w, cb, cols, sa, sb, scale, d_err);
        else
            corr_tc_tile_kernel<false, false><<<total_tiles, TC_THREADS, smem, s>>>(
                d_jobs, n_jobs, fb, nullptr, K, ld, NT, n_tiles_n, h, w, cb, cols, sa, sb, 1.f, d_err);
        return cudaGetLastError();
    }
    uint32_t acc_cols = 32;
    while (acc_cols < (uint32_t)NT) acc_cols <<= 1;
    // two accumulators per CTA; at most 512 / (2 acc_cols) CTAs per SM fit in TMEM, enforced through the shared
    // memory request so that no CTA waits in tcgen05.alloc
    const int max_ctas = 512 / (2 * (int)acc_cols);
    // ring depths: as many slots as the shared memory of one of those CTAs holds (B: 2..12); the rings run on across
    // tiles, so even a single-tap contraction keeps several tiles' operands in flight
    const size_t per_cta = (size_t)kMaxDynamicSmem / (size_t)max_ctas - 1024;
    int sa = 2, sb = 2;
    corr_tc_rings(NT, split, fp8, w, per_cta, 12, &sa, &sb);
    size_t smem = corr_tc_smem_bytes(NT, split, fp8, sa, sb);
    const size_t floor_bytes = 233472 / (size_t)(max_ctas + 1);
    if (smem < floor_bytes) smem = floor_bytes;
    if (smem > (size_t)kMaxDynamicSmem) return cudaErrorInvalidValue;
    const void *fn = split ? reinterpret_cast<const void *>(corr_tc_persistent_kernel<true, false>)
                     : fp8 ? reinterpret_cast<const void *>(corr_tc_persistent_kernel<false, true>)
                           : reinterpret_cast<const void *>(corr_tc_persistent_kernel<false, false>);
    cudaError_t e = allow_max_dynamic_smem(fn, split ? 5 : fp8 ? 6 : 4);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, TC_THREADS_P, smem);
    if (e != cudaSuccess) return e;
    per_sm = std::max(1, std::min(per_sm, max_ctas));
    const int grid = std::min(total_tiles, sm_count() * per_sm);
    note_launches(1);
    if (split)
        corr_tc_persistent_kernel<true, false><<<grid, TC_THREADS_P, smem, s>>>(d_jobs, n_jobs, total_tiles, fb, fl, K, ld, NT,
                                                                     n_tiles_n, h, w, cb, acc_cols, sa, sb, 1.f, d_err);
    else if (fp8)
        corr_tc_persistent_kernel<false, true><<<grid, TC_THREADS_P, smem, s>>>(d_jobs, n_jobs, total_tiles, fb, nullptr, K, ld,
                                                                     NT, n_tiles_n, h, w, cb, acc_cols, sa, sb, scale,
                                                                     d_err);
    else
        corr_tc_persistent_kernel<false, false><<<grid, TC_THREADS_P, smem, s>>>(d_jobs, n_jobs, total_tiles, fb, nullptr, K, ld,
                                                                      NT, n_tiles_n, h, w, cb, acc_cols, sa, sb, 1.f,
                                                                      d_err);
    return cudaGetLastError();
}

cudaError_t launch_to_bf16_planar(const ConvJob *d_jobs, int n_jobs, long long total, cudaStream_t s)
{
    if (total <= 0 || n_jobs <= 0) return cudaSuccess;
    note_launches(1);
    to_bf16_planar_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(d_jobs, n_jobs, total);
    return cudaGetLastError();
}

cudaError_t launch_to_fp8_planar(const ConvJob *d_jobs, int n_jobs, long long total, float scale, cudaStream_t s)
{
    if (total <= 0 || n_jobs <= 0) return cudaSuccess;
    note_launches(1);
    to_fp8_planar_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(d_jobs, n_jobs, total, scale);
    return cudaGetLastError();
}


// Tensor map over one BF16 planar array: dims {8 channels, cells, chunks}, box {8, 144, 4}, zero fill outside.
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

namespace {

// dims {elems per 16-byte chunk, cells, chunks}, box {elems, 144, the chunks of one tap (32 channels)}, zero fill
// outside; strides in bytes
EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !p)
            return nullptr;
        fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

bool encode_tmap(CUtensorMap *map, CUtensorMapDataType type, int elems, void *base, long long cells, int chunks)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint32_t tap_chunks = (cuuint32_t)(FD / elems);
    if (chunks < (int)tap_chunks || chunks % tap_chunks) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)elems, (cuuint64_t)cells, (cuuint64_t)chunks};
    const cuuint64_t strides[2] = {16, (cuuint64_t)cells * 16};
    const cuuint32_t box[3] = {(cuuint32_t)elems, (cuuint32_t)TC_MS, tap_chunks};
    const cuuint32_t estr[3] = {1, 1, 1};
    return fn(map, type, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool encode_level_tmap(CUtensorMap *map, const uint16_t *planar, long long cells, int chunks)
{
    return encode_tmap(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 8, const_cast<uint16_t *>(planar), cells, chunks);
}

bool encode_level_tmap_tiles(CUtensorMap *map, const uint16_t *planar, int H, int W, int box_w, int box_h)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn || H <= 0 || W <= 0) return false;
    const cuuint64_t dims[4] = {8, (cuuint64_t)W, (cuuint64_t)H, 4};
    const cuuint64_t strides[3] = {16, (cuuint64_t)W * 16, (cuuint64_t)H * W * 16};
    const cuuint32_t box[4] = {8, (cuuint32_t)box_w, (cuuint32_t)box_h, 4};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<uint16_t *>(planar), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool encode_level_tmap_fp8(CUtensorMap *map, const uint8_t *planar, long long cells)
{
    return encode_tmap(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 16, const_cast<uint8_t *>(planar), cells, 2);
}

}  // namespace tdpm
