// Step 1, decomposed form, per-filter mode, fused on the tensor cores (Sec. 4): the channel stage
//   Z_r[y][x] = sum_c c_r[c] phi[y][x][c]
// and the separable passes with the recombination
//   S_k[y][x] = sum_{r of k} lambda_r sum_dx b_r[dx] sum_dy a_r[dy] Z_r[y+dy][x+dx]
// in one kernel, so that the rank-1 maps Z_r never leave the SM.
//
// A CTA takes one spatial tile of one level (its record: job, origin, valid output rows) and one filter group (consecutive filters whose terms, at most nmax of
// them, form one MMA of width N). The tile is 32 columns x TYZ = 4*MT rows of Z (32 - (w-1) output columns,
// TY = TYZ - h + 1 output rows). Its features arrive as MT TMA boxes {8 ch, 32 columns, 4 rows, 4 chunks} of the
// level's BF16 planar copy [4][H][W][8], each of which lands in shared memory as a 128-row K-major A operand
// (row m = 32 * row + column). One thread issues the copies and then, per M tile, the MMAs Z = phi C_group into
// TMEM (columns t * nmax ...); the eight warps move Z from TMEM to shared memory (warp w reads lane quadrant w % 4,
// i.e. row 4t + w % 4 of every M tile), over the feature tiles the MMAs no longer need, release TMEM, and run the
// separable passes from shared memory: a warp owns one filter and a block of output rows, lane l column x0 + l; the
// y pass slides an h-deep window down the column, the x pass takes T_r at columns x .. x+w-1 from lanes l .. l+w-1
// by shuffles, and lambda_r times the result accumulates over the filter's terms. The MMA sequence per M tile is
// that of the channel-stage kernel (per K step hi*hi, then hi*lo, lo*hi for split operands) and the multiply-add
// order of the passes is that of the unfused separable kernel, so both forms give identical maps.
// Rows and columns beyond the level are zero-filled by the TMA; they reach only outputs beyond Ho x Wo, which are not
// written. Every mbarrier wait is bounded (the context's error flag is raised on expiry) and the CTA lets its own
// copies and MMAs finish before it releases TMEM and exits.
#include <algorithm>

#include "internal.h"
#include "tc_ptx.h"

namespace tdpm {
namespace {

constexpr int ZS_WARPS = 8, ZS_THREADS = 32 * ZS_WARPS;
constexpr uint32_t ZS_A_TILE = 128 * 64;  // one M tile of one operand part: 4 chunks x 128 rows x 16 bytes

template <int HH>
struct ZsShape {
    static constexpr int MT = HH <= 7 ? 4 : 6;  // M tiles (4 Z rows each)
    static constexpr int TYZ = 4 * MT;          // Z rows of a tile
    static constexpr int TY = TYZ - HH + 1;     // output rows of a tile
};

__host__ __device__ constexpr uint32_t zs_union_bytes(int mt, int npart, int nmax)
{
    return (uint32_t)(mt * npart) * ZS_A_TILE > (uint32_t)nmax * 4 * mt * 32 * 4
               ? (uint32_t)(mt * npart) * ZS_A_TILE
               : (uint32_t)nmax * 4 * mt * 32 * 4;
}

// Per-term factors in shared memory: a_r[0..h), b_r[0..w), lambda_r, padded to a multiple of 4 floats (float4 loads).
template <int HH, int WW>
struct ZsFactors {
    static constexpr int STRIDE = (HH + WW + 1 + 3) & ~3;
};

// A filter group's packed record: factors [nmax][STRIDE] floats, then the rank offsets of its filters minus t0
// (nmax + 2 ints), rounded up to 16 bytes (one bulk copy).
template <int HH, int WW>
__host__ __device__ constexpr uint32_t zs_record_bytes(int nmax)
{
    return ((uint32_t)nmax * ZsFactors<HH, WW>::STRIDE * 4 + (uint32_t)(nmax + 2) * 4 + 15) & ~15u;
}

// One task of the separable passes: filter terms [tb, te) of the group, output rows i0 .. i0+RB-1 of the tile (ni of
// them valid), lane = column. Rows past the tile's valid ones are computed and not stored, so the unrolled row loop
// has no branch and the rows' multiply-add chains interleave; their Z reads run at most two rows past the term's
// TYZ rows, which stays inside the CTA's shared memory (the next term, or the bank staging that follows Z).
template <int HH, int WW, int TYZ, int RB>
__device__ __forceinline__ void zs_task(const float *Z, const float *fs, int tb, int te, int i0, int ni, int lane,
                                        float *o, int Wo, bool store)
{
    constexpr int FS = ZsFactors<HH, WW>::STRIDE;
    float acc[RB];
#pragma unroll
    for (int i = 0; i < RB; ++i) acc[i] = 0.f;
    for (int tr = tb; tr < te; ++tr) {
        float f[FS];
#pragma unroll
        for (int i = 0; i < FS; i += 4) {
            const float4 v = *reinterpret_cast<const float4 *>(fs + tr * FS + i);
            f[i] = v.x; f[i + 1] = v.y; f[i + 2] = v.z; f[i + 3] = v.w;
        }
        const float *a = f, *bb = f + HH;
        const float l = f[HH + WW];
        const float *z = Z + (tr * TYZ + i0) * 32 + lane;
        float win[HH];
#pragma unroll
        for (int i = 0; i < HH - 1; ++i) win[i] = z[i * 32];
#pragma unroll
        for (int i = 0; i < RB; ++i) {
            win[(i + HH - 1) % HH] = z[(i + HH - 1) * 32];
            float tv = 0.f;
#pragma unroll
            for (int dy = 0; dy < HH; ++dy) tv = fmaf(a[dy], win[(i + dy) % HH], tv);
            float u = 0.f;
#pragma unroll
            for (int dx = 0; dx < WW; ++dx) u = fmaf(bb[dx], dx ? __shfl_down_sync(0xffffffffu, tv, dx) : tv, u);
            acc[i] = fmaf(l, u, acc[i]);
        }
    }
    if (store) {
#pragma unroll
        for (int i = 0; i < RB; ++i)
            if (i < ni) o[(size_t)i * Wo] = acc[i];
    }
}

template <int HH, int WW, bool SPLIT>
__global__ void __launch_bounds__(ZS_THREADS, 3)
    zsep_tc_kernel(const ZsJob *__restrict__ jobs, const ZsTile *__restrict__ tiles, const ZsGroup *__restrict__ fgs,
                   int n_fg, const uint8_t *__restrict__ cbank, const uint8_t *__restrict__ cbank_lo, int ld,
                   const uint8_t *__restrict__ frec, int nmax, uint32_t tmem_cols, int *err)
{
    using S = ZsShape<HH>;
    constexpr int MT = S::MT, TYZ = S::TYZ, TY = S::TY;
    constexpr int SW = 32 - (WW - 1);  // output columns of a tile
    constexpr int RB2 = (TY + 1) / 2, RB4 = (TY + 3) / 4;
    constexpr uint32_t NPART = SPLIT ? 2 : 1;
    extern __shared__ __align__(1024) uint8_t sm[];
    uint8_t *uni = sm;                                                  // feature tiles, then Z [nmax][TYZ][32]
    uint8_t *bsm = sm + zs_union_bytes(MT, NPART, nmax);                // [NPART][4][nmax][16 bytes]
    constexpr int FS = ZsFactors<HH, WW>::STRIDE;
    const uint32_t rec = zs_record_bytes<HH, WW>(nmax);
    float *fs = reinterpret_cast<float *>(bsm + NPART * 4 * nmax * 16);  // the group's record: factors [nmax][FS],
    int *ro = reinterpret_cast<int *>(fs + nmax * FS);                  // then the rank offsets of its filters - t0
    uint64_t *bars = reinterpret_cast<uint64_t *>(bsm + NPART * 4 * nmax * 16 + rec);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2);
    const uint32_t full = smem_u32(bars), done = smem_u32(bars + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int fgi = blockIdx.x % n_fg, tile = blockIdx.x / n_fg;  // the filter groups of a tile are neighbours
    const ZsTile TL = tiles[tile];
    const ZsGroup G = fgs[fgi];
    const ZsJob *J = jobs + TL.job;
    const int N = (G.n + 15) & ~15;

    if (warp == 0) {
        if (lane == 0) {
            // the copies start before the TMEM allocation and the block barrier
            mbar_init(full, 1);
            mbar_init(done, 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            mbar_expect_tx(full, MT * NPART * ZS_A_TILE + NPART * 4 * (uint32_t)N * 16 + rec);
#pragma unroll
            for (int t = 0; t < MT; ++t) {
                const uint32_t dst = smem_u32(uni + t * NPART * ZS_A_TILE);
                tma_load_4d(dst, &J->tmap, 0, TL.x0, TL.y0 + 4 * t, 0, full);
                if (SPLIT) tma_load_4d(dst + ZS_A_TILE, &J->tmap_lo, 0, TL.x0, TL.y0 + 4 * t, 0, full);
            }
            bulk_load(smem_u32(fs), frec + (size_t)fgi * rec, rec, full);
            const uint32_t bdst = smem_u32(bsm);
#pragma unroll
            for (int kc = 0; kc < 4; ++kc) {
                const size_t off = ((size_t)kc * ld + G.t0) * 16;
                bulk_load(bdst + kc * N * 16, cbank + off, (uint32_t)N * 16, full);
                if (SPLIT) bulk_load(bdst + 4 * N * 16 + kc * N * 16, cbank_lo + off, (uint32_t)N * 16, full);
            }
        }
        __syncwarp();
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    if (threadIdx.x == 0) {
        mbar_wait(full, 0, err);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t idesc = instr_desc(128, N);
        const uint32_t bdst = smem_u32(bsm);
#pragma unroll
        for (int t = 0; t < MT; ++t) {
            const uint32_t acc = tmem + (uint32_t)(t * nmax);
            const uint32_t a_base = smem_u32(uni + t * NPART * ZS_A_TILE);
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
                const uint64_t ad = smem_desc(a_base + ks * 2 * 2048, 2048, 128);
                const uint64_t bd = smem_desc(bdst + ks * 2 * N * 16, (uint32_t)N * 16, 128);
                mma_bf16(acc, ad, bd, idesc, ks != 0);
                if (SPLIT) {
                    const uint64_t ad_lo = smem_desc(a_base + ZS_A_TILE + ks * 2 * 2048, 2048, 128);
                    const uint64_t bd_lo = smem_desc(bdst + 4 * N * 16 + ks * 2 * N * 16, (uint32_t)N * 16, 128);
                    mma_bf16(acc, ad, bd_lo, idesc, 1u);
                    mma_bf16(acc, ad_lo, bd, idesc, 1u);
                }
            }
        }
        mma_commit(done);
    }
    mbar_wait(full, 0, err);  // the factor record (complete before the MMAs were issued)
    mbar_wait(done, 0, err);
    __syncwarp();  // warp 0 reconverges (lane 0 issued the MMAs) before the warp-wide TMEM loads
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    // TMEM -> shared memory: warp w reads lane quadrant q = w % 4 (Z row 4t + q of M tile t, column = lane) and half of
    // the columns (terms), two 16-column loads per wait
    float *Z = reinterpret_cast<float *>(uni);
    {
        const int q = warp & 3, cw = nmax >> 1, cb = (warp >> 2) * cw;
        const uint32_t tq = tmem + ((uint32_t)(q * 32) << 16);
        for (int c0 = cb; c0 < cb + cw && c0 < G.n; c0 += 16) {
#pragma unroll 1
            for (int t = 0; t < MT; t += 2) {
                uint32_t r[32];
                tmem_ld16x2(tq + (uint32_t)(t * nmax + c0), tq + (uint32_t)((t + 1) * nmax + c0), r);
                float *zr = Z + (c0 * TYZ + 4 * t + q) * 32 + lane;
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    zr[j * TYZ * 32] = __uint_as_float(r[j]);
                    zr[j * TYZ * 32 + 4 * 32] = __uint_as_float(r[16 + j]);
                }
            }
        }
    }
    if (threadIdx.x == 0) {
        // only reached with copies or MMAs in flight when a wait above gave up
        mbar_drain(full, 0);
        mbar_drain(done, 0);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");

    // separable passes: tasks (filter, block of RB output rows) over the warps; two row blocks per filter when the
    // group has four or more filters, four otherwise
    const int nf = G.k1 - G.k0;
    const int Ho = J->Ho, Wo = J->Wo;
    const int x = TL.x0 + lane;
    const bool col_ok = lane < SW && x < Wo;
    float *out0 = J->out + (size_t)TL.y0 * Wo + x;
    if (nf >= 4) {
        for (int task = warp; task < 2 * nf; task += ZS_WARPS) {
            const int f = task >> 1, i0 = (task & 1) * RB2;
            if (i0 >= TL.rows) continue;  // warp-uniform
            zs_task<HH, WW, TYZ, RB2>(Z, fs, ro[f], ro[f + 1], i0, min(RB2, TL.rows - i0), lane,
                                      out0 + ((size_t)(G.k0 + f) * Ho + i0) * Wo, Wo, col_ok);
        }
    } else {
        for (int task = warp; task < 4 * nf; task += ZS_WARPS) {
            const int f = task >> 2, i0 = (task & 3) * RB4;
            if (i0 >= TL.rows) continue;
            zs_task<HH, WW, TYZ, RB4>(Z, fs, ro[f], ro[f + 1], i0, min(RB4, TL.rows - i0), lane,
                                      out0 + ((size_t)(G.k0 + f) * Ho + i0) * Wo, Wo, col_ok);
        }
    }
}

// Persistent form: one CTA per SM walks the items (tile, filter group) blockIdx.x, blockIdx.x + gridDim.x, ...
// with a producer warp running ahead of sixteen compute warps.
//   producer (warp 16): per item, once the MMAs of the item `stages` back have read its feature / bank stage, the
//     TMA boxes and bank rows into that stage; once the compute warps are done with the item two back, the group's
//     packed factor record (one bulk copy) and the tile record into the buffers of the item's parity; then lane 0
//     issues the item's MMAs into the TMEM accumulator of its parity and commits. The next item's tile and group
//     records are loaded one item early.
//   compute (warps 0-15): per item, wait for its factors and MMAs, drain the accumulator into the Z buffer of the
//     item's parity (warp w: lane quadrant w % 4, M tile w / 4), a named barrier, the separable passes (tasks: filter
//     x row block), then free the item's accumulator and factor buffer. With two Z buffers that is the only barrier
//     per item; with one, a second barrier guards Z before the next drain.
// Every wait is bounded; the results are those of the tile form.
constexpr int ZP_CWARPS = 16, ZP_THREADS = 32 * (ZP_CWARPS + 1);

struct ZsMeta {          // per-item tile record staged by the producer
    float *out;          // output of the group's first filter at the tile's origin
    int plane, Wo, x0, rows, nf, n;
};

template <int HH, int WW, bool SPLIT>
__global__ void __launch_bounds__(ZP_THREADS, 1)
    zsep_tc_persistent_kernel(const ZsJob *__restrict__ jobs, const ZsTile *__restrict__ tiles,
                              const ZsGroup *__restrict__ fgs, int n_fg, int n_items,
                              const uint8_t *__restrict__ cbank, const uint8_t *__restrict__ cbank_lo, int ld,
                              const uint8_t *__restrict__ frec, int nmax, int stages, int zbufs, uint32_t tmem_cols,
                              int *err)
{
    using S = ZsShape<HH>;
    constexpr int MT = S::MT, TYZ = S::TYZ, TY = S::TY;
    constexpr int SW = 32 - (WW - 1);
    constexpr int RB4 = (TY + 3) / 4, RB8 = (TY + 7) / 8;
    constexpr uint32_t NPART = SPLIT ? 2 : 1;
    constexpr int FS = ZsFactors<HH, WW>::STRIDE;
    const uint32_t rec = zs_record_bytes<HH, WW>(nmax);
    const uint32_t phi_bytes = MT * NPART * ZS_A_TILE, b_bytes = NPART * 4 * (uint32_t)nmax * 16;
    const uint32_t stage_bytes = phi_bytes + b_bytes, z_bytes = (uint32_t)nmax * TYZ * 32 * 4;
    extern __shared__ __align__(1024) uint8_t sm[];
    uint8_t *stage0 = sm;                                               // [stages][phi | bank rows]
    float *Z0 = reinterpret_cast<float *>(sm + stages * stage_bytes);   // [zbufs][nmax][TYZ][32]
    uint8_t *fr0 = sm + stages * stage_bytes + zbufs * z_bytes;         // [2][record]: factors [nmax][FS], rank offsets
    ZsMeta *meta = reinterpret_cast<ZsMeta *>(fr0 + 2 * rec);           // [2]
    uint64_t *bars = reinterpret_cast<uint64_t *>(meta + 2);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 8);
    const uint32_t full0 = smem_u32(bars);                              // [stages <= 2]
    const uint32_t done0 = smem_u32(bars + 2), ffull0 = smem_u32(bars + 4), free0 = smem_u32(bars + 6);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t acc_cols = (uint32_t)(MT * nmax);

    if (threadIdx.x == 0) {
        for (int b = 0; b < 2; ++b) {
            mbar_init(full0 + 8 * b, 1);
            mbar_init(done0 + 8 * b, 1);
            mbar_init(ffull0 + 8 * b, 1);
            mbar_init(free0 + 8 * b, 32 * ZP_CWARPS);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == ZP_CWARPS) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == ZP_CWARPS) {
        // ------------------------------------------------------------------------------------------- producer
        if (lane == 0) {
            int item = blockIdx.x;
            ZsTile TL{};
            ZsGroup G{};
            if (item < n_items) {
                TL = tiles[item / n_fg];
                G = fgs[item % n_fg];
            }
            int k = 0;
            for (; item < n_items; item += gridDim.x, ++k) {
                const int b = k & 1, st = stages == 2 ? b : 0;
                const ZsJob *J = jobs + TL.job;
                const int N = (G.n + 15) & ~15;
                // the stage is free once the MMAs of the item `stages` back have completed
                if (k >= stages) mbar_wait(done0 + 8 * ((k - stages) & 1), ((k - stages) >> 1) & 1, err);
                const uint32_t full = full0 + 8 * st;
                const uint32_t sdst = smem_u32(stage0 + st * stage_bytes), bdst = sdst + phi_bytes;
                mbar_expect_tx(full, phi_bytes + NPART * 4 * (uint32_t)N * 16);
#pragma unroll
                for (int t = 0; t < MT; ++t) {
                    const uint32_t dst = sdst + t * NPART * ZS_A_TILE;
                    tma_load_4d(dst, &J->tmap, 0, TL.x0, TL.y0 + 4 * t, 0, full);
                    if (SPLIT) tma_load_4d(dst + ZS_A_TILE, &J->tmap_lo, 0, TL.x0, TL.y0 + 4 * t, 0, full);
                }
#pragma unroll
                for (int kc = 0; kc < 4; ++kc) {
                    const size_t off = ((size_t)kc * ld + G.t0) * 16;
                    bulk_load(bdst + kc * N * 16, cbank + off, (uint32_t)N * 16, full);
                    if (SPLIT) bulk_load(bdst + 4 * N * 16 + kc * N * 16, cbank_lo + off, (uint32_t)N * 16, full);
                }
                // factor record and tile record of parity b: free once the compute warps finished item k-2
                if (k >= 2) mbar_wait(free0 + 8 * b, ((k - 2) >> 1) & 1, err);
                const int Wo = J->Wo, plane = J->Ho * Wo;
                meta[b] = ZsMeta{J->out + (size_t)G.k0 * plane + (size_t)TL.y0 * Wo + TL.x0, plane, Wo, TL.x0, TL.rows,
                                 G.k1 - G.k0, G.n};
                const uint32_t ff = ffull0 + 8 * b;
                mbar_expect_tx(ff, rec);  // also this thread's arrival, after its tile record store
                bulk_load(smem_u32(fr0 + b * rec), frec + (size_t)(item % n_fg) * rec, rec, ff);
                // the next item's records, while this item's copies land
                const int nxt = item + gridDim.x;
                if (nxt < n_items) {
                    TL = tiles[nxt / n_fg];
                    G = fgs[nxt % n_fg];
                }
                mbar_wait(full, (k / stages) & 1, err);
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t idesc = instr_desc(128, N);
#pragma unroll
                for (int t = 0; t < MT; ++t) {
                    const uint32_t acc = tmem + (uint32_t)b * acc_cols + (uint32_t)(t * nmax);
                    const uint32_t a_base = sdst + t * NPART * ZS_A_TILE;
#pragma unroll
                    for (int ks = 0; ks < 2; ++ks) {
                        const uint64_t ad = smem_desc(a_base + ks * 2 * 2048, 2048, 128);
                        const uint64_t bd = smem_desc(bdst + ks * 2 * N * 16, (uint32_t)N * 16, 128);
                        mma_bf16(acc, ad, bd, idesc, ks != 0);
                        if (SPLIT) {
                            const uint64_t ad_lo = smem_desc(a_base + ZS_A_TILE + ks * 2 * 2048, 2048, 128);
                            const uint64_t bd_lo =
                                smem_desc(bdst + 4 * N * 16 + ks * 2 * N * 16, (uint32_t)N * 16, 128);
                            mma_bf16(acc, ad, bd_lo, idesc, 1u);
                            mma_bf16(acc, ad_lo, bd, idesc, 1u);
                        }
                    }
                }
                mma_commit(done0 + 8 * b);
            }
            // only waits when a bounded wait gave up with copies or MMAs in flight: the last phase of every barrier
            // (a barrier's earlier phases are complete once a later one is)
            for (int j = k - 2 < 0 ? 0 : k - 2; j < k; ++j) {
                if (stages == 2 || j == k - 1) mbar_drain(full0 + 8 * (stages == 2 ? (j & 1) : 0), (j / stages) & 1);
                mbar_drain(ffull0 + 8 * (j & 1), (j >> 1) & 1);
                mbar_drain(done0 + 8 * (j & 1), (j >> 1) & 1);
            }
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------------------------------------- compute
        const int q = warp & 3;
        int k = 0;
        for (int item = blockIdx.x; item < n_items; item += gridDim.x, ++k) {
            const int b = k & 1;
            float *Z = Z0 + (zbufs == 2 ? b : 0) * (z_bytes / 4);
            mbar_wait(ffull0 + 8 * b, (k >> 1) & 1, err);
            const ZsMeta M = meta[b];
            mbar_wait(done0 + 8 * b, (k >> 1) & 1, err);
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (zbufs == 1 && k > 0) asm volatile("bar.sync 1, %0;" ::"r"(32 * ZP_CWARPS) : "memory");  // Z read
            const uint32_t tq = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)b * acc_cols;
            for (int t = warp >> 2; t < MT; t += 4) {
                for (int c0 = 0; c0 < M.n; c0 += 32) {
                    uint32_t r[32];
                    tmem_ld16x2(tq + (uint32_t)(t * nmax + c0), tq + (uint32_t)(t * nmax + c0 + 16), r);
                    float *zr = Z + (c0 * TYZ + 4 * t + q) * 32 + lane;
#pragma unroll
                    for (int j = 0; j < 32; ++j) zr[j * TYZ * 32] = __uint_as_float(r[j]);
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            asm volatile("bar.sync 1, %0;" ::"r"(32 * ZP_CWARPS) : "memory");  // Z complete
            const float *fs = reinterpret_cast<const float *>(fr0 + b * rec);
            const int *ro = reinterpret_cast<const int *>(fs + nmax * FS);
            const bool col_ok = lane < SW && M.x0 + lane < M.Wo;
            float *out0 = M.out + lane;
            if (M.nf >= 4) {
                for (int task = warp; task < 4 * M.nf; task += ZP_CWARPS) {
                    const int f = task >> 2, i0 = (task & 3) * RB4;
                    if (i0 >= M.rows) continue;  // warp-uniform
                    zs_task<HH, WW, TYZ, RB4>(Z, fs, ro[f], ro[f + 1], i0, min(RB4, M.rows - i0), lane,
                                              out0 + (size_t)f * M.plane + (size_t)i0 * M.Wo, M.Wo, col_ok);
                }
            } else {
                for (int task = warp; task < 8 * M.nf; task += ZP_CWARPS) {
                    const int f = task >> 3, i0 = (task & 7) * RB8;
                    if (i0 >= M.rows) continue;
                    zs_task<HH, WW, TYZ, RB8>(Z, fs, ro[f], ro[f + 1], i0, min(RB8, M.rows - i0), lane,
                                              out0 + (size_t)f * M.plane + (size_t)i0 * M.Wo, M.Wo, col_ok);
                }
            }
            mbar_arrive(free0 + 8 * b);  // this thread is done with the item's accumulator, factors and tile record
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == ZP_CWARPS)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
}

template <int HH, int WW>
size_t zs_persistent_bytes(bool split, int nmax, int stages, int zbufs)
{
    const int mt = ZsShape<HH>::MT, npart = split ? 2 : 1;
    return (size_t)stages * ((size_t)mt * npart * ZS_A_TILE + (size_t)npart * 4 * nmax * 16) +
           (size_t)zbufs * nmax * 4 * mt * 32 * 4 + 2 * (size_t)zs_record_bytes<HH, WW>(nmax) + 2 * sizeof(ZsMeta) +
           8 * 8 + 16;
}

size_t zsep_persistent_smem_bytes(int h, int w, bool split, int nmax, int stages, int zbufs)
{
    if (h == 6) return zs_persistent_bytes<6, 6>(split, nmax, stages, zbufs);
    if (h == 5) return zs_persistent_bytes<5, 11>(split, nmax, stages, zbufs);
    if (h == 7) return zs_persistent_bytes<7, 7>(split, nmax, stages, zbufs);
    return zs_persistent_bytes<11, 5>(split, nmax, stages, zbufs);
}

size_t zsep_smem_bytes(int h, int w, bool split, int nmax)
{
    const int mt = h <= 7 ? 4 : 6, npart = split ? 2 : 1;
    const size_t rec = h == 6 ? zs_record_bytes<6, 6>(nmax) : h == 5 ? zs_record_bytes<5, 11>(nmax)
                     : h == 7 ? zs_record_bytes<7, 7>(nmax) : zs_record_bytes<11, 5>(nmax);
    return (size_t)zs_union_bytes(mt, npart, nmax) + (size_t)npart * 4 * nmax * 16 + rec + 2 * 8 + 16;
}

}  // namespace

bool zsep_shape(int h, int w)
{
    return (h == 6 && w == 6) || (h == 5 && w == 11) || (h == 7 && w == 7) || (h == 11 && w == 5);
}

void zsep_tile(int h, int w, int *tile_cols, int *tile_rows)
{
    *tile_cols = 32 - (w - 1);
    *tile_rows = (h <= 7 ? 16 : 24) - h + 1;
}

int zsep_nmax(int max_rank) { return max_rank <= 32 ? 32 : max_rank <= 64 ? 64 : 0; }

int zsep_record_bytes(int h, int w, int nmax)
{
    if (h == 6) return (int)zs_record_bytes<6, 6>(nmax);
    if (h == 5) return (int)zs_record_bytes<5, 11>(nmax);
    if (h == 7) return (int)zs_record_bytes<7, 7>(nmax);
    return (int)zs_record_bytes<11, 5>(nmax);
}

int zsep_factor_stride(int h, int w) { return (h + w + 1 + 3) & ~3; }

bool zsep_form_fits(int h, int w, bool split, int nmax, int form)
{
    if (form == ZSEP_TILE) return true;
    const int mt = h <= 7 ? 4 : 6;
    const int stages = form == ZSEP_PERSIST_S2 || form == ZSEP_PERSIST_S2Z2 ? 2 : 1;
    const int zbufs = form == ZSEP_PERSIST_Z2 || form == ZSEP_PERSIST_S2Z2 ? 2 : 1;
    return 2 * mt * nmax <= 512 &&
           zsep_persistent_smem_bytes(h, w, split, nmax, stages, zbufs) <= (size_t)kMaxDynamicSmem;
}

namespace {
int zs_sm_count()
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

cudaError_t launch_zsep_tc(const ZsJob *d_jobs, const ZsTile *d_tiles, int tiles, const ZsGroup *d_fg, int n_fg,
                           const void *cbank, const void *cbank_lo, int ld, const void *d_frec, int nmax, int h, int w,
                           int *d_err, cudaStream_t s, int form)
{
    if (tiles <= 0 || n_fg <= 0) return cudaSuccess;
    if (!zsep_shape(h, w) || (nmax != 32 && nmax != 64) || !d_frec) return cudaErrorInvalidValue;
    if ((long long)tiles * n_fg > 0x7fffffffll) return cudaErrorInvalidValue;
    const bool split = cbank_lo != nullptr;
    const int mt = h <= 7 ? 4 : 6;
    if (form != ZSEP_TILE) {
        if (!zsep_form_fits(h, w, split, nmax, form) || !d_frec) return cudaErrorInvalidValue;
        const int stages = form == ZSEP_PERSIST_S2 || form == ZSEP_PERSIST_S2Z2 ? 2 : 1;
        const int zbufs = form == ZSEP_PERSIST_Z2 || form == ZSEP_PERSIST_S2Z2 ? 2 : 1;
        uint32_t pcols = 32;
        while (pcols < (uint32_t)(2 * mt * nmax)) pcols <<= 1;
        const size_t psmem = zsep_persistent_smem_bytes(h, w, split, nmax, stages, zbufs);
        const uint8_t *fr = static_cast<const uint8_t *>(d_frec);
        const int n_items = tiles * n_fg;
        const unsigned pgrid = (unsigned)std::min(n_items, zs_sm_count());
        const uint8_t *pcb = static_cast<const uint8_t *>(cbank), *pcl = static_cast<const uint8_t *>(cbank_lo);
        cudaError_t pe = cudaSuccess;
#define TDPM_ZSEPP(HH, WW, SP, SLOT)                                                                              \
    do {                                                                                                          \
        pe = allow_max_dynamic_smem(reinterpret_cast<const void *>(zsep_tc_persistent_kernel<HH, WW, SP>), SLOT); \
        if (pe != cudaSuccess) return pe;                                                                         \
        note_launches(1);                                                                                         \
        zsep_tc_persistent_kernel<HH, WW, SP><<<pgrid, ZP_THREADS, psmem, s>>>(                                   \
            d_jobs, d_tiles, d_fg, n_fg, n_items, pcb, pcl, ld, fr, nmax, stages, zbufs, pcols, d_err);           \
    } while (0)
        if (split) {
            if (h == 6) TDPM_ZSEPP(6, 6, true, 16);
            else if (h == 5) TDPM_ZSEPP(5, 11, true, 17);
            else if (h == 7) TDPM_ZSEPP(7, 7, true, 18);
            else TDPM_ZSEPP(11, 5, true, 19);
        } else {
            if (h == 6) TDPM_ZSEPP(6, 6, false, 20);
            else if (h == 5) TDPM_ZSEPP(5, 11, false, 21);
            else if (h == 7) TDPM_ZSEPP(7, 7, false, 22);
            else TDPM_ZSEPP(11, 5, false, 23);
        }
#undef TDPM_ZSEPP
        return cudaGetLastError();
    }
    uint32_t cols = 32;
    while (cols < (uint32_t)(mt * nmax)) cols <<= 1;
    // at most 512 / cols CTAs per SM fit in TMEM: enforced through the shared memory request, so that no CTA waits
    // in tcgen05.alloc behind another CTA of this launch
    const int max_ctas = 512 / (int)cols;
    size_t smem = zsep_smem_bytes(h, w, split, nmax);
    const size_t floor_bytes = 233472 / (size_t)(max_ctas + 1);
    if (smem < floor_bytes) smem = floor_bytes;
    if (smem > (size_t)kMaxDynamicSmem) return cudaErrorInvalidValue;
    const uint8_t *cb = static_cast<const uint8_t *>(cbank), *cl = static_cast<const uint8_t *>(cbank_lo);
    const unsigned grid = (unsigned)((long long)tiles * n_fg);
    cudaError_t e = cudaSuccess;
#define TDPM_ZSEP(HH, WW, SP, SLOT)                                                                               \
    do {                                                                                                          \
        e = allow_max_dynamic_smem(reinterpret_cast<const void *>(zsep_tc_kernel<HH, WW, SP>), SLOT);           \
        if (e != cudaSuccess) return e;                                                                           \
        note_launches(1);                                                                                         \
        zsep_tc_kernel<HH, WW, SP><<<grid, ZS_THREADS, smem, s>>>(d_jobs, d_tiles, d_fg, n_fg, cb, cl, ld,        \
                                                                  static_cast<const uint8_t *>(d_frec), nmax,    \
                                                                  cols, d_err);                                   \
    } while (0)
    if (split) {
        if (h == 6) TDPM_ZSEP(6, 6, true, 8);
        else if (h == 5) TDPM_ZSEP(5, 11, true, 9);
        else if (h == 7) TDPM_ZSEP(7, 7, true, 10);
        else TDPM_ZSEP(11, 5, true, 11);
    } else {
        if (h == 6) TDPM_ZSEP(6, 6, false, 12);
        else if (h == 5) TDPM_ZSEP(5, 11, false, 13);
        else if (h == 7) TDPM_ZSEP(7, 7, false, 14);
        else TDPM_ZSEP(11, 5, false, 15);
    }
#undef TDPM_ZSEP
    return cudaGetLastError();
}

}  // namespace tdpm
