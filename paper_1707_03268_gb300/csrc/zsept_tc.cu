// Step 1, decomposed form, per-filter mode (Sec. 4), with the CP terms on the tensor cores' M dimension:
//   Z_r[y][x]   = sum_c c_r[c] phi[y][x][c]                     (tcgen05 MMA: M = 128 terms, N = 256 cells, K = 32)
//   S_k[y][x]   = sum_{r of k} sum_dy (lambda_r a_r[dy]) sum_dx b_r[dx] Z_r[y+dy][x+dx]
//
// A work item is (spatial tile, term group). The tile is 16 x 16 cells of a level (TY = 17 - h output rows, TX =
// 17 - w output columns); the term group is consecutive filters of the shape group with at most 128 terms between
// them. One thread issues the tile's TMA box {8 ch, 16 columns, 16 rows, 4 chunks} (it lands as the K-major B operand,
// cell n = 16 * row + column), the group's 128 channel-factor rows (the A operand) and its factor record, then the MMAs
// into a 256-column TMEM accumulator: lane t holds Z of term t for every cell of the tile. Thread (warp w, lane l)
// then owns term t = 32 (w % 4) + l and half of the output columns (w / 4): it reads Z row by row from its own TMEM
// lane (one 32x32b.x16 load per row, the next row's load in flight), takes the x pass of the row in registers and
// accumulates the y pass into a ring of h output rows; both passes stay inside the thread. The sum over a filter's
// terms is the only exchange: every RR finished output rows the threads write their terms' contributions to shared
// memory and the CTA adds them per (filter, row, column) in a fixed order (four interleaved partial sums over the
// filter's terms, then their pairwise sum), and stores the filter maps.
// The CTA is persistent over a contiguous range of items, tile-major, so a tile's features are loaded once for all
// its term groups; the next group's A rows and record are prefetched during the current item's passes. Every mbarrier
// wait is bounded (the context's error flag is raised on expiry) and the CTA lets its copies and MMAs finish before it
// releases TMEM and exits.
#include <algorithm>

#include "internal.h"
#include "tc_ptx.h"

namespace tdpm {
namespace {

constexpr int ZT_THREADS = 256;
constexpr int ZT_T = 16;                 // tile side in cells
constexpr int ZT_N = ZT_T * ZT_T;        // cells per tile (MMA N)
constexpr int ZT_M = 128;                // terms per group (MMA M)
constexpr int ZT_FS = 16;                // floats per term in the factor record
constexpr int ZT_RR = 4;                 // output rows per reduction round
constexpr int ZT_RS = 12;                // floats per (term, row) in the reduction buffer
constexpr int ZT_TS = ZT_RR * ZT_RS + 1; // floats per term in the reduction buffer (odd: the lanes' rows fall in
                                         // different banks)
constexpr uint32_t ZT_FEAT = 4 * ZT_N * 16;   // one operand part of the tile: 4 chunks x 256 cells x 16 bytes
constexpr uint32_t ZT_ABANK = 4 * ZT_M * 16;  // one operand part of the group's A rows
constexpr uint32_t ZT_TMEM_COLS = ZT_N;

// Group record: factors [ZT_FS][128] floats (rows 0..h-1: lambda_r a_r[dy]; rows h..h+w-1: b_r[dx]; column = term
// lane), then ints: nf, k0 (the group's first filter in its shape group), lanes[0..nf] (filter f owns lanes
// [lanes[f], lanes[f+1])), rounded up to 16 bytes.
__host__ __device__ constexpr uint32_t zt_record_bytes() { return (ZT_M * ZT_FS * 4 + (ZT_M + 3) * 4 + 15) & ~15u; }

__host__ __device__ constexpr uint32_t zt_smem_bytes(bool split)
{
    const uint32_t np = split ? 2 : 1;
    return np * ZT_FEAT + 2 * np * ZT_ABANK + 2 * zt_record_bytes() + ((ZT_M * ZT_TS * 4 + 15) & ~15) + 64;
}

__device__ __forceinline__ void zt_ld16_nowait(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

// Waits for this thread's TMEM loads; the registers are tied to the wait so that no use moves above it.
__device__ __forceinline__ void zt_ld_wait(uint32_t (&r)[16])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15])
                 :
                 : "memory");
}

// One Z row of a thread's half of the output columns: the x pass (b_r), the y pass into the ring of HH output rows
// (lambda_r a_r, increasing dy), and the output row it completes into the term's reduction rows. C0: the half's first
// output column and NC its number of columns (the first NC of the NCM accumulator columns).
template <int HH, int WW, int NC, int NCM, int TY, int C0>
__device__ __forceinline__ void zt_row(int y, const uint32_t (&zc)[16], const float (&a)[HH], const float (&bb)[WW],
                                       float (&acc)[HH][NCM], float *red_t)
{
    float X[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        float u = 0.f;
#pragma unroll
        for (int dx = 0; dx < WW; ++dx) u = fmaf(bb[dx], __uint_as_float(zc[C0 + c + dx]), u);
        X[c] = u;
    }
#pragma unroll
    for (int dy = 0; dy < HH; ++dy) {
        const int o = y - dy;
        if (o >= 0 && o < TY) {
#pragma unroll
            for (int c = 0; c < NC; ++c) acc[o % HH][c] = dy == 0 ? a[0] * X[c] : fmaf(a[dy], X[c], acc[o % HH][c]);
        }
    }
    const int o = y - (HH - 1);
    if (o >= 0) {
        float *rr = red_t + (o % ZT_RR) * ZT_RS + C0;
#pragma unroll
        for (int c = 0; c < NC; ++c) rr[c] = acc[o % HH][c];
    }
}

template <int HH, int WW, bool SPLIT>
__global__ void __launch_bounds__(ZT_THREADS, 2)
    zsept_tc_kernel(const ZsJob *__restrict__ jobs, const ZsTile *__restrict__ tiles, int n_tiles, int n_tg,
                    const uint8_t *__restrict__ grec, const uint8_t *__restrict__ cbank,
                    const uint8_t *__restrict__ cbank_lo, int ld, const int *__restrict__ group_t0, int *err)
{
    constexpr int TX = ZT_T - WW + 1, TY = ZT_T - HH + 1;
    constexpr int NC = (TX + 1) / 2;  // output columns of the first half; the second half takes the other TX - NC
    constexpr uint32_t NP = SPLIT ? 2 : 1;
    constexpr uint32_t REC = zt_record_bytes();
    extern __shared__ __align__(1024) uint8_t sm[];
    uint8_t *feat = sm;                                        // [NP][4][256][16 B]
    uint8_t *abank = sm + NP * ZT_FEAT;                        // [2][NP][4][128][16 B]
    uint8_t *recs = abank + 2 * NP * ZT_ABANK;                 // [2][REC]
    float *red = reinterpret_cast<float *>(recs + 2 * REC);    // [128][TS]: [RR][RS] per term
    uint64_t *bars = reinterpret_cast<uint64_t *>(recs + 2 * REC + ((ZT_M * ZT_TS * 4 + 15) & ~15));
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 4);
    const uint32_t feat_full = smem_u32(bars), mma_done = smem_u32(bars + 1);
    const uint32_t g_full0 = smem_u32(bars + 2);  // [2]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long n_items = (long long)n_tiles * n_tg;
    const long long per = (n_items + gridDim.x - 1) / gridDim.x;
    const long long ibeg = (long long)blockIdx.x * per, iend = ibeg + per < n_items ? ibeg + per : n_items;
    const int n_local = ibeg < iend ? (int)(iend - ibeg) : 0;

    if (threadIdx.x == 0) {
        mbar_init(feat_full, 1);
        mbar_init(mma_done, 1);
        mbar_init(g_full0, 1);
        mbar_init(g_full0 + 8, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(ZT_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    // the group records and A rows of local item k into buffer k & 1 (thread 0)
    auto issue_group = [&](int k) {
        const int g = (int)((ibeg + k) % n_tg), b = k & 1;
        const uint32_t bar = g_full0 + 8 * b;
        mbar_expect_tx(bar, NP * ZT_ABANK + REC);
        bulk_load(smem_u32(recs + b * REC), grec + (size_t)g * REC, REC, bar);
        const int t0 = group_t0[g];
        const uint32_t dst = smem_u32(abank + b * NP * ZT_ABANK);
#pragma unroll
        for (int kc = 0; kc < 4; ++kc) {
            const size_t off = ((size_t)kc * ld + t0) * 16;
            bulk_load(dst + kc * ZT_M * 16, cbank + off, ZT_M * 16, bar);
            if (SPLIT) bulk_load(dst + ZT_ABANK + kc * ZT_M * 16, cbank_lo + off, ZT_M * 16, bar);
        }
    };
    if (threadIdx.x == 0 && n_local > 0) issue_group(0);

    int prev_tile = -1;
    uint32_t feat_phase = 0;
    const int q = warp & 3, hf = warp >> 2;
    const int t = 32 * q + lane;                // this thread's term lane
    const uint32_t tq = tmem + ((uint32_t)(32 * q) << 16);

    for (int k = 0; k < n_local; ++k) {
        const long long item = ibeg + k;
        const int tile = (int)(item / n_tg), b = k & 1;
        const ZsTile TL = tiles[tile];
        const ZsJob *J = jobs + TL.job;
        if (threadIdx.x == 0) {
            if (tile != prev_tile) {
                // the MMAs of the previous item have read the old tile (all threads waited for them)
                mbar_expect_tx(feat_full, NP * ZT_FEAT);
                tma_load_4d(smem_u32(feat), &J->tmap, 0, TL.x0, TL.y0, 0, feat_full);
                if (SPLIT) tma_load_4d(smem_u32(feat + ZT_FEAT), &J->tmap_lo, 0, TL.x0, TL.y0, 0, feat_full);
            }
            if (k + 1 < n_local) issue_group(k + 1);  // its buffer was last read by item k - 1, now finished
            if (tile != prev_tile) {
                mbar_wait(feat_full, feat_phase, err);
                feat_phase ^= 1u;
            }
            mbar_wait(g_full0 + 8 * b, (uint32_t)(k >> 1) & 1u, err);
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t idesc = instr_desc(ZT_M, ZT_N);
            const uint32_t a0 = smem_u32(abank + b * NP * ZT_ABANK), b0 = smem_u32(feat);
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
                const uint64_t ad = smem_desc(a0 + ks * 2 * ZT_M * 16, ZT_M * 16, 128);
                const uint64_t bd = smem_desc(b0 + ks * 2 * ZT_N * 16, ZT_N * 16, 128);
                mma_bf16(tmem, ad, bd, idesc, ks != 0);
                if (SPLIT) {
                    const uint64_t ad_lo = smem_desc(a0 + ZT_ABANK + ks * 2 * ZT_M * 16, ZT_M * 16, 128);
                    const uint64_t bd_lo = smem_desc(b0 + ZT_FEAT + ks * 2 * ZT_N * 16, ZT_N * 16, 128);
                    mma_bf16(tmem, ad, bd_lo, idesc, 1u);
                    mma_bf16(tmem, ad_lo, bd, idesc, 1u);
                }
            }
            mma_commit(mma_done);
        }
        prev_tile = tile;
        mbar_wait(g_full0 + 8 * b, (uint32_t)(k >> 1) & 1u, err);  // the record (complete before the MMAs)
        mbar_wait(mma_done, (uint32_t)k & 1u, err);
        __syncwarp();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

        // this thread's factors: a_r scaled by lambda_r, b_r (factor-major: the lanes read consecutive words)
        const float *fr = reinterpret_cast<const float *>(recs + b * REC) + t;
        float a[HH], bb[WW];
#pragma unroll
        for (int i = 0; i < HH; ++i) a[i] = fr[i * ZT_M];
#pragma unroll
        for (int i = 0; i < WW; ++i) bb[i] = fr[(HH + i) * ZT_M];
        const int *ri = reinterpret_cast<const int *>(recs + b * REC + ZT_M * ZT_FS * 4);
        const int nf = ri[0], kf0 = ri[1];
        const int *lanes = ri + 2;
        const int Ho = J->Ho, Wo = J->Wo;
        float *out = J->out;

        float acc[HH][NC];
        // the passes of Z row y (held in zc) for this thread's half, and the reduction round it completes
        auto row_step = [&](const int y, const uint32_t(&zc)[16]) {
            // warp-uniform branch; each half has constant indices
            if (hf) zt_row<HH, WW, TX - NC, NC, TY, NC>(y, zc, a, bb, acc, red + t * ZT_TS);
            else zt_row<HH, WW, NC, NC, TY, 0>(y, zc, a, bb, acc, red + t * ZT_TS);
            const int o = y - (HH - 1);  // output row completed by this Z row
            if (o >= 0) {
                if (o % ZT_RR == ZT_RR - 1 || o == TY - 1) {
                    // reduction round over output rows [rb, o]
                    const int rb = o - o % ZT_RR, nr = o - rb + 1;
                    __syncthreads();
                    const int total = nf * nr * TX;
                    for (int j = threadIdx.x; j < total; j += ZT_THREADS) {
                        const int c = j % TX, tmp = j / TX;
                        const int r = rb + tmp % nr, f = tmp / nr;
                        const int l0 = lanes[f], n = lanes[f + 1] - l0;
                        const float *src = red + l0 * ZT_TS + (r % ZT_RR) * ZT_RS + c;
                        // four partial sums over the terms l0 + 4 i + m, then (s0 + s1) + (s2 + s3): a fixed order
                        float s0 = src[0], s1 = 0.f, s2 = 0.f, s3 = 0.f;
                        if (n > 1) s1 = src[ZT_TS];
                        if (n > 2) s2 = src[2 * ZT_TS];
                        if (n > 3) s3 = src[3 * ZT_TS];
                        int l = 4;
                        for (; l + 3 < n; l += 4) {
                            s0 += src[l * ZT_TS];
                            s1 += src[(l + 1) * ZT_TS];
                            s2 += src[(l + 2) * ZT_TS];
                            s3 += src[(l + 3) * ZT_TS];
                        }
                        if (l < n) s0 += src[l * ZT_TS];
                        if (l + 1 < n) s1 += src[(l + 1) * ZT_TS];
                        if (l + 2 < n) s2 += src[(l + 2) * ZT_TS];
                        const float s = (s0 + s1) + (s2 + s3);
                        const int yy = TL.y0 + r, xx = TL.x0 + c;
                        if (r < TL.rows && xx < Wo) out[((size_t)(kf0 + f) * Ho + yy) * Wo + xx] = s;
                    }
                    // the last round's barrier also ends the item: every TMEM read of it is complete (the last row's
                    // load was waited for) before the next item's MMAs overwrite the accumulator
                    if (o == TY - 1) asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    __syncthreads();
                    if (o == TY - 1) asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                }
            }
        };
        // two row buffers in turn: the next row's TMEM load is in flight during the current row's passes
        static_assert(ZT_T % 2 == 0, "rows are taken in pairs");
        uint32_t z0[16], z1[16];
        zt_ld16_nowait(tq, z0);
        zt_ld_wait(z0);
#pragma unroll
        for (int y = 0; y < ZT_T; y += 2) {
            zt_ld16_nowait(tq + 16 * (y + 1), z1);
            row_step(y, z0);
            zt_ld_wait(z1);
            if (y + 2 < ZT_T) zt_ld16_nowait(tq + 16 * (y + 2), z0);
            row_step(y + 1, z1);
            if (y + 2 < ZT_T) zt_ld_wait(z0);
        }
        static_assert(TY - 1 + HH - 1 == ZT_T - 1, "the last Z row completes the last output row and its round");
    }
    if (threadIdx.x == 0 && n_local > 0) {
        // only reached with copies or MMAs in flight when a wait above gave up
        mbar_drain(mma_done, (uint32_t)(n_local - 1) & 1u);
        if (n_local > 1) mbar_drain(g_full0 + 8 * ((n_local - 1) & 1), (uint32_t)((n_local - 1) >> 1) & 1u);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ZT_TMEM_COLS)
                     : "memory");
}

int zt_sm_count()
{
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

}  // namespace

bool zsept_shape(int h, int w) { return (h == 6 && w == 6) || (h == 7 && w == 7); }
int zsept_tile_side() { return ZT_T; }
int zsept_terms() { return ZT_M; }
int zsept_record_bytes() { return (int)zt_record_bytes(); }
int zsept_factor_stride() { return ZT_FS; }

cudaError_t launch_zsept_tc(const ZsJob *d_jobs, const ZsTile *d_tiles, int n_tiles, int n_tg, const void *d_grec,
                            const int *d_group_t0, const void *cbank, const void *cbank_lo, int ld, int h, int w,
                            int *d_err, cudaStream_t s)
{
    if (n_tiles <= 0 || n_tg <= 0) return cudaSuccess;
    if (!zsept_shape(h, w) || !d_grec || !d_group_t0) return cudaErrorInvalidValue;
    const bool split = cbank_lo != nullptr;
    // at most two CTAs per SM: their accumulators fill TMEM; the request keeps a third one off the SM
    const size_t smem = std::max<size_t>(zt_smem_bytes(split), 233472 / 3 + 1024);
    if (smem > (size_t)kMaxDynamicSmem) return cudaErrorInvalidValue;
    const long long n_items = (long long)n_tiles * n_tg;
    const unsigned grid = (unsigned)std::min<long long>(n_items, 2ll * zt_sm_count());
    const uint8_t *gr = static_cast<const uint8_t *>(d_grec);
    const uint8_t *cb = static_cast<const uint8_t *>(cbank), *cl = static_cast<const uint8_t *>(cbank_lo);
    cudaError_t e = cudaSuccess;
#define TDPM_ZT(HH, WW, SP, SLOT)                                                                                  \
    do {                                                                                                           \
        e = allow_max_dynamic_smem(reinterpret_cast<const void *>(zsept_tc_kernel<HH, WW, SP>), SLOT);             \
        if (e != cudaSuccess) return e;                                                                            \
        note_launches(1);                                                                                          \
        zsept_tc_kernel<HH, WW, SP><<<grid, ZT_THREADS, smem, s>>>(d_jobs, d_tiles, n_tiles, n_tg, gr, cb, cl, ld, \
                                                                    d_group_t0, d_err);                            \
    } while (0)
    if (split) {
        if (h == 6) TDPM_ZT(6, 6, true, 32);
        else TDPM_ZT(7, 7, true, 33);
    } else {
        if (h == 6) TDPM_ZT(6, 6, false, 34);
        else TDPM_ZT(7, 7, false, 35);
    }
#undef TDPM_ZT
    return cudaGetLastError();
}

}  // namespace tdpm
