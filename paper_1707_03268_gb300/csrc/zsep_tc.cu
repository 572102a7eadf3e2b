// Step 1, decomposed form, per-filter mode, fused on the tensor cores (Sec. 4): the channel stage
//   Z_r[y][x] = sum_c c_r[c] phi[y][x][c]
// and the separable passes with the recombination
//   S_k[y][x] = sum_{r of k} lambda_r sum_dx b_r[dx] sum_dy a_r[dy] Z_r[y+dy][x+dx]
// in one kernel, so that the rank-1 maps Z_r never leave the SM.
//
// A CTA takes one spatial tile of one level and one filter group (consecutive filters whose terms, at most nmax of
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

__device__ __forceinline__ int zs_find_job(const ZsJob *jobs, int n, int idx)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].begin <= idx) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__host__ __device__ constexpr uint32_t zs_union_bytes(int mt, int npart, int nmax)
{
    return (uint32_t)(mt * npart) * ZS_A_TILE > (uint32_t)nmax * 4 * mt * 32 * 4
               ? (uint32_t)(mt * npart) * ZS_A_TILE
               : (uint32_t)nmax * 4 * mt * 32 * 4;
}

template <int HH, int WW, bool SPLIT>
__global__ void __launch_bounds__(ZS_THREADS, 3)
    zsep_tc_kernel(const ZsJob *__restrict__ jobs, int n_jobs, const ZsGroup *__restrict__ fgs, int n_fg,
                   const uint8_t *__restrict__ cbank, const uint8_t *__restrict__ cbank_lo, int ld,
                   const float *__restrict__ A, const float *__restrict__ B, const float *__restrict__ lam,
                   const int *__restrict__ rank_off, int R, int nmax, uint32_t tmem_cols, int *err)
{
    using S = ZsShape<HH>;
    constexpr int MT = S::MT, TYZ = S::TYZ, TY = S::TY;
    constexpr int SW = 32 - (WW - 1);  // output columns of a tile
    constexpr uint32_t NPART = SPLIT ? 2 : 1;
    extern __shared__ __align__(1024) uint8_t sm[];
    uint8_t *uni = sm;                                                  // feature tiles, then Z [nmax][TYZ][32]
    uint8_t *bsm = sm + zs_union_bytes(MT, NPART, nmax);                // [NPART][4][nmax][16 bytes]
    float *fa = reinterpret_cast<float *>(bsm + NPART * 4 * nmax * 16);  // a_r [HH][nmax]
    float *fb = fa + HH * nmax;                                         // b_r [WW][nmax]
    float *fl = fb + WW * nmax;                                         // lambda_r [nmax]
    uint64_t *bars = reinterpret_cast<uint64_t *>(fl + nmax);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2);
    const uint32_t full = smem_u32(bars), done = smem_u32(bars + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int fgi = blockIdx.x % n_fg, tile = blockIdx.x / n_fg;  // the filter groups of a tile are neighbours
    const ZsJob *J = jobs + zs_find_job(jobs, n_jobs, tile);
    const int lt = tile - J->begin;
    const int x0 = (lt % J->tiles_x) * SW, y0 = (lt / J->tiles_x) * TY;
    const ZsGroup G = fgs[fgi];
    const int N = (G.n + 15) & ~15;

    if (threadIdx.x == 0) {
        mbar_init(full, 1);
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

    if (threadIdx.x == 0) {
        mbar_expect_tx(full, MT * NPART * ZS_A_TILE + NPART * 4 * (uint32_t)N * 16);
#pragma unroll
        for (int t = 0; t < MT; ++t) {
            const uint32_t dst = smem_u32(uni + t * NPART * ZS_A_TILE);
            tma_load_4d(dst, &J->tmap, 0, x0, y0 + 4 * t, 0, full);
            if (SPLIT) tma_load_4d(dst + ZS_A_TILE, &J->tmap_lo, 0, x0, y0 + 4 * t, 0, full);
        }
        const uint32_t bdst = smem_u32(bsm);
#pragma unroll
        for (int kc = 0; kc < 4; ++kc) {
            const size_t off = ((size_t)kc * ld + G.t0) * 16;
            bulk_load(bdst + kc * N * 16, cbank + off, (uint32_t)N * 16, full);
            if (SPLIT) bulk_load(bdst + 4 * N * 16 + kc * N * 16, cbank_lo + off, (uint32_t)N * 16, full);
        }
        mbar_wait(full, 0, err);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t idesc = instr_desc(128, N);
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
    // the group's factors, while the copies and MMAs run (zero beyond its terms)
    for (int i = threadIdx.x; i < (HH + WW + 1) * nmax; i += ZS_THREADS) {
        const int row = i / nmax, j = i - row * nmax;
        const int r = G.t0 + j;
        float v = 0.f;
        if (j < G.n) v = row < HH ? __ldg(A + (size_t)row * R + r)
                         : row < HH + WW ? __ldg(B + (size_t)(row - HH) * R + r) : __ldg(lam + r);
        fa[i] = v;  // fa, fb and fl are contiguous
    }
    mbar_wait(done, 0, err);
    __syncwarp();  // warp 0 reconverges (lane 0 issued the copies and MMAs) before the warp-wide TMEM loads
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    // TMEM -> shared memory: warp w reads lane quadrant q = w % 4 (Z row 4t + q of M tile t, column = lane) and half of
    // the columns (terms)
    float *Z = reinterpret_cast<float *>(uni);
    {
        const int q = warp & 3, cw = nmax >> 1, cb = (warp >> 2) * cw;
        for (int c0 = cb; c0 < cb + cw && c0 < G.n; c0 += 16) {
#pragma unroll
            for (int t = 0; t < MT; ++t) {
                uint32_t r[16];
                tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(t * nmax + c0), r);
                float *zr = Z + ((size_t)c0 * TYZ + 4 * t + q) * 32 + lane;
#pragma unroll
                for (int j = 0; j < 16; ++j) zr[(size_t)j * TYZ * 32] = __uint_as_float(r[j]);
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

    // separable passes: tasks (filter, block of output rows), spread over the warps
    const int nf = G.k1 - G.k0;
    const int n_rows = min(TY, J->Ho - y0);
    const int nrb = max(1, ZS_WARPS / nf);
    const int SR = (n_rows + nrb - 1) / nrb;
    const int Ho = J->Ho, Wo = J->Wo;
    const int x = x0 + lane;
    for (int task = warp; task < nf * nrb; task += ZS_WARPS) {
        const int f = task / nrb, rb = task - f * nrb;
        const int i0 = rb * SR, ni = min(SR, n_rows - i0);
        if (ni <= 0) continue;  // warp-uniform
        const int k = G.k0 + f;
        const int tb = __ldg(rank_off + k) - G.t0, te = __ldg(rank_off + k + 1) - G.t0;
        float acc[TY];
#pragma unroll
        for (int i = 0; i < TY; ++i) acc[i] = 0.f;
        for (int tr = tb; tr < te; ++tr) {
            float a[HH], bb[WW];
#pragma unroll
            for (int i = 0; i < HH; ++i) a[i] = fa[i * nmax + tr];
#pragma unroll
            for (int i = 0; i < WW; ++i) bb[i] = fb[i * nmax + tr];
            const float l = fl[tr];
            const float *z = Z + ((size_t)tr * TYZ + i0) * 32 + lane;
            float win[HH];
#pragma unroll
            for (int i = 0; i < HH - 1; ++i) win[i] = z[i * 32];
#pragma unroll
            for (int i = 0; i < TY; ++i) {
                if (i < ni) {  // warp-uniform
                    win[(i + HH - 1) % HH] = z[(i + HH - 1) * 32];
                    float tv = 0.f;
#pragma unroll
                    for (int dy = 0; dy < HH; ++dy) tv = fmaf(a[dy], win[(i + dy) % HH], tv);
                    float u = 0.f;
#pragma unroll
                    for (int dx = 0; dx < WW; ++dx)
                        u = fmaf(bb[dx], dx ? __shfl_down_sync(0xffffffffu, tv, dx) : tv, u);
                    acc[i] = fmaf(l, u, acc[i]);
                }
            }
        }
        if (lane < SW && x < Wo) {
            float *o = J->out + (size_t)k * Ho * Wo + (size_t)(y0 + i0) * Wo + x;
#pragma unroll
            for (int i = 0; i < TY; ++i)
                if (i < ni) o[(size_t)i * Wo] = acc[i];
        }
    }
}

size_t zsep_smem_bytes(int h, int w, bool split, int nmax)
{
    const int mt = h <= 7 ? 4 : 6, npart = split ? 2 : 1;
    return (size_t)zs_union_bytes(mt, npart, nmax) + (size_t)npart * 4 * nmax * 16 + (size_t)(h + w + 1) * nmax * 4 +
           2 * 8 + 16;
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

cudaError_t launch_zsep_tc(const ZsJob *d_jobs, int n_jobs, int tiles, const ZsGroup *d_fg, int n_fg,
                           const void *cbank, const void *cbank_lo, int ld, const float *A, const float *B,
                           const float *lam, const int *rank_off, int R, int nmax, int h, int w, int *d_err,
                           cudaStream_t s)
{
    if (tiles <= 0 || n_fg <= 0) return cudaSuccess;
    if (!zsep_shape(h, w) || (nmax != 32 && nmax != 64)) return cudaErrorInvalidValue;
    if ((long long)tiles * n_fg > 0x7fffffffll) return cudaErrorInvalidValue;
    const bool split = cbank_lo != nullptr;
    const int mt = h <= 7 ? 4 : 6;
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
        zsep_tc_kernel<HH, WW, SP><<<grid, ZS_THREADS, smem, s>>>(d_jobs, n_jobs, d_fg, n_fg, cb, cl, ld, A, B,   \
                                                                  lam, rank_off, R, nmax, cols, d_err);           \
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
