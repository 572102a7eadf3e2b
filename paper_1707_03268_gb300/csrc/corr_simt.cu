// SIMT correlation kernels (FP32 arithmetic):
//   corr_f32_kernel  step 1, full form (Sec. 2 score equation): register-tiled direct correlation, the FP32 GPU
//                    baseline the decomposed form is measured against;
//   zproj_kernel     step 1, decomposed form, channel stage Z_r = phi o c_r (Sec. 4, correlation with the L-vector);
//   sep_kernel       step 1, decomposed form, the 1-D passes along y (a_r) and x (b_r) and the recombination
//                    S_k = sum_r Lambda[k][r] U_r (Sec. 4, I o T = sum_r ((I o a_r) o b_r) o c_r).
#include <cuda_bf16.h>

#include "internal.h"

namespace tdpm {
namespace {

template <class Job>
__device__ __forceinline__ int find_job(const Job *jobs, int n, long long idx)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((long long)jobs[mid].begin <= idx) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ------------------------------------------------------------------------------------------------------------ K8
// CTA tile: CT_TY rows x CT_TX columns of output positions x CT_TK filters. Thread (tx, tf) owns the CT_TY positions
// of column x0+tx and the 8 filters k0+8tf..k0+8tf+7: 64 FP32 accumulators. The level's halo tile sits in shared
// memory channel-planar ([c][row][col]); filter taps are staged CT_TAPS at a time as [tap][c][filter].
constexpr int CT_TX = 16, CT_TY = 8, CT_TK = 64, CT_THREADS = 128, CT_TAPS = 4;

__global__ void __launch_bounds__(CT_THREADS) corr_f32_kernel(const CorrJob *__restrict__ jobs, int n_jobs,
                                                              const float *__restrict__ filt_t, int K, int Kpad,
                                                              int h, int w)
{
    extern __shared__ __align__(16) float sm[];
    const int HX = CT_TX + w - 1, HY = CT_TY + h - 1;
    const int plane = HY * HX;
    float *halo = sm;
    float *fs = sm + ((FD * plane + 3) & ~3);

    const int ji = find_job(jobs, n_jobs, blockIdx.x);
    const CorrJob J = jobs[ji];
    int local = blockIdx.x - J.begin;
    const int k_tiles = Kpad / CT_TK;
    const int kt = local % k_tiles;
    local /= k_tiles;
    const int x0 = (local % J.tiles_x) * CT_TX, y0 = (local / J.tiles_x) * CT_TY, k0 = kt * CT_TK;

    for (int i = threadIdx.x; i < plane * 8; i += CT_THREADS) {
        const int c4 = i & 7, cell = i >> 3;
        const int r = cell / HX, q = cell - r * HX;
        const int gy = y0 + r, gx = x0 + q;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (gy < J.H && gx < J.W) v = __ldg(reinterpret_cast<const float4 *>(J.feat + ((size_t)gy * J.W + gx) * FD) + c4);
        float *dst = halo + (c4 * 4) * plane + cell;
        dst[0] = v.x; dst[plane] = v.y; dst[2 * plane] = v.z; dst[3 * plane] = v.w;
    }

    const int tx = threadIdx.x & 15, tf = threadIdx.x >> 4;
    float acc[CT_TY][8];
#pragma unroll
    for (int r = 0; r < CT_TY; ++r)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[r][j] = 0.f;

    const int ntaps = h * w;
    for (int t0 = 0; t0 < ntaps; t0 += CT_TAPS) {
        const int nt = min(CT_TAPS, ntaps - t0);
        __syncthreads();
        for (int i = threadIdx.x; i < nt * FD * (CT_TK / 4); i += CT_THREADS) {
            const int k4 = i & 15, tc = i >> 4;
            reinterpret_cast<float4 *>(fs + tc * CT_TK)[k4] =
                __ldg(reinterpret_cast<const float4 *>(filt_t + (size_t)(t0 * FD + tc) * Kpad + k0) + k4);
        }
        __syncthreads();
        for (int tl = 0; tl < nt; ++tl) {
            const int tap = t0 + tl, dy = tap / w, dx = tap - dy * w;
            const float *hb = halo + dy * HX + tx + dx;
            const float *fb = fs + tl * FD * CT_TK + tf * 8;
#pragma unroll 4
            for (int c = 0; c < FD; ++c) {
                float a[CT_TY];
#pragma unroll
                for (int r = 0; r < CT_TY; ++r) a[r] = hb[c * plane + r * HX];
                const float4 b0 = *reinterpret_cast<const float4 *>(fb + c * CT_TK);
                const float4 b1 = *reinterpret_cast<const float4 *>(fb + c * CT_TK + 4);
                const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
                for (int r = 0; r < CT_TY; ++r)
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[r][j] = fmaf(a[r], b[j], acc[r][j]);
            }
        }
    }

    const int x = x0 + tx;
    if (x >= J.Wo) return;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int k = k0 + tf * 8 + j;
        if (k >= K) break;
        float *o = J.out + (size_t)k * J.Ho * J.Wo + x;
#pragma unroll
        for (int r = 0; r < CT_TY; ++r)
            if (y0 + r < J.Ho) o[(size_t)(y0 + r) * J.Wo] = acc[r][j];
    }
}

// ------------------------------------------------------------------------------------------------------------ K2
// One thread per cell, ZP_RCHUNK projections per CTA: z_r = sum_c C[c][r] phi[cell][c] (FP32 path).
constexpr int ZP_CELLS = 128, ZP_RCHUNK = 64;

__global__ void __launch_bounds__(ZP_CELLS) zproj_kernel(const ZJob *__restrict__ jobs, int n_jobs,
                                                         const float *__restrict__ Ct, int R)
{
    __shared__ __align__(16) float cs[ZP_RCHUNK][FD];
    const int ji = find_job(jobs, n_jobs, blockIdx.x);
    const ZJob J = jobs[ji];
    const int local = blockIdx.x - J.begin;
    const int r_chunks = (R + ZP_RCHUNK - 1) / ZP_RCHUNK;
    const int rc = local % r_chunks, ct = local / r_chunks;
    const int r0 = rc * ZP_RCHUNK, nr = min(ZP_RCHUNK, R - r0);
    for (int i = threadIdx.x; i < ZP_RCHUNK * FD; i += ZP_CELLS) {
        const int r = i / FD;
        cs[r][i % FD] = r < nr ? Ct[(size_t)(r0 + r) * FD + (i % FD)] : 0.f;
    }
    const int cell = ct * ZP_CELLS + threadIdx.x;
    float f[FD];
    if (cell < J.cells) {
        const float4 *src = reinterpret_cast<const float4 *>(J.feat + (size_t)cell * FD);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const float4 v = __ldg(src + i);
            f[4 * i] = v.x; f[4 * i + 1] = v.y; f[4 * i + 2] = v.z; f[4 * i + 3] = v.w;
        }
    }
    __syncthreads();
    if (cell >= J.cells) return;
    for (int r = 0; r < nr; ++r) {
        float z = 0.f;
#pragma unroll
        for (int c = 0; c < FD; ++c) z = fmaf(cs[r][c], f[c], z);
        J.Z[(size_t)(r0 + r) * J.cells + cell] = z;
    }
}

// ------------------------------------------------------------------------------------------------------------ K3/K4
// CTA tile: SQ_T x SQ_T output positions of one filter (per-filter mode) or of SQ_FC_JOINT filters (joint mode).
// For every rank-1 term r of those filters the CTA copies the Z_r halo ((SQ_T+h-1) x (SQ_T+w-1) cells) into shared
// memory with cp.async (zero fill outside the map), double-buffered so term r+1 is in flight while term r is
// processed. y pass: each work item forms 4 rows of one column of T = a_r o_y Z_r from h+3 loads; x pass: each
// thread forms U_r = b_r o_x T at 4 consecutive columns of one row from w+3 loads, then adds Lambda[k][r] * U_r to
// each filter's accumulators. HH / WW are the filter sides when known at compile time (0: runtime sides).
// TERMS: the CTA owns 8 consecutive terms instead of 8 filters; its "weights" are the unit vectors, so the
// accumulators hold U_r exactly, and they are stored as BF16 planar (16 bytes per cell: the 8 terms' values).
constexpr int SQ_T = 32, SQ_THREADS = 256, SQ_MAXHW = 16, SQ_HALO = SQ_T + SQ_MAXHW - 1, SQ_FC_JOINT = 8;
constexpr int SQ_TS_STRIDE = 65;  // == 1 (mod 32): the x pass's 4 rows x 8 column groups per warp hit distinct banks

__device__ __forceinline__ void cp_async_f32(float *dst, const float *src, bool pred)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    const int n = pred ? 4 : 0;
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(n) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <int FC, int HH, int WW, bool TERMS>
__global__ void __launch_bounds__(SQ_THREADS) sep_kernel(const SepJob *__restrict__ jobs, int n_jobs,
                                                         const float *__restrict__ A, const float *__restrict__ B,
                                                         const float *__restrict__ lam,
                                                         const int *__restrict__ rank_off, int K, int R, int h_rt,
                                                         int w_rt)
{
    constexpr int MH = HH ? HH : SQ_MAXHW, MW = WW ? WW : SQ_MAXHW;
    const int h = HH ? HH : h_rt, w = WW ? WW : w_rt;
    __shared__ float zs[2][SQ_HALO][SQ_HALO + 1];
    __shared__ float ts[SQ_T][SQ_TS_STRIDE];
    __shared__ float coef[2][2 * SQ_MAXHW + FC];

    const int tid = threadIdx.x;
    const int ji = find_job(jobs, n_jobs, blockIdx.x);
    const SepJob J = jobs[ji];
    int local = blockIdx.x - J.begin;
    const int f_chunks = (FC == 1) ? K : (K + FC - 1) / FC;
    const int fc = local % f_chunks;
    local /= f_chunks;
    const int x0 = (local % J.tiles_x) * SQ_T, y0 = (local / J.tiles_x) * SQ_T;
    const int k0 = fc * FC;
    int r_begin = 0, r_end = R;
    if (FC == 1) { r_begin = rank_off[k0]; r_end = rank_off[k0 + 1]; }
    if (TERMS) { r_begin = min(k0, R); r_end = min(k0 + FC, R); }
    const int HY = SQ_T + h - 1, HX = SQ_T + w - 1;
    const size_t plane = (size_t)J.H * J.W;
    const int lx = tid % SQ_T, ly = tid / SQ_T;  // 32 x 8 layout for the copies

    auto load_term = [&](int r, int buf) {
        const float *Zr = J.Z + (size_t)r * plane;
        for (int yy = ly; yy < HY; yy += SQ_THREADS / SQ_T) {
            const int gy = y0 + yy;
            for (int xx = lx; xx < HX; xx += SQ_T) {
                const int gx = x0 + xx;
                const bool in = gy < J.H && gx < J.W;
                cp_async_f32(&zs[buf][yy][xx], in ? Zr + (size_t)gy * J.W + gx : Zr, in);
            }
        }
        if (tid < h) coef[buf][tid] = __ldg(A + (size_t)tid * R + r);
        else if (tid < h + w) coef[buf][tid] = __ldg(B + (size_t)(tid - h) * R + r);
        else if (tid < h + w + FC) {
            const int f = tid - h - w;
            if (TERMS)
                coef[buf][tid] = (f == r - k0) ? 1.f : 0.f;
            else
                coef[buf][tid] =
                    (FC == 1) ? __ldg(lam + r) : ((k0 + f < K) ? __ldg(lam + (size_t)(k0 + f) * R + r) : 0.f);
        }
        cp_async_commit();
    };

    // x pass ownership: row xr, columns xc .. xc+3
    const int xr = tid / 8, xc = (tid % 8) * 4;
    float acc[FC][4];
#pragma unroll
    for (int f = 0; f < FC; ++f)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[f][j] = 0.f;

    if (r_begin < r_end) load_term(r_begin, 0);
    for (int r = r_begin; r < r_end; ++r) {
        const int buf = (r - r_begin) & 1;
        if (r + 1 < r_end) {
            load_term(r + 1, buf ^ 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const float *a = coef[buf], *b = coef[buf] + h, *lf = coef[buf] + h + w;
        // y pass: items (column xx, row group g of 4 rows)
        for (int item = tid; item < HX * (SQ_T / 4); item += SQ_THREADS) {
            const int g = item / HX, xx = item - g * HX, y = g * 4;
            float z[4 + MH - 1];
#pragma unroll
            for (int k = 0; k < 4 + MH - 1; ++k)
                if (HH || k < 4 + h - 1) z[k] = zs[buf][y + k][xx];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float t = 0.f;
#pragma unroll
                for (int dy = 0; dy < MH; ++dy)
                    if (HH || dy < h) t = fmaf(a[dy], z[j + dy], t);
                ts[y + j][xx] = t;
            }
        }
        __syncthreads();
        {
            float tv[4 + MW - 1];
#pragma unroll
            for (int k = 0; k < 4 + MW - 1; ++k)
                if (WW || k < 4 + w - 1) tv[k] = ts[xr][xc + k];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float u = 0.f;
#pragma unroll
                for (int dx = 0; dx < MW; ++dx)
                    if (WW || dx < w) u = fmaf(b[dx], tv[j + dx], u);
#pragma unroll
                for (int f = 0; f < FC; ++f) acc[f][j] = fmaf(lf[f], u, acc[f][j]);
            }
        }
        __syncthreads();
    }
    const int y = y0 + xr;
    if (y >= J.Ho) return;
    if (TERMS) {
        static_assert(!TERMS || FC == 8, "one planar chunk of 8 terms per CTA");
        const size_t cells = (size_t)J.Ho * J.Wo;
        const size_t row = ((size_t)fc * cells + (size_t)y * J.Wo) * 8;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int x = x0 + xc + j;
            if (x >= J.Wo) break;
            uint32_t hv[4], lv[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const __nv_bfloat16 h0 = __float2bfloat16_rn(acc[2 * q][j]), h1 = __float2bfloat16_rn(acc[2 * q + 1][j]);
                hv[q] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
                const __nv_bfloat16 l0 = __float2bfloat16_rn(acc[2 * q][j] - __bfloat162float(h0));
                const __nv_bfloat16 l1 = __float2bfloat16_rn(acc[2 * q + 1][j] - __bfloat162float(h1));
                lv[q] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
            }
            *reinterpret_cast<uint4 *>(J.U + row + (size_t)x * 8) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
            if (J.U_lo) *reinterpret_cast<uint4 *>(J.U_lo + row + (size_t)x * 8) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
        }
        return;
    }
#pragma unroll
    for (int f = 0; f < FC; ++f) {
        if (k0 + f >= K) break;
        float *o = J.out + ((size_t)(k0 + f) * J.Ho + y) * J.Wo;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (x0 + xc + j < J.Wo) o[x0 + xc + j] = acc[f][j];
    }
}

// Per-filter mode, warp form (no block barrier). A warp owns one filter k and a block of SW_ROWS output rows x
// (32 - (w-1)) output columns. For each of the filter's terms, lane l copies the block's SW_ROWS + h - 1 values of Z_r
// in column x0 + l into the warp's own shared-memory buffer with cp.async (double-buffered: term r+1 is in flight while
// term r is computed; the waits are per warp). The y pass slides an h-deep window down the column (one shared load
// per row), the x pass takes T_r at columns x .. x+w-1 from lanes l .. l+w-1 by shuffles, and lambda_r U_r
// accumulates in registers across the filter's terms. The multiply-add order (dy ascending, then dx ascending, then
// the terms) is that of sep_kernel, so both give identical results.
constexpr int SW_ROWS = 8, SW_WARPS = 4;

template <int HH, int WW>
__global__ void __launch_bounds__(SW_WARPS * 32, 7) sep_warp_kernel(const SepJob *__restrict__ jobs, int n_jobs,
                                                                long long total, const float *__restrict__ A,
                                                                const float *__restrict__ B,
                                                                const float *__restrict__ lam,
                                                                const int *__restrict__ rank_off, int K, int R)
{
    constexpr int SW = 32 - (WW - 1);  // output columns per warp
    constexpr int NZ = SW_ROWS + HH - 1;
    __shared__ float zs[SW_WARPS][2][NZ][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long task = (long long)blockIdx.x * SW_WARPS + warp;
    if (task >= total) return;
    const SepJob &J = jobs[find_job(jobs, n_jobs, task)];
    long long local = task - J.begin;
    const int k = (int)(local % K);
    local /= K;
    const int sx = (int)(local % J.tiles_x), sy = (int)(local / J.tiles_x);
    const int x0 = sx * SW, y0 = sy * SW_ROWS;
    const int x = x0 + lane;
    const int W = J.W;
    const size_t plane = (size_t)J.H * W;
    // Rows: output row y < Ho reads Z rows y .. y+h-1 <= H-1, so no row is out of range (rows past the block's last
    // needed row repeat it). Columns: a lane past the last column reads column W-1 instead; its T only reaches
    // outputs at x >= Wo, which are not written.
    const int xc = x < W ? x : W - 1;
    const int n_out = min(SW_ROWS, J.Ho - y0), n_in = n_out + HH - 1;  // output rows, Z rows of the block
    const float *zbase = J.Z + (size_t)y0 * W + xc;
    float(*buf)[NZ][32] = zs[warp];
    auto issue = [&](int r, int b) {
        const float *zp = zbase + (size_t)r * plane;
        // an opaque copy of the row stride: the row offsets are recomputed per term, not held live across the loop
        int ws = W;
        asm volatile("" : "+r"(ws));
        // a running row pointer: each address depends on the previous one, so none is precomputed and held
#pragma unroll
        for (int i = 0; i < NZ; ++i) {
            cp_async_f32(&buf[b][i][lane], zp, true);
            if (i < n_in - 1) zp += ws;
        }
        cp_async_commit();
    };
    float acc[SW_ROWS];
#pragma unroll
    for (int i = 0; i < SW_ROWS; ++i) acc[i] = 0.f;
    const int r_begin = rank_off[k], r_end = rank_off[k + 1];
    if (r_begin < r_end) issue(r_begin, 0);
    for (int r = r_begin; r < r_end; ++r) {
        const int b = (r - r_begin) & 1;
        float a[HH], bb[WW];
#pragma unroll
        for (int i = 0; i < HH; ++i) a[i] = __ldg(A + (size_t)i * R + r);
#pragma unroll
        for (int i = 0; i < WW; ++i) bb[i] = __ldg(B + (size_t)i * R + r);
        const float l = __ldg(lam + r);
        if (r + 1 < r_end) {
            issue(r + 1, b ^ 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncwarp();
        const float(*z)[32] = buf[b];
        float win[HH];
#pragma unroll
        for (int i = 0; i < HH - 1; ++i) win[i] = z[i][lane];
#pragma unroll
        for (int i = 0; i < SW_ROWS; ++i) {
            if (i < n_out) {  // warp-uniform
                win[(i + HH - 1) % HH] = z[i + HH - 1][lane];
                float tv = 0.f;
#pragma unroll
                for (int dy = 0; dy < HH; ++dy) tv = fmaf(a[dy], win[(i + dy) % HH], tv);
                float u = 0.f;
#pragma unroll
                for (int dx = 0; dx < WW; ++dx) u = fmaf(bb[dx], dx ? __shfl_down_sync(0xffffffffu, tv, dx) : tv, u);
                acc[i] = fmaf(l, u, acc[i]);
            }
        }
        __syncwarp();  // every lane is done with buffer b before it is refilled (two terms later)
    }
    if (lane >= SW || x >= J.Wo) return;
    float *o = J.out + (size_t)k * J.Ho * J.Wo + x;
#pragma unroll
    for (int i = 0; i < SW_ROWS; ++i)
        if (i < n_out) o[(size_t)(y0 + i) * J.Wo] = acc[i];
}

template <int FC, bool TERMS>
cudaError_t launch_sep_fc(const SepJob *d_jobs, int n_jobs, int total_tiles, const float *A, const float *B,
                          const float *lam, const int *rank_off, int K, int R, int h, int w, cudaStream_t s)
{
#define TDPM_SEP(HH, WW) \
    sep_kernel<FC, HH, WW, TERMS><<<total_tiles, SQ_THREADS, 0, s>>>(d_jobs, n_jobs, A, B, lam, rank_off, K, R, h, w)
    if (h == 6 && w == 6) TDPM_SEP(6, 6);
    else if (h == 5 && w == 11) TDPM_SEP(5, 11);
    else if (h == 7 && w == 7) TDPM_SEP(7, 7);
    else if (h == 11 && w == 5) TDPM_SEP(11, 5);
    else TDPM_SEP(0, 0);
#undef TDPM_SEP
    return cudaGetLastError();
}

}  // namespace

int corr_f32_tile_x() { return CT_TX; }
int corr_f32_tile_y() { return CT_TY; }
int corr_f32_tile_k() { return CT_TK; }

cudaError_t launch_corr_f32(const CorrJob *d_jobs, int n_jobs, int total_tiles, const float *filt_t, int K, int Kpad,
                            int h, int w, cudaStream_t s)
{
    if (total_tiles <= 0) return cudaSuccess;
    const int plane = (CT_TY + h - 1) * (CT_TX + w - 1);
    const size_t smem = sizeof(float) * (((FD * plane + 3) & ~3) + CT_TAPS * FD * CT_TK);
    cudaError_t e = allow_max_dynamic_smem(reinterpret_cast<const void *>(corr_f32_kernel), 1);
    if (e != cudaSuccess) return e;
    note_launches(1);
    corr_f32_kernel<<<total_tiles, CT_THREADS, smem, s>>>(d_jobs, n_jobs, filt_t, K, Kpad, h, w);
    return cudaGetLastError();
}

int zproj_simt_cells_per_tile() { return ZP_CELLS; }
int zproj_simt_r_chunk() { return ZP_RCHUNK; }

cudaError_t launch_zproj_simt(const ZJob *d_jobs, int n_jobs, int total_tiles, const float *Ct, int R, cudaStream_t s)
{
    if (total_tiles <= 0) return cudaSuccess;
    note_launches(1);
    zproj_kernel<<<total_tiles, ZP_CELLS, 0, s>>>(d_jobs, n_jobs, Ct, R);
    return cudaGetLastError();
}

// The filter shapes with a compiled warp form of the per-filter mode.
bool sep_warp_shape(int h, int w)
{
    return (h == 6 && w == 6) || (h == 5 && w == 11) || (h == 7 && w == 7) || (h == 11 && w == 5);
}

bool sep_uses_warp_form(int mode, int h, int w) { return mode == SEP_PER_FILTER && sep_warp_shape(h, w); }

long long sep_job_items(int mode, int h, int w, int Ho, int Wo, int K, int *tiles_x, int *tiles_y)
{
    if (sep_uses_warp_form(mode, h, w)) {
        const int sw = 32 - (w - 1);
        *tiles_x = (Wo + sw - 1) / sw;
        *tiles_y = (Ho + SW_ROWS - 1) / SW_ROWS;
        return (long long)*tiles_x * *tiles_y * K;
    }
    *tiles_x = (Wo + SQ_T - 1) / SQ_T;
    *tiles_y = (Ho + SQ_T - 1) / SQ_T;
    const int fpc = mode == SEP_PER_FILTER ? 1 : SQ_FC_JOINT;
    return (long long)*tiles_x * *tiles_y * ((K + fpc - 1) / fpc);
}

cudaError_t launch_sep(const SepJob *d_jobs, int n_jobs, long long total_items, const float *A, const float *B,
                       const float *lam, const int *rank_off, int K, int R, int h, int w, int mode, cudaStream_t s)
{
    if (total_items <= 0) return cudaSuccess;
    if (h < 1 || h > SQ_MAXHW || w < 1 || w > SQ_MAXHW) return cudaErrorInvalidValue;
    if (mode == SEP_TERMS && (K % SQ_FC_JOINT != 0 || K < R)) return cudaErrorInvalidValue;
    note_launches(1);
    if (sep_uses_warp_form(mode, h, w)) {
        const unsigned blocks = (unsigned)((total_items + SW_WARPS - 1) / SW_WARPS);
#define TDPM_SEPW(HH, WW)                                                                                       \
    sep_warp_kernel<HH, WW><<<blocks, SW_WARPS * 32, 0, s>>>(d_jobs, n_jobs, total_items, A, B, lam, rank_off, K, R)
        if (h == 6 && w == 6) TDPM_SEPW(6, 6);
        else if (h == 5 && w == 11) TDPM_SEPW(5, 11);
        else if (h == 7 && w == 7) TDPM_SEPW(7, 7);
        else TDPM_SEPW(11, 5);
#undef TDPM_SEPW
        return cudaGetLastError();
    }
    if (total_items > 0x7fffffffll) return cudaErrorInvalidValue;
    const int total_tiles = (int)total_items;
    if (mode == SEP_TERMS)
        return launch_sep_fc<SQ_FC_JOINT, true>(d_jobs, n_jobs, total_tiles, A, B, lam, rank_off, K, R, h, w, s);
    if (mode == SEP_JOINT)
        return launch_sep_fc<SQ_FC_JOINT, false>(d_jobs, n_jobs, total_tiles, A, B, lam, rank_off, K, R, h, w, s);
    return launch_sep_fc<1, false>(d_jobs, n_jobs, total_tiles, A, B, lam, rank_off, K, R, h, w, s);
}

}  // namespace tdpm
