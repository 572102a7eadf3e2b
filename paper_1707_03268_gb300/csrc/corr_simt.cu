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

__device__ __forceinline__ float bf16_to_f32(uint16_t v) { return __uint_as_float(((uint32_t)v) << 16); }

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
// One thread per cell, ZP_RCHUNK projections per CTA: z_r = sum_c C[c][r] phi[cell][c].
constexpr int ZP_CELLS = 128, ZP_RCHUNK = 64;

__global__ void __launch_bounds__(ZP_CELLS) zproj_kernel(const ZJob *__restrict__ jobs, int n_jobs,
                                                         const float *__restrict__ Ct, int R, int bf16)
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
        if (bf16) {
            const uint4 *src = reinterpret_cast<const uint4 *>(J.feat_bf + (size_t)cell * FD);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const uint4 u = __ldg(src + i);
                const uint32_t wv[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    f[i * 8 + 2 * j] = bf16_to_f32((uint16_t)(wv[j] & 0xffffu));
                    f[i * 8 + 2 * j + 1] = bf16_to_f32((uint16_t)(wv[j] >> 16));
                }
            }
        } else {
            const float4 *src = reinterpret_cast<const float4 *>(J.feat + (size_t)cell * FD);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const float4 v = __ldg(src + i);
                f[4 * i] = v.x; f[4 * i + 1] = v.y; f[4 * i + 2] = v.z; f[4 * i + 3] = v.w;
            }
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
// CTA tile: SP_TY x SP_TX output positions, one per thread, for FC filters. For every rank-1 term r the CTA stages
// the Z_r halo, runs the y pass with a_r into shared memory, the x pass with b_r in registers, and adds
// Lambda[k][r] * U_r to each filter's accumulator.
constexpr int SP_TX = 32, SP_TY = 8, SP_THREADS = SP_TX * SP_TY, SP_FC_JOINT = 16, SP_MAXHW = 16;

template <int FC>
__global__ void __launch_bounds__(SP_THREADS) sep_kernel(const SepJob *__restrict__ jobs, int n_jobs,
                                                         const float *__restrict__ A, const float *__restrict__ B,
                                                         const float *__restrict__ lam,
                                                         const int *__restrict__ rank_off, int K, int R, int h, int w)
{
    extern __shared__ __align__(16) float sm[];
    const int HX = SP_TX + w - 1, HY = SP_TY + h - 1;
    float *zh = sm;                // [HY][HX]
    float *th = zh + HY * HX;      // [SP_TY][HX]
    float *co = th + SP_TY * HX;   // a[h], b[w], lam[FC]

    const int ji = find_job(jobs, n_jobs, blockIdx.x);
    const SepJob J = jobs[ji];
    int local = blockIdx.x - J.begin;
    const int f_chunks = (FC == 1) ? K : (K + FC - 1) / FC;
    const int fc = local % f_chunks;
    local /= f_chunks;
    const int x0 = (local % J.tiles_x) * SP_TX, y0 = (local / J.tiles_x) * SP_TY;
    const int k0 = fc * FC;
    int r_begin = 0, r_end = R;
    if (FC == 1) { r_begin = rank_off[k0]; r_end = rank_off[k0 + 1]; }

    const int tx = threadIdx.x % SP_TX, ty = threadIdx.x / SP_TX;
    const size_t plane = (size_t)J.H * J.W;
    float acc[FC];
#pragma unroll
    for (int f = 0; f < FC; ++f) acc[f] = 0.f;

    for (int r = r_begin; r < r_end; ++r) {
        __syncthreads();
        const float *Zr = J.Z + (size_t)r * plane;
        for (int i = threadIdx.x; i < HY * HX; i += SP_THREADS) {
            const int yy = i / HX, xx = i - yy * HX;
            const int gy = y0 + yy, gx = x0 + xx;
            zh[i] = (gy < J.H && gx < J.W) ? __ldg(Zr + (size_t)gy * J.W + gx) : 0.f;
        }
        if (threadIdx.x < h) co[threadIdx.x] = A[threadIdx.x * R + r];
        else if (threadIdx.x < h + w) co[threadIdx.x] = B[(threadIdx.x - h) * R + r];
        else if (threadIdx.x < h + w + FC) {
            const int f = threadIdx.x - h - w;
            co[threadIdx.x] = (FC == 1) ? lam[r] : ((k0 + f < K) ? lam[(size_t)(k0 + f) * R + r] : 0.f);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < SP_TY * HX; i += SP_THREADS) {
            const int yy = i / HX, xx = i - yy * HX;
            float t = 0.f;
            for (int dy = 0; dy < h; ++dy) t = fmaf(co[dy], zh[(yy + dy) * HX + xx], t);
            th[i] = t;
        }
        __syncthreads();
        float u = 0.f;
        for (int dx = 0; dx < w; ++dx) u = fmaf(co[h + dx], th[ty * HX + tx + dx], u);
#pragma unroll
        for (int f = 0; f < FC; ++f) acc[f] = fmaf(co[h + w + f], u, acc[f]);
    }
    const int y = y0 + ty, x = x0 + tx;
    if (y >= J.Ho || x >= J.Wo) return;
#pragma unroll
    for (int f = 0; f < FC; ++f)
        if (k0 + f < K) J.out[((size_t)(k0 + f) * J.Ho + y) * J.Wo + x] = acc[f];
}

__global__ void to_bf16_kernel(const float *__restrict__ src, uint16_t *__restrict__ dst, long long n)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        __nv_bfloat16 b = __float2bfloat16_rn(src[i]);
        dst[i] = *reinterpret_cast<uint16_t *>(&b);
    }
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
    cudaError_t e = cudaFuncSetAttribute(corr_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    note_launches(1);
    corr_f32_kernel<<<total_tiles, CT_THREADS, smem, s>>>(d_jobs, n_jobs, filt_t, K, Kpad, h, w);
    return cudaGetLastError();
}

int zproj_simt_cells_per_tile() { return ZP_CELLS; }
int zproj_simt_r_chunk() { return ZP_RCHUNK; }

cudaError_t launch_zproj_simt(const ZJob *d_jobs, int n_jobs, int total_tiles, const float *Ct, int R, bool bf16_feat,
                              cudaStream_t s)
{
    if (total_tiles <= 0) return cudaSuccess;
    note_launches(1);
    zproj_kernel<<<total_tiles, ZP_CELLS, 0, s>>>(d_jobs, n_jobs, Ct, R, bf16_feat ? 1 : 0);
    return cudaGetLastError();
}

int sep_tile_x() { return SP_TX; }
int sep_tile_y() { return SP_TY; }
int sep_filters_per_cta(bool joint) { return joint ? SP_FC_JOINT : 1; }

cudaError_t launch_sep_simt(const SepJob *d_jobs, int n_jobs, int total_tiles, const float *A, const float *B,
                            const float *lam, const int *rank_off, int K, int R, int h, int w, bool joint,
                            cudaStream_t s)
{
    if (total_tiles <= 0) return cudaSuccess;
    if (h > SP_MAXHW || w > SP_MAXHW) return cudaErrorInvalidValue;
    const int HX = SP_TX + w - 1, HY = SP_TY + h - 1;
    const size_t smem = sizeof(float) * (HY * HX + SP_TY * HX + h + w + SP_FC_JOINT);
    note_launches(1);
    if (joint)
        sep_kernel<SP_FC_JOINT><<<total_tiles, SP_THREADS, smem, s>>>(d_jobs, n_jobs, A, B, lam, rank_off, K, R, h, w);
    else
        sep_kernel<1><<<total_tiles, SP_THREADS, smem, s>>>(d_jobs, n_jobs, A, B, lam, rank_off, K, R, h, w);
    return cudaGetLastError();
}

cudaError_t launch_to_bf16(const float *src, uint16_t *dst, long long n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    note_launches(1);
    to_bf16_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

}  // namespace tdpm
