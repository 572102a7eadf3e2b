// The feature extraction block (Sec. 2): an image's 32-channel HOG pyramid on the device, in the DPM form the paper
// scores (Felzenszwalb et al., PAMI 2010, Sec. 6). Four stages, each one launch over every image or level of the
// pyramid:
//   resize    area-averaging resample (octave 0 from the 8-bit image at the lam scales 2^(-i/lam); each further
//             octave halves the previous one), with per-axis tap tables built on the host in FP64;
//   gradient  per pixel the colour channel with the largest squared central-difference gradient and the nearest of
//             18 oriented directions, both decided in FP32 with every product and sum rounded once (no contraction),
//             and the magnitude;
//   histogram per cell, a gather of the bilinear votes of the 2 sbin x 2 sbin pixels around it into 18 bins held in
//             shared memory (no atomics: each cell sums its votes in a fixed order);
//   features  per interior cell, the four block normalisations of its 3x3 neighbourhood's energies, truncation at 0.2
//             and the 18 + 9 + 4 (+ one zero) channel projection, written as FP32 NHWC levels ready for scoring.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "ctx.h"

namespace tdpm {
namespace {

constexpr float HOG_TRUNC = 0.2f;
constexpr float HOG_EPS = 1e-4f;
constexpr int HOG_HIST_THREADS = 128;

__constant__ float c_ux[9], c_uy[9];

// ------------------------------------------------------------------------------------------------------ resize
// out[y][x][c] = sum_t wy[t] sum_u wx[u] in[y0 + t][x0 + u][c], the taps of every output row and column from tables.
template <typename TIn>
__global__ void hog_resize_kernel(const HogResizeJob *__restrict__ jobs)
{
    const HogResizeJob J = jobs[blockIdx.y];
    const long long n = (long long)J.ho * J.wo;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int y = (int)(p / J.wo), x = (int)(p - (long long)y * J.wo);
    const HogTap ty = J.ytaps[y], tx = J.xtaps[x];
    const TIn *src = static_cast<const TIn *>(J.src);
    float acc[3] = {0.f, 0.f, 0.f};
    for (int t = 0; t < ty.n; ++t) {
        const float wy = J.weights[ty.w + t];
        float row[3] = {0.f, 0.f, 0.f};
        const TIn *s = src + ((size_t)(ty.i0 + t) * J.w + tx.i0) * 3;
        for (int u = 0; u < tx.n; ++u) {
            const float wx = J.weights[tx.w + u];
#pragma unroll
            for (int c = 0; c < 3; ++c) row[c] = fmaf(wx, (float)s[u * 3 + c], row[c]);
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[c] = fmaf(wy, row[c], acc[c]);
    }
    float *d = J.dst + (size_t)p * 3;
    d[0] = acc[0];
    d[1] = acc[1];
    d[2] = acc[2];
}

// ---------------------------------------------------------------------------------------------------- gradient
__global__ void hog_grad_kernel(const HogImage *__restrict__ imgs)
{
    const HogImage I = imgs[blockIdx.y];
    const long long n = (long long)I.h * I.w;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int y = (int)(p / I.w), x = (int)(p - (long long)y * I.w);
    float mag = 0.f;
    int bin = 0;
    if (x >= 1 && y >= 1 && x <= I.w - 2 && y <= I.h - 2) {
        const float *c0 = I.img + ((size_t)y * I.w + x) * 3;
        const long long row = (long long)I.w * 3;
        float bv = -1.f, gx = 0.f, gy = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float dx = __fsub_rn(c0[3 + c], c0[c - 3]);
            const float dy = __fsub_rn(c0[row + c], c0[(long long)c - row]);
            const float v = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
            if (v > bv) {  // strictly larger: the first channel wins ties
                bv = v;
                gx = dx;
                gy = dy;
            }
        }
        float best = 0.f;
#pragma unroll
        for (int o = 0; o < 9; ++o) {
            const float d = __fadd_rn(__fmul_rn(c_ux[o], gx), __fmul_rn(c_uy[o], gy));
            if (d > best) {
                best = d;
                bin = o;
            }
            if (-d > best) {
                best = -d;
                bin = o + 9;
            }
        }
        mag = sqrtf(bv);
    }
    I.mag[p] = mag;
    I.bin[p] = (uint8_t)bin;
}

// --------------------------------------------------------------------------------------------------- histogram
// 2 sbin threads per cell, one per row of the 2 sbin x 2 sbin pixels that vote into it: each sums its row's votes into
// its own 18 bins in shared memory ([bin][thread]: a warp's updates of one bin fall in distinct banks), then the rows
// are added in a fixed tree order and the first thread writes the cell's bins and its energy
// E = sum_{o<9} (h_o + h_{o+9})^2.
__global__ void __launch_bounds__(HOG_HIST_THREADS) hog_hist_kernel(const HogLevelJob *__restrict__ jobs)
{
    __shared__ float hs[18][HOG_HIST_THREADS];
    const HogLevelJob J = jobs[blockIdx.y];
    const int t = threadIdx.x;
    const int s = J.sbin, hs2 = s / 2, tpc = 2 * s;  // threads per cell (tpc divides the block)
    const int cpb = HOG_HIST_THREADS / tpc;
    const long long n_cells = (long long)J.cy * J.cx;
    if ((long long)blockIdx.x * cpb >= n_cells) return;  // uniform per block
    const int r = t % tpc;
    const long long cell = (long long)blockIdx.x * cpb + t / tpc;
#pragma unroll
    for (int o = 0; o < 18; ++o) hs[o][t] = 0.f;
    if (cell < n_cells) {
        const int Y = (int)(cell / J.cx), X = (int)(cell - (long long)Y * J.cx);
        const int y = Y * s - hs2 + r;
        if (y >= 1 && y <= J.cy * s - 2) {
            const float inv = 1.f / (float)s;  // s is a power of two: exact
            const float yp = ((float)y + 0.5f) * inv - 0.5f;
            const int iy = (int)floorf(yp);
            const float fy = yp - (float)iy;
            const float wy = iy == Y ? 1.f - fy : fy;
            const int yy = min(y, J.h - 2);
            const float *mrow = J.mag + (size_t)yy * J.w;
            const uint8_t *brow = J.bin + (size_t)yy * J.w;
            const int x_lo = max(1, X * s - hs2), x_hi = min(J.cx * s - 2, X * s + s + hs2 - 1);
            for (int x = x_lo; x <= x_hi; ++x) {
                const float xp = ((float)x + 0.5f) * inv - 0.5f;
                const int ix = (int)floorf(xp);
                const float fx = xp - (float)ix;
                const float wx = ix == X ? 1.f - fx : fx;
                const int xx = min(x, J.w - 2);
                hs[brow[xx]][t] += wy * wx * mrow[xx];
            }
        }
    }
    __syncthreads();
    for (int st = s; st >= 1; st >>= 1) {  // rows r and r + st of the same cell, in a fixed order
        if (r < st)
#pragma unroll
            for (int o = 0; o < 18; ++o) hs[o][t] += hs[o][t + st];
        __syncthreads();
    }
    if (r == 0 && cell < n_cells) {
        float *out = J.hist + (size_t)cell * 18;
        float e = 0.f;
#pragma unroll
        for (int o = 0; o < 18; ++o) out[o] = hs[o][t];
#pragma unroll
        for (int o = 0; o < 9; ++o) {
            const float v = hs[o][t] + hs[o + 9][t];
            e = fmaf(v, v, e);
        }
        J.energy[cell] = e;
    }
}

// ---------------------------------------------------------------------------------------------------- features
__global__ void hog_feat_kernel(const HogLevelJob *__restrict__ jobs)
{
    const HogLevelJob J = jobs[blockIdx.y];
    const int oy = J.cy - 2, ox = J.cx - 2;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (oy <= 0 || ox <= 0 || p >= (long long)oy * ox) return;
    const int y = (int)(p / ox), x = (int)(p - (long long)y * ox);
    const int Y = y + 1, X = x + 1;
    float E[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) E[a][b] = J.energy[(size_t)(Y - 1 + a) * J.cx + (X - 1 + b)];
    // blocks with top-left corner (Y, X), (Y, X - 1), (Y - 1, X), (Y - 1, X - 1)
    float n[4];
    n[0] = rsqrtf(E[1][1] + E[1][2] + E[2][1] + E[2][2] + HOG_EPS);
    n[1] = rsqrtf(E[1][0] + E[1][1] + E[2][0] + E[2][1] + HOG_EPS);
    n[2] = rsqrtf(E[0][1] + E[0][2] + E[1][1] + E[1][2] + HOG_EPS);
    n[3] = rsqrtf(E[0][0] + E[0][1] + E[1][0] + E[1][1] + HOG_EPS);
    float h[18];
    {
        const float2 *h2 = reinterpret_cast<const float2 *>(J.hist + ((size_t)Y * J.cx + X) * 18);
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const float2 v = h2[q];
            h[2 * q] = v.x;
            h[2 * q + 1] = v.y;
        }
    }
    float f[32];
    float tex[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int o = 0; o < 18; ++o) {
        const float v = h[o];
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float t = fminf(v * n[k], HOG_TRUNC);
            acc += t;
            tex[k] += t;
        }
        f[o] = 0.5f * acc;
    }
#pragma unroll
    for (int o = 0; o < 9; ++o) {
        const float v = h[o] + h[o + 9];
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < 4; ++k) acc += fminf(v * n[k], HOG_TRUNC);
        f[18 + o] = 0.5f * acc;
    }
    const float inv_sqrt18 = 0.23570226039551584f;  // 1 / sqrt(18)
#pragma unroll
    for (int k = 0; k < 4; ++k) f[27 + k] = tex[k] * inv_sqrt18;
    f[31] = 0.f;
    float4 *d = reinterpret_cast<float4 *>(J.out + (size_t)p * 32);
#pragma unroll
    for (int q = 0; q < 8; ++q) d[q] = make_float4(f[4 * q], f[4 * q + 1], f[4 * q + 2], f[4 * q + 3]);
}

}  // namespace

cudaError_t hog_set_orientations(const float *ux, const float *uy)
{
    cudaError_t e = cudaMemcpyToSymbol(c_ux, ux, sizeof(float) * 9);
    return e == cudaSuccess ? cudaMemcpyToSymbol(c_uy, uy, sizeof(float) * 9) : e;
}

cudaError_t launch_hog_resize(const HogResizeJob *d_jobs, int n_jobs, long long max_pixels, bool from_u8,
                              cudaStream_t s)
{
    if (n_jobs <= 0 || max_pixels <= 0) return cudaSuccess;
    const dim3 grid((unsigned)((max_pixels + 255) / 256), (unsigned)n_jobs);
    note_launches(1);
    if (from_u8) hog_resize_kernel<uint8_t><<<grid, 256, 0, s>>>(d_jobs);
    else hog_resize_kernel<float><<<grid, 256, 0, s>>>(d_jobs);
    return cudaGetLastError();
}

int hog_hist_blocks(int cy, int cx, int sbin)
{
    const long long cpb = HOG_HIST_THREADS / (2 * sbin);
    return (int)(((long long)cy * cx + cpb - 1) / cpb);
}

cudaError_t launch_hog_grad(const HogImage *d_imgs, int n_imgs, long long max_pixels, cudaStream_t s)
{
    if (n_imgs <= 0 || max_pixels <= 0) return cudaSuccess;
    note_launches(1);
    hog_grad_kernel<<<dim3((unsigned)((max_pixels + 255) / 256), (unsigned)n_imgs), 256, 0, s>>>(d_imgs);
    return cudaGetLastError();
}

cudaError_t launch_hog_levels(const HogLevelJob *d_jobs, int n_jobs, long long max_hist_blocks, long long max_out_cells,
                              cudaStream_t s)
{
    if (n_jobs <= 0) return cudaSuccess;
    note_launches(2);
    if (max_hist_blocks > 0)
        hog_hist_kernel<<<dim3((unsigned)max_hist_blocks, (unsigned)n_jobs), HOG_HIST_THREADS, 0, s>>>(d_jobs);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || max_out_cells <= 0) return e;
    hog_feat_kernel<<<dim3((unsigned)((max_out_cells + 127) / 128), (unsigned)n_jobs), 128, 0, s>>>(d_jobs);
    return cudaGetLastError();
}

}  // namespace tdpm

namespace tdpm {

// ================================================================================================== host side
namespace {

struct Bumper {
    size_t off = 0;
    size_t take(size_t bytes)
    {
        const size_t o = (off + 255) & ~(size_t)255;
        off = o + bytes;
        return o;
    }
};

int hog_cells(int n, int s) { return (2 * n + s) / (2 * s); }  // floor(n / s + 1/2)
int resized(int n, double s) { return (int)std::floor(n * s + 0.5); }

struct HogPlanH {
    int lam = 0;
    std::vector<std::pair<int, int>> img;  // image sizes; image k * lam + i is octave k, scale step i
    std::vector<int> lvl_img, lvl_sbin;
};

// Levels of the pyramid: lam part levels (sbin / 2 on octave 0), then root levels (sbin) octave by octave while both
// sides keep at least min_cells cells.
tdpm_status hog_plan(int H, int W, int sbin, int lam, int min_cells, HogPlanH &P)
{
    if (H < 16 || W < 16 || H > 16384 || W > 16384) return fail(TDPM_ERR_ARG, "image sides must be in [16, 16384]");
    if (sbin != 4 && sbin != 8 && sbin != 16) return fail(TDPM_ERR_ARG, "sbin must be 4, 8 or 16");
    if (lam < 1 || lam > 64) return fail(TDPM_ERR_ARG, "lambda must be in [1, 64]");
    if (min_cells < 1 || min_cells > 4096) return fail(TDPM_ERR_ARG, "min_cells must be in [1, 4096]");
    P = HogPlanH{};
    P.lam = lam;
    for (int i = 0; i < lam; ++i) {
        const double sc = std::pow(2.0, -(double)i / lam);
        P.img.push_back(i == 0 ? std::make_pair(H, W) : std::make_pair(resized(H, sc), resized(W, sc)));
    }
    for (int i = 0; i < lam; ++i) {
        P.lvl_img.push_back(i);
        P.lvl_sbin.push_back(sbin / 2);
    }
    int last = lam - 1;
    bool done = false;
    for (int k = 0; k < 32 && !done; ++k)
        for (int i = 0; i < lam; ++i) {
            const int idx = k * lam + i;
            if (idx >= (int)P.img.size()) {
                const auto &src = P.img[idx - lam];
                P.img.push_back({resized(src.first, 0.5), resized(src.second, 0.5)});
            }
            const auto &hw = P.img[idx];
            if (hw.first < 3 || hw.second < 3 || hog_cells(hw.first, sbin) - 2 < min_cells ||
                hog_cells(hw.second, sbin) - 2 < min_cells) {
                done = true;
                break;
            }
            P.lvl_img.push_back(idx);
            P.lvl_sbin.push_back(sbin);
            last = std::max(last, idx);
        }
    if ((int)P.lvl_img.size() == lam) return fail(TDPM_ERR_ARG, "image too small for one root level");
    P.img.resize(last + 1);
    for (int j = 0; j < lam; ++j) {
        const auto &hw = P.img[j];
        if (hog_cells(hw.first, sbin / 2) - 2 < 1 || hog_cells(hw.second, sbin / 2) - 2 < 1)
            return fail(TDPM_ERR_ARG, "image too small for the part levels");
    }
    return TDPM_OK;
}

void level_shape(const HogPlanH &P, int j, int &cy, int &cx)
{
    const auto &hw = P.img[P.lvl_img[j]];
    cy = hog_cells(hw.first, P.lvl_sbin[j]);
    cx = hog_cells(hw.second, P.lvl_sbin[j]);
}

// Taps of one axis resampled by s (area averaging; weights normalised over the covered part of each interval).
void axis_taps(int n_in, int n_out, double s, std::vector<HogTap> &T, std::vector<float> &Wt)
{
    T.clear();
    for (int j = 0; j < n_out; ++j) {
        const double a = j / s, b = std::min((j + 1) / s, (double)n_in);
        HogTap t{(int)std::floor(a), 0, (int)Wt.size()};
        std::vector<double> ov;
        for (int i = (int)std::floor(a); i < (int)std::ceil(b); ++i) {
            const double o = std::min(b, i + 1.0) - std::max(a, (double)i);
            if (o > 0.0) ov.push_back(o);
            else if (ov.empty()) t.i0 = i + 1;
        }
        double sum = 0.0;
        for (double o : ov) sum += o;
        for (double o : ov) Wt.push_back((float)(o / sum));
        t.n = (int)ov.size();
        T.push_back(t);
    }
}

// Drops the cached pyramid tables and graph (the scratch is about to change).
void hog_forget(tdpm_ctx *ctx)
{
    ctx->hog_key.clear();
    if (ctx->hog_graph) cudaGraphExecDestroy(ctx->hog_graph);
    ctx->hog_graph = nullptr;
    ctx->hog_graph_kernels = 0;
    ctx->hog_uses = 0;
}

tdpm_status hog_prepare(tdpm_ctx *ctx, cudaStream_t s, size_t need, char *&base)
{
    static std::atomic<bool> orient_set[64];
    int dev = ctx->device;
    if (dev >= 0 && dev < 64 && !orient_set[dev].load()) {
        float ux[9], uy[9];
        for (int o = 0; o < 9; ++o) {
            ux[o] = (float)std::cos(o * M_PI / 9.0);
            uy[o] = (float)std::sin(o * M_PI / 9.0);
        }
        CUDA_TRY(hog_set_orientations(ux, uy));
        orient_set[dev].store(true);
    }
    if (!ctx->hog_done) CUDA_TRY(cudaEventCreateWithFlags(&ctx->hog_done, cudaEventDisableTiming));
    else CUDA_TRY(cudaStreamWaitEvent(s, ctx->hog_done, 0));  // the previous call's work has left the scratch
    if (need > ctx->hog_cap) {
        if (ctx->d_hog) {
            CUDA_TRY(cudaEventSynchronize(ctx->hog_done));
            cudaFree(ctx->d_hog);
            ctx->used -= std::min(ctx->used, ctx->hog_cap);
            ctx->d_hog = nullptr;
            ctx->hog_cap = 0;
        }
        if (ctx->budget && ctx->used + need > ctx->budget) return fail(TDPM_ERR_OOM, "HOG scratch exceeds the budget");
        CUDA_TRY(cudaMalloc(&ctx->d_hog, need));
        ctx->hog_cap = need;
        ctx->used += need;
        hog_forget(ctx);
    }
    base = static_cast<char *>(ctx->d_hog);
    return TDPM_OK;
}

}  // namespace

}  // namespace tdpm

using namespace tdpm;

tdpm_status tdpm_hog_pyramid_shape(int32_t img_h, int32_t img_w, int32_t sbin, int32_t lambda, int32_t min_cells,
                                   int32_t *n_levels, int32_t *level_hw, int32_t max_levels, size_t *out_bytes)
{
    clear_error();
    if (!n_levels || !out_bytes) return fail(TDPM_ERR_ARG, "NULL argument");
    HogPlanH P;
    tdpm_status st = hog_plan(img_h, img_w, sbin, lambda, min_cells, P);
    if (st) return st;
    const int L = (int)P.lvl_img.size();
    *n_levels = L;
    size_t bytes = 0;
    for (int j = 0; j < L; ++j) {
        int cy, cx;
        level_shape(P, j, cy, cx);
        if (level_hw && j < max_levels) {
            level_hw[2 * j] = cy - 2;
            level_hw[2 * j + 1] = cx - 2;
        }
        bytes += (size_t)(cy - 2) * (cx - 2) * 32 * sizeof(float);
    }
    *out_bytes = bytes;
    if (level_hw && max_levels < L) return fail(TDPM_ERR_CAPACITY, "more levels than max_levels");
    return TDPM_OK;
}

namespace {

// Device layout of one pyramid call inside the scratch: images, gradients, cell histograms, then the tables (resize
// jobs, images, levels first, so that their offsets follow from the plan alone; then the taps and their weights).
struct HogLayout {
    std::vector<size_t> img_off, mag_off, bin_off, hist_off, energy_off;
    size_t rj_off = 0, im_off = 0, lv_off = 0, taps_off = 0, bytes_fixed = 0;
    long long max_px = 0, max_hist_blocks = 0, max_out = 0;
    std::vector<long long> oct_max;  // per octave: the largest image
};

HogLayout hog_layout(const HogPlanH &P)
{
    const int NI = (int)P.img.size(), L = (int)P.lvl_img.size();
    HogLayout Y;
    Bumper b;
    Y.img_off.resize(NI);
    Y.mag_off.resize(NI);
    Y.bin_off.resize(NI);
    Y.hist_off.resize(L);
    Y.energy_off.resize(L);
    for (int k = 0; k < NI; ++k) Y.img_off[k] = b.take(sizeof(float) * 3 * (size_t)P.img[k].first * P.img[k].second);
    for (int k = 0; k < NI; ++k) Y.mag_off[k] = b.take(sizeof(float) * (size_t)P.img[k].first * P.img[k].second);
    for (int k = 0; k < NI; ++k) Y.bin_off[k] = b.take((size_t)P.img[k].first * P.img[k].second);
    for (int j = 0; j < L; ++j) {
        int cy, cx;
        level_shape(P, j, cy, cx);
        Y.hist_off[j] = b.take(sizeof(float) * 18 * (size_t)cy * cx);
        Y.energy_off[j] = b.take(sizeof(float) * (size_t)cy * cx);
        Y.max_hist_blocks = std::max(Y.max_hist_blocks, (long long)hog_hist_blocks(cy, cx, P.lvl_sbin[j]));
        Y.max_out = std::max(Y.max_out, (long long)(cy - 2) * (cx - 2));
    }
    Y.rj_off = b.take(sizeof(HogResizeJob) * NI);
    Y.im_off = b.take(sizeof(HogImage) * NI);
    Y.lv_off = b.take(sizeof(HogLevelJob) * L);
    Y.taps_off = b.take(0);
    Y.bytes_fixed = Y.taps_off;
    for (int k = 0; k < NI; ++k) {
        const long long px = (long long)P.img[k].first * P.img[k].second;
        Y.max_px = std::max(Y.max_px, px);
        const size_t oct = (size_t)(k / P.lam);
        if (Y.oct_max.size() <= oct) Y.oct_max.push_back(0);
        Y.oct_max[oct] = std::max(Y.oct_max[oct], px);
    }
    return Y;
}

// The pyramid's launches: octave 0 from the 8-bit image, each further octave from the previous one, gradients of
// every image, cells and features of every level.
cudaError_t hog_enqueue(const HogPlanH &P, const HogLayout &Y, char *base, cudaStream_t s)
{
    const int NI = (int)P.img.size(), L = (int)P.lvl_img.size();
    const auto *d_rj = reinterpret_cast<const HogResizeJob *>(base + Y.rj_off);
    cudaError_t e = launch_hog_resize(d_rj, std::min(NI, P.lam), Y.oct_max[0], true, s);
    for (int k0 = P.lam, oct = 1; e == cudaSuccess && k0 < NI; k0 += P.lam, ++oct)
        e = launch_hog_resize(d_rj + k0, std::min(P.lam, NI - k0), Y.oct_max[oct], false, s);
    if (e == cudaSuccess) e = launch_hog_grad(reinterpret_cast<const HogImage *>(base + Y.im_off), NI, Y.max_px, s);
    if (e == cudaSuccess)
        e = launch_hog_levels(reinterpret_cast<const HogLevelJob *>(base + Y.lv_off), L, Y.max_hist_blocks, Y.max_out,
                              s);
    return e;
}

}  // namespace

tdpm_status tdpm_hog_pyramid(tdpm_ctx *ctx, const uint8_t *d_image, int32_t img_h, int32_t img_w, int32_t sbin,
                             int32_t lambda, int32_t min_cells, float *d_out, size_t out_bytes, tdpm_level *levels,
                             int32_t max_levels, int32_t *n_levels, void *stream)
{
    clear_error();
    if (!ctx || !d_image || !d_out || !levels || !n_levels) return fail(TDPM_ERR_ARG, "NULL argument");
    if (reinterpret_cast<uintptr_t>(d_out) % 16) return fail(TDPM_ERR_ARG, "d_out must be 16-byte aligned");
    HogPlanH P;
    tdpm_status st = hog_plan(img_h, img_w, sbin, lambda, min_cells, P);
    if (st) return st;
    const int L = (int)P.lvl_img.size(), NI = (int)P.img.size();
    *n_levels = L;
    if (max_levels < L) return fail(TDPM_ERR_CAPACITY, "more levels than max_levels");
    std::vector<size_t> out_off(L);
    size_t need_out = 0;
    for (int j = 0; j < L; ++j) {
        int cy, cx;
        level_shape(P, j, cy, cx);
        out_off[j] = need_out;
        levels[j].H = cy - 2;
        levels[j].W = cx - 2;
        levels[j].data = d_out + need_out / sizeof(float);
        need_out += (size_t)(cy - 2) * (cx - 2) * 32 * sizeof(float);
    }
    if (out_bytes < need_out) return fail(TDPM_ERR_CAPACITY, "d_out holds " + std::to_string(out_bytes) +
                                                                   " bytes, the pyramid needs " + std::to_string(need_out));
    std::lock_guard<std::mutex> lk(ctx->mu);
    if ((st = set_device(ctx))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const HogLayout Y = hog_layout(P);
    const std::string key = std::to_string(img_h) + "x" + std::to_string(img_w) + ":" + std::to_string(sbin) + ":" +
                            std::to_string(lambda) + ":" + std::to_string(min_cells) + ":" +
                            std::to_string(reinterpret_cast<uintptr_t>(d_image)) + ":" +
                            std::to_string(reinterpret_cast<uintptr_t>(d_out));
    if (!ctx->hog_key.empty() && key == ctx->hog_key && ctx->d_hog) {
        // the same call again: the tables on the device are current; from the second repeat on, one graph launch
        char *base = static_cast<char *>(ctx->d_hog);
        CUDA_TRY(cudaStreamWaitEvent(s, ctx->hog_done, 0));
        if (!ctx->hog_graph && ctx->hog_uses >= 2 && ctx->use_graphs) {
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                int captured = 0;
                t_capture_launches = &captured;
                const cudaError_t eq = hog_enqueue(P, Y, base, ctx->cap_stream);
                t_capture_launches = nullptr;
                e = cudaStreamEndCapture(ctx->cap_stream, &g);
                if (eq != cudaSuccess) e = eq;
                ctx->hog_graph_kernels = captured;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&ctx->hog_graph, g, 0);
            if (g) cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                cudaGetLastError();
                ctx->hog_graph = nullptr;
            }
        }
        if (ctx->hog_graph) {
            CUDA_TRY(cudaGraphLaunch(ctx->hog_graph, s));
            note_launches(ctx->hog_graph_kernels);
        } else {
            CUDA_TRY(hog_enqueue(P, Y, base, s));
        }
        ctx->hog_uses++;
        CUDA_TRY(cudaEventRecord(ctx->hog_done, s));
        return TDPM_OK;
    }
    // host tables: resize jobs with their taps, images, levels
    std::vector<HogResizeJob> rj(NI);
    std::vector<HogTap> taps_all;
    std::vector<float> wts;
    std::vector<size_t> ytap_off(NI), xtap_off(NI);
    for (int k = 0; k < NI; ++k) {
        const int oct = k / P.lam, i = k % P.lam;
        const double sc = oct == 0 ? (i == 0 ? 1.0 : std::pow(2.0, -(double)i / P.lam)) : 0.5;
        const int hin = oct == 0 ? img_h : P.img[k - P.lam].first, win = oct == 0 ? img_w : P.img[k - P.lam].second;
        std::vector<HogTap> T;
        ytap_off[k] = taps_all.size();
        axis_taps(hin, P.img[k].first, sc, T, wts);
        taps_all.insert(taps_all.end(), T.begin(), T.end());
        xtap_off[k] = taps_all.size();
        axis_taps(win, P.img[k].second, sc, T, wts);
        taps_all.insert(taps_all.end(), T.begin(), T.end());
        rj[k].h = hin;
        rj[k].w = win;
        rj[k].ho = P.img[k].first;
        rj[k].wo = P.img[k].second;
    }
    const size_t w_off = align256(Y.taps_off + sizeof(HogTap) * taps_all.size());
    const size_t total = w_off + sizeof(float) * wts.size();
    char *base = nullptr;
    hog_forget(ctx);
    if ((st = hog_prepare(ctx, s, total, base))) return st;
    std::vector<HogImage> im(NI);
    for (int k = 0; k < NI; ++k) {
        rj[k].src = k < P.lam ? static_cast<const void *>(d_image) : static_cast<const void *>(base + Y.img_off[k - P.lam]);
        rj[k].dst = reinterpret_cast<float *>(base + Y.img_off[k]);
        rj[k].ytaps = reinterpret_cast<const HogTap *>(base + Y.taps_off) + ytap_off[k];
        rj[k].xtaps = reinterpret_cast<const HogTap *>(base + Y.taps_off) + xtap_off[k];
        rj[k].weights = reinterpret_cast<const float *>(base + w_off);
        im[k] = HogImage{rj[k].dst, P.img[k].first, P.img[k].second, reinterpret_cast<float *>(base + Y.mag_off[k]),
                         reinterpret_cast<uint8_t *>(base + Y.bin_off[k])};
    }
    std::vector<HogLevelJob> lj(L);
    for (int j = 0; j < L; ++j) {
        const int k = P.lvl_img[j];
        int cy, cx;
        level_shape(P, j, cy, cx);
        lj[j] = HogLevelJob{im[k].mag, im[k].bin, P.img[k].first, P.img[k].second, P.lvl_sbin[j], cy, cx,
                            reinterpret_cast<float *>(base + Y.hist_off[j]),
                            reinterpret_cast<float *>(base + Y.energy_off[j]), d_out + out_off[j] / sizeof(float)};
    }
    // one transfer of every table, from pinned memory when the context has room for it
    std::vector<char> blob(total - Y.rj_off);
    std::memcpy(blob.data() + (Y.rj_off - Y.rj_off), rj.data(), sizeof(HogResizeJob) * NI);
    std::memcpy(blob.data() + (Y.im_off - Y.rj_off), im.data(), sizeof(HogImage) * NI);
    std::memcpy(blob.data() + (Y.lv_off - Y.rj_off), lj.data(), sizeof(HogLevelJob) * L);
    if (!taps_all.empty())
        std::memcpy(blob.data() + (Y.taps_off - Y.rj_off), taps_all.data(), sizeof(HogTap) * taps_all.size());
    if (!wts.empty()) std::memcpy(blob.data() + (w_off - Y.rj_off), wts.data(), sizeof(float) * wts.size());
    CUDA_TRY(cudaMemcpyAsync(base + Y.rj_off, blob.data(), blob.size(), cudaMemcpyHostToDevice, s));
    CUDA_TRY(hog_enqueue(P, Y, base, s));
    CUDA_TRY(cudaEventRecord(ctx->hog_done, s));
    ctx->hog_key = key;
    ctx->hog_uses = 1;
    return TDPM_OK;
}

tdpm_status tdpm_hog_features(tdpm_ctx *ctx, const float *d_img, int32_t h, int32_t w, int32_t sbin, float *d_out,
                              size_t out_bytes, int32_t *out_h, int32_t *out_w, void *stream)
{
    clear_error();
    if (!ctx || !d_img || !d_out || !out_h || !out_w) return fail(TDPM_ERR_ARG, "NULL argument");
    if (h < 3 || w < 3 || h > 16384 || w > 16384) return fail(TDPM_ERR_ARG, "image sides must be in [3, 16384]");
    if (sbin != 2 && sbin != 4 && sbin != 8 && sbin != 16) return fail(TDPM_ERR_ARG, "sbin must be 2, 4, 8 or 16");
    if (reinterpret_cast<uintptr_t>(d_out) % 16) return fail(TDPM_ERR_ARG, "d_out must be 16-byte aligned");
    const int cy = hog_cells(h, sbin), cx = hog_cells(w, sbin);
    *out_h = std::max(cy - 2, 0);
    *out_w = std::max(cx - 2, 0);
    const size_t need_out = (size_t)(*out_h) * (*out_w) * 32 * sizeof(float);
    if (out_bytes < need_out) return fail(TDPM_ERR_CAPACITY, "d_out too small");
    if (cy < 1 || cx < 1) return TDPM_OK;
    std::lock_guard<std::mutex> lk(ctx->mu);
    tdpm_status st = set_device(ctx);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    Bumper b;
    const size_t mag_off = b.take(sizeof(float) * (size_t)h * w), bin_off = b.take((size_t)h * w),
                 hist_off = b.take(sizeof(float) * 18 * (size_t)cy * cx),
                 energy_off = b.take(sizeof(float) * (size_t)cy * cx), im_off = b.take(sizeof(HogImage)),
                 lv_off = b.take(sizeof(HogLevelJob));
    char *base = nullptr;
    hog_forget(ctx);
    if ((st = hog_prepare(ctx, s, b.off, base))) return st;
    HogImage im{d_img, h, w, reinterpret_cast<float *>(base + mag_off), reinterpret_cast<uint8_t *>(base + bin_off)};
    HogLevelJob lj{im.mag, im.bin, h, w, sbin, cy, cx, reinterpret_cast<float *>(base + hist_off),
                   reinterpret_cast<float *>(base + energy_off), d_out};
    char blob[512];
    static_assert(sizeof(HogImage) + sizeof(HogLevelJob) + 256 <= sizeof(blob), "blob");
    std::memcpy(blob, &im, sizeof im);
    std::memcpy(blob + (lv_off - im_off), &lj, sizeof lj);
    CUDA_TRY(cudaMemcpyAsync(base + im_off, blob, lv_off - im_off + sizeof lj, cudaMemcpyHostToDevice, s));
    CUDA_TRY(launch_hog_grad(reinterpret_cast<const HogImage *>(base + im_off), 1, (long long)h * w, s));
    CUDA_TRY(launch_hog_levels(reinterpret_cast<const HogLevelJob *>(base + lv_off), 1, hog_hist_blocks(cy, cx, sbin),
                               (long long)(*out_h) * (*out_w), s));
    CUDA_TRY(cudaEventRecord(ctx->hog_done, s));
    CUDA_TRY(cudaStreamSynchronize(s));  // the blob above lives on this stack frame
    return TDPM_OK;
}

tdpm_status tdpm_resize(tdpm_ctx *ctx, const float *d_src, int32_t h, int32_t w, double scale, float *d_dst,
                        size_t dst_bytes, int32_t *out_h, int32_t *out_w, void *stream)
{
    clear_error();
    if (!ctx || !d_src || !d_dst || !out_h || !out_w) return fail(TDPM_ERR_ARG, "NULL argument");
    if (!(scale > 0.0 && scale <= 1.0)) return fail(TDPM_ERR_ARG, "scale must be in (0, 1]");
    if (h < 1 || w < 1 || h > 16384 || w > 16384) return fail(TDPM_ERR_ARG, "image sides must be in [1, 16384]");
    const int ho = resized(h, scale), wo = resized(w, scale);
    *out_h = ho;
    *out_w = wo;
    if (ho < 1 || wo < 1) return fail(TDPM_ERR_ARG, "the resized image is empty");
    if (dst_bytes < sizeof(float) * 3 * (size_t)ho * wo) return fail(TDPM_ERR_CAPACITY, "d_dst too small");
    std::lock_guard<std::mutex> lk(ctx->mu);
    tdpm_status st = set_device(ctx);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<HogTap> ty, tx;
    std::vector<float> wts;
    axis_taps(h, ho, scale, ty, wts);
    axis_taps(w, wo, scale, tx, wts);
    Bumper b;
    const size_t j_off = b.take(sizeof(HogResizeJob)), ty_off = b.take(sizeof(HogTap) * ty.size()),
                 tx_off = b.take(sizeof(HogTap) * tx.size()), w_off = b.take(sizeof(float) * wts.size());
    char *base = nullptr;
    hog_forget(ctx);
    if ((st = hog_prepare(ctx, s, b.off, base))) return st;
    HogResizeJob J{d_src, h, w, d_dst, ho, wo, reinterpret_cast<const HogTap *>(base + ty_off),
                   reinterpret_cast<const HogTap *>(base + tx_off), reinterpret_cast<const float *>(base + w_off)};
    std::vector<char> blob(b.off);
    std::memcpy(blob.data() + j_off, &J, sizeof J);
    std::memcpy(blob.data() + ty_off, ty.data(), sizeof(HogTap) * ty.size());
    std::memcpy(blob.data() + tx_off, tx.data(), sizeof(HogTap) * tx.size());
    std::memcpy(blob.data() + w_off, wts.data(), sizeof(float) * wts.size());
    CUDA_TRY(cudaMemcpyAsync(base, blob.data(), blob.size(), cudaMemcpyHostToDevice, s));
    CUDA_TRY(launch_hog_resize(reinterpret_cast<const HogResizeJob *>(base + j_off), 1, (long long)ho * wo, false, s));
    CUDA_TRY(cudaEventRecord(ctx->hog_done, s));
    return TDPM_OK;
}
