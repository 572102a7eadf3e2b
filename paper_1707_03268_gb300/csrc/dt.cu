// Step 2: generalised distance transform with argmax (Sec. 2 argmax equation),
//   D[p] = max_q f[q] - (lin*(q-p) + quad*(q-p)^2),  the smallest maximising q,
// run as an x pass over every row of a part score map and a y pass over every sampled column of its result.
//
// The scan of one output p (dt_scan): the candidates q within +-DT_R0 of p are evaluated in increasing index order
// (the first strict maximum is the smallest maximiser), with the costs of those displacements taken once per line.
// Then the result is checked against the line maximum M: on each side, beyond the cost's vertex, a cost above
// (M - best) + margin at distance DT_R0 + 1 rules out every farther candidate (its f[q] - cost <= M - cost < best -
// margin). With DPM-like deformation costs most outputs finish there (away from the line ends the window needs no
// bounds checks); an output whose window is wider continues outward, four distances per step, over the window that
// its first result bounds (left candidates win ties, right ones must be strictly better). The margin covers FP32
// rounding of the evaluated values, so the result is the brute-force one.
//
// x pass: one CTA per (job, 8 rows), one warp per row: the row is staged in shared memory, and the lanes take the
//         sampled columns p = x_off + x_step*k; results V[y][k], IV[y][k] (row-major [H][nx]: the lanes of a warp
//         store contiguous words).
// y pass: one CTA per (job, 8 consecutive sampled columns): the 8 columns of V are staged transposed in shared
//         memory, one warp per column takes the sampled rows p = y_off + y_step*i, and the results are staged and
//         written back as rows of 8: D[i][k], A[i][k] = (qy << 16) | IV[qy][k].
// Both passes find their job with a 32-ary warp search (the jobs' xbegin / ybegin count CTAs).
//
// Fused form (dt_xy_kernel, the one the scoring path runs): one CTA per (job, strip of 32 sampled columns). The x pass
// (warp per row, the row staged in shared memory, lane = sampled column of the strip) writes V and IV column-major
// into shared memory (odd column stride: conflict-free), with per-warp column maxima; the y pass takes lane = column,
// warp = sampled row, so each warp writes 32 consecutive results. The intermediate never reaches device memory; the
// scans and line maxima are those of the two-pass form, so the results are identical.
#include "internal.h"

namespace tdpm {
namespace {

constexpr int DT_WARPS = 8;
constexpr int DT_R0 = 4;

// Candidate window [lo, hi] of output p for a line of length n with maximum mx.
__device__ __forceinline__ void dt_window(float lin, float quad, float mx, float fp, int p, int n, int &lo, int &hi)
{
    const float T = (mx - fp) + 1e-5f * (1.f + fabsf(mx) + fabsf(fp));
    const float s = sqrtf(fmaf(4.f * quad, T, lin * lin));
    const float inv = 0.5f / quad;
    const float dlo = (-lin - s) * inv, dhi = (-lin + s) * inv;
    lo = (dlo > -(float)n) ? p + (int)floorf(dlo) - 1 : 0;
    hi = (dhi < (float)n) ? p + (int)ceilf(dhi) + 1 : n - 1;
    lo = max(lo, 0);
    hi = min(hi, n - 1);
}

// Per-line constants of the scan.
struct DtLine {
    float lin, quad, mx;
    float cst[2 * DT_R0 + 1];  // cost of displacement k - DT_R0
    float cl1, cr1;            // costs at -(DT_R0+1) and +(DT_R0+1)
    bool past_l, past_r;       // DT_R0+1 lies beyond the vertex of the left / right cost
};

__device__ __forceinline__ void dt_line_init(DtLine &c, float lin, float quad, float mx)
{
    c.lin = lin;
    c.quad = quad;
    c.mx = mx;
#pragma unroll
    for (int k = 0; k <= 2 * DT_R0; ++k) {
        const float dd = (float)(k - DT_R0);
        c.cst[k] = fmaf(quad, dd * dd, lin * dd);
    }
    const float f1 = (float)(DT_R0 + 1);
    c.cl1 = fmaf(quad, f1 * f1, -lin * f1);
    c.cr1 = fmaf(quad, f1 * f1, lin * f1);
    c.past_l = f1 >= lin / (2.f * quad);
    c.past_r = f1 >= -lin / (2.f * quad);
}

// The transformed value and smallest maximiser of output p of line L (length n).
__device__ __forceinline__ void dt_scan(const DtLine &c, const float *L, int n, int p, float &best_out, int &arg_out)
{
    // the window's values (minus infinity outside the line), then its first maximum by a pairwise tree: a right
    // operand (larger indices) replaces a left one only when strictly greater, exactly as in a left-to-right scan, so
    // the smallest maximiser wins; the tree's depth is 4 instead of a chain of 9 dependent compares
    static_assert(DT_R0 == 4, "the reduction tree below is written for a 9-candidate window");
    float v[2 * DT_R0 + 1];
    if (p >= DT_R0 && p + DT_R0 < n) {
        const float *Lp = L + (p - DT_R0);  // interior: the whole window is inside the line
#pragma unroll
        for (int k = 0; k <= 2 * DT_R0; ++k) v[k] = Lp[k] - c.cst[k];
    } else {
#pragma unroll
        for (int k = 0; k <= 2 * DT_R0; ++k) {
            const int q = p + k - DT_R0;
            v[k] = q >= 0 && q < n ? L[q] - c.cst[k] : -INFINITY;
        }
    }
    auto first_max = [](float &va, int &ka, float vb, int kb) {
        if (vb > va) {
            va = vb;
            ka = kb;
        }
    };
    int k0 = 0, k2 = 2, k4 = 4, k6 = 6;
    float b0 = v[0], b2 = v[2], b4 = v[4], b6 = v[6];
    first_max(b0, k0, v[1], 1);
    first_max(b2, k2, v[3], 3);
    first_max(b4, k4, v[5], 5);
    first_max(b6, k6, v[7], 7);
    first_max(b0, k0, b2, k2);
    first_max(b4, k4, b6, k6);
    first_max(b0, k0, b4, k4);
    first_max(b0, k0, v[8], 8);
    float best = b0;
    int arg = p + k0 - DT_R0;
    const float T = (c.mx - best) + 1e-5f * (1.f + fabsf(c.mx) + fabsf(best));
    const bool done_l = p - DT_R0 - 1 < 0 || (c.past_l && c.cl1 > T);
    const bool done_r = p + DT_R0 + 1 >= n || (c.past_r && c.cr1 > T);
    if (!(done_l && done_r)) {
        int lo, hi;
        dt_window(c.lin, c.quad, c.mx, best, p, n, lo, hi);
        // the window of the first result holds every candidate that can still win (a better value would only narrow
        // it); four distances per step, at each distance the left candidate first: it is the smallest index seen so
        // far and also wins a tie, the right one must be strictly better
        const int dmax = max(p - lo, hi - p);
        for (int d0 = DT_R0 + 1; d0 <= dmax; d0 += 4) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int d = d0 + u;
                const float fd = (float)d;
                const float vl = p - d >= lo ? L[p - d] - fmaf(c.quad, fd * fd, -c.lin * fd) : -INFINITY;
                const float vr = p + d <= hi ? L[p + d] - fmaf(c.quad, fd * fd, c.lin * fd) : -INFINITY;
                if (vl >= best) {
                    best = vl;
                    arg = p - d;
                }
                if (vr > best) {
                    best = vr;
                    arg = p + d;
                }
            }
        }
    }
    best_out = best;
    arg_out = arg;
}

// Job of CTA b: the last job whose first CTA is <= b (the first CTAs increase strictly). A 32-ary search by one warp:
// each lane probes one of 32 evenly spaced jobs of the remaining range and a ballot keeps the last one at or below
// b, so a range of n jobs takes about log32(n) dependent loads. All lanes return the same job.
template <bool XPASS>
__device__ __forceinline__ int cta_job(const DtJob *jobs, int n, int b, int lane)
{
    int lo = 0, hi = n - 1;  // invariant: first(lo) <= b
    while (lo < hi) {
        const int stride = (hi - lo + 32) / 32;
        const int probe = lo + lane * stride;
        const bool ok = probe <= hi && (XPASS ? jobs[probe].xbegin : jobs[probe].ybegin) <= b;
        const int k = __popc(__ballot_sync(0xffffffffu, ok));  // >= 1: lane 0 probes lo
        lo += (k - 1) * stride;
        hi = min(hi, lo + stride - 1);
    }
    return lo;
}

__global__ void __launch_bounds__(DT_WARPS * 32) dt_x_kernel(const DtJob *__restrict__ jobs, int n_jobs, int nmax)
{
    extern __shared__ float lines[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // every warp finds the job itself (no block barrier); the job's fields in registers: stores through its pointers
    // could alias the job table otherwise
    const DtJob J = jobs[cta_job<true>(jobs, n_jobs, blockIdx.x, lane)];
    const int line = (blockIdx.x - J.xbegin) * DT_WARPS + warp;
    if (line >= J.H) return;
    const int n = J.W;
    const float *in = J.S + (size_t)line * n;
    float *L = lines + (size_t)warp * nmax;
    float mx = -INFINITY;
    for (int q = lane; q < n; q += 32) {
        const float v = __ldg(in + q);
        L[q] = v;
        mx = fmaxf(mx, v);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    __syncwarp();
    DtLine c;
    dt_line_init(c, J.lx, J.qx, mx);
    float *V = J.V + (size_t)line * J.nx;
    int32_t *IV = J.IV + (size_t)line * J.nx;
    for (int k = lane; k < J.nx; k += 32) {
        float best;
        int arg;
        dt_scan(c, L, n, J.x_off + J.x_step * k, best, arg);
        V[k] = best;
        IV[k] = arg;
    }
}

// shared memory: 8 columns of length H (stride colstride, odd) and the staged results (8 x ny values and argmaxes)
__global__ void __launch_bounds__(DT_WARPS * 32) dt_y_kernel(const DtJob *__restrict__ jobs, int n_jobs, int colstride,
                                                             int outstride)
{
    extern __shared__ float sm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const DtJob J = jobs[cta_job<false>(jobs, n_jobs, blockIdx.x, lane)];
    const int k0 = (blockIdx.x - J.ybegin) * DT_WARPS;
    const int ncols = min(DT_WARPS, J.nx - k0);
    const int H = J.H, nx = J.nx, ny = J.ny;
    float *col = sm;                                              // [8][colstride]
    float *outD = sm + DT_WARPS * colstride;                      // [8][outstride]
    int32_t *outA = reinterpret_cast<int32_t *>(outD + DT_WARPS * outstride);
    // stage the 8 columns transposed: rows of V are read 8 words at a time
    for (int idx = threadIdx.x; idx < H * DT_WARPS; idx += DT_WARPS * 32) {
        const int y = idx >> 3, c = idx & 7;
        if (c < ncols) col[c * colstride + y] = J.V[(size_t)y * nx + k0 + c];
    }
    __syncthreads();
    if (warp < ncols) {
        const float *L = col + warp * colstride;
        float mx = -INFINITY;
        for (int q = lane; q < H; q += 32) mx = fmaxf(mx, L[q]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        DtLine c;
        dt_line_init(c, J.ly, J.qy, mx);
        const int k = k0 + warp;
        for (int i = lane; i < ny; i += 32) {
            float best;
            int arg;
            dt_scan(c, L, H, J.y_off + J.y_step * i, best, arg);
            outD[warp * outstride + i] = best;
            outA[warp * outstride + i] = (arg << 16) | J.IV[(size_t)arg * nx + k];
        }
    }
    __syncthreads();
    // write rows of 8 results
    for (int idx = threadIdx.x; idx < ny * DT_WARPS; idx += DT_WARPS * 32) {
        const int i = idx >> 3, c = idx & 7;
        if (c < ncols) {
            J.D[(size_t)i * nx + k0 + c] = outD[c * outstride + i];
            J.A[(size_t)i * nx + k0 + c] = outA[c * outstride + i];
        }
    }
}

constexpr int DT_KS = 32;  // sampled columns per CTA of the fused form

__device__ __forceinline__ void dt_cp_async4(float *dst, const float *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void dt_cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void dt_cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// shared memory: V and IV of the strip [32][hstride] each (hstride odd, >= H), nbuf staged rows per warp
// [nbuf][wmax] (two: the next row is copied in with cp.async while the current one is scanned; one: it is refilled
// after use), and the warps' partial column maxima [8][32]. cta_jobs: the job of every CTA (null: searched in the
// jobs' xbegin).
__global__ void __launch_bounds__(DT_WARPS * 32, 4) dt_xy_kernel(const DtJob *__restrict__ jobs, int n_jobs,
                                                              const int *__restrict__ cta_jobs, int hstride, int wmax,
                                                              int nbuf)
{
    extern __shared__ float sm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ji = cta_jobs ? __ldg(cta_jobs + blockIdx.x) : cta_job<true>(jobs, n_jobs, blockIdx.x, lane);
    const DtJob J = jobs[ji];  // xbegin: first CTA (strip) of the job
    const int k0 = (blockIdx.x - J.xbegin) * DT_KS;
    const int ncols = min(DT_KS, J.nx - k0);
    float *Vs = sm;
    int32_t *IVs = reinterpret_cast<int32_t *>(sm + DT_KS * hstride);
    float *rows = sm + 2 * DT_KS * hstride + nbuf * warp * wmax;
    float *pmax = sm + 2 * DT_KS * hstride + nbuf * DT_WARPS * wmax;
    const int H = J.H, n = J.W;
    const bool active = lane < ncols;
    const int px = J.x_off + J.x_step * (k0 + lane);  // this lane's sampled column
    float cmax = -INFINITY;                           // its column maximum over this warp's rows
    DtLine cx;
    dt_line_init(cx, J.lx, J.qx, 0.f);  // per-line constants; the line maximum is set per row
    auto fetch = [&](int y, float *dst) {
        const float *in = J.S + (size_t)y * n;
        for (int q = lane; q < n; q += 32) dt_cp_async4(dst + q, in + q);
        dt_cp_commit();
    };
    if (warp < H) fetch(warp, rows);
    int buf = 0;
    for (int y = warp; y < H; y += DT_WARPS) {
        float *L = rows + buf * wmax;
        if (nbuf == 2 && y + DT_WARPS < H) {
            fetch(y + DT_WARPS, rows + (buf ^ 1) * wmax);
            dt_cp_wait<1>();
        } else {
            dt_cp_wait<0>();
        }
        __syncwarp();
        float mx = -INFINITY;
        for (int q = lane; q < n; q += 32) mx = fmaxf(mx, L[q]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (active) {
            cx.mx = mx;
            float best;
            int arg;
            dt_scan(cx, L, n, px, best, arg);
            Vs[lane * hstride + y] = best;
            IVs[lane * hstride + y] = arg;
            cmax = fmaxf(cmax, best);
        }
        __syncwarp();  // every lane is done with this buffer before it is refilled
        if (nbuf == 2) buf ^= 1;
        else if (y + DT_WARPS < H) fetch(y + DT_WARPS, rows);
    }
    pmax[warp * 32 + lane] = cmax;
    __syncthreads();
    if (!active) return;
    float mx = pmax[lane];
#pragma unroll
    for (int w = 1; w < DT_WARPS; ++w) mx = fmaxf(mx, pmax[w * 32 + lane]);
    DtLine c;
    dt_line_init(c, J.ly, J.qy, mx);
    const float *col = Vs + lane * hstride;
    const int32_t *icol = IVs + lane * hstride;
    const int k = k0 + lane;
    for (int i = warp; i < J.ny; i += DT_WARPS) {
        float best;
        int arg;
        dt_scan(c, col, H, J.y_off + J.y_step * i, best, arg);
        J.D[(size_t)i * J.nx + k] = best;
        J.A[(size_t)i * J.nx + k] = (arg << 16) | icol[arg];
    }
}

}  // namespace

int dt_lines_per_cta() { return DT_WARPS; }
int dt_strip_columns() { return DT_KS; }
int dt_job_strips(int nx) { return (nx + DT_KS - 1) / DT_KS; }

size_t dt_fused_smem_bytes(int max_W, int max_H, int nbuf)
{
    return sizeof(float) * (2 * (size_t)DT_KS * (size_t)(max_H | 1) + (size_t)nbuf * DT_WARPS * max_W + DT_WARPS * 32);
}

cudaError_t launch_dt_fused(const DtJob *d_jobs, int n_jobs, const int *d_cta_jobs, int ctas, int max_W, int max_H,
                            cudaStream_t s)
{
    if (n_jobs <= 0 || ctas <= 0) return cudaSuccess;
    if (max_W > kDtMaxSide || max_H > kDtMaxSide || max_W < 1 || max_H < 1) return cudaErrorInvalidValue;
    const int nbuf = dt_fused_smem_bytes(max_W, max_H, 2) <= (size_t)kMaxDynamicSmem ? 2 : 1;
    const size_t smem = dt_fused_smem_bytes(max_W, max_H, nbuf);
    if (smem > (size_t)kMaxDynamicSmem) return cudaErrorInvalidValue;
    cudaError_t e = allow_max_dynamic_smem(reinterpret_cast<const void *>(dt_xy_kernel), 6 + 18);
    if (e != cudaSuccess) return e;
    note_launches(1);
    dt_xy_kernel<<<ctas, DT_WARPS * 32, smem, s>>>(d_jobs, n_jobs, d_cta_jobs, max_H | 1, max_W, nbuf);
    return cudaGetLastError();
}

cudaError_t launch_dt(const DtJob *d_jobs, int n_jobs, int x_ctas, int y_ctas, int max_W, int max_H, cudaStream_t s)
{
    if (n_jobs <= 0) return cudaSuccess;
    if (max_W > kDtMaxSide || max_H > kDtMaxSide) return cudaErrorInvalidValue;
    const size_t smem_x = sizeof(float) * DT_WARPS * (size_t)max_W;
    // y pass: a column has H <= max_H values; outputs per column ny <= H
    const int colstride = max_H | 1, outstride = max_H | 1;
    const size_t smem_y = sizeof(float) * DT_WARPS * (size_t)(colstride + 2 * outstride);
    cudaError_t e = allow_max_dynamic_smem(reinterpret_cast<const void *>(dt_y_kernel), 7);
    if (e != cudaSuccess) return e;
    note_launches((x_ctas > 0) + (y_ctas > 0));
    if (x_ctas > 0) dt_x_kernel<<<x_ctas, DT_WARPS * 32, smem_x, s>>>(d_jobs, n_jobs, max_W);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (y_ctas > 0) dt_y_kernel<<<y_ctas, DT_WARPS * 32, smem_y, s>>>(d_jobs, n_jobs, colstride, outstride);
    return cudaGetLastError();
}

}  // namespace tdpm
