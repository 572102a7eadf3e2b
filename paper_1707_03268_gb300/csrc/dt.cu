// Step 2: generalised distance transform with argmax (Sec. 2 argmax equation),
//   D[p] = max_q f[q] - (lin*(q-p) + quad*(q-p)^2),  the smallest maximising q,
// run as an x pass over every row of a part score map and a y pass over every sampled column of its result.
//
// One warp owns one line: it stages the line in shared memory and reduces its maximum M. Each lane then takes output
// positions p and scans the candidates q in increasing order, keeping the first strict maximum, exactly like the
// brute-force definition. The scan is restricted to the window where the deformation cost is at most
// (M - f[p]) + margin: any q outside it has f[q] - cost <= M - cost < f[p] - margin, so it can never beat the
// candidate q = p (whose value is f[p] exactly). The margin covers FP32 rounding of the evaluated values, so the
// window never changes the result of the full scan, in exact or in FP32 arithmetic; it only skips hopeless
// candidates (for the default deformation costs the window spans a few to a few tens of cells).
//
// x pass: line = row y of S (length W); outputs at p = x_off + x_step*k, written transposed: V[k][y], IV[k][y].
// y pass: line = row k of V (length H, contiguous); outputs at p = y_off + y_step*i: D[i][k], A[i][k] =
//         (qy << 16) | IV[k][qy].
#include "internal.h"

namespace tdpm {
namespace {

constexpr int DT_WARPS = 8;

__device__ __forceinline__ int find_line_job(const DtJob *jobs, int n, int idx, bool xpass)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const int b = xpass ? jobs[mid].xbegin : jobs[mid].ybegin;
        if (b <= idx) lo = mid; else hi = mid - 1;
    }
    return lo;
}

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

template <bool XPASS>
__global__ void __launch_bounds__(DT_WARPS * 32) dt_line_kernel(const DtJob *__restrict__ jobs, int n_jobs,
                                                                int total_lines, int nmax)
{
    extern __shared__ float lines[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gl = blockIdx.x * DT_WARPS + warp;
    if (gl >= total_lines) return;
    const DtJob &J = jobs[find_line_job(jobs, n_jobs, gl, XPASS)];
    const int line = gl - (XPASS ? J.xbegin : J.ybegin);
    const int n = XPASS ? J.W : J.H;
    const float *in = XPASS ? J.S + (size_t)line * J.W : J.V + (size_t)line * J.H;
    const float lin = XPASS ? J.lx : J.ly, quad = XPASS ? J.qx : J.qy;
    const int off = XPASS ? J.x_off : J.y_off, step = XPASS ? J.x_step : J.y_step, m = XPASS ? J.nx : J.ny;
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

    for (int i = lane; i < m; i += 32) {
        const int p = off + step * i;
        // start from q = p and walk outwards; every improvement of the best value shrinks the window
        float best = L[p];
        int arg = p, lo, hi;
        dt_window(lin, quad, mx, best, p, n, lo, hi);
        for (int d = 1; p - d >= lo || p + d <= hi; ++d) {
            const float fd = (float)d;
            if (p - d >= lo) {
                // smallest index seen so far: it also wins a tie
                const float v = L[p - d] - fmaf(quad, fd * fd, -lin * fd);
                if (v >= best) {
                    best = v;
                    arg = p - d;
                    dt_window(lin, quad, mx, best, p, n, lo, hi);
                }
            }
            if (p + d <= hi) {
                const float v = L[p + d] - fmaf(quad, fd * fd, lin * fd);
                if (v > best) {
                    best = v;
                    arg = p + d;
                    dt_window(lin, quad, mx, best, p, n, lo, hi);
                }
            }
        }
        if (XPASS) {
            J.V[(size_t)i * J.H + line] = best;
            J.IV[(size_t)i * J.H + line] = arg;
        } else {
            J.D[(size_t)i * J.nx + line] = best;
            J.A[(size_t)i * J.nx + line] = (arg << 16) | J.IV[(size_t)line * J.H + arg];
        }
    }
}

}  // namespace

cudaError_t launch_dt(const DtJob *d_jobs, int n_jobs, int x_lines, int y_lines, int max_W, int max_H, cudaStream_t s)
{
    if (n_jobs <= 0) return cudaSuccess;
    if (max_W > 800 || max_H > 800) return cudaErrorInvalidValue;
    const size_t smem_x = sizeof(float) * DT_WARPS * (size_t)max_W;
    const size_t smem_y = sizeof(float) * DT_WARPS * (size_t)max_H;
    note_launches((x_lines > 0) + (y_lines > 0));
    if (x_lines > 0)
        dt_line_kernel<true><<<(x_lines + DT_WARPS - 1) / DT_WARPS, DT_WARPS * 32, smem_x, s>>>(d_jobs, n_jobs, x_lines,
                                                                                                max_W);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (y_lines > 0)
        dt_line_kernel<false><<<(y_lines + DT_WARPS - 1) / DT_WARPS, DT_WARPS * 32, smem_y, s>>>(d_jobs, n_jobs,
                                                                                                 y_lines, max_H);
    return cudaGetLastError();
}

}  // namespace tdpm
