// Step 2: generalised distance transform with argmax (Sec. 2 argmax equation),
//   D[p] = max_q f[q] - (lin*(q-p) + quad*(q-p)^2), smallest maximising q,
// run as an x pass over every row of a part score map and a y pass over every sampled column of its result.
//
// One thread owns one line and builds the upper envelope of the parabolas q -> f[q] - cost(q - p) in increasing q.
// Because quad > 0, candidate r > q beats q (strictly) exactly for p above one threshold, so each envelope entry stores
// the first integer p where it starts to win. That breakpoint comes from the closed-form intersection and is then
// corrected by direct comparison of the two candidates' values at the neighbouring integers, so the envelope makes
// the same decisions as a brute-force scan that keeps the first strict maximum. Entries live in shared memory in a
// [entry][lane] layout (one 32-bit word per lane per row: conflict-free whatever entry each lane touches).
//
// x pass: a warp owns 32 consecutive rows; 32x32 blocks of the map are staged through shared memory so the global
// reads and writes stay coalesced. y pass: a warp owns 32 consecutive sampled columns; its reads of V are coalesced.
#include "internal.h"

namespace tdpm {
namespace {

struct Line {
    float lin, quad;
    int n;
};

__device__ __forceinline__ float dt_cost(float lin, float quad, int d)
{
    const float fd = (float)d;
    return fmaf(quad, fd * fd, lin * fd);
}

// candidate r (value fr) strictly beats q (value fq) at p
__device__ __forceinline__ bool dt_beats(const Line &L, int r, float fr, int q, float fq, int p)
{
    return (fr - dt_cost(L.lin, L.quad, r - p)) > (fq - dt_cost(L.lin, L.quad, q - p));
}

// first integer p in [0, n] at which r > q strictly beats q (n: never inside the line)
__device__ __forceinline__ int dt_break(const Line &L, int q, float fq, int r, float fr)
{
    const float num = (fq - fr) + L.lin * (float)(r - q) + L.quad * (float)(r * r - q * q);
    const float den = 2.f * L.quad * (float)(r - q);
    const float s = num / den;
    int p;
    if (!(s < (float)L.n)) p = L.n;  // also catches NaN
    else if (s < 0.f) p = 0;
    else p = (int)floorf(s) + 1;
    if (p > L.n) p = L.n;
    for (int it = 0; it < 2 && p > 0 && dt_beats(L, r, fr, q, fq, p - 1); ++it) --p;
    for (int it = 0; it < 2 && p < L.n && !dt_beats(L, r, fr, q, fq, p); ++it) ++p;
    return p;
}

// envelope storage: ENVP[k*32+lane] = v | (z << 16); ENVF[k*32+lane] = f[v]
struct Env {
    int *P;
    float *F;
    int lane;
    int top;
    __device__ __forceinline__ int v(int k) const { return P[k * 32 + lane] & 0xffff; }
    __device__ __forceinline__ int z(int k) const { return P[k * 32 + lane] >> 16; }
    __device__ __forceinline__ float f(int k) const { return F[k * 32 + lane]; }
    __device__ __forceinline__ void push(int q, int zq, float fq)
    {
        ++top;
        P[top * 32 + lane] = q | (zq << 16);
        F[top * 32 + lane] = fq;
    }
    __device__ __forceinline__ void insert(const Line &L, int q, float fq)
    {
        int s = 0;
        while (top >= 0) {
            s = dt_break(L, v(top), f(top), q, fq);
            if (s <= z(top)) --top; else break;
        }
        if (top < 0) push(q, 0, fq);
        else if (s < L.n) push(q, s, fq);
    }
};

template <class Job>
__device__ __forceinline__ int find_begin(const Job *jobs, int n, int idx, bool xpass)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const int b = xpass ? jobs[mid].xbegin : jobs[mid].ybegin;
        if (b <= idx) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(32) dt_x_kernel(const DtJob *__restrict__ jobs, int n_jobs, int nmax)
{
    extern __shared__ __align__(16) int dsm[];
    int *envp = dsm;
    float *envf = reinterpret_cast<float *>(dsm + nmax * 32);
    float *tile = reinterpret_cast<float *>(dsm + 2 * nmax * 32);   // [32][33]
    int *tilei = dsm + 2 * nmax * 32 + 32 * 33;                      // [32][33]
    const int lane = threadIdx.x;
    const int gw = blockIdx.x;
    const DtJob J = jobs[find_begin(jobs, n_jobs, gw, true)];
    const int row0 = (gw - J.xbegin) * 32, row = row0 + lane;
    const bool active = row < J.H;
    const Line L{J.lx, J.qx, J.W};
    Env E{envp, envf, lane, -1};

    for (int c0 = 0; c0 < J.W; c0 += 32) {
        const int col = c0 + lane;
        for (int i = 0; i < 32; ++i) {
            const int r = row0 + i;
            tile[lane * 33 + i] = (r < J.H && col < J.W) ? __ldg(J.S + (size_t)r * J.W + col) : 0.f;
        }
        __syncwarp();
        const int cend = min(32, J.W - c0);
        if (active)
            for (int j = 0; j < cend; ++j) E.insert(L, c0 + j, tile[j * 33 + lane]);
        __syncwarp();
    }

    int kk = 0;
    for (int k0 = 0; k0 < J.nx; k0 += 32) {
        const int kend = min(32, J.nx - k0);
        if (active) {
            for (int j = 0; j < kend; ++j) {
                const int p = J.x_off + J.x_step * (k0 + j);
                while (kk < E.top && E.z(kk + 1) <= p) ++kk;
                const int q = E.v(kk);
                tile[j * 33 + lane] = E.f(kk) - dt_cost(L.lin, L.quad, q - p);
                tilei[j * 33 + lane] = q;
            }
        }
        __syncwarp();
        const int k = k0 + lane;
        for (int i = 0; i < 32; ++i) {
            const int r = row0 + i;
            if (r < J.H && lane < kend) {
                J.V[(size_t)r * J.nx + k] = tile[lane * 33 + i];
                J.IV[(size_t)r * J.nx + k] = tilei[lane * 33 + i];
            }
        }
        __syncwarp();
    }
}

__global__ void __launch_bounds__(32) dt_y_kernel(const DtJob *__restrict__ jobs, int n_jobs, int nmax)
{
    extern __shared__ __align__(16) int dsm[];
    int *envp = dsm;
    float *envf = reinterpret_cast<float *>(dsm + nmax * 32);
    const int lane = threadIdx.x;
    const int gw = blockIdx.x;
    const DtJob J = jobs[find_begin(jobs, n_jobs, gw, false)];
    const int k = (gw - J.ybegin) * 32 + lane;
    if (k >= J.nx) return;
    const Line L{J.ly, J.qy, J.H};
    Env E{envp, envf, lane, -1};
    for (int q = 0; q < J.H; ++q) E.insert(L, q, __ldg(J.V + (size_t)q * J.nx + k));
    int kk = 0;
    for (int i = 0; i < J.ny; ++i) {
        const int p = J.y_off + J.y_step * i;
        while (kk < E.top && E.z(kk + 1) <= p) ++kk;
        const int q = E.v(kk);
        J.D[(size_t)i * J.nx + k] = E.f(kk) - dt_cost(L.lin, L.quad, q - p);
        J.A[(size_t)i * J.nx + k] = (q << 16) | J.IV[(size_t)q * J.nx + k];
    }
}

}  // namespace

cudaError_t launch_dt(const DtJob *d_jobs, int n_jobs, int x_warps, int y_warps, int max_W, int max_H, cudaStream_t s)
{
    if (n_jobs <= 0) return cudaSuccess;
    const size_t smem_x = sizeof(int) * (2 * (size_t)max_W * 32 + 2 * 32 * 33);
    const size_t smem_y = sizeof(int) * (2 * (size_t)max_H * 32);
    if (smem_x > 220 * 1024 || smem_y > 220 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(dt_x_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_x);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(dt_y_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_y);
    if (e != cudaSuccess) return e;
    note_launches((x_warps > 0) + (y_warps > 0));
    if (x_warps > 0) dt_x_kernel<<<x_warps, 32, smem_x, s>>>(d_jobs, n_jobs, max_W);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (y_warps > 0) dt_y_kernel<<<y_warps, 32, smem_y, s>>>(d_jobs, n_jobs, max_H);
    return cudaGetLastError();
}

}  // namespace tdpm
