// Steps 3 and 4: shift-and-sum of the transformed part maps into the root map (Sec. 2 score equation; Algorithm 1,
// step 13) and the threshold (Algorithm 1, steps 15-16).
//
// assemble_kernel  s[y][x] = root[y][x] + bias + sum_i D_i[y][x]  (D_i already sampled at 2y+vy, 2x+vx)
// detect kernels   deterministic stream compaction: per-block counts, one scan, per-block ordered writes, so the
//                  records come out ordered by (image, component, level, y, x) with no sort and no float atomics.
#include "internal.h"

namespace tdpm {
namespace {

constexpr int AS_THREADS = 256;
constexpr int DET_THREADS = 256;

__device__ __forceinline__ int find_pos_job(const AsmJob *jobs, int n, long long idx)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].begin <= idx) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(AS_THREADS) assemble_kernel(const AsmJob *__restrict__ jobs, int n_jobs,
                                                              long long total)
{
    const long long idx = (long long)blockIdx.x * AS_THREADS + threadIdx.x;
    if (idx >= total) return;
    const AsmJob &J = jobs[find_pos_job(jobs, n_jobs, idx)];
    const int local = (int)(idx - J.begin);
    const int y = local / J.X, x = local - y * J.X;
    float s = J.root[(size_t)y * J.root_W + x] + J.bias;
    for (int i = 0; i < J.n_parts; ++i) s += J.D[i][local];
    J.out[local] = s;
}

// threshold of job ji: job_tau[ji] when given (one per (image, component) of the scores set), else tau
__device__ __forceinline__ float job_threshold(const float *job_tau, int ji, float tau)
{
    return job_tau ? job_tau[ji] : tau;
}

__global__ void __launch_bounds__(DET_THREADS) detect_count_kernel(const AsmJob *__restrict__ jobs, int n_jobs,
                                                                   long long total, float tau,
                                                                   const float *__restrict__ job_tau, int *counts)
{
    const long long idx = (long long)blockIdx.x * DET_THREADS + threadIdx.x;
    bool hit = false;
    if (idx < total) {
        const int ji = find_pos_job(jobs, n_jobs, idx);
        const AsmJob &J = jobs[ji];
        hit = J.out[idx - J.begin] >= job_threshold(job_tau, ji, tau);
    }
    const int c = __syncthreads_count(hit);
    if (threadIdx.x == 0) counts[blockIdx.x] = c;
}

// exclusive scan of n block counts by one CTA; total written to *d_total
__global__ void __launch_bounds__(1024) detect_scan_kernel(const int *counts, int *offsets, int n, long long *d_total)
{
    __shared__ long long warp_sums[32];
    __shared__ long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int base = 0; base < n; base += 1024) {
        const int i = base + threadIdx.x;
        long long v = i < n ? counts[i] : 0;
        long long incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            const long long t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) warp_sums[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            long long ws = warp_sums[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const long long t = __shfl_up_sync(0xffffffffu, ws, o);
                if (lane >= o) ws += t;
            }
            warp_sums[lane] = ws;  // inclusive over warps
        }
        __syncthreads();
        const long long before = carry + (wid > 0 ? warp_sums[wid - 1] : 0) + incl - v;
        if (i < n) offsets[i] = (int)before;
        __syncthreads();
        if (threadIdx.x == 1023) carry = before + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) *d_total = carry;
}

__global__ void __launch_bounds__(DET_THREADS) detect_write_kernel(const AsmJob *__restrict__ jobs, int n_jobs,
                                                                   long long total, float tau,
                                                                   const float *__restrict__ job_tau,
                                                                   const int *__restrict__ offsets,
                                                                   tdpm_detection *__restrict__ out,
                                                                   long long capacity, int model)
{
    __shared__ int warp_counts[DET_THREADS / 32];
    const long long idx = (long long)blockIdx.x * DET_THREADS + threadIdx.x;
    int ji = 0;
    bool hit = false;
    if (idx < total) {
        ji = find_pos_job(jobs, n_jobs, idx);
        hit = jobs[ji].out[idx - jobs[ji].begin] >= job_threshold(job_tau, ji, tau);
    }
    const unsigned ballot = __ballot_sync(0xffffffffu, hit);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) warp_counts[wid] = __popc(ballot);
    __syncthreads();
    if (!hit) return;
    int before = 0;
    for (int w = 0; w < wid; ++w) before += warp_counts[w];
    before += __popc(ballot & ((1u << lane) - 1u));
    const long long slot = (long long)offsets[blockIdx.x] + before;
    if (slot >= capacity) return;
    const AsmJob &J = jobs[ji];
    const int local = (int)(idx - J.begin);
    tdpm_detection d;
    d.image = J.image;
    d.model = model;
    d.component = J.comp;
    d.level = J.level;
    d.y = local / J.X;
    d.x = local - d.y * J.X;
    d.score = J.out[local];
    d.n_parts = J.n_parts;
    for (int i = 0; i < MAXP; ++i) {
        const int a = i < J.n_parts ? J.A[i][local] : 0;
        d.part_y[i] = i < J.n_parts ? (a >> 16) : 0;
        d.part_x[i] = i < J.n_parts ? (a & 0xffff) : 0;
    }
    out[slot] = d;
}

}  // namespace

int detect_positions_per_block() { return DET_THREADS; }

cudaError_t launch_assemble(const AsmJob *d_jobs, int n_jobs, long long total, cudaStream_t s)
{
    if (total <= 0) return cudaSuccess;
    note_launches(1);
    assemble_kernel<<<(unsigned)((total + AS_THREADS - 1) / AS_THREADS), AS_THREADS, 0, s>>>(d_jobs, n_jobs, total);
    return cudaGetLastError();
}

cudaError_t launch_detect_count(const AsmJob *d_jobs, int n_jobs, long long total, float tau, const float *d_job_tau,
                                int *d_block_counts, int *d_block_offsets, int n_blocks, long long *d_total,
                                cudaStream_t s)
{
    if (total <= 0 || n_blocks <= 0) return cudaMemsetAsync(d_total, 0, sizeof(long long), s);
    note_launches(2);
    detect_count_kernel<<<n_blocks, DET_THREADS, 0, s>>>(d_jobs, n_jobs, total, tau, d_job_tau, d_block_counts);
    detect_scan_kernel<<<1, 1024, 0, s>>>(d_block_counts, d_block_offsets, n_blocks, d_total);
    return cudaGetLastError();
}

cudaError_t launch_detect_write(const AsmJob *d_jobs, int n_jobs, long long total, float tau, const float *d_job_tau,
                                const int *d_block_offsets, int n_blocks, tdpm_detection *d_out, long long capacity,
                                int model, cudaStream_t s)
{
    if (total <= 0 || n_blocks <= 0) return cudaSuccess;
    note_launches(1);
    detect_write_kernel<<<n_blocks, DET_THREADS, 0, s>>>(d_jobs, n_jobs, total, tau, d_job_tau, d_block_offsets, d_out,
                                                        capacity, model);
    return cudaGetLastError();
}

}  // namespace tdpm
