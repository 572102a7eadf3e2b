// Convolution shortening (Sec. 4, Algorithm 1): a root hypothesis gamma is given up as soon as the partial sum of a
// filter's first q CP terms at gamma falls below that filter's threshold t_q. Filters are visited in model order
// (root, then parts); a part is tested at its anchor, (2y + vy, 2x + vx) on the level lambda below. Term r of filter
// k at window phi is lambda_r * sum_{dy,dx,c} phi[dy][dx][c] a_r[dy] b_r[dx] c_r[c].
//
// One warp per hypothesis, lane = channel: every term is one pass over the window of the filter under test (sum over
// cells of a[dy] b[dx] phi, per lane) and one butterfly reduction of c_r[c] times that over the lanes. The first term
// reads the window from global memory; a hypothesis that survives it has the window staged in the warp's slice of
// shared memory for the rest (filters of up to CASC_MAX_CELLS cells; larger ones keep reading global memory). The exit is uniform across the warp. The thresholds come from the same device function run
// without exits at positive examples, so a positive's own partial sums are never below them.
#include <algorithm>

#include "internal.h"

namespace tdpm {
namespace {

constexpr int CASC_WARPS = 4;
constexpr int CASC_MAX_CELLS = 64;  // h * w staged in shared memory (8 KB per warp)

__device__ __forceinline__ float warp_sum_all(float v)
{
    // xor butterfly: every lane ends with the same (bit-identical) value
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Partial sums of one filter at one window, in the filter's term order, with an early exit when thr is not null.
// Returns the number of terms evaluated; *pruned is set when a partial sum fell below its threshold. partial (lane
// 0 writes; may be null) receives every evaluated partial sum. The first term reads the window from global memory
// (most hypotheses stop there); a hypothesis that goes on has its window staged in the warp's shared memory first
// (swin, when not null). The arithmetic is the same either way.
__device__ int casc_filter(const CascFilter &F, const float *__restrict__ gwin, int gstride, float *swin,
                           const float *thr, float *partial, bool *pruned)
{
    const int lane = threadIdx.x & 31;
    const float *win = gwin;
    int stride = gstride;
    float p = 0.f;
    for (int q = 0; q < F.nterms; ++q) {
        if (q == 1 && swin) {
            __syncwarp();
            for (int dy = 0; dy < F.h; ++dy)
                for (int dx = 0; dx < F.w; ++dx)
                    swin[(dy * F.w + dx) * 32 + lane] = __ldg(gwin + (size_t)dy * gstride + dx * 32 + lane);
            __syncwarp();
            win = swin;
            stride = F.w * 32;
        }
        const int r = F.order[q];
        float acc = 0.f;
        for (int dy = 0; dy < F.h; ++dy) {
            const float ay = __ldg(F.A + (size_t)dy * F.R + r);
            const float *row = win + (size_t)dy * stride;
            for (int dx = 0; dx < F.w; ++dx) acc = fmaf(ay * __ldg(F.B + (size_t)dx * F.R + r), row[dx * 32 + lane], acc);
        }
        const float v = warp_sum_all(__ldg(F.Ct + (size_t)r * 32 + lane) * acc);
        p = fmaf(__ldg(F.lam + r), v, p);
        if (partial && lane == 0) partial[q] = p;
        if (thr && p < thr[q]) {
            *pruned = true;
            return q + 1;
        }
    }
    return F.nterms;
}

__global__ void __launch_bounds__(CASC_WARPS * 32) cascade_kernel(CascArgs a)
{
    __shared__ __align__(16) float s_win[CASC_WARPS][CASC_MAX_CELLS * 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float *mywin = s_win[wid];
    unsigned long long evaluated = 0, total = 0, pruned_n = 0, bad = 0;
    for (long long i = (long long)blockIdx.x * CASC_WARPS + wid; i < a.n; i += (long long)gridDim.x * CASC_WARPS) {
        const tdpm_detection d = a.rec[i];
        const int first = a.comp_first[d.component], cnt = a.comp_count[d.component];
        bool pruned = false;
        for (int s = 0; s < cnt; ++s) {
            const CascFilter F = a.filt[first + s];
            total += F.nterms;
            if (pruned) continue;
            const int lev = F.part ? d.level - a.img_lam[d.image] : d.level;
            const int y0 = F.part ? 2 * d.y + F.vy : d.y, x0 = F.part ? 2 * d.x + F.vx : d.x;
            bool inside = lev >= 0 && lev < a.max_levels;
            CascLevel L{};
            if (inside) {
                L = a.levels[(size_t)d.image * a.max_levels + lev];
                inside = L.data && y0 >= 0 && x0 >= 0 && y0 + F.h <= L.H && x0 + F.w <= L.W;
            }
            if (!inside) {  // cannot happen for the library's own records; counted, never read out of bounds
                bad += 1;
                break;
            }
            const float *gwin = L.data + ((size_t)y0 * L.W + x0) * 32;
            float *part = a.partials ? a.partials + ((size_t)i * a.max_slots + s) * a.max_terms : nullptr;
            evaluated += casc_filter(F, gwin, L.W * 32, F.h * F.w <= CASC_MAX_CELLS ? mywin : nullptr,
                                     a.apply_thr ? F.thr : nullptr, part, &pruned);
        }
        if (lane == 0) {
            if (a.alive) a.alive[i] = pruned ? 0 : 1;
            pruned_n += pruned ? 1 : 0;
        }
    }
    if (lane == 0 && a.stats) {
        atomicAdd(a.stats + 0, evaluated);
        atomicAdd(a.stats + 1, total);
        atomicAdd(a.stats + 2, pruned_n);
        if (bad) atomicAdd(a.stats + 3, bad);
    }
}

}  // namespace

cudaError_t launch_cascade(const CascArgs &args, cudaStream_t s)
{
    if (args.n <= 0) return cudaSuccess;
    int sms = 152, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long want = (args.n + CASC_WARPS - 1) / CASC_WARPS;
    const unsigned blocks = (unsigned)std::min<long long>(want, (long long)sms * 8);
    note_launches(1);
    cascade_kernel<<<blocks, CASC_WARPS * 32, 0, s>>>(args);
    return cudaGetLastError();
}

}  // namespace tdpm
