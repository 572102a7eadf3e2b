// Greedy non-maximum suppression of detection records, per (image, class). The paper has no NMS; this is the DPM
// convention, kept exact so that it can be checked against the FP64 oracle:
//   * a detection's box is its component's root filter (h0 x w0 cells) at its level, whose cells measure cell[level]
//     image pixels: [x c, x c + w0 c) x [y c, y c + h0 c), in FP64 with each product and sum rounded once;
//   * within a group detections are taken by score, highest first, ties by record order; each one not yet
//     suppressed is kept and suppresses every later one whose box it covers by more than `overlap` of that later
//     box's own area.
// Steps, all in this file's kernels: group sizes (atomics); group offsets by a one-CTA scan; every record's sort key
// (score descending, then record index) scattered into its group's range; one CTA per group sorts its range with a
// bitonic network (in shared memory when it fits) and lays out the boxes in that order; the overlap test of every
// pair of every group runs once on the whole GPU into 64-bit masks, and one warp per group walks its detections in
// order, OR-ing the masks of the kept ones (above 16,384 detections, where the masks would grow past 32 MB, the
// group's CTA walks its boxes itself, a block barrier after each kept one); the kept flags go back to record order
// and the kept records are compacted in that order (per-block counts, a one-CTA scan of them, an ordered write).
#include <algorithm>

#include "internal.h"

namespace tdpm {
namespace {

struct NmsBox {
    double x1, y1, x2, y2;
};

constexpr int NMS_THREADS = 1024;        // per-group CTA and the scan CTA
constexpr int NMS_SORT_SMEM = 16384;     // groups up to this size sort in shared memory (8 bytes a key)
constexpr int NMS_BOX_SMEM = 3584;       // groups up to this size keep their boxes in shared memory
constexpr int NMS_FLAG_SMEM = 16384;     // ... and their kept flags (after the boxes)
constexpr int NMS_SMEM_BYTES = NMS_SORT_SMEM * 8;
constexpr int NMS_FLAG_OFF = NMS_BOX_SMEM * 32;
static_assert(NMS_BOX_SMEM * 32 + NMS_FLAG_SMEM <= NMS_SMEM_BYTES, "boxes and flags reuse the sort buffer");
constexpr int NMS_CBLOCK = 1024;         // records per compaction block (one thread each)

__device__ __forceinline__ int nms_group(const tdpm_detection &d, const int32_t *cls, int n_classes)
{
    return d.image * n_classes + (cls ? cls[d.component] : 0);
}

__global__ void nms_count_kernel(const tdpm_detection *__restrict__ rec, long long n, const int32_t *__restrict__ cls,
                                 int n_classes, int *__restrict__ counts)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicAdd(counts + nms_group(rec[i], cls, n_classes), 1);
}

// Exclusive scan of m ints by one CTA of NMS_THREADS threads, in chunks of NMS_THREADS with a running carry; the sum
// goes to *total when total is not null.
__global__ void __launch_bounds__(NMS_THREADS) nms_scan_kernel(const int *__restrict__ in, int m, int *__restrict__ out,
                                                              long long *__restrict__ total)
{
    __shared__ int warp_sum[NMS_THREADS / 32];
    __shared__ long long carry_s;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    if (t == 0) carry_s = 0;
    __syncthreads();
    for (int base = 0; base < m; base += NMS_THREADS) {
        const int v = base + t < m ? in[base + t] : 0;
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_sum[w] = x;
        __syncthreads();
        if (w == 0) {
            int s = warp_sum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            warp_sum[lane] = s;  // inclusive over warps
        }
        __syncthreads();
        const long long carry = carry_s;
        const int before = (w ? warp_sum[w - 1] : 0) + x - v;
        if (base + t < m) out[base + t] = (int)(carry + before);
        __syncthreads();
        if (t == NMS_THREADS - 1) carry_s = carry + before + v;
        __syncthreads();
    }
    if (t == 0 && total) *total = carry_s;
}

// Each record's key in its group's range: (score descending, record index ascending) as one unsigned 64-bit key.
__global__ void nms_scatter_kernel(const tdpm_detection *__restrict__ rec, long long n, const int32_t *__restrict__ cls,
                                   int n_classes, const int *__restrict__ offsets, int *__restrict__ cursor,
                                   unsigned long long *__restrict__ keys)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int g = nms_group(rec[i], cls, n_classes);
    uint32_t u = __float_as_uint(rec[i].score);
    u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);  // increasing with the score
    keys[offsets[g] + atomicAdd(cursor + g, 1)] = ((unsigned long long)(~u) << 32) | (unsigned long long)(uint32_t)i;
}

// Ascending bitonic sort of a[0, cnt) by the CTA: the network for the next power of two P >= cnt in the form whose
// every comparator puts the smaller key at the lower index (each merge opens with the mirrored compare). The missing
// keys a[cnt, P) count as +infinity; they never move, so the comparators that touch them are skipped.
__device__ void nms_bitonic(unsigned long long *a, int cnt)
{
    int P = 1;
    while (P < cnt) P <<= 1;
    for (int k = 2; k <= P; k <<= 1) {
        const int hk = k >> 1;
        for (int t = threadIdx.x; t < P / 2; t += blockDim.x) {
            const int blk = t / hk, pos = t - blk * hk;
            const int i = blk * k + pos, j = blk * k + k - 1 - pos;
            if (j < cnt) {
                const unsigned long long x = a[i], y = a[j];
                if (y < x) {
                    a[i] = y;
                    a[j] = x;
                }
            }
        }
        __syncthreads();
        for (int h = hk >> 1; h >= 1; h >>= 1) {
            for (int t = threadIdx.x; t < P / 2; t += blockDim.x) {
                const int i = (t / h) * 2 * h + (t % h), j = i + h;
                if (j < cnt) {
                    const unsigned long long x = a[i], y = a[j];
                    if (y < x) {
                        a[i] = y;
                        a[j] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
}

__device__ __forceinline__ NmsBox nms_box(const tdpm_detection &d, const int32_t *root_h, const int32_t *root_w,
                                          const double *cell, int max_levels)
{
    const double c = cell[(size_t)d.image * max_levels + d.level];
    const double x1 = __dmul_rn((double)d.x, c), y1 = __dmul_rn((double)d.y, c);
    return NmsBox{x1, y1, __dadd_rn(x1, __dmul_rn((double)root_w[d.component], c)),
                  __dadd_rn(y1, __dmul_rn((double)root_h[d.component], c))};
}

// The same decision as nms_covers without the FP64 division where it cannot matter: with prod = fl(overlap * area),
// inter >= prod (1 + 2^-50) implies fl(inter / area) > overlap and inter <= prod (1 - 2^-50) implies the opposite
// (every rounding involved is within 2^-53 relative, and overlap is a double, so a quotient 2^-51 above it rounds
// above it); only the band in between divides.
__device__ __forceinline__ bool nms_covers_fast(const NmsBox &a, const NmsBox &b, double overlap)
{
    const double iw = __dsub_rn(fmin(a.x2, b.x2), fmax(a.x1, b.x1));
    const double ih = __dsub_rn(fmin(a.y2, b.y2), fmax(a.y1, b.y1));
    if (!(iw > 0.0 && ih > 0.0)) return false;
    const double area = __dmul_rn(__dsub_rn(b.x2, b.x1), __dsub_rn(b.y2, b.y1));
    const double inter = __dmul_rn(iw, ih);
    const double prod = __dmul_rn(overlap, area);
    if (inter >= prod * (1.0 + 0x1p-50)) return true;
    if (inter <= prod * (1.0 - 0x1p-50)) return false;
    return __ddiv_rn(inter, area) > overlap;
}

// More than `overlap` of box b's own area covered by box a.
__device__ __forceinline__ bool nms_covers(const NmsBox &a, const NmsBox &b, double overlap)
{
    const double iw = __dsub_rn(fmin(a.x2, b.x2), fmax(a.x1, b.x1));
    const double ih = __dsub_rn(fmin(a.y2, b.y2), fmax(a.y1, b.y1));
    if (!(iw > 0.0 && ih > 0.0)) return false;
    const double area = __dmul_rn(__dsub_rn(b.x2, b.x1), __dsub_rn(b.y2, b.y1));
    return __ddiv_rn(__dmul_rn(iw, ih), area) > overlap;
}

// One CTA per group: sort the group's keys, then keep[off + p] for its detections in sorted order p. A detection's
// flag is final once every earlier one has been processed; the block barrier after each kept detection publishes
// its suppressions (global and shared writes of the block are visible to the block after the barrier).
__global__ void __launch_bounds__(NMS_THREADS) nms_group_kernel(
    const tdpm_detection *__restrict__ rec, unsigned long long *__restrict__ keys, const int *__restrict__ offsets,
    const int *__restrict__ counts, const int32_t *__restrict__ root_h, const int32_t *__restrict__ root_w,
    const double *__restrict__ cell, int max_levels, NmsBox *__restrict__ gboxes, double overlap, uint8_t *keep,
    int *__restrict__ pos_group, bool walk)
{
    extern __shared__ __align__(16) unsigned char nms_smem[];
    const int g = blockIdx.x;
    const int cnt = counts[g], off = offsets[g];
    if (cnt == 0) return;
    unsigned long long *gk = keys + off;
    if (cnt <= NMS_SORT_SMEM) {
        auto *sk = reinterpret_cast<unsigned long long *>(nms_smem);
        for (int p = threadIdx.x; p < cnt; p += blockDim.x) sk[p] = gk[p];
        __syncthreads();
        nms_bitonic(sk, cnt);
        for (int p = threadIdx.x; p < cnt; p += blockDim.x) gk[p] = sk[p];
        __syncthreads();  // the sort buffer is reused for the boxes below
    } else {
        nms_bitonic(gk, cnt);
    }
    static_assert(sizeof(NmsBox) == 32, "box layout");
    if (!walk) {
        // boxes in sorted order and each position's group, for the overlap masks and the walk that follow
        for (int p = threadIdx.x; p < cnt; p += blockDim.x) {
            gboxes[off + p] = nms_box(rec[(uint32_t)gk[p]], root_h, root_w, cell, max_levels);
            pos_group[off + p] = g;
        }
        return;
    }
    NmsBox *box = cnt <= NMS_BOX_SMEM ? reinterpret_cast<NmsBox *>(nms_smem) : gboxes + off;
    // the flags every thread reads at each step of the walk: shared memory when they fit
    uint8_t *kf = cnt <= NMS_FLAG_SMEM ? nms_smem + NMS_FLAG_OFF : keep + off;
    for (int p = threadIdx.x; p < cnt; p += blockDim.x) {
        kf[p] = 1;
        box[p] = nms_box(rec[(uint32_t)gk[p]], root_h, root_w, cell, max_levels);
    }
    __syncthreads();
    for (int i = 0; i < cnt; ++i) {
        if (!kf[i]) continue;  // the same value for every thread: written before the last barrier
        const NmsBox bi = box[i];
        for (int j = i + 1 + threadIdx.x; j < cnt; j += blockDim.x)
            if (kf[j] && nms_covers(bi, box[j], overlap)) kf[j] = 0;
        __syncthreads();
    }
    if (kf != keep + off)
        for (int p = threadIdx.x; p < cnt; p += blockDim.x) keep[off + p] = kf[p];
}

// Overlap masks: bit j - 64 w of mask[P][w] is set when sorted detection P covers the later detection j of its group,
// for every pair of every group at once: one thread per (P, j), each warp's 32 decisions gathered by a ballot into
// half a mask word.
__global__ void nms_mask_kernel(const NmsBox *__restrict__ boxes, const int *__restrict__ pos_group,
                                const int *__restrict__ offsets, const int *__restrict__ counts, long long n, int W,
                                double overlap, unsigned *__restrict__ mask32)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long per_row = (long long)W * 64;
    bool c = false;
    if (t < n * per_row) {
        const int P = (int)(t / per_row), j = (int)(t - (long long)P * per_row);
        const int g = pos_group[P], off = offsets[g], cnt = counts[g];
        if (j < cnt && j > P - off) c = nms_covers_fast(boxes[P], boxes[off + j], overlap);
    }
    const unsigned bits = __ballot_sync(0xffffffffu, c);  // n * W * 64 is a multiple of 32: no partial warps
    if ((threadIdx.x & 31) == 0 && t < n * per_row) mask32[t >> 5] = bits;
}

// One warp per group walks its detections in score order: one not yet removed is kept and removes every detection
// its mask row covers. The rows are staged 64 at a time in shared memory (from the block's own word on); the block's
// removal word is held in a register, so a step that finds its detection removed costs a bit test.
__global__ void __launch_bounds__(32) nms_walk_kernel(const unsigned long long *__restrict__ mask,
                                                      const int *__restrict__ offsets, const int *__restrict__ counts,
                                                      int W, uint8_t *__restrict__ keep)
{
    extern __shared__ unsigned long long walk_smem[];
    unsigned long long *removed = walk_smem, *blk = walk_smem + W;  // W words, then 64 x W
    const int g = blockIdx.x, lane = threadIdx.x;
    const int cnt = counts[g], off = offsets[g];
    if (cnt == 0) return;
    const int words = (cnt + 63) / 64;
    for (int w = lane; w < words; w += 32) removed[w] = 0;
    for (int b = 0; b < words; ++b) {
        const int rows = min(64, cnt - 64 * b), nw = words - b;
        __syncwarp();
        const int total = rows * nw;  // blk[r * nw + w] = row r's word b + w; eight loads in flight per lane
        for (int k0 = lane; k0 < total; k0 += 32 * 8) {
            unsigned long long v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int k = k0 + 32 * u;
                if (k < total) {
                    const int r = k / nw;
                    v[u] = mask[(size_t)(off + 64 * b + r) * W + b + (k - r * nw)];
                }
            }
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (k0 + 32 * u < total) blk[k0 + 32 * u] = v[u];
        }
        __syncwarp();
        unsigned long long cur = removed[b];
        for (int r = 0; r < rows; ++r) {
            if ((cur >> r) & 1ull) continue;  // the same for every lane
            cur |= blk[r * nw];
            for (int w = 1 + lane; w < nw; w += 32) removed[b + w] |= blk[r * nw + w];
        }
        // a row's bit is final once the rows before it are done: later rows only set later bits
        for (int r = lane; r < rows; r += 32) keep[off + 64 * b + r] = ((cur >> r) & 1ull) ? 0 : 1;
    }
}

// The kept flags in record order.
__global__ void nms_mark_kernel(const unsigned long long *__restrict__ keys, const uint8_t *__restrict__ keep,
                                long long n, uint8_t *__restrict__ kept)
{
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) kept[(uint32_t)keys[p]] = keep[p];
}

size_t align256z(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

namespace {
// Flagged records per block of NMS_CBLOCK.
__global__ void __launch_bounds__(NMS_CBLOCK) compact_count_kernel(const uint8_t *__restrict__ kept, long long n,
                                                                   int *__restrict__ bcount)
{
    __shared__ int ws[NMS_CBLOCK / 32];
    const long long i = (long long)blockIdx.x * NMS_CBLOCK + threadIdx.x;
    const unsigned b = __ballot_sync(0xffffffffu, i < n && kept[i]);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = __popc(b);
    __syncthreads();
    if (threadIdx.x < 32) {
        int s = ws[threadIdx.x];
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) bcount[blockIdx.x] = s;
    }
}

// The flagged records of each block at the block's offset, in record order.
__global__ void __launch_bounds__(NMS_CBLOCK) compact_write_kernel(const tdpm_detection *__restrict__ rec,
                                                                   const uint8_t *__restrict__ kept, long long n,
                                                                   const int *__restrict__ boff,
                                                                   tdpm_detection *__restrict__ out)
{
    __shared__ int ws[NMS_CBLOCK / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long i = (long long)blockIdx.x * NMS_CBLOCK + threadIdx.x;
    const bool k = i < n && kept[i];
    const unsigned b = __ballot_sync(0xffffffffu, k);
    if (lane == 0) ws[w] = __popc(b);
    __syncthreads();
    int before = 0;
    for (int v = 0; v < w; ++v) before += ws[v];
    if (k) out[boff[blockIdx.x] + before + __popc(b & ((1u << lane) - 1u))] = rec[i];
}

}  // namespace

size_t compact_scratch_bytes(long long n)
{
    const size_t nb = ((size_t)std::max<long long>(n, 1) + NMS_CBLOCK - 1) / NMS_CBLOCK;
    return 2 * align256z(4 * nb);
}

cudaError_t launch_compact_records(const tdpm_detection *d_rec, const uint8_t *d_flags, long long n, void *d_scratch,
                                   size_t scratch_bytes, tdpm_detection *d_out, long long *d_n_out, cudaStream_t s)
{
    if (n <= 0) return cudaMemsetAsync(d_n_out, 0, sizeof(long long), s);
    if (n > (1ll << 30) || scratch_bytes < compact_scratch_bytes(n)) return cudaErrorInvalidValue;
    const int nb = (int)((n + NMS_CBLOCK - 1) / NMS_CBLOCK);
    auto *bcount = static_cast<int *>(d_scratch);
    auto *boff = reinterpret_cast<int *>(static_cast<char *>(d_scratch) + align256z(4 * (size_t)nb));
    note_launches(3);
    compact_count_kernel<<<nb, NMS_CBLOCK, 0, s>>>(d_flags, n, bcount);
    nms_scan_kernel<<<1, NMS_THREADS, 0, s>>>(bcount, nb, boff, d_n_out);
    compact_write_kernel<<<nb, NMS_CBLOCK, 0, s>>>(d_rec, d_flags, n, boff, d_out);
    return cudaGetLastError();
}

constexpr long long NMS_MASK_MAX = 16384;  // up to this many detections the overlaps go through masks

size_t nms_scratch_bytes(long long n, int n_groups)
{
    const size_t nn = (size_t)std::max<long long>(n, 1);
    const size_t W = (nn + 63) / 64;
    const size_t mask_b = n <= NMS_MASK_MAX ? align256z(8 * nn * W) : 0;
    return align256z(8 * nn) + align256z(sizeof(NmsBox) * nn) + 2 * align256z(nn) + align256z(4 * nn) + mask_b +
           3 * align256z(4 * (size_t)std::max(n_groups, 1)) + compact_scratch_bytes(n);
}

cudaError_t launch_nms(const tdpm_detection *d_rec, long long n, const int32_t *d_cls, int n_classes, int n_images,
                       const int32_t *d_root_h, const int32_t *d_root_w, const double *d_cell, int max_levels,
                       double overlap, void *d_scratch, size_t scratch_bytes, tdpm_detection *d_out,
                       long long *d_n_out, cudaStream_t s)
{
    if (n <= 0) return cudaMemsetAsync(d_n_out, 0, sizeof(long long), s);
    if (n > (1ll << 30) || n_classes < 1 || n_images < 1 || (long long)n_images * n_classes > 0x7fffffffll)
        return cudaErrorInvalidValue;
    const int n_groups = n_images * n_classes;
    if (scratch_bytes < nms_scratch_bytes(n, n_groups)) return cudaErrorInvalidValue;
    char *p = static_cast<char *>(d_scratch);
    auto take = [&](size_t b) {
        char *q = p;
        p += align256z(b);
        return q;
    };
    auto *keys = reinterpret_cast<unsigned long long *>(take(8 * (size_t)n));
    auto *boxes = reinterpret_cast<NmsBox *>(take(sizeof(NmsBox) * (size_t)n));
    auto *keep = reinterpret_cast<uint8_t *>(take((size_t)n));
    auto *kept = reinterpret_cast<uint8_t *>(take((size_t)n));
    auto *pos_group = reinterpret_cast<int *>(take(4 * (size_t)n));
    const bool use_mask = n <= NMS_MASK_MAX;
    const int W = (int)((n + 63) / 64);
    auto *mask = use_mask ? reinterpret_cast<unsigned long long *>(take(8 * (size_t)n * W)) : nullptr;
    auto *counts = reinterpret_cast<int *>(take(4 * (size_t)n_groups));
    auto *offsets = reinterpret_cast<int *>(take(4 * (size_t)n_groups));
    auto *cursor = reinterpret_cast<int *>(take(4 * (size_t)n_groups));
    void *cscratch = p;
    const size_t cbytes = scratch_bytes - (size_t)(p - static_cast<char *>(d_scratch));
    cudaError_t e = allow_max_dynamic_smem(reinterpret_cast<const void *>(nms_group_kernel), 25);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(counts, 0, 4 * (size_t)n_groups, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(cursor, 0, 4 * (size_t)n_groups, s)) != cudaSuccess) return e;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    note_launches(use_mask ? 7 : 5);
    nms_count_kernel<<<blocks, 256, 0, s>>>(d_rec, n, d_cls, n_classes, counts);
    nms_scan_kernel<<<1, NMS_THREADS, 0, s>>>(counts, n_groups, offsets, nullptr);
    nms_scatter_kernel<<<blocks, 256, 0, s>>>(d_rec, n, d_cls, n_classes, offsets, cursor, keys);
    // sort each group; then either masks of every pair on the whole GPU and a one-warp walk per group, or (very
    // large inputs) the walk inside the group's CTA
    nms_group_kernel<<<n_groups, NMS_THREADS, NMS_SMEM_BYTES, s>>>(d_rec, keys, offsets, counts, d_root_h, d_root_w,
                                                                   d_cell, max_levels, boxes, overlap, keep, pos_group,
                                                                   !use_mask);
    if (use_mask) {
        const long long items = n * W * 64;
        nms_mask_kernel<<<(unsigned)((items + 255) / 256), 256, 0, s>>>(boxes, pos_group, offsets, counts, n, W,
                                                                         overlap, reinterpret_cast<unsigned *>(mask));
        e = allow_max_dynamic_smem(reinterpret_cast<const void *>(nms_walk_kernel), 26);
        if (e != cudaSuccess) return e;
        nms_walk_kernel<<<n_groups, 32, 8 * (size_t)W * 65, s>>>(mask, offsets, counts, W, keep);
    }
    nms_mark_kernel<<<blocks, 256, 0, s>>>(keys, keep, n, kept);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return launch_compact_records(d_rec, kept, n, cscratch, cbytes, d_out, d_n_out, s);
}

}  // namespace tdpm
