// tdpm_dt_noalloc: the distance transform of tdpm_dt with its scratch in a fixed device array, for callers that
// cannot allocate device memory (see include/tdpm.h).
//
// The scratch (job record, x-pass values and argmax) lives in a file-scope __device__ array that every GPU loading
// the library holds until the process exits. Host code cannot use the array's name as a device address, so the first
// call on each device looks the address up with cudaGetSymbolAddress (with that device current) and keeps it.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "ctx.h"

namespace tdpm {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(4) << 20;  // 4 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_dt_scratch[kNoAllocScratchBytes];

std::mutex g_setup_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of g_dt_scratch on the current device (looked up once per device).
tdpm_status scratch_address(void **out)
{
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(TDPM_ERR_ARG, "device index above the supported range");
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_dt_scratch);
        if (e != cudaSuccess || !p)
            return fail(TDPM_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return TDPM_OK;
}

// Writes the job record into the scratch array. The record travels as a kernel parameter, so the call makes no copy
// from host memory: nothing waits for the stream, and no host buffer has to outlive the call.
__global__ void dt_store_job_kernel(DtJob J, DtJob *dst) { *dst = J; }

}  // namespace
}  // namespace tdpm

using namespace tdpm;

extern "C" {

size_t tdpm_dt_noalloc_max_elements(void)
{
    return (kNoAllocScratchBytes - align256(sizeof(DtJob)) - 256) / (sizeof(float) + sizeof(int32_t));
}

tdpm_status tdpm_dt_noalloc(const float *S, int32_t H, int32_t W, const float d[4], int32_t x_off, int32_t x_step,
                            int32_t nx, int32_t y_off, int32_t y_step, int32_t ny, float *D, int32_t *arg,
                            void *stream)
{
    clear_error();
    if (!S || !d || !D || !arg) return fail(TDPM_ERR_ARG, "NULL argument");
    if (H <= 0 || W <= 0 || H > kDtMaxSide || W > kDtMaxSide)
        return fail(TDPM_ERR_ARG, "map sides must be in [1, " + std::to_string(kDtMaxSide) + "]");
    for (int k = 0; k < 4; ++k)
        if (!std::isfinite(d[k])) return fail(TDPM_ERR_ARG, "non-finite deformation coefficient");
    if (!(d[1] > 0.f) || !(d[3] > 0.f)) return fail(TDPM_ERR_ARG, "quadratic coefficients must be > 0");
    if (nx <= 0 || ny <= 0 || x_step <= 0 || y_step <= 0 || x_off < 0 || y_off < 0 ||
        (long long)x_off + (long long)x_step * (nx - 1) >= W || (long long)y_off + (long long)y_step * (ny - 1) >= H)
        return fail(TDPM_ERR_ARG, "sampled positions outside the map");
    if ((size_t)H * (size_t)nx > tdpm_dt_noalloc_max_elements())
        return fail(TDPM_ERR_ARG, "H * nx = " + std::to_string((size_t)H * nx) +
                                      " exceeds the fixed scratch of tdpm_dt_noalloc (" +
                                      std::to_string(tdpm_dt_noalloc_max_elements()) + " elements)");
    void *base = nullptr;
    tdpm_status st = scratch_address(&base);
    if (st) return st;
    char *sb = reinterpret_cast<char *>(base);
    const size_t v_off = align256(sizeof(DtJob));
    const size_t iv_off = v_off + align256(sizeof(float) * (size_t)H * nx);
    DtJob J{};
    J.S = S; J.H = H; J.W = W;
    J.lx = d[0]; J.qx = d[1]; J.ly = d[2]; J.qy = d[3];
    J.x_off = x_off; J.x_step = x_step; J.nx = nx;
    J.y_off = y_off; J.y_step = y_step; J.ny = ny;
    J.V = reinterpret_cast<float *>(sb + v_off);
    J.IV = reinterpret_cast<int32_t *>(sb + iv_off);
    J.D = D; J.A = arg;
    J.xbegin = 0; J.ybegin = 0;
    cudaStream_t s = (cudaStream_t)stream;
    note_launches(1);
    dt_store_job_kernel<<<1, 1, 0, s>>>(J, reinterpret_cast<DtJob *>(sb));
    CUDA_TRY(cudaGetLastError());
    const int lpc = dt_lines_per_cta();
    CUDA_TRY(launch_dt(reinterpret_cast<const DtJob *>(sb), 1, (H + lpc - 1) / lpc, (nx + lpc - 1) / lpc, W, H, s));
    return TDPM_OK;
}

}  // extern "C"
