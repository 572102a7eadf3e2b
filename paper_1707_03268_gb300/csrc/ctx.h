// Host-side state of a tdpm context (shared by model.cu and pipeline.cu; not part of the C-ABI).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace tdpm {

tdpm_status fail(tdpm_status st, const std::string &msg);
void clear_error();

#define CUDA_TRY(expr)                                                                                           \
    do {                                                                                                         \
        cudaError_t _e = (expr);                                                                                 \
        if (_e != cudaSuccess) return ::tdpm::fail(TDPM_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
    } while (0)

inline size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// ------------------------------------------------------------------------------------------------------ model
struct FilterH {
    int h, w, role, comp, part, group, gidx;
    std::vector<float> data;  // [h][w][32]
};

struct PartH {
    int fid, vy, vx;
    float d[4];
};

struct CompH {
    int root_fid;
    float bias;
    std::vector<PartH> parts;
};

// Filters of one role (root / part) and one shape. Device copies of the full filters and, once decomposed, of the
// CP factors (Sec. 4): A [h][R], B [w][R], C [32][R], Lambda [K][R].
struct Group {
    int role = 0, h = 0, w = 0, K = 0;
    std::vector<int> fids;
    int Kpad = 0;                        // FP32 SIMT layout padding (multiple of 64)
    float *d_filt_t = nullptr;           // [h*w*32][Kpad] FP32
    int Npad_tc = 0;                     // tensor-core bank rows (K padded for every candidate N tiling)
    uint8_t *d_filt_fp8 = nullptr;       // [h*w][2][Npad_tc][16] E4M3 bytes of the filters times fp8_scale
    float fp8_scale = 1.f;               // per-tensor scale of that bank (448 / max |filter value|)
    uint16_t *d_filt_tc = nullptr;       // [h*w][4][Npad_tc][8] BF16 (hi part: bf16(x))
    uint16_t *d_filt_tc_lo = nullptr;    // lo part bf16(x - bf16(x)), same layout (split-BF16 precision)
    // decomposition, FP64 master copies
    int R = 0, joint = 0;
    std::vector<double> A, B, C, Lam;
    std::vector<int> rank_off;           // per-filter mode: filter k owns terms [rank_off[k], rank_off[k+1])
    std::vector<double> rel_err;         // per filter
    // FP32 device copies (the 1-D passes run in FP32 for every precision)
    float *d_A = nullptr, *d_B = nullptr, *d_Ct = nullptr, *d_lam = nullptr;
    int *d_rank_off = nullptr;
    int Rpad_tc = 0;                     // rows of the channel-factor bank
    uint16_t *d_C_tc = nullptr;          // [1][4][Rpad_tc][8] BF16: the channel factor as a 1x1 "filter bank"
    uint16_t *d_C_tc_lo = nullptr;       // its lo part
    uint8_t *d_C_fp8 = nullptr;          // [1][2][Rpad_tc][16] E4M3 channel factor times C_fp8_scale
    float C_fp8_scale = 1.f;
    // joint mode on tensor cores: per-term maps U_r are recombined by S = Lambda U as a GEMM over Upad terms
    int Upad = 0;                        // R rounded up to a multiple of 32 (zero terms beyond R)
    int Npad_lam = 0;                    // rows of the Lambda bank
    uint16_t *d_lam_tc = nullptr;        // [Upad/32][4][Npad_lam][8] BF16: Lambda as a bank of K "filters"
    uint16_t *d_lam_tc_lo = nullptr;     // its lo part

    void free_factors();
    void free_all();
};

struct Model {
    std::vector<FilterH> filters;
    std::vector<CompH> comps;
    std::vector<Group> groups;
    bool decomposed = false;
    int decomp_mode = 0;
    int version = 0;                     // bumped whenever the factors change (invalidates cached plans)
};

// ------------------------------------------------------------------------------------------------------ scores
struct MapRef {
    size_t off = 0;  // byte offset in the arena
    int rows = 0, cols = 0;
};

struct Plan;  // pipeline.cu

// One device arena (score maps, intermediates, job tables) with its pinned host copy of the job tables and, once
// captured, a CUDA graph of the whole enqueue for the plan it was last filled for.
struct Arena {
    char *dev = nullptr;
    char *host = nullptr;
    size_t bytes = 0, host_bytes = 0;
    uint64_t plan_uid = 0;               // plan whose job tables the host blob currently holds (0: none)
    std::vector<const void *> levels;    // level pointers patched into the blob
    cudaGraphExec_t graph = nullptr;
    int graph_kernels = 0;               // kernel launches captured in `graph` (counted again at each replay)
    int uses = 0;
    bool blob_on_device = false;         // the device copy of the job tables matches the host blob
};

struct Scores {
    int model_id = 0;
    std::shared_ptr<Plan> plan;
    Arena arena;
    cudaEvent_t done = nullptr;
};

struct Pending {
    std::string name;
    cudaEvent_t a, b;
};

}  // namespace tdpm

constexpr int kSideStreams = 4;

namespace tdpm {
struct Server;  // serve.cpp
}

struct tdpm_ctx {
    int device = 0;
    size_t budget = 0, used = 0;
    std::mutex mu;
    int next_id = 1;
    std::map<int, std::unique_ptr<tdpm::Model>> models;
    std::map<int, std::unique_ptr<tdpm::Scores>> scores;
    std::map<std::string, std::shared_ptr<tdpm::Plan>> plans;
    std::vector<tdpm::Arena> free_arenas;
    cudaStream_t cap_stream = nullptr;   // private stream for graph capture
    // the shape groups' correlation chains are independent: they run on side streams forked from (and joined back
    // into) the caller's stream, as parallel branches of a captured graph
    std::vector<cudaStream_t> side;
    cudaEvent_t fork_ev = nullptr;
    std::vector<cudaEvent_t> join_ev;
    tdpm::Server *server = nullptr;      // the serving loop, when started
    // device buffer the detection records are written to before their copy to the caller: one per context, grown on
    // demand (tdpm_detect calls are serialised by the context lock and finish before they return)
    tdpm_detection *d_records = nullptr;
    size_t rec_cap = 0;
    float *d_job_tau = nullptr;          // per-job thresholds of the current tdpm_detect_thresholds call
    size_t tau_cap = 0;
    int *d_err = nullptr;                // raised by bounded device waits
    int *h_err = nullptr;                // pinned mirror
    long long *h_total = nullptr;        // pinned: detection count read back with the records
    std::unordered_map<uint64_t, size_t> det_last;  // plan uid -> detections of its last read-back (copy size hint)
    void *d_nms = nullptr;               // grow-only scratch of tdpm_detect_nms
    size_t nms_cap = 0;
    void *d_hog = nullptr;               // grow-only scratch of the HOG pyramid calls (images, gradients, cells, tables)
    size_t hog_cap = 0;
    cudaEvent_t hog_done = nullptr;      // recorded after each HOG call's work; the next one waits before reusing d_hog
    std::string hog_key;                 // the pyramid call whose job tables d_hog holds ("" after any other HOG call)
    cudaGraphExec_t hog_graph = nullptr; // that call's launches, captured once it repeats
    int hog_graph_kernels = 0, hog_uses = 0;
    bool use_graphs = true;
    bool fuse = true;                    // fused channel stage + separable passes where possible (tdpm_set_fusion)
    int zsep_form = -1;                  // fused kernel form forced by TDPM_ZSEP_FORM (-1: default / tuned)
    bool autotune = true;                // time the N tilings of a new plan's tensor-core launches (TDPM_AUTOTUNE=0: off)
    std::map<std::string, int> tune_cache;  // shape class of a tensor-core launch -> chosen N tile width
    // profiling
    bool prof = false;
    std::vector<tdpm::Pending> pending;
    std::vector<std::pair<std::string, std::pair<double, long long>>> stages;
    std::vector<cudaEvent_t> event_pool;
};

namespace tdpm {

tdpm_status set_device(tdpm_ctx *ctx);
Model *get_model(tdpm_ctx *ctx, int id);
void free_scores(tdpm_ctx *ctx, Scores &s);
void arena_free(tdpm_ctx *ctx, Arena &a);
void drop_plans_of_model(tdpm_ctx *ctx, int model_id);
// Device bytes of the arena a batch needs (makes, or finds, and caches its plan).
tdpm_status batch_arena_bytes(tdpm_ctx *ctx, int32_t model_id, const tdpm_pyramid *pyrs, int32_t n_images,
                              const uint8_t *mask, int32_t form, int32_t precision, size_t *bytes);
// Stop the server thread (finishing its requests) and free it; the caller must not hold ctx->mu.
void server_free(tdpm_ctx *ctx);

template <class T>
tdpm_status upload(T **dst, const std::vector<T> &src)
{
    CUDA_TRY(cudaMalloc(dst, sizeof(T) * std::max<size_t>(src.size(), 1)));
    if (!src.empty()) CUDA_TRY(cudaMemcpy(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice));
    return TDPM_OK;
}

uint16_t bf16_bits(float x);
float bf16_round(float x);
uint8_t e4m3_bits(float x);  // E4M3 encoding, round to nearest even, saturated at +-448
inline bool valid_precision(int p)
{
    return p == TDPM_PREC_FP32 || p == TDPM_PREC_BF16 || p == TDPM_PREC_FP8 || p == TDPM_PREC_BF16X3;
}

}  // namespace tdpm
