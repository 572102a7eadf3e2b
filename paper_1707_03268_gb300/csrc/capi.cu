// C-ABI of libtdpm: context, model, decomposition, pyramid scoring and detection (declarations in include/tdpm.h).
//
// A scores set plans every stage of one pyramid on the host (job tables for each launch, map offsets in one device
// arena), uploads the tables with a single copy and enqueues one launch per stage: correlation per shape group
// (all levels in one launch), the two distance-transform passes over all part maps, and the assembly.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "als.h"
#include "internal.h"

using namespace tdpm;

namespace {

thread_local std::string g_err;

tdpm_status fail(tdpm_status st, const std::string &msg)
{
    g_err = msg;
    return st;
}

#define CUDA_TRY(expr)                                                                                   \
    do {                                                                                                 \
        cudaError_t _e = (expr);                                                                         \
        if (_e != cudaSuccess) return fail(TDPM_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
    } while (0)

float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

int fdiv2(int a) { return a >= 0 ? a / 2 : -((-a + 1) / 2); }

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// ------------------------------------------------------------------------------------------------------ model
struct FilterH {
    int h, w, role, comp, part, group, gidx;
    std::vector<float> data;
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

struct Group {
    int role = 0, h = 0, w = 0, K = 0, Kpad = 0;
    std::vector<int> fids;
    float *d_filt_t = nullptr;          // [h*w*32][Kpad] FP32
    // decomposition (Sec. 4): A [h][R], B [w][R], C [32][R], Lam [K][R], FP64 master copies
    int R = 0, joint = 0;
    std::vector<double> A, B, C, Lam;
    std::vector<int> rank_off;          // per-filter mode: filter k owns terms [rank_off[k], rank_off[k+1])
    std::vector<double> rel_err;        // per filter
    float *d_A[2] = {nullptr, nullptr}, *d_B[2] = {nullptr, nullptr}, *d_Ct[2] = {nullptr, nullptr},
          *d_lam[2] = {nullptr, nullptr};
    int *d_rank_off = nullptr;

    void free_factors()
    {
        for (int p = 0; p < 2; ++p) {
            cudaFree(d_A[p]); cudaFree(d_B[p]); cudaFree(d_Ct[p]); cudaFree(d_lam[p]);
            d_A[p] = d_B[p] = d_Ct[p] = d_lam[p] = nullptr;
        }
        cudaFree(d_rank_off);
        d_rank_off = nullptr;
    }
};

struct Model {
    std::vector<FilterH> filters;
    std::vector<CompH> comps;
    std::vector<Group> groups;
    bool decomposed = false;
    int decomp_mode = 0;
};

// ------------------------------------------------------------------------------------------------------ scores
struct MapRef {
    size_t off = 0;  // byte offset in the arena
    int rows = 0, cols = 0;
};

struct Arena {
    char *dev = nullptr;
    char *host = nullptr;  // pinned staging for the job tables
    size_t bytes = 0, host_bytes = 0;
};

struct Scores {
    int model_id = 0;
    Arena arena;
    std::map<std::pair<int, int>, MapRef> filter_maps, final_maps, dt_maps, arg_maps;
    AsmJob *d_asm = nullptr;
    int n_asm = 0;
    long long total = 0;
    int n_det_blocks = 0;
    int *d_counts = nullptr, *d_offsets = nullptr;
    long long *d_total = nullptr;
    tdpm_detection *d_records = nullptr;
    size_t rec_cap = 0;
    cudaEvent_t done = nullptr;
};

}  // namespace

namespace {
struct Pending {
    std::string name;
    cudaEvent_t a, b;
};
std::atomic<unsigned long long> g_launches{0};
}  // namespace

void tdpm::note_launches(int n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }

struct tdpm_ctx {
    int device = 0;
    bool prof = false;
    std::vector<Pending> pending;
    std::vector<std::pair<std::string, std::pair<double, long long>>> stages;
    std::vector<cudaEvent_t> event_pool;
    size_t budget = 0, used = 0;
    std::mutex mu;
    int next_id = 1;
    std::map<int, std::unique_ptr<Model>> models;
    std::map<int, std::unique_ptr<Scores>> scores;
    std::vector<Arena> free_arenas;
};

namespace {

tdpm_status set_device(tdpm_ctx *ctx)
{
    CUDA_TRY(cudaSetDevice(ctx->device));
    return TDPM_OK;
}

void arena_free(tdpm_ctx *ctx, Arena &a)
{
    if (a.dev) cudaFree(a.dev);
    if (a.host) cudaFreeHost(a.host);
    ctx->used -= std::min(ctx->used, a.bytes);
    a = Arena{};
}

tdpm_status arena_get(tdpm_ctx *ctx, size_t bytes, size_t host_bytes, Arena &out)
{
    for (size_t i = 0; i < ctx->free_arenas.size(); ++i) {
        Arena &a = ctx->free_arenas[i];
        if (a.bytes >= bytes && a.bytes <= bytes + bytes / 4 + (1 << 20) && a.host_bytes >= host_bytes) {
            out = a;
            ctx->free_arenas.erase(ctx->free_arenas.begin() + i);
            return TDPM_OK;
        }
    }
    while (ctx->budget && ctx->used + bytes > ctx->budget && !ctx->free_arenas.empty()) {
        arena_free(ctx, ctx->free_arenas.back());
        ctx->free_arenas.pop_back();
    }
    if (ctx->budget && ctx->used + bytes > ctx->budget)
        return fail(TDPM_ERR_OOM, "scores need " + std::to_string(bytes) + " bytes; budget " +
                                      std::to_string(ctx->budget) + ", in use " + std::to_string(ctx->used));
    Arena a;
    cudaError_t e = cudaMalloc(&a.dev, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(TDPM_ERR_OOM, std::string("cudaMalloc arena: ") + cudaGetErrorString(e));
    }
    e = cudaMallocHost(&a.host, host_bytes);
    if (e != cudaSuccess) {
        cudaFree(a.dev);
        return fail(TDPM_ERR_OOM, std::string("cudaMallocHost staging: ") + cudaGetErrorString(e));
    }
    a.bytes = bytes;
    a.host_bytes = host_bytes;
    ctx->used += bytes;
    out = a;
    return TDPM_OK;
}

void arena_put(tdpm_ctx *ctx, Arena &a)
{
    if (!a.dev) return;
    ctx->free_arenas.push_back(a);
    a = Arena{};
    while (ctx->free_arenas.size() > 8) {
        arena_free(ctx, ctx->free_arenas.front());
        ctx->free_arenas.erase(ctx->free_arenas.begin());
    }
}

Model *get_model(tdpm_ctx *ctx, int id)
{
    auto it = ctx->models.find(id);
    return it == ctx->models.end() ? nullptr : it->second.get();
}

Scores *get_scores(tdpm_ctx *ctx, int id)
{
    auto it = ctx->scores.find(id);
    return it == ctx->scores.end() ? nullptr : it->second.get();
}

cudaEvent_t prof_event(tdpm_ctx *ctx)
{
    if (!ctx->event_pool.empty()) {
        cudaEvent_t e = ctx->event_pool.back();
        ctx->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Bracket one stage with CUDA events on its stream when the context profiles (no-op otherwise).
struct Prof {
    tdpm_ctx *ctx;
    cudaStream_t s;
    const char *name;
    cudaEvent_t a = nullptr;
    Prof(tdpm_ctx *c, cudaStream_t st, const char *n) : ctx(c), s(st), name(n)
    {
        if (ctx->prof && (a = prof_event(ctx))) cudaEventRecord(a, s);
    }
    void end()
    {
        if (!a) return;
        cudaEvent_t b = prof_event(ctx);
        if (b) {
            cudaEventRecord(b, s);
            ctx->pending.push_back(Pending{name, a, b});
        } else {
            ctx->event_pool.push_back(a);
        }
        a = nullptr;
    }
};

void prof_collect(tdpm_ctx *ctx)
{
    for (Pending &p : ctx->pending) {
        float ms = 0.f;
        cudaEventSynchronize(p.b);
        cudaEventElapsedTime(&ms, p.a, p.b);
        size_t i = 0;
        while (i < ctx->stages.size() && ctx->stages[i].first != p.name) ++i;
        if (i == ctx->stages.size()) ctx->stages.push_back({p.name, {0.0, 0}});
        ctx->stages[i].second.first += ms;
        ctx->stages[i].second.second += 1;
        ctx->event_pool.push_back(p.a);
        ctx->event_pool.push_back(p.b);
    }
    ctx->pending.clear();
}

template <class T>
tdpm_status upload(T **dst, const std::vector<T> &src)
{
    CUDA_TRY(cudaMalloc(dst, sizeof(T) * std::max<size_t>(src.size(), 1)));
    if (!src.empty()) CUDA_TRY(cudaMemcpy(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice));
    return TDPM_OK;
}

// Upload the FP32 and BF16-rounded device copies of a group's factors.
tdpm_status upload_factors(Group &g)
{
    g.free_factors();
    const int R = g.R, K = (int)g.fids.size();
    for (int p = 0; p < 2; ++p) {
        auto cvt = [p](double v) { return p ? bf16_round((float)v) : (float)v; };
        std::vector<float> A(g.A.size()), B(g.B.size()), Ct((size_t)R * FD), lam;
        for (size_t i = 0; i < A.size(); ++i) A[i] = cvt(g.A[i]);
        for (size_t i = 0; i < B.size(); ++i) B[i] = cvt(g.B[i]);
        for (int r = 0; r < R; ++r)
            for (int c = 0; c < FD; ++c) Ct[(size_t)r * FD + c] = cvt(g.C[(size_t)c * R + r]);
        if (g.joint) {
            lam.resize((size_t)K * R);
            for (size_t i = 0; i < lam.size(); ++i) lam[i] = cvt(g.Lam[i]);
        } else {
            lam.resize(R);
            for (int k = 0; k < K; ++k)
                for (int r = g.rank_off[k]; r < g.rank_off[k + 1]; ++r) lam[r] = cvt(g.Lam[(size_t)k * R + r]);
        }
        tdpm_status st;
        if ((st = upload(&g.d_A[p], A)) || (st = upload(&g.d_B[p], B)) || (st = upload(&g.d_Ct[p], Ct)) ||
            (st = upload(&g.d_lam[p], lam)))
            return st;
    }
    std::vector<int> ro = g.rank_off;
    if (ro.empty()) ro.assign(K + 1, 0);
    return upload(&g.d_rank_off, ro);
}

void free_model(Model &m)
{
    for (Group &g : m.groups) {
        cudaFree(g.d_filt_t);
        g.d_filt_t = nullptr;
        g.free_factors();
    }
}

void free_scores(tdpm_ctx *ctx, Scores &s)
{
    if (s.done) {
        cudaEventSynchronize(s.done);
        cudaEventDestroy(s.done);
        s.done = nullptr;
    }
    if (s.d_records) {
        cudaFree(s.d_records);
        ctx->used -= std::min(ctx->used, s.rec_cap * sizeof(tdpm_detection));
        s.d_records = nullptr;
    }
    arena_put(ctx, s.arena);
}

// ------------------------------------------------------------------------------------------------ planning
struct Bump {
    size_t off = 0;
    size_t take(size_t bytes)
    {
        const size_t o = align256(off);
        off = o + bytes;
        return o;
    }
};

}  // namespace

namespace {
const char kMagic[8] = {'T', 'D', 'P', 'M', 'F', 'A', 'C', '1'};

uint64_t fnv1a(const std::vector<char> &b)
{
    uint64_t h = 1469598103934665603ull;
    for (char c : b) {
        h ^= (uint8_t)c;
        h *= 1099511628211ull;
    }
    return h;
}

template <class T>
void put(std::vector<char> &b, const T &v)
{
    const char *p = reinterpret_cast<const char *>(&v);
    b.insert(b.end(), p, p + sizeof(T));
}

template <class T>
void put_vec(std::vector<char> &b, const std::vector<T> &v)
{
    const char *p = reinterpret_cast<const char *>(v.data());
    b.insert(b.end(), p, p + sizeof(T) * v.size());
}

struct Reader {
    const std::vector<char> &b;
    size_t pos = 0;
    bool ok = true;
    template <class T>
    T get()
    {
        T v{};
        if (pos + sizeof(T) > b.size()) { ok = false; return v; }
        std::memcpy(&v, b.data() + pos, sizeof(T));
        pos += sizeof(T);
        return v;
    }
    template <class T>
    void get_vec(std::vector<T> &v, size_t n)
    {
        if (pos + sizeof(T) * n > b.size()) { ok = false; return; }
        v.resize(n);
        std::memcpy(v.data(), b.data() + pos, sizeof(T) * n);
        pos += sizeof(T) * n;
    }
};
}  // namespace

// =================================================================================================== ABI
extern "C" {

const char *tdpm_last_error(void) { return g_err.c_str(); }

const char *tdpm_version(void)
{
    static std::string v = std::string("libtdpm sm_103a cuda ") + std::to_string(CUDART_VERSION);
    return v.c_str();
}

tdpm_status tdpm_create(tdpm_ctx **out, int32_t device, size_t mem_budget_bytes)
{
    g_err.clear();
    if (!out) return fail(TDPM_ERR_ARG, "out is NULL");
    *out = nullptr;
    int n = 0;
    CUDA_TRY(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n) return fail(TDPM_ERR_ARG, "device index out of range");
    CUDA_TRY(cudaSetDevice(device));
    tdpm_ctx *c = new (std::nothrow) tdpm_ctx;
    if (!c) return fail(TDPM_ERR_OOM, "host allocation failed");
    c->device = device;
    c->budget = mem_budget_bytes;
    *out = c;
    return TDPM_OK;
}

void tdpm_destroy(tdpm_ctx *ctx)
{
    if (!ctx) return;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        cudaSetDevice(ctx->device);
        for (auto &kv : ctx->scores) free_scores(ctx, *kv.second);
        ctx->scores.clear();
        for (auto &kv : ctx->models) free_model(*kv.second);
        ctx->models.clear();
        for (Arena &a : ctx->free_arenas) arena_free(ctx, a);
        ctx->free_arenas.clear();
        prof_collect(ctx);
        for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
        ctx->event_pool.clear();
    }
    delete ctx;
}

tdpm_status tdpm_load_model(tdpm_ctx *ctx, const tdpm_model_desc *desc, int32_t *model_id)
{
    g_err.clear();
    if (!ctx || !desc || !model_id) return fail(TDPM_ERR_ARG, "NULL argument");
    if (desc->n_components <= 0 || !desc->components) return fail(TDPM_ERR_ARG, "model has no components");
    std::lock_guard<std::mutex> lk(ctx->mu);
    tdpm_status st = set_device(ctx);
    if (st) return st;
    auto m = std::make_unique<Model>();
    auto add_filter = [&](const tdpm_filter &f, int role, int comp, int part, int *fid) -> tdpm_status {
        if (f.h <= 0 || f.w <= 0 || !f.data) return fail(TDPM_ERR_ARG, "filter with non-positive size or NULL data");
        if (f.h > 64 || f.w > 64) return fail(TDPM_ERR_ARG, "filter side above 64 cells");
        FilterH F;
        F.h = f.h; F.w = f.w; F.role = role; F.comp = comp; F.part = part;
        F.data.assign(f.data, f.data + (size_t)f.h * f.w * FD);
        int g = -1;
        for (size_t i = 0; i < m->groups.size(); ++i)
            if (m->groups[i].role == role && m->groups[i].h == f.h && m->groups[i].w == f.w) g = (int)i;
        if (g < 0) {
            Group G;
            G.role = role; G.h = f.h; G.w = f.w;
            m->groups.push_back(G);
            g = (int)m->groups.size() - 1;
        }
        F.group = g;
        F.gidx = (int)m->groups[g].fids.size();
        *fid = (int)m->filters.size();
        m->groups[g].fids.push_back(*fid);
        m->filters.push_back(std::move(F));
        return TDPM_OK;
    };
    for (int c = 0; c < desc->n_components; ++c) {
        const tdpm_component &C = desc->components[c];
        if (C.n_parts < 0 || C.n_parts > TDPM_MAX_PARTS) return fail(TDPM_ERR_ARG, "n_parts out of range");
        if (C.n_parts > 0 && !C.parts) return fail(TDPM_ERR_ARG, "parts is NULL");
        CompH ch;
        ch.bias = C.bias;
        if ((st = add_filter(C.root, 0, c, -1, &ch.root_fid))) return st;
        for (int i = 0; i < C.n_parts; ++i) {
            const tdpm_part &P = C.parts[i];
            if (!(P.deform[1] > 0.f) || !(P.deform[3] > 0.f))
                return fail(TDPM_ERR_ARG, "quadratic deformation coefficients must be > 0");
            if (!std::isfinite(P.deform[0]) || !std::isfinite(P.deform[2]) || !std::isfinite(P.deform[1]) ||
                !std::isfinite(P.deform[3]))
                return fail(TDPM_ERR_ARG, "deformation coefficients must be finite");
            if (P.anchor_y < 0 || P.anchor_x < 0) return fail(TDPM_ERR_ARG, "negative anchor");
            PartH ph;
            ph.vy = P.anchor_y; ph.vx = P.anchor_x;
            std::memcpy(ph.d, P.deform, sizeof(ph.d));
            if ((st = add_filter(P.filter, 1, c, i, &ph.fid))) return st;
            ch.parts.push_back(ph);
        }
        m->comps.push_back(std::move(ch));
    }
    for (Group &g : m->groups) {
        g.K = (int)g.fids.size();
        g.Kpad = (g.K + corr_f32_tile_k() - 1) / corr_f32_tile_k() * corr_f32_tile_k();
        const int taps = g.h * g.w;
        std::vector<float> ft((size_t)taps * FD * g.Kpad, 0.f);
        for (int k = 0; k < g.K; ++k) {
            const FilterH &F = m->filters[g.fids[k]];
            for (int t = 0; t < taps; ++t)
                for (int c = 0; c < FD; ++c) ft[((size_t)t * FD + c) * g.Kpad + k] = F.data[(size_t)t * FD + c];
        }
        if ((st = upload(&g.d_filt_t, ft))) {
            free_model(*m);
            return st;
        }
    }
    const int id = ctx->next_id++;
    ctx->models[id] = std::move(m);
    *model_id = id;
    return TDPM_OK;
}

tdpm_status tdpm_model_info(tdpm_ctx *ctx, int32_t model_id, int32_t *n_filters, int32_t *n_groups)
{
    g_err.clear();
    if (!ctx) return fail(TDPM_ERR_ARG, "ctx is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    Model *m = get_model(ctx, model_id);
    if (!m) return fail(TDPM_ERR_STATE, "unknown model id");
    if (n_filters) *n_filters = (int)m->filters.size();
    if (n_groups) *n_groups = (int)m->groups.size();
    return TDPM_OK;
}

tdpm_status tdpm_group_info(tdpm_ctx *ctx, int32_t model_id, int32_t group, int32_t *role, int32_t *h, int32_t *w,
                            int32_t *n_filters, int32_t *rank, int32_t *filter_ids, int32_t capacity)
{
    g_err.clear();
    if (!ctx) return fail(TDPM_ERR_ARG, "ctx is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    Model *m = get_model(ctx, model_id);
    if (!m) return fail(TDPM_ERR_STATE, "unknown model id");
    if (group < 0 || group >= (int)m->groups.size()) return fail(TDPM_ERR_ARG, "group out of range");
    const Group &g = m->groups[group];
    if (role) *role = g.role;
    if (h) *h = g.h;
    if (w) *w = g.w;
    if (n_filters) *n_filters = g.K;
    if (rank) *rank = m->decomposed ? g.R : 0;
    if (filter_ids)
        for (int i = 0; i < std::min(capacity, g.K); ++i) filter_ids[i] = g.fids[i];
    return TDPM_OK;
}

tdpm_status tdpm_decompose(tdpm_ctx *ctx, int32_t model_id, int32_t rank, int32_t mode, int32_t max_iters, double tol,
                           uint64_t seed, tdpm_decomp_report *report)
{
    g_err.clear();
    if (!ctx) return fail(TDPM_ERR_ARG, "ctx is NULL");
    if (rank <= 0) return fail(TDPM_ERR_ARG, "rank must be > 0");
    if (mode != TDPM_DECOMP_PER_FILTER && mode != TDPM_DECOMP_JOINT) return fail(TDPM_ERR_ARG, "bad mode");
    if (max_iters <= 0) return fail(TDPM_ERR_ARG, "max_iters must be > 0");
    std::lock_guard<std::mutex> lk(ctx->mu);
    tdpm_status st = set_device(ctx);
    if (st) return st;
    Model *m = get_model(ctx, model_id);
    if (!m) return fail(TDPM_ERR_STATE, "unknown model id");
    long long total_iters = 0;
    for (Group &g : m->groups) {
        const int K = g.K, h = g.h, w = g.w, hw = h * w;
        g.joint = mode == TDPM_DECOMP_JOINT;
        g.rel_err.assign(K, 0.0);
        if (!g.joint) {
            std::vector<CpResult> res(K);
            std::vector<int> Rk(K);
            const bool exact = rank >= hw;
            if (!exact) {
                const unsigned nt = std::max(1u, std::min<unsigned>(std::thread::hardware_concurrency(), (unsigned)K));
                std::vector<std::thread> pool;
                for (unsigned t = 0; t < nt; ++t)
                    pool.emplace_back([&, t]() {
                        for (int k = (int)t; k < K; k += (int)nt) {
                            const FilterH &F = m->filters[g.fids[k]];
                            std::vector<double> T(F.data.begin(), F.data.end());
                            res[k] = cp_als(T.data(), {h, w, FD}, rank, max_iters, tol, seed + (uint64_t)g.fids[k]);
                        }
                    });
                for (auto &th : pool) th.join();
            }
            g.rank_off.assign(K + 1, 0);
            for (int k = 0; k < K; ++k) {
                Rk[k] = exact ? hw : rank;
                g.rank_off[k + 1] = g.rank_off[k] + Rk[k];
            }
            g.R = g.rank_off[K];
            const int R = g.R;
            g.A.assign((size_t)h * R, 0.0);
            g.B.assign((size_t)w * R, 0.0);
            g.C.assign((size_t)FD * R, 0.0);
            g.Lam.assign((size_t)K * R, 0.0);
            for (int k = 0; k < K; ++k) {
                const FilterH &F = m->filters[g.fids[k]];
                const int off = g.rank_off[k];
                if (exact) {
                    // Sec. 4 CP form with R = h*w: a_r = e_dy, b_r = e_dx, c_r = F[dy][dx][:]
                    for (int dy = 0; dy < h; ++dy)
                        for (int dx = 0; dx < w; ++dx) {
                            const int r = off + dy * w + dx;
                            g.A[(size_t)dy * R + r] = 1.0;
                            g.B[(size_t)dx * R + r] = 1.0;
                            for (int c = 0; c < FD; ++c)
                                g.C[(size_t)c * R + r] = F.data[((size_t)dy * w + dx) * FD + c];
                            g.Lam[(size_t)k * R + r] = 1.0;
                        }
                } else {
                    const CpResult &cr = res[k];
                    total_iters += cr.iters;
                    for (int j = 0; j < rank; ++j) {
                        const int r = off + j;
                        for (int dy = 0; dy < h; ++dy) g.A[(size_t)dy * R + r] = cr.U[0][(size_t)dy * rank + j];
                        for (int dx = 0; dx < w; ++dx) g.B[(size_t)dx * R + r] = cr.U[1][(size_t)dx * rank + j];
                        for (int c = 0; c < FD; ++c) g.C[(size_t)c * R + r] = cr.U[2][(size_t)c * rank + j];
                        g.Lam[(size_t)k * R + r] = cr.weights[j];
                    }
                }
            }
        } else {
            const size_t fsz = (size_t)hw * FD;
            const bool exact = (long long)rank >= (long long)hw * FD;
            if (exact) {
                const int R = (int)fsz;
                g.R = R;
                g.A.assign((size_t)h * R, 0.0);
                g.B.assign((size_t)w * R, 0.0);
                g.C.assign((size_t)FD * R, 0.0);
                g.Lam.assign((size_t)K * R, 0.0);
                for (int dy = 0; dy < h; ++dy)
                    for (int dx = 0; dx < w; ++dx)
                        for (int c = 0; c < FD; ++c) {
                            const int r = (dy * w + dx) * FD + c;
                            g.A[(size_t)dy * R + r] = 1.0;
                            g.B[(size_t)dx * R + r] = 1.0;
                            g.C[(size_t)c * R + r] = 1.0;
                            for (int k = 0; k < K; ++k) g.Lam[(size_t)k * R + r] = m->filters[g.fids[k]].data[r];
                        }
            } else {
                std::vector<double> T((size_t)K * fsz);
                for (int k = 0; k < K; ++k) {
                    const FilterH &F = m->filters[g.fids[k]];
                    std::copy(F.data.begin(), F.data.end(), T.begin() + (size_t)k * fsz);
                }
                CpResult cr = cp_als(T.data(), {K, h, w, FD}, rank, max_iters, tol, seed + 7919ull * (uint64_t)(&g - &m->groups[0]));
                total_iters += cr.iters;
                const int R = rank;
                g.R = R;
                g.A.assign(cr.U[1].begin(), cr.U[1].end());
                g.B.assign(cr.U[2].begin(), cr.U[2].end());
                g.C.assign(cr.U[3].begin(), cr.U[3].end());
                g.Lam.assign((size_t)K * R, 0.0);
                for (int k = 0; k < K; ++k)
                    for (int r = 0; r < R; ++r) g.Lam[(size_t)k * R + r] = cr.U[0][(size_t)k * R + r] * cr.weights[r];
            }
            g.rank_off.assign(K + 1, 0);
        }
        // per-filter relative error of the reconstruction F_k = sum_r Lam[k][r] a_r (x) b_r (x) c_r
        const int R = g.R;
        for (int k = 0; k < K; ++k) {
            const FilterH &F = m->filters[g.fids[k]];
            int r0 = 0, r1 = R;
            if (!g.joint) { r0 = g.rank_off[k]; r1 = g.rank_off[k + 1]; }
            double e2 = 0.0, n2 = 0.0;
            for (int dy = 0; dy < h; ++dy)
                for (int dx = 0; dx < w; ++dx)
                    for (int c = 0; c < FD; ++c) {
                        double v = 0.0;
                        for (int r = r0; r < r1; ++r)
                            v += g.Lam[(size_t)k * R + r] * g.A[(size_t)dy * R + r] * g.B[(size_t)dx * R + r] *
                                 g.C[(size_t)c * R + r];
                        const double f = F.data[((size_t)dy * w + dx) * FD + c];
                        e2 += (f - v) * (f - v);
                        n2 += f * f;
                    }
            g.rel_err[k] = n2 > 0 ? std::sqrt(e2 / n2) : std::sqrt(e2);
        }
        if ((st = upload_factors(g))) return st;
    }
    m->decomposed = true;
    m->decomp_mode = mode;
    if (report) {
        std::memset(report, 0, sizeof(*report));
        report->n_groups = (int)m->groups.size();
        double full = 0.0, dec = 0.0, emax = 0.0, esum = 0.0;
        int nf = 0;
        for (const Group &g : m->groups) {
            report->total_rank += g.R;
            full += (double)g.K * g.h * g.w * FD;
            dec += (double)g.R * (g.h + g.w + FD) + (g.joint ? (double)g.K * g.R : 0.0);
            for (double e : g.rel_err) {
                emax = std::max(emax, e);
                esum += e;
                ++nf;
            }
        }
        report->total_iters = (int)total_iters;
        report->max_rel_error = emax;
        report->mean_rel_error = nf ? esum / nf : 0.0;
        report->gain = dec > 0 ? full / dec : 0.0;
    }
    return TDPM_OK;
}

tdpm_status tdpm_get_factors(tdpm_ctx *ctx, int32_t model_id, int32_t group, double *A, double *B, double *C,
                             double *Lambda)
{
    g_err.clear();
    if (!ctx) return fail(TDPM_ERR_ARG, "ctx is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    Model *m = get_model(ctx, model_id);
    if (!m) return fail(TDPM_ERR_STATE, "unknown model id");
    if (!m->decomposed) return fail(TDPM_ERR_STATE, "model not decomposed");
    if (group < 0 || group >= (int)m->groups.size()) return fail(TDPM_ERR_ARG, "group out of range");
    const Group &g = m->groups[group];
    if (A) std::copy(g.A.begin(), g.A.end(), A);
    if (B) std::copy(g.B.begin(), g.B.end(), B);
    if (C) std::copy(g.C.begin(), g.C.end(), C);
    if (Lambda) std::copy(g.Lam.begin(), g.Lam.end(), Lambda);
    return TDPM_OK;
}


tdpm_status tdpm_save_factors(tdpm_ctx *ctx, int32_t model_id, const char *path)
{
    g_err.clear();
    if (!ctx || !path) return fail(TDPM_ERR_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(ctx->mu);
    Model *m = get_model(ctx, model_id);
    if (!m) return fail(TDPM_ERR_STATE, "unknown model id");
    if (!m->decomposed) return fail(TDPM_ERR_STATE, "model not decomposed");
    std::vector<char> b(kMagic, kMagic + 8);
    put<uint32_t>(b, 1u);
    put<uint32_t>(b, (uint32_t)m->groups.size());
    put<int32_t>(b, m->decomp_mode);
    for (const Group &g : m->groups) {
        put<int32_t>(b, g.role); put<int32_t>(b, g.h); put<int32_t>(b, g.w); put<int32_t>(b, g.K);
        put<int32_t>(b, g.R); put<int32_t>(b, g.joint);
        std::vector<int32_t> ro(g.rank_off.begin(), g.rank_off.end());
        ro.resize(g.K + 1, 0);
        put_vec(b, ro);
        put_vec(b, g.A); put_vec(b, g.B); put_vec(b, g.C); put_vec(b, g.Lam); put_vec(b, g.rel_err);
    }
    put<uint64_t>(b, fnv1a(b));
    FILE *f = std::fopen(path, "wb");
    if (!f) return fail(TDPM_ERR_IO, std::string("cannot open ") + path);
    const size_t n = std::fwrite(b.data(), 1, b.size(), f);
    const int rc = std::fclose(f);
    if (n != b.size() || rc != 0) return fail(TDPM_ERR_IO, "short write");
    return TDPM_OK;
}

tdpm_status tdpm_load_factors(tdpm_ctx *ctx, int32_t model_id, const char *path)
{
    g_err.clear();
    if (!ctx || !path) return fail(TDPM_ERR_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(ctx->mu);
    tdpm_status st = set_device(ctx);
    if (st) return st;
    Model *m = get_model(ctx, model_id);
    if (!m) return fail(TDPM_ERR_STATE, "unknown model id");
    FILE *f = std::fopen(path, "rb");
    if (!f) return fail(TDPM_ERR_IO, std::string("cannot open ") + path);
    std::vector<char> b;
    char buf[1 << 16];
    size_t n;
    while ((n = std::fread(buf, 1, sizeof(buf), f)) > 0) b.insert(b.end(), buf, buf + n);
    std::fclose(f);
    if (b.size() < 8 + 8 + 8 || std::memcmp(b.data(), kMagic, 8) != 0) return fail(TDPM_ERR_IO, "not a factor file");
    std::vector<char> body(b.begin(), b.end() - 8);
    uint64_t sum;
    std::memcpy(&sum, b.data() + b.size() - 8, 8);
    if (sum != fnv1a(body)) return fail(TDPM_ERR_IO, "factor file checksum mismatch");
    Reader rd{body, 8};
    const uint32_t ver = rd.get<uint32_t>(), ng = rd.get<uint32_t>();
    const int32_t mode = rd.get<int32_t>();
    if (!rd.ok || ver != 1) return fail(TDPM_ERR_IO, "unsupported factor file version");
    if (ng != m->groups.size()) return fail(TDPM_ERR_IO, "factor file has a different number of shape groups");
    std::vector<Group> tmp(ng);
    for (uint32_t i = 0; i < ng; ++i) {
        Group &t = tmp[i];
        const Group &g = m->groups[i];
        t.role = rd.get<int32_t>(); t.h = rd.get<int32_t>(); t.w = rd.get<int32_t>(); t.K = rd.get<int32_t>();
        t.R = rd.get<int32_t>(); t.joint = rd.get<int32_t>();
        if (!rd.ok || t.role != g.role || t.h != g.h || t.w != g.w || t.K != g.K || t.R <= 0)
            return fail(TDPM_ERR_IO, "factor file does not match the model's shape groups");
        std::vector<int32_t> ro;
        rd.get_vec(ro, t.K + 1);
        t.rank_off.assign(ro.begin(), ro.end());
        rd.get_vec(t.A, (size_t)t.h * t.R); rd.get_vec(t.B, (size_t)t.w * t.R); rd.get_vec(t.C, (size_t)FD * t.R);
        rd.get_vec(t.Lam, (size_t)t.K * t.R); rd.get_vec(t.rel_err, (size_t)t.K);
        if (!rd.ok) return fail(TDPM_ERR_IO, "truncated factor file");
    }
    for (uint32_t i = 0; i < ng; ++i) {
        Group &g = m->groups[i];
        g.R = tmp[i].R; g.joint = tmp[i].joint;
        g.rank_off = tmp[i].rank_off;
        g.A = tmp[i].A; g.B = tmp[i].B; g.C = tmp[i].C; g.Lam = tmp[i].Lam; g.rel_err = tmp[i].rel_err;
        if ((st = upload_factors(g))) return st;
    }
    m->decomposed = true;
    m->decomp_mode = mode;
    return TDPM_OK;
}

tdpm_status tdpm_build_pyramid_scores(tdpm_ctx *ctx, int32_t model_id, const tdpm_pyramid *pyr, int32_t form,
                                      int32_t precision, void *stream, int32_t *scores_id)
{
    g_err.clear();
    if (!ctx || !pyr || !scores_id) return fail(TDPM_ERR_ARG, "NULL argument");
    if (form != TDPM_FORM_FULL && form != TDPM_FORM_DECOMPOSED) return fail(TDPM_ERR_ARG, "bad form");
    if (precision != TDPM_PREC_FP32 && precision != TDPM_PREC_BF16) return fail(TDPM_ERR_ARG, "unsupported precision");
    if (pyr->n_levels <= 0 || !pyr->levels) return fail(TDPM_ERR_ARG, "empty pyramid");
    if (pyr->lambda < 1 || pyr->lambda >= pyr->n_levels + 1) return fail(TDPM_ERR_ARG, "lambda out of range");
    std::lock_guard<std::mutex> lk(ctx->mu);
    tdpm_status st = set_device(ctx);
    if (st) return st;
    Model *m = get_model(ctx, model_id);
    if (!m) return fail(TDPM_ERR_STATE, "unknown model id");
    if (form == TDPM_FORM_DECOMPOSED && !m->decomposed)
        return fail(TDPM_ERR_STATE, "decomposed form requested before tdpm_decompose");
    if (form == TDPM_FORM_FULL && precision != TDPM_PREC_FP32)
        return fail(TDPM_ERR_ARG, "full form runs in FP32 only in this build");
    const int L = pyr->n_levels, lam = pyr->lambda;
    for (int j = 0; j < L; ++j) {
        const tdpm_level &lv = pyr->levels[j];
        if (lv.H <= 0 || lv.W <= 0 || !lv.data) return fail(TDPM_ERR_ARG, "level with non-positive size or NULL data");
        if (lv.H > 32767 || lv.W > 32767) return fail(TDPM_ERR_ARG, "level side above 32767 cells");
    }
    cudaStream_t s = (cudaStream_t)stream;
    const bool bf = precision == TDPM_PREC_BF16;
    const bool dec = form == TDPM_FORM_DECOMPOSED;

    // ---- pass 1: sizes and offsets
    Bump bump;
    auto sc = std::make_unique<Scores>();
    sc->model_id = model_id;
    std::vector<size_t> bf_off(L, 0);
    if (bf)
        for (int j = 0; j < L; ++j) bf_off[j] = bump.take(sizeof(uint16_t) * (size_t)pyr->levels[j].H * pyr->levels[j].W * FD);

    struct GroupLevel { int j; size_t out_off, z_off; int Ho, Wo; };
    std::vector<std::vector<GroupLevel>> glv(m->groups.size());
    for (size_t gi = 0; gi < m->groups.size(); ++gi) {
        const Group &g = m->groups[gi];
        const int j0 = g.role == 0 ? lam : 0, j1 = g.role == 0 ? L : L - lam;
        for (int j = j0; j < j1; ++j) {
            const int H = pyr->levels[j].H, W = pyr->levels[j].W;
            const int Ho = H - g.h + 1, Wo = W - g.w + 1;
            if (Ho <= 0 || Wo <= 0) continue;
            GroupLevel gl{j, 0, 0, Ho, Wo};
            gl.out_off = bump.take(sizeof(float) * (size_t)g.K * Ho * Wo);
            if (dec) gl.z_off = bump.take(sizeof(float) * (size_t)g.R * H * W);
            glv[gi].push_back(gl);
            for (int k = 0; k < g.K; ++k)
                sc->filter_maps[{g.fids[k], j}] = MapRef{gl.out_off + sizeof(float) * (size_t)k * Ho * Wo, Ho, Wo};
        }
    }

    struct DtPlan { int fid, jroot, l, Hs, Ws, X, Y, vx, vy; const float *d; size_t v_off, iv_off, d_off, a_off; };
    struct AsmPlan { int c, j, Y, X; size_t out_off; std::vector<int> dt; };
    std::vector<DtPlan> dts;
    std::vector<AsmPlan> asms;
    for (size_t c = 0; c < m->comps.size(); ++c) {
        const CompH &C = m->comps[c];
        const FilterH &Rf = m->filters[C.root_fid];
        for (int j = lam; j < L; ++j) {
            const int l = j - lam;
            int Y = pyr->levels[j].H - Rf.h + 1, X = pyr->levels[j].W - Rf.w + 1;
            for (const PartH &P : C.parts) {
                const FilterH &Pf = m->filters[P.fid];
                const int Hs = pyr->levels[l].H - Pf.h + 1, Ws = pyr->levels[l].W - Pf.w + 1;
                if (Hs <= 0 || Ws <= 0) { Y = 0; X = 0; break; }
                Y = std::min(Y, fdiv2(Hs - 1 - P.vy) + 1);
                X = std::min(X, fdiv2(Ws - 1 - P.vx) + 1);
            }
            if (Y <= 0 || X <= 0) continue;
            AsmPlan ap{(int)c, j, Y, X, 0, {}};
            ap.out_off = bump.take(sizeof(float) * (size_t)Y * X);
            sc->final_maps[{(int)c, j}] = MapRef{ap.out_off, Y, X};
            for (const PartH &P : C.parts) {
                const FilterH &Pf = m->filters[P.fid];
                DtPlan dp;
                dp.fid = P.fid; dp.jroot = j; dp.l = l;
                dp.Hs = pyr->levels[l].H - Pf.h + 1; dp.Ws = pyr->levels[l].W - Pf.w + 1;
                dp.X = X; dp.Y = Y; dp.vx = P.vx; dp.vy = P.vy; dp.d = P.d;
                dp.v_off = bump.take(sizeof(float) * (size_t)dp.Hs * X);
                dp.iv_off = bump.take(sizeof(int32_t) * (size_t)dp.Hs * X);
                dp.d_off = bump.take(sizeof(float) * (size_t)Y * X);
                dp.a_off = bump.take(sizeof(int32_t) * (size_t)Y * X);
                sc->dt_maps[{P.fid, j}] = MapRef{dp.d_off, Y, X};
                sc->arg_maps[{P.fid, j}] = MapRef{dp.a_off, Y, X};
                ap.dt.push_back((int)dts.size());
                dts.push_back(dp);
            }
            asms.push_back(std::move(ap));
        }
    }
    long long total = 0;
    for (const AsmPlan &a : asms) total += (long long)a.Y * a.X;
    const int n_det_blocks = (int)((total + detect_positions_per_block() - 1) / detect_positions_per_block());
    const size_t counts_off = bump.take(sizeof(int) * std::max(1, n_det_blocks));
    const size_t offsets_off = bump.take(sizeof(int) * std::max(1, n_det_blocks));
    const size_t total_off = bump.take(sizeof(long long));

    // job tables: one blob, uploaded with one copy
    size_t jobs_begin = align256(bump.off);
    Bump jb;
    std::vector<size_t> g_jobs_off(m->groups.size()), g_sep_off(m->groups.size());
    for (size_t gi = 0; gi < m->groups.size(); ++gi) {
        g_jobs_off[gi] = jb.take(sizeof(CorrJob) * std::max<size_t>(1, glv[gi].size()) + sizeof(ZJob) * std::max<size_t>(1, glv[gi].size()));
        g_sep_off[gi] = jb.take(sizeof(SepJob) * std::max<size_t>(1, glv[gi].size()));
    }
    const size_t dt_jobs_off = jb.take(sizeof(DtJob) * std::max<size_t>(1, dts.size()));
    const size_t asm_jobs_off = jb.take(sizeof(AsmJob) * std::max<size_t>(1, asms.size()));
    const size_t blob_bytes = align256(jb.off);
    const size_t arena_bytes = jobs_begin + blob_bytes;

    if ((st = arena_get(ctx, arena_bytes, blob_bytes, sc->arena))) return st;
    char *base = sc->arena.dev;
    char *hblob = sc->arena.host;
    std::memset(hblob, 0, blob_bytes);
    char *dblob = base + jobs_begin;

    // ---- pass 2: fill the job tables with device pointers
    std::vector<int> corr_tiles(m->groups.size(), 0), z_tiles(m->groups.size(), 0), sep_tiles(m->groups.size(), 0);
    for (size_t gi = 0; gi < m->groups.size(); ++gi) {
        const Group &g = m->groups[gi];
        CorrJob *cj = reinterpret_cast<CorrJob *>(hblob + g_jobs_off[gi]);
        ZJob *zj = reinterpret_cast<ZJob *>(hblob + g_jobs_off[gi] + sizeof(CorrJob) * std::max<size_t>(1, glv[gi].size()));
        SepJob *sj = reinterpret_cast<SepJob *>(hblob + g_sep_off[gi]);
        int ct = 0, zt = 0, st2 = 0;
        for (size_t i = 0; i < glv[gi].size(); ++i) {
            const GroupLevel &gl = glv[gi][i];
            const tdpm_level &lv = pyr->levels[gl.j];
            const uint16_t *fbf = bf ? reinterpret_cast<const uint16_t *>(base + bf_off[gl.j]) : nullptr;
            CorrJob &c = cj[i];
            c.feat = lv.data; c.feat_bf = fbf; c.out = reinterpret_cast<float *>(base + gl.out_off);
            c.H = lv.H; c.W = lv.W; c.Ho = gl.Ho; c.Wo = gl.Wo;
            c.tiles_x = (gl.Wo + corr_f32_tile_x() - 1) / corr_f32_tile_x();
            c.tiles_y = (gl.Ho + corr_f32_tile_y() - 1) / corr_f32_tile_y();
            c.begin = ct;
            ct += c.tiles_x * c.tiles_y * (g.Kpad / corr_f32_tile_k());
            if (dec) {
                ZJob &z = zj[i];
                z.feat = lv.data; z.feat_bf = fbf; z.Z = reinterpret_cast<float *>(base + gl.z_off);
                z.cells = lv.H * lv.W;
                z.begin = zt;
                zt += ((z.cells + zproj_simt_cells_per_tile() - 1) / zproj_simt_cells_per_tile()) *
                      ((g.R + zproj_simt_r_chunk() - 1) / zproj_simt_r_chunk());
                SepJob &sp = sj[i];
                sp.Z = z.Z; sp.out = c.out; sp.H = lv.H; sp.W = lv.W; sp.Ho = gl.Ho; sp.Wo = gl.Wo;
                sp.tiles_x = (gl.Wo + sep_tile_x() - 1) / sep_tile_x();
                sp.tiles_y = (gl.Ho + sep_tile_y() - 1) / sep_tile_y();
                sp.begin = st2;
                const int fpc = sep_filters_per_cta(g.joint);
                st2 += sp.tiles_x * sp.tiles_y * (g.joint ? (g.K + fpc - 1) / fpc : g.K);
            }
        }
        corr_tiles[gi] = ct; z_tiles[gi] = zt; sep_tiles[gi] = st2;
    }
    DtJob *dj = reinterpret_cast<DtJob *>(hblob + dt_jobs_off);
    int xw = 0, yw = 0, maxW = 1, maxH = 1;
    for (size_t i = 0; i < dts.size(); ++i) {
        const DtPlan &p = dts[i];
        DtJob &d = dj[i];
        const MapRef &S = sc->filter_maps[{p.fid, p.l}];
        d.S = reinterpret_cast<const float *>(base + S.off);
        d.H = p.Hs; d.W = p.Ws;
        d.lx = p.d[0]; d.qx = p.d[1]; d.ly = p.d[2]; d.qy = p.d[3];
        d.x_off = p.vx; d.x_step = 2; d.nx = p.X;
        d.y_off = p.vy; d.y_step = 2; d.ny = p.Y;
        d.V = reinterpret_cast<float *>(base + p.v_off);
        d.IV = reinterpret_cast<int32_t *>(base + p.iv_off);
        d.D = reinterpret_cast<float *>(base + p.d_off);
        d.A = reinterpret_cast<int32_t *>(base + p.a_off);
        d.xbegin = xw; d.ybegin = yw;
        xw += (p.Hs + 31) / 32;
        yw += (p.X + 31) / 32;
        maxW = std::max(maxW, p.Ws);
        maxH = std::max(maxH, p.Hs);
    }
    AsmJob *aj = reinterpret_cast<AsmJob *>(hblob + asm_jobs_off);
    long long pos = 0;
    for (size_t i = 0; i < asms.size(); ++i) {
        const AsmPlan &p = asms[i];
        const CompH &C = m->comps[p.c];
        AsmJob &a = aj[i];
        const MapRef &Rm = sc->filter_maps[{C.root_fid, p.j}];
        a.root = reinterpret_cast<const float *>(base + Rm.off);
        a.root_W = Rm.cols;
        a.Y = p.Y; a.X = p.X; a.bias = C.bias; a.n_parts = (int)C.parts.size();
        a.comp = p.c; a.level = p.j;
        a.out = reinterpret_cast<float *>(base + p.out_off);
        for (size_t k = 0; k < p.dt.size(); ++k) {
            a.D[k] = reinterpret_cast<const float *>(base + dts[p.dt[k]].d_off);
            a.A[k] = reinterpret_cast<const int32_t *>(base + dts[p.dt[k]].a_off);
        }
        a.begin = pos;
        pos += (long long)p.Y * p.X;
    }
    sc->d_asm = reinterpret_cast<AsmJob *>(dblob + asm_jobs_off);
    sc->n_asm = (int)asms.size();
    sc->total = total;
    sc->n_det_blocks = n_det_blocks;
    sc->d_counts = reinterpret_cast<int *>(base + counts_off);
    sc->d_offsets = reinterpret_cast<int *>(base + offsets_off);
    sc->d_total = reinterpret_cast<long long *>(base + total_off);

    // ---- enqueue
    auto cuda_fail = [&](cudaError_t e, const char *what) {
        cudaStreamSynchronize(s);
        arena_put(ctx, sc->arena);
        return fail(TDPM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    };
    cudaError_t e = cudaMemcpyAsync(dblob, hblob, blob_bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "job table upload");
    if (bf) {
        Prof pr(ctx, s, "to_bf16");
        for (int j = 0; j < L; ++j) {
            const tdpm_level &lv = pyr->levels[j];
            e = launch_to_bf16(lv.data, reinterpret_cast<uint16_t *>(base + bf_off[j]), (long long)lv.H * lv.W * FD, s);
            if (e != cudaSuccess) return cuda_fail(e, "bf16 conversion");
        }
        pr.end();
    }
    for (size_t gi = 0; gi < m->groups.size(); ++gi) {
        const Group &g = m->groups[gi];
        const int nj = (int)glv[gi].size();
        if (!nj) continue;
        const CorrJob *dcj = reinterpret_cast<const CorrJob *>(dblob + g_jobs_off[gi]);
        if (!dec) {
            Prof pr(ctx, s, "corr_f32");
            e = launch_corr_f32(dcj, nj, corr_tiles[gi], g.d_filt_t, g.K, g.Kpad, g.h, g.w, s);
            if (e != cudaSuccess) return cuda_fail(e, "full correlation");
            pr.end();
        } else {
            const ZJob *dzj = reinterpret_cast<const ZJob *>(dblob + g_jobs_off[gi] + sizeof(CorrJob) * std::max<size_t>(1, glv[gi].size()));
            const SepJob *dsj = reinterpret_cast<const SepJob *>(dblob + g_sep_off[gi]);
            const int p = bf ? 1 : 0;
            Prof pz(ctx, s, "zproj");
            e = launch_zproj_simt(dzj, nj, z_tiles[gi], g.d_Ct[p], g.R, bf, s);
            if (e != cudaSuccess) return cuda_fail(e, "channel projection");
            pz.end();
            Prof ps(ctx, s, "sep");
            e = launch_sep_simt(dsj, nj, sep_tiles[gi], g.d_A[p], g.d_B[p], g.d_lam[p], g.d_rank_off, g.K, g.R, g.h,
                                g.w, g.joint != 0, s);
            if (e != cudaSuccess) return cuda_fail(e, "separable passes");
            ps.end();
        }
    }
    {
        Prof pr(ctx, s, "dt");
        e = launch_dt(reinterpret_cast<const DtJob *>(dblob + dt_jobs_off), (int)dts.size(), xw, yw, maxW, maxH, s);
        if (e != cudaSuccess) return cuda_fail(e, "distance transform");
        pr.end();
    }
    {
        Prof pr(ctx, s, "assemble");
        e = launch_assemble(sc->d_asm, sc->n_asm, total, s);
        if (e != cudaSuccess) return cuda_fail(e, "assembly");
        pr.end();
    }
    e = cudaEventCreateWithFlags(&sc->done, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e, "event");
    e = cudaEventRecord(sc->done, s);
    if (e != cudaSuccess) return cuda_fail(e, "event record");
    const int id = ctx->next_id++;
    ctx->scores[id] = std::move(sc);
    *scores_id = id;
    return TDPM_OK;
}

tdpm_status tdpm_detect(tdpm_ctx *ctx, int32_t scores_id, float tau, tdpm_detection *out, size_t capacity,
                        size_t *n_out, void *stream)
{
    g_err.clear();
    if (!ctx || !n_out || (capacity > 0 && !out)) return fail(TDPM_ERR_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(ctx->mu);
    tdpm_status st = set_device(ctx);
    if (st) return st;
    Scores *sc = get_scores(ctx, scores_id);
    if (!sc) return fail(TDPM_ERR_STATE, "unknown scores id");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t want = std::min<size_t>(capacity, (size_t)sc->total);
    if (want > sc->rec_cap) {
        if (sc->d_records) {
            cudaFree(sc->d_records);
            ctx->used -= std::min(ctx->used, sc->rec_cap * sizeof(tdpm_detection));
            sc->d_records = nullptr;
            sc->rec_cap = 0;
        }
        if (ctx->budget && ctx->used + want * sizeof(tdpm_detection) > ctx->budget)
            return fail(TDPM_ERR_OOM, "detection buffer exceeds the memory budget");
        CUDA_TRY(cudaMalloc(&sc->d_records, want * sizeof(tdpm_detection)));
        sc->rec_cap = want;
        ctx->used += want * sizeof(tdpm_detection);
    }
    CUDA_TRY(cudaStreamWaitEvent(s, sc->done, 0));
    Prof pr(ctx, s, "detect");
    CUDA_TRY(launch_detect(sc->d_asm, sc->n_asm, sc->total, tau, sc->d_counts, sc->d_offsets, sc->n_det_blocks,
                           sc->d_records, (long long)want, sc->d_total, s));
    pr.end();
    long long total = 0;
    CUDA_TRY(cudaMemcpyAsync(&total, sc->d_total, sizeof(long long), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    const size_t n = std::min<size_t>((size_t)total, want);
    if (n) CUDA_TRY(cudaMemcpy(out, sc->d_records, n * sizeof(tdpm_detection), cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaEventRecord(sc->done, s));
    *n_out = (size_t)total;
    if ((size_t)total > capacity)
        return fail(TDPM_ERR_CAPACITY, "detections exceed capacity: " + std::to_string(total));
    return TDPM_OK;
}

tdpm_status tdpm_get_maps(tdpm_ctx *ctx, int32_t scores_id, int32_t kind, int32_t index_a, int32_t index_b,
                          void *out_host, size_t capacity_bytes, int32_t *rows, int32_t *cols, void *stream)
{
    g_err.clear();
    if (!ctx || !rows || !cols) return fail(TDPM_ERR_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(ctx->mu);
    tdpm_status st = set_device(ctx);
    if (st) return st;
    Scores *sc = get_scores(ctx, scores_id);
    if (!sc) return fail(TDPM_ERR_STATE, "unknown scores id");
    const std::map<std::pair<int, int>, MapRef> *mp = nullptr;
    switch (kind) {
    case TDPM_MAP_FILTER_SCORE: mp = &sc->filter_maps; break;
    case TDPM_MAP_FINAL_SCORE: mp = &sc->final_maps; break;
    case TDPM_MAP_PART_DT: mp = &sc->dt_maps; break;
    case TDPM_MAP_PART_ARG: mp = &sc->arg_maps; break;
    default: return fail(TDPM_ERR_ARG, "bad map kind");
    }
    auto it = mp->find({index_a, index_b});
    *rows = 0;
    *cols = 0;
    if (it == mp->end()) return TDPM_OK;
    *rows = it->second.rows;
    *cols = it->second.cols;
    const size_t bytes = (size_t)it->second.rows * it->second.cols * 4;
    if (bytes > capacity_bytes || !out_host) return fail(TDPM_ERR_CAPACITY, "map needs " + std::to_string(bytes) + " bytes");
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(cudaStreamWaitEvent(s, sc->done, 0));
    CUDA_TRY(cudaMemcpyAsync(out_host, sc->arena.dev + it->second.off, bytes, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return TDPM_OK;
}

tdpm_status tdpm_release(tdpm_ctx *ctx, int32_t scores_id)
{
    g_err.clear();
    if (!ctx) return fail(TDPM_ERR_ARG, "ctx is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    tdpm_status st = set_device(ctx);
    if (st) return st;
    auto it = ctx->scores.find(scores_id);
    if (it == ctx->scores.end()) return fail(TDPM_ERR_STATE, "unknown scores id");
    free_scores(ctx, *it->second);
    ctx->scores.erase(it);
    return TDPM_OK;
}

// ------------------------------------------------------------------------------------------------ stateless ops
size_t tdpm_dt_scratch_bytes(int32_t H, int32_t nx)
{
    if (H <= 0 || nx <= 0) return 256;
    return align256(sizeof(DtJob)) + align256(sizeof(float) * (size_t)H * nx) + align256(sizeof(int32_t) * (size_t)H * nx);
}

tdpm_status tdpm_dt(const float *S, int32_t H, int32_t W, const float d[4], int32_t x_off, int32_t x_step, int32_t nx,
                    int32_t y_off, int32_t y_step, int32_t ny, float *D, int32_t *arg, void *scratch, void *stream)
{
    g_err.clear();
    if (!S || !d || !D || !arg || !scratch) return fail(TDPM_ERR_ARG, "NULL argument");
    if (H <= 0 || W <= 0 || H > 32767 || W > 32767) return fail(TDPM_ERR_ARG, "map size out of range");
    if (!(d[1] > 0.f) || !(d[3] > 0.f)) return fail(TDPM_ERR_ARG, "quadratic coefficients must be > 0");
    if (nx <= 0 || ny <= 0 || x_step <= 0 || y_step <= 0 || x_off < 0 || y_off < 0 ||
        (long long)x_off + (long long)x_step * (nx - 1) >= W || (long long)y_off + (long long)y_step * (ny - 1) >= H)
        return fail(TDPM_ERR_ARG, "sampled positions outside the map");
    DtJob J{};
    char *sb = reinterpret_cast<char *>(scratch);
    J.S = S; J.H = H; J.W = W;
    J.lx = d[0]; J.qx = d[1]; J.ly = d[2]; J.qy = d[3];
    J.x_off = x_off; J.x_step = x_step; J.nx = nx;
    J.y_off = y_off; J.y_step = y_step; J.ny = ny;
    J.V = reinterpret_cast<float *>(sb + align256(sizeof(DtJob)));
    J.IV = reinterpret_cast<int32_t *>(sb + align256(sizeof(DtJob)) + align256(sizeof(float) * (size_t)H * nx));
    J.D = D; J.A = arg;
    J.xbegin = 0; J.ybegin = 0;
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(cudaMemcpyAsync(sb, &J, sizeof(DtJob), cudaMemcpyHostToDevice, s));
    CUDA_TRY(launch_dt(reinterpret_cast<const DtJob *>(sb), 1, (H + 31) / 32, (nx + 31) / 32, W, H, s));
    return TDPM_OK;
}

tdpm_status tdpm_correlate(const float *feat, int32_t H, int32_t W, const float *filt_host, int32_t K, int32_t h,
                           int32_t w, int32_t precision, float *out, void *stream)
{
    g_err.clear();
    if (!feat || !filt_host || !out) return fail(TDPM_ERR_ARG, "NULL argument");
    if (H <= 0 || W <= 0 || K <= 0 || h <= 0 || w <= 0 || h > 64 || w > 64) return fail(TDPM_ERR_ARG, "bad sizes");
    const int Ho = H - h + 1, Wo = W - w + 1;
    if (Ho <= 0 || Wo <= 0) return TDPM_OK;
    if (precision != TDPM_PREC_FP32) return fail(TDPM_ERR_ARG, "unsupported precision in this build");
    cudaStream_t s = (cudaStream_t)stream;
    const int Kpad = (K + corr_f32_tile_k() - 1) / corr_f32_tile_k() * corr_f32_tile_k();
    const int taps = h * w;
    std::vector<float> ft((size_t)taps * FD * Kpad, 0.f);
    for (int k = 0; k < K; ++k)
        for (int t = 0; t < taps; ++t)
            for (int c = 0; c < FD; ++c) ft[((size_t)t * FD + c) * Kpad + k] = filt_host[((size_t)k * taps + t) * FD + c];
    CorrJob J{};
    J.feat = feat; J.out = out; J.H = H; J.W = W; J.Ho = Ho; J.Wo = Wo;
    J.tiles_x = (Wo + corr_f32_tile_x() - 1) / corr_f32_tile_x();
    J.tiles_y = (Ho + corr_f32_tile_y() - 1) / corr_f32_tile_y();
    J.begin = 0;
    const int tiles = J.tiles_x * J.tiles_y * (Kpad / corr_f32_tile_k());
    float *d_ft = nullptr;
    CorrJob *d_job = nullptr;
    CUDA_TRY(cudaMalloc(&d_ft, sizeof(float) * ft.size()));
    CUDA_TRY(cudaMalloc(&d_job, sizeof(CorrJob)));
    cudaError_t e = cudaMemcpyAsync(d_ft, ft.data(), sizeof(float) * ft.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_job, &J, sizeof(J), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_corr_f32(d_job, 1, tiles, d_ft, K, Kpad, h, w, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_ft);
    cudaFree(d_job);
    if (e != cudaSuccess) return fail(TDPM_ERR_CUDA, std::string("correlate: ") + cudaGetErrorString(e));
    return TDPM_OK;
}

// ------------------------------------------------------------------------------------------------ instrumentation
uint64_t tdpm_kernel_launches(void) { return g_launches.load(); }

tdpm_status tdpm_profile_enable(tdpm_ctx *ctx, int32_t enable)
{
    g_err.clear();
    if (!ctx) return fail(TDPM_ERR_ARG, "ctx is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->prof = enable != 0;
    return TDPM_OK;
}

tdpm_status tdpm_profile_read(tdpm_ctx *ctx, int32_t index, char *name, size_t name_cap, double *total_ms,
                              int64_t *launches, int32_t *n_stages)
{
    g_err.clear();
    if (!ctx) return fail(TDPM_ERR_ARG, "ctx is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    tdpm_status st = set_device(ctx);
    if (st) return st;
    prof_collect(ctx);
    if (n_stages) *n_stages = (int)ctx->stages.size();
    if (index < 0 || index >= (int)ctx->stages.size()) return TDPM_OK;
    const auto &sg = ctx->stages[index];
    if (name && name_cap) {
        std::strncpy(name, sg.first.c_str(), name_cap - 1);
        name[name_cap - 1] = 0;
    }
    if (total_ms) *total_ms = sg.second.first;
    if (launches) *launches = sg.second.second;
    return TDPM_OK;
}

tdpm_status tdpm_profile_reset(tdpm_ctx *ctx)
{
    g_err.clear();
    if (!ctx) return fail(TDPM_ERR_ARG, "ctx is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    prof_collect(ctx);
    ctx->stages.clear();
    return TDPM_OK;
}

}  // extern "C"
