// C-ABI, part 1: context lifecycle, model upload, CP decomposition (Sec. 4) and factor files.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <string>
#include <thread>
#include <vector>

#include "als.h"
#include "ctx.h"

namespace tdpm {

namespace {
thread_local std::string g_err;
}

tdpm_status fail(tdpm_status st, const std::string &msg)
{
    g_err = msg;
    return st;
}

void clear_error() { g_err.clear(); }

uint16_t bf16_bits(float x)
{
    const __nv_bfloat16 b = __float2bfloat16_rn(x);
    uint16_t u;
    std::memcpy(&u, &b, 2);
    return u;
}

float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// E4M3 (1 sign, 4 exponent bits with bias 7, 3 mantissa bits; largest finite value 448, no infinities) of x, rounded
// to nearest with ties to even and saturated to +-448: written from the format's definition.
uint8_t e4m3_bits(float x)
{
    const uint8_t sign = std::signbit(x) ? 0x80 : 0;
    double a = std::fabs((double)x);
    if (!(a == a)) return 0x7F;  // NaN
    if (a >= 448.0) return sign | 0x7E;
    int k = 0;
    std::frexp(a, &k);            // a = f * 2^k, f in [0.5, 1): leading bit at 2^(k-1)
    int E = k - 1;
    if (a == 0.0) return sign;
    if (E < -6) {
        // subnormal: multiples of 2^-9
        const double q = std::nearbyint(std::ldexp(a, 9));  // ties to even (default rounding mode)
        if (q >= 8.0) return sign | (1 << 3);                // rounds up to the smallest normal 2^-6
        return sign | (uint8_t)q;
    }
    double q = std::nearbyint(std::ldexp(a, 3 - E));  // in [8, 16]
    if (q >= 16.0) {
        q = 8.0;
        ++E;
    }
    const int e = E + 7, m = (int)q - 8;
    if (e > 15 || (e == 15 && m == 7)) return sign | 0x7E;
    return sign | (uint8_t)((e << 3) | m);
}


void Group::free_factors()
{
    cudaFree(d_A); cudaFree(d_B); cudaFree(d_Ct); cudaFree(d_lam);
    d_A = d_B = d_Ct = d_lam = nullptr;
    cudaFree(d_rank_off);
    cudaFree(d_C_tc);
    cudaFree(d_C_tc_lo);
    cudaFree(d_lam_tc);
    cudaFree(d_lam_tc_lo);
    cudaFree(d_C_fp8);
    d_C_fp8 = nullptr;
    d_rank_off = nullptr;
    d_C_tc = d_C_tc_lo = nullptr;
    d_lam_tc = d_lam_tc_lo = nullptr;
    Upad = Npad_lam = 0;
}

void Group::free_all()
{
    free_factors();
    cudaFree(d_filt_t);
    cudaFree(d_filt_tc);
    cudaFree(d_filt_tc_lo);
    cudaFree(d_filt_fp8);
    d_filt_fp8 = nullptr;
    d_filt_t = nullptr;
    d_filt_tc = d_filt_tc_lo = nullptr;
}

tdpm_status set_device(tdpm_ctx *ctx)
{
    CUDA_TRY(cudaSetDevice(ctx->device));
    return TDPM_OK;
}

Model *get_model(tdpm_ctx *ctx, int id)
{
    auto it = ctx->models.find(id);
    return it == ctx->models.end() ? nullptr : it->second.get();
}

namespace {

// Tensor-core filter banks: [taps][4 channel chunks][Npad][8] BF16, zero rows for n >= n_rows; the hi part bf16(x)
// and the lo part bf16(x - bf16(x)) of the split-BF16 operands.
// E4M3 bank [taps][2][Npad][16] bytes of value * scale, scale = 448 / max |value| (1 when all are zero).
tdpm_status upload_fp8_bank(uint8_t **dst, float *scale, int taps, int Npad, int n_rows,
                            const std::function<float(int, int, int)> &value)
{
    float mx = 0.f;
    for (int t = 0; t < taps; ++t)
        for (int n = 0; n < n_rows; ++n)
            for (int c = 0; c < FD; ++c) mx = std::max(mx, std::fabs(value(t, n, c)));
    *scale = mx > 0.f ? 448.f / mx : 1.f;
    std::vector<uint8_t> b((size_t)taps * 2 * Npad * 16, 0);
    for (int t = 0; t < taps; ++t)
        for (int n = 0; n < n_rows; ++n)
            for (int c = 0; c < FD; ++c)
                b[(((size_t)t * 2 + c / 16) * Npad + n) * 16 + (c % 16)] = e4m3_bits(value(t, n, c) * *scale);
    return upload(dst, b);
}

tdpm_status upload_tc_bank(uint16_t **dst_hi, uint16_t **dst_lo, int taps, int Npad, int n_rows,
                           const std::function<float(int, int, int)> &value)
{
    std::vector<uint16_t> hi((size_t)taps * 4 * Npad * 8, 0), lo(hi.size(), 0);
    for (int t = 0; t < taps; ++t)
        for (int n = 0; n < n_rows; ++n)
            for (int c = 0; c < FD; ++c) {
                const float x = value(t, n, c);
                const size_t i = (((size_t)t * 4 + c / 8) * Npad + n) * 8 + (c % 8);
                hi[i] = bf16_bits(x);
                lo[i] = bf16_bits(x - bf16_round(x));
            }
    tdpm_status st = upload(dst_hi, hi);
    return st ? st : upload(dst_lo, lo);
}

// Device copies of a group's factors: FP32 for the SIMT kernels (channel stage of the FP32 path, 1-D passes of every
// path, recombination of the FP32 path), the channel factor C as a BF16 1x1 bank for the tensor-core channel stage
// and, in joint mode, Lambda as a BF16 bank over Upad/32 blocks of terms for the tensor-core recombination.
tdpm_status upload_factors(Group &g)
{
    g.free_factors();
    const int R = g.R, K = (int)g.fids.size();
    {
        std::vector<float> A(g.A.begin(), g.A.end()), B(g.B.begin(), g.B.end()), Ct((size_t)R * FD), lam;
        for (int r = 0; r < R; ++r)
            for (int c = 0; c < FD; ++c) Ct[(size_t)r * FD + c] = (float)g.C[(size_t)c * R + r];
        if (g.joint) {
            lam.assign(g.Lam.begin(), g.Lam.end());
        } else {
            lam.assign(R, 0.f);
            for (int k = 0; k < K; ++k)
                for (int r = g.rank_off[k]; r < g.rank_off[k + 1]; ++r) lam[r] = (float)g.Lam[(size_t)k * R + r];
        }
        tdpm_status st;
        if ((st = upload(&g.d_A, A)) || (st = upload(&g.d_B, B)) || (st = upload(&g.d_Ct, Ct)) ||
            (st = upload(&g.d_lam, lam)))
            return st;
    }
    std::vector<int> ro = g.rank_off;
    if (ro.empty()) ro.assign(K + 1, 0);
    tdpm_status st = upload(&g.d_rank_off, ro);
    if (st) return st;
    // zero rows past the last term: the fused kernels' MMAs of a filter group read up to 128 rows from its first term
    g.Rpad_tc = std::max(corr_tc_bank_rows(R), (R + 15) / 16 * 16 + zsept_terms());
    st = upload_tc_bank(&g.d_C_tc, &g.d_C_tc_lo, 1, g.Rpad_tc, R,
                        [&](int, int r, int c) { return (float)g.C[(size_t)c * R + r]; });
    if (!st)
        st = upload_fp8_bank(&g.d_C_fp8, &g.C_fp8_scale, 1, g.Rpad_tc, R,
                             [&](int, int r, int c) { return (float)g.C[(size_t)c * R + r]; });
    if (st || !g.joint) return st;
    g.Upad = (R + 31) / 32 * 32;
    const int cb = g.Upad / 32;
    g.Npad_lam = corr_tc_bank_rows(K);
    return upload_tc_bank(&g.d_lam_tc, &g.d_lam_tc_lo, cb, g.Npad_lam, K, [&](int t, int k, int c) {
        const int r = t * FD + c;
        return r < R ? (float)g.Lam[(size_t)k * R + r] : 0.f;
    });
}

}  // namespace

}  // namespace tdpm

using namespace tdpm;

extern "C" {

const char *tdpm_last_error(void) { return g_err.c_str(); }

const char *tdpm_version(void)
{
    static std::string v = std::string("libtdpm sm_103a cudart ") + std::to_string(CUDART_VERSION);
    return v.c_str();
}

tdpm_status tdpm_create(tdpm_ctx **out, int32_t device, size_t mem_budget_bytes)
{
    clear_error();
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
    cudaError_t e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming);
    for (int i = 0; i < kSideStreams && e == cudaSuccess; ++i) {
        cudaStream_t st = nullptr;
        cudaEvent_t ev = nullptr;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e == cudaSuccess) c->side.push_back(st);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) c->join_ev.push_back(ev);
    }
    if (e == cudaSuccess) e = cudaMalloc(&c->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(c->d_err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost(&c->h_err, 16);  // error flag at 0, detection count at 8
    if (e == cudaSuccess) c->h_total = reinterpret_cast<long long *>(reinterpret_cast<char *>(c->h_err) + 8);
    if (e != cudaSuccess) {
        if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
        for (cudaStream_t st : c->side) cudaStreamDestroy(st);
        for (cudaEvent_t ev : c->join_ev) cudaEventDestroy(ev);
        if (c->fork_ev) cudaEventDestroy(c->fork_ev);
        cudaFree(c->d_err);
        delete c;
        return fail(TDPM_ERR_CUDA, std::string("context setup: ") + cudaGetErrorString(e));
    }
    *c->h_err = 0;
    const char *g = std::getenv("TDPM_GRAPHS");
    c->use_graphs = !(g && g[0] == '0');
    const char *at = std::getenv("TDPM_AUTOTUNE");
    c->autotune = !(at && at[0] == '0');
    const char *fu = std::getenv("TDPM_FUSE");
    c->fuse = !(fu && fu[0] == '0');
    const char *zf = std::getenv("TDPM_ZSEP_FORM");
    if (zf && zf[0] >= '0' && zf[0] <= '4' && zf[1] == 0) c->zsep_form = zf[0] - '0';
    *out = c;
    return TDPM_OK;
}

void tdpm_destroy(tdpm_ctx *ctx)
{
    if (!ctx) return;
    server_free(ctx);
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        cudaSetDevice(ctx->device);
        for (auto &kv : ctx->scores) free_scores(ctx, *kv.second);
        ctx->scores.clear();
        for (Arena &a : ctx->free_arenas) arena_free(ctx, a);
        ctx->free_arenas.clear();
        ctx->plans.clear();
        for (auto &kv : ctx->models)
            for (Group &g : kv.second->groups) g.free_all();
        ctx->models.clear();
        for (Pending &p : ctx->pending) {
            cudaEventDestroy(p.a);
            cudaEventDestroy(p.b);
        }
        for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
        cudaStreamDestroy(ctx->cap_stream);
        if (ctx->d_records) cudaFree(ctx->d_records);
        if (ctx->d_nms) cudaFree(ctx->d_nms);
        if (ctx->d_hog) cudaFree(ctx->d_hog);
        if (ctx->hog_done) cudaEventDestroy(ctx->hog_done);
        if (ctx->hog_graph) cudaGraphExecDestroy(ctx->hog_graph);
        if (ctx->d_job_tau) cudaFree(ctx->d_job_tau);
        for (cudaStream_t st : ctx->side) cudaStreamDestroy(st);
        for (cudaEvent_t ev : ctx->join_ev) cudaEventDestroy(ev);
        cudaEventDestroy(ctx->fork_ev);
        cudaFree(ctx->d_err);
        cudaFreeHost(ctx->h_err);
    }
    delete ctx;
}

tdpm_status tdpm_load_model(tdpm_ctx *ctx, const tdpm_model_desc *desc, int32_t *model_id)
{
    clear_error();
    if (!ctx || !desc || !model_id) return fail(TDPM_ERR_ARG, "NULL argument");
    if (desc->n_components <= 0 || !desc->components) return fail(TDPM_ERR_ARG, "model has no components");
    std::lock_guard<std::mutex> lk(ctx->mu);
    tdpm_status st = set_device(ctx);
    if (st) return st;
    auto m = std::make_unique<Model>();
    auto add_filter = [&](const tdpm_filter &f, int role, int comp, int part, int *fid) -> tdpm_status {
        if (f.h <= 0 || f.w <= 0 || !f.data) return fail(TDPM_ERR_ARG, "filter with non-positive size or NULL data");
        if (f.h > 16 || f.w > 16) return fail(TDPM_ERR_ARG, "filter side above 16 cells");
        FilterH F;
        F.h = f.h; F.w = f.w; F.role = role; F.comp = comp; F.part = part;
        F.data.assign(f.data, f.data + (size_t)f.h * f.w * FD);
        for (float v : F.data)
            if (!std::isfinite(v)) return fail(TDPM_ERR_ARG, "filter with a non-finite value");
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
        if (!std::isfinite(C.bias)) return fail(TDPM_ERR_ARG, "non-finite bias");
        CompH ch;
        ch.bias = C.bias;
        if ((st = add_filter(C.root, 0, c, -1, &ch.root_fid))) return st;
        for (int i = 0; i < C.n_parts; ++i) {
            const tdpm_part &P = C.parts[i];
            for (int k = 0; k < 4; ++k)
                if (!std::isfinite(P.deform[k])) return fail(TDPM_ERR_ARG, "deformation coefficients must be finite");
            if (!(P.deform[1] > 0.f) || !(P.deform[3] > 0.f))
                return fail(TDPM_ERR_ARG, "quadratic deformation coefficients must be > 0");
            if (P.anchor_y < 0 || P.anchor_x < 0 || P.anchor_y > 1024 || P.anchor_x > 1024)
                return fail(TDPM_ERR_ARG, "anchor out of range");
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
        g.Npad_tc = corr_tc_bank_rows(g.K);
        if ((st = upload(&g.d_filt_t, ft)) ||
            (st = upload_tc_bank(&g.d_filt_tc, &g.d_filt_tc_lo, taps, g.Npad_tc, g.K, [&](int t, int k, int c) {
                 return m->filters[g.fids[k]].data[(size_t)t * FD + c];
             })) ||
            (st = upload_fp8_bank(&g.d_filt_fp8, &g.fp8_scale, taps, g.Npad_tc, g.K, [&](int t, int k, int c) {
                 return m->filters[g.fids[k]].data[(size_t)t * FD + c];
             }))) {
            for (Group &gg : m->groups) gg.free_all();
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
    clear_error();
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
    clear_error();
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

}  // extern "C"

namespace {

// ||T - sum_j w_j u0_j (x) u1_j (x) u2_j||_F of an order-3 CP result (FP64).
double cp_abs_error(const std::vector<double> &T, const CpResult &cr, int n0, int n1, int n2)
{
    const int R = (int)cr.weights.size();
    double e2 = 0.0;
    for (int i = 0; i < n0; ++i)
        for (int j = 0; j < n1; ++j)
            for (int c = 0; c < n2; ++c) {
                double v = 0.0;
                for (int r = 0; r < R; ++r)
                    v += cr.weights[r] * cr.U[0][(size_t)i * R + r] * cr.U[1][(size_t)j * R + r] *
                         cr.U[2][(size_t)c * R + r];
                const double d = T[((size_t)i * n1 + j) * n2 + c] - v;
                e2 += d * d;
            }
    return std::sqrt(e2);
}

// Decomposition of every shape group of a model. Per filter (Sec. 4): rank `rank` for every filter or, with autorank,
// the smallest r in [1, max_rank] meeting the rank criterion ||f - CP(f, r)||_F < e (r (h+w+32) / (h w 32))^2
// (a filter meeting it at no r <= max_rank keeps max_rank); a rank >= h*w is the exact slice form (error 0). Joint:
// one CP per shape group of rank `rank`. ranks_out: the filters' ranks by filter id (per filter mode), may be null.
tdpm_status decompose_model(tdpm_ctx *ctx, int32_t model_id, int32_t rank, int32_t mode, bool autorank, double e,
                            int32_t max_rank, int32_t max_iters, double tol, uint64_t seed, int32_t *ranks_out,
                            tdpm_decomp_report *report, const int32_t *ranks_in = nullptr)
{
    std::lock_guard<std::mutex> lk(ctx->mu);
    tdpm_status st = set_device(ctx);
    if (st) return st;
    Model *m = get_model(ctx, model_id);
    if (!m) return fail(TDPM_ERR_STATE, "unknown model id");
    long long total_iters = 0;
    for (size_t gi = 0; gi < m->groups.size(); ++gi) {
        Group &g = m->groups[gi];
        const int K = g.K, h = g.h, w = g.w, hw = h * w;
        g.joint = mode == TDPM_DECOMP_JOINT;
        g.rel_err.assign(K, 0.0);
        if (!g.joint) {
            // Sec. 4: one CP per filter; a rank >= h*w uses the exact slice form a_r = e_dy, b_r = e_dx,
            // c_r = F[dy][dx][:]
            std::vector<CpResult> res(K);
            std::vector<int> Rk(K, rank >= hw ? hw : rank);
            if (ranks_in)  // one rank per filter (by filter id); at least h*w is the exact slice form
                for (int k = 0; k < K; ++k) Rk[k] = std::min(ranks_in[g.fids[k]], hw);
            const unsigned nt = std::max(1u, std::min<unsigned>(std::thread::hardware_concurrency(), (unsigned)K));
            std::vector<std::thread> pool;
            for (unsigned t = 0; t < nt; ++t)
                pool.emplace_back([&, t]() {
                    for (int k = (int)t; k < K; k += (int)nt) {
                        const FilterH &F = m->filters[g.fids[k]];
                        std::vector<double> T(F.data.begin(), F.data.end());
                        const uint64_t sd = seed + (uint64_t)g.fids[k];
                        if (!autorank) {
                            if (Rk[k] < hw) res[k] = cp_als(T.data(), {h, w, FD}, Rk[k], max_iters, tol, sd);
                            continue;
                        }
                        // the smallest rank meeting the criterion, scanning upward (the criterion's error side
                        // comes from ALS, which need not decrease in r, so no bisection)
                        const double shape = (double)(h + w + FD) / ((double)hw * FD);
                        const int top = std::min(max_rank, hw - 1);
                        bool met = false;
                        int iters = 0;
                        for (int r = 1; r <= top && !met; ++r) {
                            CpResult cr = cp_als(T.data(), {h, w, FD}, r, max_iters, tol, sd);
                            iters += cr.iters;
                            met = cp_abs_error(T, cr, h, w, FD) < e * (r * shape) * (r * shape);
                            res[k] = std::move(cr);
                            Rk[k] = r;
                        }
                        if (!met && max_rank >= hw) Rk[k] = hw;  // the exact form: error 0
                        res[k].iters = iters;
                    }
                });
            for (auto &th : pool) th.join();
            g.rank_off.assign(K + 1, 0);
            for (int k = 0; k < K; ++k) g.rank_off[k + 1] = g.rank_off[k] + Rk[k];
            g.R = g.rank_off[K];
            const int R = g.R;
            g.A.assign((size_t)h * R, 0.0);
            g.B.assign((size_t)w * R, 0.0);
            g.C.assign((size_t)FD * R, 0.0);
            g.Lam.assign((size_t)K * R, 0.0);
            for (int k = 0; k < K; ++k) {
                const FilterH &F = m->filters[g.fids[k]];
                const int off = g.rank_off[k];
                if (ranks_out) ranks_out[g.fids[k]] = Rk[k];
                if (Rk[k] >= hw) {
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
                    const int rk = Rk[k];
                    for (int j = 0; j < rk; ++j) {
                        const int r = off + j;
                        for (int dy = 0; dy < h; ++dy) g.A[(size_t)dy * R + r] = cr.U[0][(size_t)dy * rk + j];
                        for (int dx = 0; dx < w; ++dx) g.B[(size_t)dx * R + r] = cr.U[1][(size_t)dx * rk + j];
                        for (int c = 0; c < FD; ++c) g.C[(size_t)c * R + r] = cr.U[2][(size_t)c * rk + j];
                        g.Lam[(size_t)k * R + r] = cr.weights[j];
                    }
                }
            }
        } else {
            // joint: one CP of the stacked K x h x w x 32 tensor; factors a_r, b_r, c_r shared, Lambda[k][r] per filter
            const size_t fsz = (size_t)hw * FD;
            const bool exact = (long long)rank >= (long long)fsz;
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
                const CpResult cr = cp_als(T.data(), {K, h, w, FD}, rank, max_iters, tol, seed + 7919ull * gi);
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
        // relative error of every rebuilt filter F_k = sum_r Lambda[k][r] a_r (x) b_r (x) c_r
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
    m->version++;
    drop_plans_of_model(ctx, model_id);
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

}  // namespace

extern "C" {

tdpm_status tdpm_decompose(tdpm_ctx *ctx, int32_t model_id, int32_t rank, int32_t mode, int32_t max_iters, double tol,
                           uint64_t seed, tdpm_decomp_report *report)
{
    clear_error();
    if (!ctx) return fail(TDPM_ERR_ARG, "ctx is NULL");
    if (rank <= 0) return fail(TDPM_ERR_ARG, "rank must be > 0");
    if (mode != TDPM_DECOMP_PER_FILTER && mode != TDPM_DECOMP_JOINT) return fail(TDPM_ERR_ARG, "bad mode");
    if (max_iters <= 0) return fail(TDPM_ERR_ARG, "max_iters must be > 0");
    if (!(tol >= 0.0)) return fail(TDPM_ERR_ARG, "tol must be >= 0");
    return decompose_model(ctx, model_id, rank, mode, false, 0.0, 0, max_iters, tol, seed, nullptr, report);
}

tdpm_status tdpm_decompose_ranks(tdpm_ctx *ctx, int32_t model_id, const int32_t *ranks, int32_t max_iters, double tol,
                                 uint64_t seed, tdpm_decomp_report *report)
{
    clear_error();
    if (!ctx || !ranks) return fail(TDPM_ERR_ARG, "NULL argument");
    if (max_iters <= 0) return fail(TDPM_ERR_ARG, "max_iters must be > 0");
    if (!(tol >= 0.0)) return fail(TDPM_ERR_ARG, "tol must be >= 0");
    int nf = 0;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        Model *m = get_model(ctx, model_id);
        if (!m) return fail(TDPM_ERR_STATE, "unknown model id");
        nf = (int)m->filters.size();
    }
    for (int i = 0; i < nf; ++i)
        if (ranks[i] <= 0) return fail(TDPM_ERR_ARG, "every rank must be > 0");
    return decompose_model(ctx, model_id, 1, TDPM_DECOMP_PER_FILTER, false, 0.0, 0, max_iters, tol, seed, nullptr,
                           report, ranks);
}

tdpm_status tdpm_decompose_auto(tdpm_ctx *ctx, int32_t model_id, double e, int32_t max_rank, int32_t max_iters,
                                double tol, uint64_t seed, int32_t *ranks, tdpm_decomp_report *report)
{
    clear_error();
    if (!ctx) return fail(TDPM_ERR_ARG, "ctx is NULL");
    if (!(e > 0.0) || !std::isfinite(e)) return fail(TDPM_ERR_ARG, "e must be finite and > 0");
    if (max_rank <= 0) return fail(TDPM_ERR_ARG, "max_rank must be > 0");
    if (max_iters <= 0) return fail(TDPM_ERR_ARG, "max_iters must be > 0");
    if (!(tol >= 0.0)) return fail(TDPM_ERR_ARG, "tol must be >= 0");
    return decompose_model(ctx, model_id, max_rank, TDPM_DECOMP_PER_FILTER, true, e, max_rank, max_iters, tol, seed,
                           ranks, report);
}

tdpm_status tdpm_get_factors(tdpm_ctx *ctx, int32_t model_id, int32_t group, double *A, double *B, double *C,
                             double *Lambda)
{
    clear_error();
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

}  // extern "C"

// --------------------------------------------------------------------------------------------- factor files
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
        if (n > b.size() || pos + sizeof(T) * n > b.size()) { ok = false; return; }
        v.resize(n);
        std::memcpy(v.data(), b.data() + pos, sizeof(T) * n);
        pos += sizeof(T) * n;
    }
};
}  // namespace

extern "C" {

tdpm_status tdpm_save_factors(tdpm_ctx *ctx, int32_t model_id, const char *path)
{
    clear_error();
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
    clear_error();
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
    if (b.size() < 24 || std::memcmp(b.data(), kMagic, 8) != 0) return fail(TDPM_ERR_IO, "not a factor file");
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
        if (!rd.ok || t.role != g.role || t.h != g.h || t.w != g.w || t.K != g.K || t.R <= 0 || t.R > (1 << 24))
            return fail(TDPM_ERR_IO, "factor file does not match the model's shape groups");
        std::vector<int32_t> ro;
        rd.get_vec(ro, (size_t)t.K + 1);
        t.rank_off.assign(ro.begin(), ro.end());
        rd.get_vec(t.A, (size_t)t.h * t.R); rd.get_vec(t.B, (size_t)t.w * t.R); rd.get_vec(t.C, (size_t)FD * t.R);
        rd.get_vec(t.Lam, (size_t)t.K * t.R); rd.get_vec(t.rel_err, (size_t)t.K);
        if (!rd.ok) return fail(TDPM_ERR_IO, "truncated factor file");
        if (!t.joint) {
            if (t.rank_off.empty() || t.rank_off[0] != 0 || t.rank_off[t.K] != t.R)
                return fail(TDPM_ERR_IO, "corrupt term offsets");
            for (int k = 0; k < t.K; ++k)
                if (t.rank_off[k + 1] < t.rank_off[k]) return fail(TDPM_ERR_IO, "corrupt term offsets");
        }
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
    m->version++;
    drop_plans_of_model(ctx, model_id);
    return TDPM_OK;
}

}  // extern "C"
