// C-ABI, part 3: the serving loop (continuous batching over the scoring path).
//
// One server thread per context. Submitted requests are split into parts, one per (request, model); parts wait in a
// FIFO queue. The thread repeatedly
//   * forms a batch from the oldest part and every queued part with the same (model, form, precision), up to
//     max_batch_images images (requests that ask for a subset of the model's components get a per-image mask);
//   * admits it by device memory: the batch's arena size is known from its plan before anything is launched, and the
//     batches in flight together stay within the budget (the oldest in-flight batch is finished first to make room;
//     a batch that cannot fit even alone is halved, and a single image that cannot fit fails with ERR_OOM);
//   * launches it with tdpm_build_batch_scores on the next of max_inflight streams, so that it runs while earlier
//     batches are still on the device;
//   * when no new part is waiting, or all slots are busy, finishes the oldest batch in flight: tdpm_detect with the
//     lowest threshold of its requests, each record handed to its request if it clears that request's threshold.
// A request is done when all of its parts are; tdpm_poll hands its detections out. The server thread is the only
// caller of the scoring entry points while it runs (it takes the context lock through them), and user threads only
// touch the server's own queue and result table, under the server's lock.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "ctx.h"

namespace tdpm {

namespace {

uint64_t now_ns()
{
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Request {
    uint64_t ticket = 0;
    std::vector<tdpm_level> levels;  // copy of the caller's level descriptors (device data stays the caller's)
    tdpm_pyramid pyr{};
    std::vector<int32_t> models;
    std::vector<int32_t> components;  // empty: all
    int32_t form = 0, precision = 0;
    float tau = 0.f;
    uint64_t t_submit = 0, t_start = 0, t_done = 0;
    int parts_left = 0;
    int32_t status = TDPM_OK;
    int32_t batch_images = 0;
    std::vector<std::vector<tdpm_detection>> dets;  // per model, in the request's model order
    bool done = false;
};

struct Part {
    Request *req;
    int model_index;  // into req->models
};

struct Batch {
    int32_t model = 0, form = 0, precision = 0;
    size_t n_comps = 0;  // components of the model
    std::vector<Part> parts;
    int32_t scores_id = 0;
    cudaStream_t stream = nullptr;
    size_t bytes = 0;
};

}  // namespace

struct Server {
    tdpm_server_config cfg{};
    std::thread th;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Part> queue;
    std::map<uint64_t, std::unique_ptr<Request>> reqs;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::vector<cudaStream_t> streams;
};

namespace {

void complete_parts(Server *S, const Batch &b, int32_t status, std::vector<std::vector<tdpm_detection>> *per_part)
{
    std::lock_guard<std::mutex> lk(S->mu);
    const uint64_t t = now_ns();
    for (size_t i = 0; i < b.parts.size(); ++i) {
        Request *r = b.parts[i].req;
        if (status != TDPM_OK && r->status == TDPM_OK) r->status = status;
        if (per_part) r->dets[b.parts[i].model_index] = std::move((*per_part)[i]);
        r->batch_images = std::max<int32_t>(r->batch_images, (int32_t)b.parts.size());
        if (--r->parts_left == 0) {
            r->t_done = t;
            r->done = true;
        }
    }
    S->cv_done.notify_all();
}

// Read back a batch's detections (each image with its own request's threshold) and hand them to its requests.
void finish(tdpm_ctx *ctx, Server *S, Batch &b)
{
    std::vector<float> taus(b.parts.size() * b.n_comps);
    for (size_t i = 0; i < b.parts.size(); ++i)
        std::fill(taus.begin() + i * b.n_comps, taus.begin() + (i + 1) * b.n_comps, b.parts[i].req->tau);
    std::vector<tdpm_detection> buf(4096);
    size_t n = 0;
    tdpm_status st = tdpm_detect_thresholds(ctx, b.scores_id, taus.data(), buf.data(), buf.size(), &n, b.stream);
    if (st == TDPM_ERR_CAPACITY) {
        buf.resize(n);
        st = tdpm_detect_thresholds(ctx, b.scores_id, taus.data(), buf.data(), buf.size(), &n, b.stream);
    }
    tdpm_release(ctx, b.scores_id);
    if (st != TDPM_OK) {
        complete_parts(S, b, st, nullptr);
        return;
    }
    std::vector<std::vector<tdpm_detection>> per_part(b.parts.size());
    for (size_t i = 0; i < n; ++i) {
        const tdpm_detection &d = buf[i];
        if (d.image < 0 || d.image >= (int)b.parts.size()) continue;
        per_part[d.image].push_back(d);
        per_part[d.image].back().image = 0;
    }
    complete_parts(S, b, TDPM_OK, &per_part);
}

void server_loop(tdpm_ctx *ctx, Server *S)
{
    cudaSetDevice(ctx->device);
    std::deque<Batch> inflight;
    size_t inflight_bytes = 0;
    size_t slot = 0;
    const size_t budget = S->cfg.mem_budget_bytes;
    std::vector<Part> carry;  // parts of a batch that was halved to fit the budget, tried first next time
    auto retire_oldest = [&]() {
        Batch b = std::move(inflight.front());
        inflight.pop_front();
        inflight_bytes -= b.bytes;
        finish(ctx, S, b);
    };
    for (;;) {
        std::vector<Part> take;
        if (!carry.empty()) {
            take.swap(carry);
        } else {
            std::unique_lock<std::mutex> lk(S->mu);
            if (S->queue.empty() && inflight.empty()) {
                S->cv_work.wait(lk, [&] { return S->stop || !S->queue.empty(); });
                if (S->queue.empty()) break;  // stop requested and nothing left
                if (S->cfg.max_wait_us > 0 && (int)S->queue.size() < S->cfg.max_batch_images)
                    S->cv_work.wait_for(lk, std::chrono::microseconds(S->cfg.max_wait_us), [&] {
                        return S->stop || (int)S->queue.size() >= S->cfg.max_batch_images;
                    });
            }
            if (!S->queue.empty() && inflight.size() < (size_t)S->cfg.max_inflight) {
                // oldest part's key; then every queued part with the same key, in arrival order
                const Part first = S->queue.front();
                const int32_t model = first.req->models[first.model_index];
                const int32_t form = first.req->form, prec = first.req->precision;
                for (auto it = S->queue.begin(); it != S->queue.end() && (int)take.size() < S->cfg.max_batch_images;) {
                    const Request *r = it->req;
                    if (r->models[it->model_index] == model && r->form == form && r->precision == prec) {
                        take.push_back(*it);
                        it = S->queue.erase(it);
                    } else {
                        ++it;
                    }
                }
            }
        }
        if (take.empty()) {
            if (!inflight.empty()) retire_oldest();
            continue;
        }
        Batch b;
        b.model = take.front().req->models[take.front().model_index];
        b.form = take.front().req->form;
        b.precision = take.front().req->precision;
        std::vector<tdpm_pyramid> pyrs;
        for (const Part &p : take) pyrs.push_back(p.req->pyr);
        // component mask of the batch ([image][component]); none when every image wants every component
        std::vector<uint8_t> mask;
        tdpm_status st = TDPM_OK;
        bool subset = false;
        for (const Part &p : take) subset |= !p.req->components.empty();
        {
            std::lock_guard<std::mutex> lk(ctx->mu);
            const Model *m = get_model(ctx, b.model);
            b.n_comps = m ? m->comps.size() : 0;
        }
        if (!b.n_comps) st = TDPM_ERR_STATE;  // unknown model
        if (subset && st == TDPM_OK) {
            const size_t nc = b.n_comps;
            mask.assign(take.size() * nc, 1);
            for (size_t i = 0; i < take.size() && nc; ++i) {
                const auto &cs = take[i].req->components;
                if (cs.empty()) continue;
                std::fill(mask.begin() + i * nc, mask.begin() + (i + 1) * nc, 0);
                for (int32_t c : cs) {
                    if (c < 0 || (size_t)c >= nc) st = TDPM_ERR_ARG;
                    else mask[i * nc + c] = 1;
                }
            }
        }
        if (st == TDPM_OK)
            st = batch_arena_bytes(ctx, b.model, pyrs.data(), (int32_t)pyrs.size(), subset ? mask.data() : nullptr,
                                   b.form, b.precision, &b.bytes);
        if (st == TDPM_OK && budget && b.bytes > budget) {
            if (take.size() > 1) {
                // too large even alone: run the first half now, put the second half back at the head of the queue
                const size_t half = take.size() / 2;
                {
                    std::lock_guard<std::mutex> lk(S->mu);
                    S->queue.insert(S->queue.begin(), take.begin() + half, take.end());
                }
                take.resize(half);
                carry.swap(take);
                continue;
            }
            st = TDPM_ERR_OOM;
        }
        b.parts = take;
        if (st != TDPM_OK) {
            complete_parts(S, b, st, nullptr);
            continue;
        }
        while (!inflight.empty() &&
               (inflight.size() >= (size_t)S->cfg.max_inflight || (budget && inflight_bytes + b.bytes > budget)))
            retire_oldest();
        b.stream = S->streams[slot];
        slot = (slot + 1) % S->streams.size();
        {
            std::lock_guard<std::mutex> lk(S->mu);
            const uint64_t t = now_ns();
            for (const Part &p : b.parts)
                if (!p.req->t_start) p.req->t_start = t;
        }
        st = tdpm_build_batch_scores_subset(ctx, b.model, pyrs.data(), (int32_t)pyrs.size(),
                                            subset ? mask.data() : nullptr, b.form, b.precision, b.stream,
                                            &b.scores_id);
        if (st != TDPM_OK) {
            complete_parts(S, b, st, nullptr);
            continue;
        }
        inflight_bytes += b.bytes;
        inflight.push_back(std::move(b));
    }
    while (!inflight.empty()) retire_oldest();
}

}  // namespace

void server_shutdown(tdpm_ctx *ctx)
{
    Server *S = ctx->server;
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->th.joinable()) S->th.join();
    for (cudaStream_t st : S->streams) cudaStreamDestroy(st);
    S->streams.clear();
}

void server_free(tdpm_ctx *ctx)
{
    server_shutdown(ctx);
    delete ctx->server;
    ctx->server = nullptr;
}

}  // namespace tdpm

using namespace tdpm;

extern "C" {

tdpm_status tdpm_server_start(tdpm_ctx *ctx, const tdpm_server_config *cfg)
{
    clear_error();
    if (!ctx || !cfg) return fail(TDPM_ERR_ARG, "NULL argument");
    if (cfg->max_batch_images < 1 || cfg->max_batch_images > 4096)
        return fail(TDPM_ERR_ARG, "max_batch_images must be in [1, 4096]");
    if (cfg->max_inflight < 1 || cfg->max_inflight > 4) return fail(TDPM_ERR_ARG, "max_inflight must be in [1, 4]");
    if (cfg->max_wait_us < 0) return fail(TDPM_ERR_ARG, "max_wait_us must be >= 0");
    if (ctx->server && ctx->server->th.joinable()) return fail(TDPM_ERR_STATE, "server already running");
    if (!ctx->server) ctx->server = new Server;
    Server *S = ctx->server;
    S->cfg = *cfg;
    S->stop = false;
    CUDA_TRY(cudaSetDevice(ctx->device));
    for (int i = 0; i < cfg->max_inflight; ++i) {
        cudaStream_t st = nullptr;
        CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        S->streams.push_back(st);
    }
    S->th = std::thread(server_loop, ctx, S);
    return TDPM_OK;
}

tdpm_status tdpm_server_stop(tdpm_ctx *ctx)
{
    clear_error();
    if (!ctx) return fail(TDPM_ERR_ARG, "ctx is NULL");
    if (ctx->server) server_shutdown(ctx);
    return TDPM_OK;
}

tdpm_status tdpm_submit(tdpm_ctx *ctx, const tdpm_request *req, uint64_t *ticket)
{
    clear_error();
    if (!ctx || !req || !ticket || !req->pyramid || !req->model_ids) return fail(TDPM_ERR_ARG, "NULL argument");
    Server *S = ctx->server;
    if (!S || !S->th.joinable()) return fail(TDPM_ERR_STATE, "server not running");
    if (req->n_models < 1 || req->n_models > TDPM_MAX_REQUEST_MODELS)
        return fail(TDPM_ERR_ARG, "n_models must be in [1, TDPM_MAX_REQUEST_MODELS]");
    if (req->form != TDPM_FORM_FULL && req->form != TDPM_FORM_DECOMPOSED) return fail(TDPM_ERR_ARG, "bad form");
    if (!valid_precision(req->precision)) return fail(TDPM_ERR_ARG, "unsupported precision");
    if (std::isnan(req->tau)) return fail(TDPM_ERR_ARG, "tau is NaN");
    const tdpm_pyramid &py = *req->pyramid;
    if (py.n_levels <= 0 || py.n_levels > 4096 || !py.levels) return fail(TDPM_ERR_ARG, "empty pyramid");
    if (py.lambda < 1 || py.lambda > py.n_levels) return fail(TDPM_ERR_ARG, "lambda out of range");
    for (int j = 0; j < py.n_levels; ++j) {
        const tdpm_level &l = py.levels[j];
        if (l.H <= 0 || l.W <= 0 || l.H > 4096 || l.W > 4096 || !l.data)
            return fail(TDPM_ERR_ARG, "level with a bad size or NULL data");
        if (reinterpret_cast<uintptr_t>(l.data) % 16) return fail(TDPM_ERR_ARG, "level data not 16-byte aligned");
    }
    for (int i = 0; i < req->n_models; ++i)
        for (int k = 0; k < i; ++k)
            if (req->model_ids[i] == req->model_ids[k]) return fail(TDPM_ERR_ARG, "model listed twice");
    if (req->n_components < 0 || (req->n_components > 0 && !req->components))
        return fail(TDPM_ERR_ARG, "bad component list");
    for (int i = 0; i < req->n_components; ++i) {
        if (req->components[i] < 0) return fail(TDPM_ERR_ARG, "negative component id");
        for (int k = 0; k < i; ++k)
            if (req->components[i] == req->components[k]) return fail(TDPM_ERR_ARG, "component listed twice");
    }
    auto r = std::make_unique<Request>();
    r->levels.assign(py.levels, py.levels + py.n_levels);
    r->pyr = py;
    r->pyr.levels = r->levels.data();
    r->models.assign(req->model_ids, req->model_ids + req->n_models);
    if (req->n_components > 0) r->components.assign(req->components, req->components + req->n_components);
    r->form = req->form;
    r->precision = req->precision;
    r->tau = req->tau;
    r->parts_left = req->n_models;
    r->dets.resize(req->n_models);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) return fail(TDPM_ERR_STATE, "server is stopping");
        r->ticket = S->next_ticket++;
        r->t_submit = now_ns();
        for (int i = 0; i < req->n_models; ++i) S->queue.push_back(Part{r.get(), i});
        *ticket = r->ticket;
        S->reqs[r->ticket] = std::move(r);
    }
    S->cv_work.notify_one();
    return TDPM_OK;
}

tdpm_status tdpm_poll(tdpm_ctx *ctx, uint64_t ticket, int32_t timeout_ms, tdpm_detection *out, size_t capacity,
                      size_t *n_out, tdpm_result_info *info)
{
    clear_error();
    if (!ctx || !n_out || (capacity > 0 && !out)) return fail(TDPM_ERR_ARG, "NULL argument");
    Server *S = ctx->server;
    if (!S) return fail(TDPM_ERR_STATE, "no server");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return fail(TDPM_ERR_STATE, "unknown or released ticket");
    Request *r = it->second.get();
    auto ready = [&] { return r->done; };
    if (timeout_ms < 0) S->cv_done.wait(lk, ready);
    else S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready);
    *n_out = 0;
    if (!r->done) return fail(TDPM_ERR_TIMEOUT, "request not finished");
    const int32_t status = r->status;
    size_t n = 0;
    if (status == TDPM_OK)
        for (const auto &v : r->dets) n += v.size();  // a failed request hands out no records
    *n_out = n;
    if (info) {
        info->status = r->status;
        info->batch_images = r->batch_images;
        info->t_submit_ns = r->t_submit;
        info->t_start_ns = r->t_start;
        info->t_done_ns = r->t_done;
        info->n_detections = n;
    }
    if (n > capacity) return fail(TDPM_ERR_CAPACITY, "detection buffer too small");
    size_t k = 0;
    if (status == TDPM_OK)
        for (const auto &v : r->dets)
            for (const tdpm_detection &d : v) out[k++] = d;
    S->reqs.erase(it);
    if (status != TDPM_OK) return fail(status, "request failed");
    return TDPM_OK;
}

}  // extern "C"
