// C-ABI, part 2: scoring a pyramid (steps 1-3), detection (step 4), maps, instrumentation and stateless ops.
//
// A Plan is computed once per (model version, form, precision, pyramid shape): the arena layout (every score map,
// intermediate and job table at a fixed offset) and the launch list (one launch per stage over all levels). A device
// arena holds one scores set; its pinned host blob carries the job tables. Reusing an arena for the same plan only
// patches the caller's level pointers in the blob, and from the second use on the whole enqueue (table upload plus
// every kernel) is replayed as one CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <functional>
#include <string>
#include <vector>

#include "ctx.h"

namespace tdpm {

namespace {
std::atomic<unsigned long long> g_launches{0};
std::atomic<unsigned long long> g_plan_uid{1};

int fdiv2(int a) { return a >= 0 ? a / 2 : -((-a + 1) / 2); }

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

// while a thread captures a graph its launches are counted into the graph (they run at each replay, not now)
thread_local int *t_capture_launches = nullptr;

void note_launches(int n)
{
    if (t_capture_launches) *t_capture_launches += n;
    else g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed);
}

cudaError_t allow_max_dynamic_smem(const void *func, int slot)
{
    static std::atomic<bool> done[kSmemSlots][64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (slot >= 0 && slot < kSmemSlots && dev >= 0 && dev < 64 && done[slot][dev].load(std::memory_order_acquire))
        return cudaSuccess;
    // the opt-in maximum minus the kernel's own static shared memory
    cudaFuncAttributes fa{};
    e = cudaFuncGetAttributes(&fa, func);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kMaxDynamicSmem - (int)fa.sharedSizeBytes);
    if (e == cudaSuccess && slot >= 0 && slot < kSmemSlots && dev >= 0 && dev < 64)
        done[slot][dev].store(true, std::memory_order_release);
    return e;
}

struct GroupLevel {
    int j;
    size_t out_off, z_off;
    int Ho, Wo;
    size_t u_off = 0, u_lo_off = 0;  // joint form on tensor cores: per-term maps U_r, BF16 planar hi / lo
};

struct DtPlan {
    int fid, jroot, l, Hs, Ws, X, Y, vx, vy;
    float d[4];
    size_t s_off, v_off, iv_off, d_off, a_off;
};

struct AsmPlan {
    int image, c, j, Y, X, root_W;
    float bias;
    size_t out_off, root_off;
    std::vector<int> dt;
};

struct Plan {
    uint64_t uid = 0;
    int model_id = 0, form = 0, precision = 0, L = 0;  // L: levels of all images (flat index)
    int n_images = 0;
    std::vector<int> img_base, img_L, img_lam;         // per image: first flat level, level count, lambda
    bool bf = false, split = false, dec = false;  // bf: the tensor-core path (BF16, split BF16 or FP8 operands)
    bool fp8 = false;
    std::vector<std::pair<int, int>> sizes;
    size_t arena_bytes = 0, blob_off = 0, blob_bytes = 0;
    std::vector<size_t> bf_off, bf_lo_off;  // planar copies of the levels: BF16 (hi part, lo part) or E4M3
    std::vector<std::vector<GroupLevel>> glv;
    std::vector<DtPlan> dts;
    std::vector<AsmPlan> asms;
    std::map<std::pair<int, int>, MapRef> filter_maps, final_maps, dt_maps, arg_maps;
    long long total = 0;
    int n_det_blocks = 0;
    size_t counts_off = 0, offsets_off = 0, total_off = 0;
    // job tables, offsets inside the blob
    size_t conv_off = 0;
    long long conv_items = 0;
    std::vector<size_t> g_jobs_off, g_sep_off, g_rec_off;
    std::vector<int> g_tiles, g_rec_tiles;  // tensor-core launches: M tiles (the N tiling is chosen at launch)
    // tile configuration of the group's tensor-core launches (tuned or default): N tile width | persistent << 16
    std::vector<int> g_nt, g_rec_nt;
    bool tuned = false;
    std::vector<long long> g_sep_tiles;
    // decomposed per-filter groups on tensor cores with the fused kernel: no Z maps; spatial tiles in g_tiles, filter
    // groups (ZsGroup table at g_fg_off) and their width bound
    std::vector<char> g_fused;
    std::vector<size_t> g_fg_off, g_tile_off, g_frec_off;
    std::vector<std::vector<uint8_t>> g_frec;  // packed factor records of the filter groups (persistent forms)
    bool zsep_forced = false;                  // the fused kernel's form was fixed by the context (not tuned)
    std::vector<int> g_n_fg, g_nmax;
    std::vector<std::vector<ZsGroup>> g_fg;
    size_t dt_off = 0, asm_off = 0, dt_cta_off = 0;  // dt_cta_off: the job of every distance-transform CTA
    int dt_ctas = 0, max_W = 1, max_H = 1;  // CTAs of the fused distance transform (strips of sampled columns)
    std::vector<std::pair<size_t, int>> patches;  // blob offsets of caller level pointers

    // decomposed per-filter groups whose every filter is at its exact rank (h*w, the slice form): scored by the full
    // form's kernel on the original filters (the same function, in fewer flops than the slice form's passes)
    std::vector<char> g_exact;
    bool gdec(size_t gi) const { return dec && !g_exact[gi]; }
    // joint decomposition with tensor-core operands: the separable stage writes U_r and Lambda U runs as a GEMM
    bool rec_tc(const Group &g) const { return bf && dec && g.joint; }
    int sep_mode(const Group &g) const { return rec_tc(g) ? SEP_TERMS : (g.joint ? SEP_JOINT : SEP_PER_FILTER); }
    int sep_k(const Group &g) const { return rec_tc(g) ? g.Upad : g.K; }
};

namespace {

// mask: null (every component of every image) or [n][components], nonzero = score that component on that image
std::string plan_key(int model_id, const Model &m, int form, int prec, const tdpm_pyramid *pyrs, int n,
                     const uint8_t *mask, bool fuse, int zsep_form)
{
    std::string k = std::to_string(model_id) + ":" + std::to_string(m.version) + ":" + std::to_string(form) + ":" +
                    std::to_string(prec) + ":" + std::to_string(n) + (fuse ? ":f" : ":u") + std::to_string(zsep_form);
    for (int i = 0; i < n; ++i) {
        k += "|" + std::to_string(pyrs[i].lambda);
        for (int j = 0; j < pyrs[i].n_levels; ++j)
            k += ":" + std::to_string(pyrs[i].levels[j].H) + "x" + std::to_string(pyrs[i].levels[j].W);
        if (mask) {
            k += "/";
            for (size_t c = 0; c < m.comps.size(); ++c) k += mask[(size_t)i * m.comps.size() + c] ? '1' : '0';
        }
    }
    return k;
}

// The terms-on-M fused kernel serves the shapes it has unless TDPM_ZSEPT=0 (then the tile kernel below does), or
// unless a form of the tile kernel is forced (TDPM_ZSEP_FORM).
bool zsept_enabled()
{
    static const bool on = [] {
        const char *e = getenv("TDPM_ZSEPT");
        return !(e && e[0] == '0');
    }();
    return on;
}

// The untuned form of the tensor-core correlation launches: TDPM_CORR_FORM=tile or =persistent fixes it for every
// precision (a profiling and testing aid; the tuner, when on, still times both) and for tdpm_correlate; -1 when unset.
// Read at each plan build and each tdpm_correlate call.
int corr_form_override()
{
    const char *e = getenv("TDPM_CORR_FORM");
    if (!e) return -1;
    if (!strcmp(e, "tile")) return 0;
    if (!strcmp(e, "persistent")) return 1;
    return -1;
}

// The filter groups of a per-filter decomposed shape group for the fused kernel: consecutive filters while their
// terms fit nmax (and the bank rows an MMA of the rounded-up width reads exist). Empty when the group cannot be fused.
std::vector<ZsGroup> fused_groups(const Group &g, int *nmax_out)
{
    std::vector<ZsGroup> out;
    if (g.joint || !zsep_shape(g.h, g.w) || (int)g.rank_off.size() != g.K + 1) return out;
    int max_rank = 0;
    for (int k = 0; k < g.K; ++k) max_rank = std::max(max_rank, g.rank_off[k + 1] - g.rank_off[k]);
    const int nmax = zsep_nmax(max_rank);
    if (!nmax || max_rank <= 0) return out;
    for (int k0 = 0; k0 < g.K;) {
        const int t0 = g.rank_off[k0];
        int k1 = k0 + 1;
        while (k1 < g.K && g.rank_off[k1 + 1] - t0 <= nmax) ++k1;
        const int n = g.rank_off[k1] - t0;
        if (t0 + (n + 15) / 16 * 16 > g.Rpad_tc) return {};
        out.push_back(ZsGroup{k0, k1, t0, n});
        k0 = k1;
    }
    *nmax_out = nmax;
    return out;
}

std::shared_ptr<Plan> make_plan(const Model &m, int model_id, const tdpm_pyramid *pyrs, int n_images, int form,
                                int prec, const uint8_t *mask, bool fuse, int zsep_form)
{
    auto P = std::make_shared<Plan>();
    P->uid = g_plan_uid.fetch_add(1);
    P->model_id = model_id; P->form = form; P->precision = prec;
    P->n_images = n_images;
    for (int i = 0; i < n_images; ++i) {
        P->img_base.push_back((int)P->sizes.size());
        P->img_L.push_back(pyrs[i].n_levels);
        P->img_lam.push_back(pyrs[i].lambda);
        for (int j = 0; j < pyrs[i].n_levels; ++j) P->sizes.push_back({pyrs[i].levels[j].H, pyrs[i].levels[j].W});
    }
    P->L = (int)P->sizes.size();
    P->bf = prec == TDPM_PREC_BF16 || prec == TDPM_PREC_BF16X3 || prec == TDPM_PREC_FP8;
    P->fp8 = prec == TDPM_PREC_FP8;
    P->split = prec == TDPM_PREC_BF16X3;
    P->dec = form == TDPM_FORM_DECOMPOSED;
    const int L = P->L;
    Bump bump;
    if (P->bf) {
        P->bf_off.resize(L);
        const size_t elem = P->fp8 ? 1 : sizeof(uint16_t);
        for (int j = 0; j < L; ++j) P->bf_off[j] = bump.take(elem * (size_t)P->sizes[j].first * P->sizes[j].second * FD);
        if (P->split) {
            P->bf_lo_off.resize(L);
            for (int j = 0; j < L; ++j)
                P->bf_lo_off[j] = bump.take(sizeof(uint16_t) * (size_t)P->sizes[j].first * P->sizes[j].second * FD);
        }
    }
    P->glv.resize(m.groups.size());
    const size_t ngr = m.groups.size();
    P->g_exact.assign(ngr, 0);
    for (size_t gi = 0; gi < ngr && P->dec; ++gi) {
        const Group &g = m.groups[gi];
        bool exact = !g.joint && (int)g.rank_off.size() == g.K + 1;
        for (int k = 0; k < g.K && exact; ++k) exact = g.rank_off[k + 1] - g.rank_off[k] >= g.h * g.w;
        P->g_exact[gi] = exact;
    }
    P->g_fused.assign(ngr, 0); P->g_fg_off.assign(ngr, 0); P->g_tile_off.assign(ngr, 0); P->g_frec_off.assign(ngr, 0);
    P->g_frec.assign(ngr, {}); P->g_n_fg.assign(ngr, 0); P->g_nmax.assign(ngr, 0);
    P->g_fg.assign(ngr, {});
    for (size_t gi = 0; gi < ngr; ++gi) {
        // the fused kernel: BF16 or split-BF16 operands, per-filter factors, a compiled shape
        if (!fuse || !P->bf || P->fp8 || !P->dec) break;
        if (P->g_exact[gi]) continue;
        {
            // terms on the M dimension (6x6 and 7x7 filters): term groups of consecutive filters, <= 128 terms each
            const Group &g = m.groups[gi];
            std::vector<ZsGroup> tg;
            if (!g.joint && zsept_shape(g.h, g.w) && (int)g.rank_off.size() == g.K + 1 && zsep_form < 0 &&
                zsept_enabled()) {
                const int M = zsept_terms();
                bool ok = true;
                for (int k0 = 0; k0 < g.K && ok;) {
                    const int t0 = g.rank_off[k0];
                    int k1 = k0;
                    while (k1 < g.K && g.rank_off[k1 + 1] - t0 <= M) ++k1;
                    if (k1 == k0 || t0 + M > g.Rpad_tc) ok = false;  // a filter above 128 terms, or a short bank
                    else tg.push_back(ZsGroup{k0, k1, t0, g.rank_off[k1] - t0});
                    k0 = k1;
                }
                if (!ok) tg.clear();
            }
            if (!tg.empty()) {
                P->g_fg[gi] = tg;
                P->g_fused[gi] = 2;
                P->g_n_fg[gi] = (int)tg.size();
                P->g_nmax[gi] = zsept_terms();
                const int rec = zsept_record_bytes(), M = zsept_terms();
                std::vector<uint8_t> &out = P->g_frec[gi];
                out.assign((size_t)rec * tg.size(), 0);
                for (size_t f = 0; f < tg.size(); ++f) {
                    const ZsGroup &G = tg[f];
                    float *fv = reinterpret_cast<float *>(out.data() + f * rec);
                    int *ri = reinterpret_cast<int *>(fv + (size_t)M * zsept_factor_stride());
                    for (int k = G.k0; k < G.k1; ++k)
                        for (int r = g.rank_off[k]; r < g.rank_off[k + 1]; ++r) {
                            const int l = r - G.t0;
                            const double lam = g.Lam[(size_t)k * g.R + r];
                            for (int i = 0; i < g.h; ++i) fv[(size_t)i * M + l] = (float)(lam * g.A[(size_t)i * g.R + r]);
                            for (int i = 0; i < g.w; ++i) fv[(size_t)(g.h + i) * M + l] = (float)g.B[(size_t)i * g.R + r];
                        }
                    ri[0] = G.k1 - G.k0;
                    ri[1] = G.k0;
                    for (int i = 0; i <= G.k1 - G.k0; ++i) ri[2 + i] = g.rank_off[G.k0 + i] - G.t0;
                }
                continue;
            }
        }
        int nmax = 0;
        P->g_fg[gi] = fused_groups(m.groups[gi], &nmax);
        if (P->g_fg[gi].empty()) continue;
        P->g_fused[gi] = 1;
        P->g_n_fg[gi] = (int)P->g_fg[gi].size();
        P->g_nmax[gi] = nmax;
        // packed factor records: the same FP32 values as the group's device factor copies
        const Group &g = m.groups[gi];
        const int rec = zsep_record_bytes(g.h, g.w, nmax), fs = zsep_factor_stride(g.h, g.w);
        std::vector<uint8_t> &out = P->g_frec[gi];
        out.assign((size_t)rec * P->g_fg[gi].size(), 0);
        for (size_t f = 0; f < P->g_fg[gi].size(); ++f) {
            const ZsGroup &G = P->g_fg[gi][f];
            float *fv = reinterpret_cast<float *>(out.data() + f * rec);
            int *ro = reinterpret_cast<int *>(fv + (size_t)nmax * fs);
            for (int k = G.k0; k < G.k1; ++k)
                for (int r = g.rank_off[k]; r < g.rank_off[k + 1]; ++r) {
                    float *t = fv + (size_t)(r - G.t0) * fs;
                    for (int i = 0; i < g.h; ++i) t[i] = (float)g.A[(size_t)i * g.R + r];
                    for (int i = 0; i < g.w; ++i) t[g.h + i] = (float)g.B[(size_t)i * g.R + r];
                    t[g.h + g.w] = (float)g.Lam[(size_t)k * g.R + r];
                }
            for (int i = 0; i <= G.k1 - G.k0; ++i) ro[i] = g.rank_off[G.k0 + i] - G.t0;
        }
    }
    for (size_t gi = 0; gi < m.groups.size(); ++gi) {
        const Group &g = m.groups[gi];
        for (int im = 0; im < n_images; ++im) {
            // roots score levels [lambda, L) of each image, parts levels [0, L - lambda)
            const int base = P->img_base[im], lam = P->img_lam[im], Li = P->img_L[im];
            const int j0 = base + (g.role == 0 ? lam : 0), j1 = base + (g.role == 0 ? Li : Li - lam);
            for (int j = j0; j < j1; ++j) {
                const int H = P->sizes[j].first, W = P->sizes[j].second;
                const int Ho = H - g.h + 1, Wo = W - g.w + 1;
                if (Ho <= 0 || Wo <= 0) continue;
                GroupLevel gl{j, 0, 0, Ho, Wo};
                gl.out_off = bump.take(sizeof(float) * (size_t)g.K * Ho * Wo);
                if (P->gdec(gi) && !P->g_fused[gi]) gl.z_off = bump.take(sizeof(float) * (size_t)g.R * H * W);
                if (P->rec_tc(g)) {
                    gl.u_off = bump.take(sizeof(uint16_t) * (size_t)g.Upad * Ho * Wo);
                    if (P->split) gl.u_lo_off = bump.take(sizeof(uint16_t) * (size_t)g.Upad * Ho * Wo);
                }
                P->glv[gi].push_back(gl);
                for (int k = 0; k < g.K; ++k)
                    P->filter_maps[{g.fids[k], j}] = MapRef{gl.out_off + sizeof(float) * (size_t)k * Ho * Wo, Ho, Wo};
            }
        }
    }
    for (int im = 0; im < n_images; ++im)
    for (size_t c = 0; c < m.comps.size(); ++c) {
        if (mask && !mask[(size_t)im * m.comps.size() + c]) continue;  // component not asked for on this image
        const CompH &C = m.comps[c];
        const FilterH &Rf = m.filters[C.root_fid];
        const int base = P->img_base[im], lam = P->img_lam[im], Li = P->img_L[im];
        for (int j = base + lam; j < base + Li; ++j) {
            const int l = j - lam;
            // root positions where the root and every anchored part placement fit
            int Y = P->sizes[j].first - Rf.h + 1, X = P->sizes[j].second - Rf.w + 1;
            for (const PartH &Pp : C.parts) {
                const FilterH &Pf = m.filters[Pp.fid];
                const int Hs = P->sizes[l].first - Pf.h + 1, Ws = P->sizes[l].second - Pf.w + 1;
                if (Hs <= 0 || Ws <= 0) { Y = 0; X = 0; break; }
                Y = std::min(Y, fdiv2(Hs - 1 - Pp.vy) + 1);
                X = std::min(X, fdiv2(Ws - 1 - Pp.vx) + 1);
            }
            if (Y <= 0 || X <= 0) continue;
            AsmPlan ap;
            ap.image = im; ap.c = (int)c; ap.j = j; ap.Y = Y; ap.X = X; ap.bias = C.bias;
            const MapRef &Rm = P->filter_maps.at({C.root_fid, j});
            ap.root_off = Rm.off;
            ap.root_W = Rm.cols;
            ap.out_off = bump.take(sizeof(float) * (size_t)Y * X);
            P->final_maps[{(int)c, j}] = MapRef{ap.out_off, Y, X};
            for (const PartH &Pp : C.parts) {
                const FilterH &Pf = m.filters[Pp.fid];
                DtPlan dp;
                dp.fid = Pp.fid; dp.jroot = j; dp.l = l;
                dp.Hs = P->sizes[l].first - Pf.h + 1; dp.Ws = P->sizes[l].second - Pf.w + 1;
                dp.X = X; dp.Y = Y; dp.vx = Pp.vx; dp.vy = Pp.vy;
                std::memcpy(dp.d, Pp.d, sizeof(dp.d));
                dp.s_off = P->filter_maps.at({Pp.fid, l}).off;
                dp.v_off = dp.iv_off = 0;  // the fused distance transform keeps V and IV in shared memory
                dp.d_off = bump.take(sizeof(float) * (size_t)Y * X);
                dp.a_off = bump.take(sizeof(int32_t) * (size_t)Y * X);
                P->dt_maps[{Pp.fid, j}] = MapRef{dp.d_off, Y, X};
                P->arg_maps[{Pp.fid, j}] = MapRef{dp.a_off, Y, X};
                ap.dt.push_back((int)P->dts.size());
                P->dts.push_back(dp);
            }
            P->asms.push_back(std::move(ap));
        }
    }
    for (const AsmPlan &a : P->asms) P->total += (long long)a.Y * a.X;
    P->n_det_blocks = (int)((P->total + detect_positions_per_block() - 1) / detect_positions_per_block());
    P->counts_off = bump.take(sizeof(int) * std::max(1, P->n_det_blocks));
    P->offsets_off = bump.take(sizeof(int) * std::max(1, P->n_det_blocks));
    P->total_off = bump.take(sizeof(long long));
    P->blob_off = align256(bump.off);

    // job tables inside the blob
    Bump jb;
    if (P->bf) {
        P->conv_off = jb.take(sizeof(ConvJob) * L);
        for (int j = 0; j < L; ++j) P->conv_items += (P->fp8 ? 2ll : 4ll) * P->sizes[j].first * P->sizes[j].second;
    }
    const size_t ng = m.groups.size();
    P->g_jobs_off.assign(ng, 0); P->g_sep_off.assign(ng, 0); P->g_tiles.assign(ng, 0); P->g_sep_tiles.assign(ng, 0);
    P->g_rec_off.assign(ng, 0); P->g_rec_tiles.assign(ng, 0);
    P->g_nt.assign(ng, 0); P->g_rec_nt.assign(ng, 0);
    for (size_t gi = 0; gi < ng; ++gi) {
        const Group &g = m.groups[gi];
        const size_t nj = std::max<size_t>(1, P->glv[gi].size());
        const size_t job_bytes = P->g_fused[gi] ? sizeof(ZsJob)
                                 : P->bf        ? sizeof(TcJob)
                                                : (P->gdec(gi) ? sizeof(ZJob) : sizeof(CorrJob));
        P->g_jobs_off[gi] = jb.take(job_bytes * nj);
        if (P->g_fused[gi] == 2) {
            P->g_fg_off[gi] = jb.take(sizeof(int) * P->g_fg[gi].size());  // first term of every term group
            const int T = zsept_tile_side(), tc = T - g.w + 1, tr = T - g.h + 1;
            long long tiles = 0;
            for (const GroupLevel &gl : P->glv[gi])
                tiles += (long long)((gl.Wo + tc - 1) / tc) * ((gl.Ho + tr - 1) / tr);
            P->g_tiles[gi] = (int)std::min<long long>(tiles, 0x7fffffff);
            P->g_tile_off[gi] = jb.take(sizeof(ZsTile) * std::max(1, P->g_tiles[gi]));
            P->g_frec_off[gi] = jb.take(P->g_frec[gi].size());
            P->g_nt[gi] = 0;
            continue;
        }
        if (P->g_fused[gi]) {
            P->g_fg_off[gi] = jb.take(sizeof(ZsGroup) * P->g_fg[gi].size());
            int tc, tr;
            zsep_tile(g.h, g.w, &tc, &tr);
            long long tiles = 0;
            for (const GroupLevel &gl : P->glv[gi])
                tiles += (long long)((gl.Wo + tc - 1) / tc) * ((gl.Ho + tr - 1) / tr);
            P->g_tiles[gi] = (int)std::min<long long>(tiles, 0x7fffffff);
            P->g_tile_off[gi] = jb.take(sizeof(ZsTile) * std::max(1, P->g_tiles[gi]));
            P->g_frec_off[gi] = jb.take(P->g_frec[gi].size());
            // untuned: one CTA per item (the tuner's usual choice for the large part groups)
            P->g_nt[gi] = ZSEP_TILE;
            if (zsep_form >= 0 && zsep_form_fits(g.h, g.w, P->split, P->g_nmax[gi], zsep_form)) {
                P->g_nt[gi] = zsep_form;  // fixed by the context
                P->zsep_forced = true;
            }
            continue;
        }
        if (P->gdec(gi)) P->g_sep_off[gi] = jb.take(sizeof(SepJob) * nj);
        if (P->rec_tc(g)) P->g_rec_off[gi] = jb.take(sizeof(TcJob) * nj);
        int tiles = 0, rec_tiles = 0;
        long long sep_tiles = 0;
        for (const GroupLevel &gl : P->glv[gi]) {
            const int H = P->sizes[gl.j].first, W = P->sizes[gl.j].second;
            if (P->bf) {
                const long long span = P->gdec(gi) ? (long long)H * W : (long long)(gl.Ho - 1) * W + gl.Wo;
                tiles += (int)((span + corr_tc_tile_m() - 1) / corr_tc_tile_m());
            } else if (P->gdec(gi)) {
                tiles += ((H * W + zproj_simt_cells_per_tile() - 1) / zproj_simt_cells_per_tile()) *
                         ((g.R + zproj_simt_r_chunk() - 1) / zproj_simt_r_chunk());
            } else {
                tiles += ((gl.Wo + corr_f32_tile_x() - 1) / corr_f32_tile_x()) *
                         ((gl.Ho + corr_f32_tile_y() - 1) / corr_f32_tile_y()) * (g.Kpad / corr_f32_tile_k());
            }
            if (P->gdec(gi)) {
                int tx, ty;
                sep_tiles += sep_job_items(P->sep_mode(g), g.h, g.w, gl.Ho, gl.Wo, P->sep_k(g), &tx, &ty);
            }
            if (P->rec_tc(g))
                rec_tiles += (int)(((long long)gl.Ho * gl.Wo + corr_tc_tile_m() - 1) / corr_tc_tile_m());
        }
        P->g_tiles[gi] = tiles;
        P->g_sep_tiles[gi] = sep_tiles;
        P->g_rec_tiles[gi] = rec_tiles;
        // untuned: the balanced width; the persistent form for split operands (three MMAs per step keep the tensor
        // cores busy enough for the accumulator double buffer to pay), the tile form otherwise
        const int form = corr_form_override();
        const int persist = (form < 0 ? P->split : form == 1) ? kTcPersistent : 0;
        P->g_nt[gi] = (P->gdec(gi) ? corr_tc_default_nt(g.R, 1) : corr_tc_default_nt(g.K, g.h * g.w)) | persist;
        P->g_rec_nt[gi] = P->rec_tc(g) ? corr_tc_default_nt(g.K, g.Upad / FD) | persist : 0;
    }
    P->dt_off = jb.take(sizeof(DtJob) * std::max<size_t>(1, P->dts.size()));
    for (const DtPlan &p : P->dts) {
        P->max_W = std::max(P->max_W, p.Ws);
        P->max_H = std::max(P->max_H, p.Hs);
    }
    // one distance-transform CTA per strip of sampled columns (maps above the supported side are refused later)
    for (const DtPlan &p : P->dts) P->dt_ctas += dt_job_strips(p.X);
    P->dt_cta_off = jb.take(sizeof(int) * (size_t)std::max(1, P->dt_ctas));
    P->asm_off = jb.take(sizeof(AsmJob) * std::max<size_t>(1, P->asms.size()));
    P->blob_bytes = align256(jb.off);
    P->arena_bytes = P->blob_off + P->blob_bytes;
    return P;
}

// Write every job table of the plan into the arena's host blob (device pointers into this arena).
tdpm_status fill_blob(const Plan &P, const Model &m, const std::vector<const tdpm_level *> &lv, Arena &A)
{
    char *base = A.dev;
    char *hb = A.host;
    std::memset(hb, 0, P.blob_bytes);
    const_cast<Plan &>(P).patches.clear();
    std::vector<std::pair<size_t, int>> patches;
    if (P.bf) {
        ConvJob *cj = reinterpret_cast<ConvJob *>(hb + P.conv_off);
        long long begin = 0;
        for (int j = 0; j < P.L; ++j) {
            cj[j].src = lv[j]->data;
            patches.push_back({P.conv_off + sizeof(ConvJob) * j + offsetof(ConvJob, src), j});
            cj[j].dst = reinterpret_cast<uint16_t *>(base + P.bf_off[j]);
            cj[j].dst_lo = P.split ? reinterpret_cast<uint16_t *>(base + P.bf_lo_off[j]) : nullptr;
            cj[j].cells = (long long)P.sizes[j].first * P.sizes[j].second;
            cj[j].begin = begin;
            begin += (P.fp8 ? 2 : 4) * cj[j].cells;
        }
    }
    for (size_t gi = 0; gi < m.groups.size(); ++gi) {
        const Group &g = m.groups[gi];
        if (P.g_fused[gi]) {
            const bool zt = P.g_fused[gi] == 2;
            int tc, tr, bw = 32, bh = 4;
            if (zt) {
                bw = bh = zsept_tile_side();
                tc = bw - g.w + 1;
                tr = bh - g.h + 1;
            } else {
                zsep_tile(g.h, g.w, &tc, &tr);
            }
            ZsTile *tl = reinterpret_cast<ZsTile *>(hb + P.g_tile_off[gi]);
            for (size_t i = 0; i < P.glv[gi].size(); ++i) {
                const GroupLevel &gl = P.glv[gi][i];
                const int H = P.sizes[gl.j].first, W = P.sizes[gl.j].second;
                ZsJob &z = reinterpret_cast<ZsJob *>(hb + P.g_jobs_off[gi])[i];
                if (!encode_level_tmap_tiles(&z.tmap, reinterpret_cast<const uint16_t *>(base + P.bf_off[gl.j]), H, W,
                                             bw, bh) ||
                    (P.split && !encode_level_tmap_tiles(&z.tmap_lo,
                                                         reinterpret_cast<const uint16_t *>(base + P.bf_lo_off[gl.j]),
                                                         H, W, bw, bh)))
                    return fail(TDPM_ERR_CUDA, "cuTensorMapEncodeTiled failed");
                z.out = reinterpret_cast<float *>(base + gl.out_off);
                z.H = H; z.W = W; z.Ho = gl.Ho; z.Wo = gl.Wo;
                for (int y0 = 0; y0 < gl.Ho; y0 += tr)
                    for (int x0 = 0; x0 < gl.Wo; x0 += tc) *tl++ = ZsTile{(int)i, x0, y0, std::min(tr, gl.Ho - y0)};
            }
            if (zt) {
                int *t0s = reinterpret_cast<int *>(hb + P.g_fg_off[gi]);
                for (size_t f = 0; f < P.g_fg[gi].size(); ++f) t0s[f] = P.g_fg[gi][f].t0;
            } else {
                std::memcpy(hb + P.g_fg_off[gi], P.g_fg[gi].data(), sizeof(ZsGroup) * P.g_fg[gi].size());
            }
            std::memcpy(hb + P.g_frec_off[gi], P.g_frec[gi].data(), P.g_frec[gi].size());
            continue;
        }
        int begin = 0, rec_begin = 0;
        long long sep_begin = 0;
        for (size_t i = 0; i < P.glv[gi].size(); ++i) {
            const GroupLevel &gl = P.glv[gi][i];
            const int H = P.sizes[gl.j].first, W = P.sizes[gl.j].second;
            float *out = reinterpret_cast<float *>(base + gl.out_off);
            if (P.bf) {
                TcJob &t = reinterpret_cast<TcJob *>(hb + P.g_jobs_off[gi])[i];
                const bool ok = P.fp8 ? encode_level_tmap_fp8(&t.tmap, reinterpret_cast<const uint8_t *>(base + P.bf_off[gl.j]),
                                                              (long long)H * W)
                                      : encode_level_tmap(&t.tmap, reinterpret_cast<const uint16_t *>(base + P.bf_off[gl.j]),
                                                          (long long)H * W);
                if (!ok) return fail(TDPM_ERR_CUDA, "cuTensorMapEncodeTiled failed");
                if (P.split && !encode_level_tmap(&t.tmap_lo, reinterpret_cast<const uint16_t *>(base + P.bf_lo_off[gl.j]),
                                                  (long long)H * W))
                    return fail(TDPM_ERR_CUDA, "cuTensorMapEncodeTiled failed");
                const bool gd = P.gdec(gi);
                t.out = gd ? reinterpret_cast<float *>(base + gl.z_off) : out;
                t.H = H; t.W = W;
                t.Ho = gd ? H : gl.Ho;
                t.Wo = gd ? W : gl.Wo;
                t.begin = begin;
                const long long span = gd ? (long long)H * W : (long long)(gl.Ho - 1) * W + gl.Wo;
                begin += (int)((span + corr_tc_tile_m() - 1) / corr_tc_tile_m());
            } else if (P.gdec(gi)) {
                ZJob &z = reinterpret_cast<ZJob *>(hb + P.g_jobs_off[gi])[i];
                z.feat = lv[gl.j]->data;
                patches.push_back({P.g_jobs_off[gi] + sizeof(ZJob) * i + offsetof(ZJob, feat), gl.j});
                z.Z = reinterpret_cast<float *>(base + gl.z_off);
                z.cells = H * W;
                z.begin = begin;
                begin += ((z.cells + zproj_simt_cells_per_tile() - 1) / zproj_simt_cells_per_tile()) *
                         ((g.R + zproj_simt_r_chunk() - 1) / zproj_simt_r_chunk());
            } else {
                CorrJob &c = reinterpret_cast<CorrJob *>(hb + P.g_jobs_off[gi])[i];
                c.feat = lv[gl.j]->data;
                patches.push_back({P.g_jobs_off[gi] + sizeof(CorrJob) * i + offsetof(CorrJob, feat), gl.j});
                c.out = out;
                c.H = H; c.W = W; c.Ho = gl.Ho; c.Wo = gl.Wo;
                c.tiles_x = (gl.Wo + corr_f32_tile_x() - 1) / corr_f32_tile_x();
                c.tiles_y = (gl.Ho + corr_f32_tile_y() - 1) / corr_f32_tile_y();
                c.begin = begin;
                begin += c.tiles_x * c.tiles_y * (g.Kpad / corr_f32_tile_k());
            }
            if (P.gdec(gi)) {
                SepJob &sp = reinterpret_cast<SepJob *>(hb + P.g_sep_off[gi])[i];
                sp.Z = reinterpret_cast<const float *>(base + gl.z_off);
                sp.out = out;
                sp.U = P.rec_tc(g) ? reinterpret_cast<uint16_t *>(base + gl.u_off) : nullptr;
                sp.U_lo = P.rec_tc(g) && P.split ? reinterpret_cast<uint16_t *>(base + gl.u_lo_off) : nullptr;
                sp.H = H; sp.W = W; sp.Ho = gl.Ho; sp.Wo = gl.Wo;
                sp.begin = sep_begin;
                sep_begin += sep_job_items(P.sep_mode(g), g.h, g.w, gl.Ho, gl.Wo, P.sep_k(g), &sp.tiles_x, &sp.tiles_y);
            }
            if (P.rec_tc(g)) {
                // recombination S_k = sum_r Lambda[k][r] U_r: a 1x1 tap over the Ho x Wo grid with Upad input terms
                TcJob &t = reinterpret_cast<TcJob *>(hb + P.g_rec_off[gi])[i];
                const long long cells = (long long)gl.Ho * gl.Wo;
                if (!encode_level_tmap(&t.tmap, reinterpret_cast<const uint16_t *>(base + gl.u_off), cells, g.Upad / 8))
                    return fail(TDPM_ERR_CUDA, "cuTensorMapEncodeTiled failed");
                if (P.split && !encode_level_tmap(&t.tmap_lo, reinterpret_cast<const uint16_t *>(base + gl.u_lo_off),
                                                  cells, g.Upad / 8))
                    return fail(TDPM_ERR_CUDA, "cuTensorMapEncodeTiled failed");
                t.out = out;
                t.H = gl.Ho; t.W = gl.Wo; t.Ho = gl.Ho; t.Wo = gl.Wo;
                t.begin = rec_begin;
                rec_begin += (int)((cells + corr_tc_tile_m() - 1) / corr_tc_tile_m());
            }
        }
    }
    DtJob *dj = reinterpret_cast<DtJob *>(hb + P.dt_off);
    int xw = 0;
    for (size_t i = 0; i < P.dts.size(); ++i) {
        const DtPlan &p = P.dts[i];
        DtJob &d = dj[i];
        d.S = reinterpret_cast<const float *>(base + p.s_off);
        d.H = p.Hs; d.W = p.Ws;
        d.lx = p.d[0]; d.qx = p.d[1]; d.ly = p.d[2]; d.qy = p.d[3];
        d.x_off = p.vx; d.x_step = 2; d.nx = p.X;
        d.y_off = p.vy; d.y_step = 2; d.ny = p.Y;
        d.V = nullptr;
        d.IV = nullptr;
        d.D = reinterpret_cast<float *>(base + p.d_off);
        d.A = reinterpret_cast<int32_t *>(base + p.a_off);
        d.xbegin = xw;  // first CTA (strip of sampled columns) of the job in the fused launch
        d.ybegin = 0;
        const int strips = dt_job_strips(p.X);
        int *cj = reinterpret_cast<int *>(hb + P.dt_cta_off) + xw;
        for (int t = 0; t < strips; ++t) cj[t] = (int)i;
        xw += strips;
    }
    AsmJob *aj = reinterpret_cast<AsmJob *>(hb + P.asm_off);
    long long pos = 0;
    for (size_t i = 0; i < P.asms.size(); ++i) {
        const AsmPlan &p = P.asms[i];
        AsmJob &a = aj[i];
        a.root = reinterpret_cast<const float *>(base + p.root_off);
        a.root_W = p.root_W;
        a.Y = p.Y; a.X = p.X; a.bias = p.bias; a.n_parts = (int)p.dt.size();
        a.image = p.image; a.comp = p.c; a.level = p.j - P.img_base[p.image];
        a.out = reinterpret_cast<float *>(base + p.out_off);
        for (size_t k = 0; k < p.dt.size(); ++k) {
            a.D[k] = reinterpret_cast<const float *>(base + P.dts[p.dt[k]].d_off);
            a.A[k] = reinterpret_cast<const int32_t *>(base + P.dts[p.dt[k]].a_off);
        }
        a.begin = pos;
        pos += (long long)p.Y * p.X;
    }
    const_cast<Plan &>(P).patches = patches;
    A.levels.assign(lv.size(), nullptr);
    for (size_t j = 0; j < lv.size(); ++j) A.levels[j] = lv[j]->data;
    return TDPM_OK;
}

// The plan's features in the tensor-core operand format (BF16 planar, with lo parts for split operands, or E4M3).
cudaError_t launch_convert(const Plan &P, char *dblob, cudaStream_t s)
{
    const ConvJob *cj = reinterpret_cast<const ConvJob *>(dblob + P.conv_off);
    return P.fp8 ? launch_to_fp8_planar(cj, P.L, P.conv_items, kFp8FeatureScale, s)
                 : launch_to_bf16_planar(cj, P.L, P.conv_items, s);
}

// A shape group's tensor-core contraction over its m_tiles M tiles: the full correlation, or the channel stage of the
// decomposed form, with the bank of the plan's operand format (FP8 results rescaled by the two per-tensor scales).
// code: N tile width | kTcPersistent for the persistent form.
cudaError_t launch_group_tc(const Plan &P, size_t gi, const Group &g, const TcJob *jobs, int nj, int m_tiles, int code,
                            int *err, cudaStream_t s)
{
    const int nt = code & 0xffff;
    const bool pers = (code & kTcPersistent) != 0;
    if (P.gdec(gi)) {
        if (P.fp8)
            return launch_corr_tc(jobs, nj, m_tiles, g.d_C_fp8, nullptr, g.R, g.Rpad_tc, nt, 1, 1, 1, err, s, true,
                                  1.f / (g.C_fp8_scale * kFp8FeatureScale), pers);
        return launch_corr_tc(jobs, nj, m_tiles, g.d_C_tc, P.split ? g.d_C_tc_lo : nullptr, g.R, g.Rpad_tc, nt, 1, 1,
                              1, err, s, false, 1.f, pers);
    }
    if (P.fp8)
        return launch_corr_tc(jobs, nj, m_tiles, g.d_filt_fp8, nullptr, g.K, g.Npad_tc, nt, g.h, g.w, 1, err, s, true,
                              1.f / (g.fp8_scale * kFp8FeatureScale), pers);
    return launch_corr_tc(jobs, nj, m_tiles, g.d_filt_tc, P.split ? g.d_filt_tc_lo : nullptr, g.K, g.Npad_tc, nt, g.h,
                          g.w, 1, err, s, false, 1.f, pers);
}

// The joint recombination S = Lambda U of a group (code as for launch_group_tc).
cudaError_t launch_group_recomb(const Plan &P, const Group &g, const TcJob *jobs, int nj, int m_tiles, int code,
                                int *err, cudaStream_t s)
{
    return launch_corr_tc(jobs, nj, m_tiles, g.d_lam_tc, P.split ? g.d_lam_tc_lo : nullptr, g.K, g.Npad_lam,
                          code & 0xffff, 1, 1, g.Upad / FD, err, s, false, 1.f, (code & kTcPersistent) != 0);
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

// Every stage of the plan on stream s.
// Every stage of the plan on stream s (the job tables must already be on the device).
cudaError_t enqueue(tdpm_ctx *ctx, const Plan &P, const Model &m, const Arena &A, cudaStream_t s)
{
    char *dblob = A.dev + P.blob_off;
    cudaError_t e = cudaSuccess;
    if (P.bf) {
        Prof pr(ctx, s, P.fp8 ? "to_fp8" : "to_bf16");
        e = launch_convert(P, dblob, s);
        if (e != cudaSuccess) return e;
        pr.end();
    }
    // step 1 for one shape group, on stream gs
    auto run_group = [&](size_t gi, cudaStream_t gs) -> cudaError_t {
        const Group &g = m.groups[gi];
        const int nj = (int)P.glv[gi].size();
        cudaError_t e = cudaSuccess;
        const char *jobs = dblob + P.g_jobs_off[gi];
        if (P.g_fused[gi] == 2) {
            Prof pr(ctx, gs, "zsep_tc");
            e = launch_zsept_tc(reinterpret_cast<const ZsJob *>(jobs),
                                reinterpret_cast<const ZsTile *>(dblob + P.g_tile_off[gi]), P.g_tiles[gi],
                                P.g_n_fg[gi], dblob + P.g_frec_off[gi],
                                reinterpret_cast<const int *>(dblob + P.g_fg_off[gi]), g.d_C_tc,
                                P.split ? g.d_C_tc_lo : nullptr, g.Rpad_tc, g.h, g.w, ctx->d_err, gs);
            if (e != cudaSuccess) return e;
            pr.end();
            return cudaSuccess;
        }
        if (P.g_fused[gi]) {
            Prof pr(ctx, gs, "zsep_tc");
            e = launch_zsep_tc(reinterpret_cast<const ZsJob *>(jobs),
                               reinterpret_cast<const ZsTile *>(dblob + P.g_tile_off[gi]), P.g_tiles[gi],
                               reinterpret_cast<const ZsGroup *>(dblob + P.g_fg_off[gi]), P.g_n_fg[gi], g.d_C_tc,
                               P.split ? g.d_C_tc_lo : nullptr, g.Rpad_tc, dblob + P.g_frec_off[gi], P.g_nmax[gi], g.h,
                               g.w, ctx->d_err, gs, P.g_nt[gi]);
            if (e != cudaSuccess) return e;
            pr.end();
            return cudaSuccess;
        }
        if (P.bf) {
            Prof pr(ctx, gs, P.gdec(gi) ? "zproj_tc" : "corr_tc");
            e = launch_group_tc(P, gi, g, reinterpret_cast<const TcJob *>(jobs), nj, P.g_tiles[gi], P.g_nt[gi], ctx->d_err,
                                gs);
            if (e != cudaSuccess) return e;
            pr.end();
        } else if (P.gdec(gi)) {
            Prof pr(ctx, gs, "zproj_f32");
            e = launch_zproj_simt(reinterpret_cast<const ZJob *>(jobs), nj, P.g_tiles[gi], g.d_Ct, g.R, gs);
            if (e != cudaSuccess) return e;
            pr.end();
        } else {
            Prof pr(ctx, gs, "corr_f32");
            e = launch_corr_f32(reinterpret_cast<const CorrJob *>(jobs), nj, P.g_tiles[gi], g.d_filt_t, g.K, g.Kpad,
                                g.h, g.w, gs);
            if (e != cudaSuccess) return e;
            pr.end();
        }
        if (P.gdec(gi)) {
            Prof pr(ctx, gs, "sep");
            e = launch_sep(reinterpret_cast<const SepJob *>(dblob + P.g_sep_off[gi]), nj, P.g_sep_tiles[gi], g.d_A,
                           g.d_B, g.d_lam, g.d_rank_off, P.sep_k(g), g.R, g.h, g.w, P.sep_mode(g), gs);
            if (e != cudaSuccess) return e;
            pr.end();
        }
        if (P.rec_tc(g)) {
            Prof pr(ctx, gs, "recomb_tc");
            e = launch_group_recomb(P, g, reinterpret_cast<const TcJob *>(dblob + P.g_rec_off[gi]), nj,
                                    P.g_rec_tiles[gi], P.g_rec_nt[gi], ctx->d_err, gs);
            if (e != cudaSuccess) return e;
            pr.end();
        }
        return cudaSuccess;
    };
    std::vector<size_t> busy;
    for (size_t gi = 0; gi < m.groups.size(); ++gi)
        if (!P.glv[gi].empty()) busy.push_back(gi);
    if (ctx->prof || busy.size() < 2 || ctx->side.empty()) {
        // serial on the caller's stream (always when profiling, so that every stage is timed on its own)
        for (size_t gi : busy)
            if ((e = run_group(gi, s)) != cudaSuccess) return e;
    } else {
        // fork: every side stream waits for the work already on s; the group with the most jobs stays on s
        if ((e = cudaEventRecord(ctx->fork_ev, s)) != cudaSuccess) return e;
        const size_t ns = std::min(ctx->side.size(), busy.size() - 1);
        for (size_t i = 0; i < ns; ++i)
            if ((e = cudaStreamWaitEvent(ctx->side[i], ctx->fork_ev, 0)) != cudaSuccess) return e;
        size_t big = 0;
        for (size_t i = 1; i < busy.size(); ++i)
            if (P.g_tiles[busy[i]] > P.g_tiles[busy[big]]) big = i;
        size_t next = 0;
        for (size_t i = 0; i < busy.size(); ++i) {
            cudaStream_t gs = i == big ? s : ctx->side[(next++) % ns];
            if ((e = run_group(busy[i], gs)) != cudaSuccess) return e;
        }
        // join
        for (size_t i = 0; i < ns; ++i) {
            if ((e = cudaEventRecord(ctx->join_ev[i], ctx->side[i])) != cudaSuccess) return e;
            if ((e = cudaStreamWaitEvent(s, ctx->join_ev[i], 0)) != cudaSuccess) return e;
        }
    }
    {
        Prof pr(ctx, s, "dt");
        e = launch_dt_fused(reinterpret_cast<const DtJob *>(dblob + P.dt_off), (int)P.dts.size(),
                            reinterpret_cast<const int *>(dblob + P.dt_cta_off), P.dt_ctas, P.max_W, P.max_H, s);
        if (e != cudaSuccess) return e;
        pr.end();
    }
    {
        Prof pr(ctx, s, "assemble");
        e = launch_assemble(reinterpret_cast<const AsmJob *>(dblob + P.asm_off), (int)P.asms.size(), P.total, s);
        if (e != cudaSuccess) return e;
        pr.end();
    }
    return cudaSuccess;
}

// Autotuner for the tensor-core launches (N tile width). A new plan's candidates are timed on its own inputs, on the
// caller's stream, before its first real enqueue (whose launches then overwrite every output). The choice is cached in
// the context per shape class: (launch kind, N, K blocks, split operands, M tiles rounded up to a power of two), so
// later plans of the same class (other images, a server's batches) reuse it without timing.
std::string tune_key(const char *kind, int N, int kblocks, const char *operands, int m_tiles)
{
    int b = 1;
    while (b < m_tiles) b <<= 1;
    return std::string(kind) + ":" + std::to_string(N) + ":" + std::to_string(kblocks) + ":" + operands + ":" +
           std::to_string(b);
}

cudaError_t autotune_plan(tdpm_ctx *ctx, Plan &P, const Model &m, Arena &A, cudaStream_t s)
{
    P.tuned = true;
    if (!P.bf) return cudaSuccess;
    char *dblob = A.dev + P.blob_off;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaError_t e = cudaEventCreate(&ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&ev1);
    bool staged = false;
    // time one candidate: a warm-up launch, then three timed ones
    auto time_ms = [&](const std::function<cudaError_t()> &launch, float *ms) -> cudaError_t {
        cudaError_t r = launch();
        if (r == cudaSuccess) r = cudaEventRecord(ev0, s);
        for (int i = 0; i < 3 && r == cudaSuccess; ++i) r = launch();
        if (r == cudaSuccess) r = cudaEventRecord(ev1, s);
        if (r == cudaSuccess) r = cudaEventSynchronize(ev1);
        if (r == cudaSuccess) r = cudaEventElapsedTime(ms, ev0, ev1);
        return r;
    };
    // time every candidate configuration code (or, with none given, every balanced N tile width in the tile and the
    // persistent form) and keep the fastest
    auto choose = [&](const std::string &key, int N, const std::function<cudaError_t(int)> &launch_nt,
                      int *chosen, std::vector<int> codes = {}) -> cudaError_t {
        auto it = ctx->tune_cache.find(key);
        if (it != ctx->tune_cache.end()) {
            *chosen = it->second;
            return cudaSuccess;
        }
        if (!staged) {
            staged = true;
            cudaError_t r = cudaSuccess;
            if (!A.blob_on_device) r = cudaMemcpyAsync(dblob, A.host, P.blob_bytes, cudaMemcpyHostToDevice, s);
            if (r == cudaSuccess) A.blob_on_device = true;
            if (r == cudaSuccess) r = launch_convert(P, dblob, s);
            if (r != cudaSuccess) return r;
        }
        if (codes.empty()) {
            int cand[4];
            const int nc = corr_tc_nt_candidates(N, cand);
            for (int i = 0; i < nc; ++i)
                for (int pers = 0; pers < 2; ++pers) codes.push_back(cand[i] | (pers ? kTcPersistent : 0));
        }
        float best = 0.f;
        bool first = true;
        for (int code : codes) {
            float ms = 0.f;
            const cudaError_t r = time_ms([&] { return launch_nt(code); }, &ms);
            if (r != cudaSuccess) return r;
            if (first || ms < best) {
                best = ms;
                *chosen = code;
                first = false;
            }
        }
        ctx->tune_cache[key] = *chosen;
        return cudaSuccess;
    };
    for (size_t gi = 0; gi < m.groups.size() && e == cudaSuccess; ++gi) {
        const Group &g = m.groups[gi];
        const int nj = (int)P.glv[gi].size();
        if (!nj) continue;
        if (P.g_fused[gi] == 2) continue;  // one form
        if (P.g_fused[gi] && P.zsep_forced) continue;
        if (P.g_fused[gi]) {
            // the fused kernel: its forms (one CTA per item, or persistent with one or two feature stages / Z buffers)
            std::vector<int> forms;
            for (int f : {ZSEP_TILE, ZSEP_PERSIST_S2, ZSEP_PERSIST_Z2, ZSEP_PERSIST_S2Z2, ZSEP_PERSIST_S1})
                if (zsep_form_fits(g.h, g.w, P.split, P.g_nmax[gi], f)) forms.push_back(f);
            const std::string key = tune_key("zsep", g.h * 16 + g.w, P.g_nmax[gi], P.split ? "x3" : "x1",
                                             P.g_tiles[gi] * P.g_n_fg[gi]);
            e = choose(key, 0, [&](int form) {
                return launch_zsep_tc(reinterpret_cast<const ZsJob *>(dblob + P.g_jobs_off[gi]),
                                      reinterpret_cast<const ZsTile *>(dblob + P.g_tile_off[gi]), P.g_tiles[gi],
                                      reinterpret_cast<const ZsGroup *>(dblob + P.g_fg_off[gi]), P.g_n_fg[gi],
                                      g.d_C_tc, P.split ? g.d_C_tc_lo : nullptr, g.Rpad_tc, dblob + P.g_frec_off[gi],
                                      P.g_nmax[gi], g.h, g.w, ctx->d_err, s, form);
            }, &P.g_nt[gi], forms);
            continue;
        }
        const TcJob *jobs = reinterpret_cast<const TcJob *>(dblob + P.g_jobs_off[gi]);
        const char *op = P.fp8 ? "f8" : P.split ? "x3" : "x1";
        if (P.gdec(gi))
            e = choose(tune_key("zproj", g.R, 1, op, P.g_tiles[gi]), g.R,
                       [&](int nt) { return launch_group_tc(P, gi, g, jobs, nj, P.g_tiles[gi], nt, ctx->d_err, s); },
                       &P.g_nt[gi]);
        else
            e = choose(tune_key("corr", g.K, g.h * g.w, op, P.g_tiles[gi]), g.K,
                       [&](int nt) { return launch_group_tc(P, gi, g, jobs, nj, P.g_tiles[gi], nt, ctx->d_err, s); },
                       &P.g_nt[gi]);
        if (e == cudaSuccess && P.rec_tc(g)) {
            const TcJob *rj = reinterpret_cast<const TcJob *>(dblob + P.g_rec_off[gi]);
            e = choose(tune_key("recomb", g.K, g.Upad / FD, P.split ? "x3" : "x1", P.g_rec_tiles[gi]), g.K,
                       [&](int code) { return launch_group_recomb(P, g, rj, nj, P.g_rec_tiles[gi], code, ctx->d_err, s); },
                       &P.g_rec_nt[gi]);
        }
    }
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    return e;
}

// Arena sizes are rounded up to one of four sizes per octave, so that plans of similar size (a server's batches of
// different images) reuse each other's arenas instead of allocating: cudaMalloc and cudaFree can stall the device.
size_t arena_bucket(size_t bytes)
{
    if (bytes <= (1u << 20)) return 1u << 20;
    int e = 0;
    while ((bytes >> e) > 7) ++e;          // bytes >> e in [4, 7]
    const size_t unit = (size_t)1 << e;    // a quarter of the octave's base size
    return (bytes + unit - 1) / unit * unit;
}

tdpm_status arena_get(tdpm_ctx *ctx, const Plan &P, Arena &out)
{
    const size_t bytes = P.arena_bytes, host_bytes = P.blob_bytes;
    for (size_t i = 0; i < ctx->free_arenas.size(); ++i)
        if (ctx->free_arenas[i].plan_uid == P.uid) {
            out = ctx->free_arenas[i];
            ctx->free_arenas.erase(ctx->free_arenas.begin() + i);
            return TDPM_OK;
        }
    for (size_t i = 0; i < ctx->free_arenas.size(); ++i) {
        Arena &a = ctx->free_arenas[i];
        if (a.bytes >= bytes && a.bytes <= arena_bucket(bytes) + arena_bucket(bytes) / 4 && a.host_bytes >= host_bytes) {
            out = a;
            ctx->free_arenas.erase(ctx->free_arenas.begin() + i);
            out.plan_uid = 0;
            if (out.graph) {
                cudaGraphExecDestroy(out.graph);
                out.graph = nullptr;
            }
            out.uses = 0;
            return TDPM_OK;
        }
    }
    size_t alloc = arena_bucket(bytes);
    if (ctx->budget && alloc > ctx->budget) alloc = bytes;
    while (ctx->budget && ctx->used + alloc > ctx->budget && !ctx->free_arenas.empty()) {
        arena_free(ctx, ctx->free_arenas.back());
        ctx->free_arenas.pop_back();
    }
    if (ctx->budget && ctx->used + alloc > ctx->budget)
        return fail(TDPM_ERR_OOM, "scores need " + std::to_string(alloc) + " bytes; budget " +
                                      std::to_string(ctx->budget) + ", in use " + std::to_string(ctx->used));
    Arena a;
    cudaError_t e = cudaMalloc(&a.dev, alloc);
    while (e == cudaErrorMemoryAllocation && !ctx->free_arenas.empty()) {
        // device memory exhausted: give back the cached arenas, oldest first, and try again
        cudaGetLastError();
        arena_free(ctx, ctx->free_arenas.front());
        ctx->free_arenas.erase(ctx->free_arenas.begin());
        e = cudaMalloc(&a.dev, alloc);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(TDPM_ERR_OOM, std::string("cudaMalloc arena: ") + cudaGetErrorString(e));
    }
    const size_t host_alloc = arena_bucket(host_bytes);
    e = cudaMallocHost(&a.host, host_alloc);
    if (e != cudaSuccess) {
        cudaFree(a.dev);
        return fail(TDPM_ERR_OOM, std::string("cudaMallocHost staging: ") + cudaGetErrorString(e));
    }
    a.bytes = alloc;
    a.host_bytes = host_alloc;
    ctx->used += alloc;
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

Scores *get_scores(tdpm_ctx *ctx, int id)
{
    auto it = ctx->scores.find(id);
    return it == ctx->scores.end() ? nullptr : it->second.get();
}

// Read and clear the device error flag (bounded waits that expired); call after the stream has been synchronised.
tdpm_status check_device_flag(tdpm_ctx *ctx)
{
    int v = 0;
    CUDA_TRY(cudaMemcpy(&v, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (v) {
        cudaMemset(ctx->d_err, 0, sizeof(int));
        return fail(TDPM_ERR_TIMEOUT, "a bounded device wait expired; results of the last scoring are invalid");
    }
    return TDPM_OK;
}

}  // namespace

void arena_free(tdpm_ctx *ctx, Arena &a)
{
    if (a.graph) cudaGraphExecDestroy(a.graph);
    if (a.dev) cudaFree(a.dev);
    if (a.host) cudaFreeHost(a.host);
    ctx->used -= std::min(ctx->used, a.bytes);
    a = Arena{};
}

void free_scores(tdpm_ctx *ctx, Scores &s)
{
    if (s.done) {
        cudaEventSynchronize(s.done);
        cudaEventDestroy(s.done);
        s.done = nullptr;
    }
    arena_put(ctx, s.arena);
}

void drop_plans_of_model(tdpm_ctx *ctx, int model_id)
{
    for (auto it = ctx->plans.begin(); it != ctx->plans.end();) {
        if (it->second->model_id == model_id) {
            for (Arena &a : ctx->free_arenas)
                if (a.plan_uid == it->second->uid) {
                    a.plan_uid = 0;
                    if (a.graph) cudaGraphExecDestroy(a.graph);
                    a.graph = nullptr;
                }
            it = ctx->plans.erase(it);
        } else {
            ++it;
        }
    }
}

// Device bytes of the arena a batch needs, as allocated (its plan is made, or found, and cached). Used by the server's
// admission and by tdpm_scores_bytes.
tdpm_status batch_arena_bytes(tdpm_ctx *ctx, int32_t model_id, const tdpm_pyramid *pyrs, int32_t n_images,
                              const uint8_t *mask, int32_t form, int32_t precision, size_t *bytes)
{
    std::lock_guard<std::mutex> lk(ctx->mu);
    Model *m = get_model(ctx, model_id);
    if (!m) return fail(TDPM_ERR_STATE, "unknown model id");
    if (form == TDPM_FORM_DECOMPOSED && !m->decomposed)
        return fail(TDPM_ERR_STATE, "decomposed form requested before tdpm_decompose");
    const std::string key = plan_key(model_id, *m, form, precision, pyrs, n_images, mask, ctx->fuse, ctx->zsep_form);
    auto pit = ctx->plans.find(key);
    if (pit == ctx->plans.end()) {
        auto plan = make_plan(*m, model_id, pyrs, n_images, form, precision, mask, ctx->fuse, ctx->zsep_form);
        if (ctx->plans.size() > 256) ctx->plans.clear();
        pit = ctx->plans.emplace(key, plan).first;
    }
    *bytes = arena_bucket(pit->second->arena_bytes);  // what arena_get allocates for it
    return TDPM_OK;
}

// Step 4 for tdpm_detect (one threshold) and tdpm_detect_thresholds (tau_table: host [images][components]).
tdpm_status detect_impl(tdpm_ctx *ctx, int32_t scores_id, float tau, const float *tau_table, tdpm_detection *out,
                        size_t capacity, size_t *n_out, void *stream)
{
    if (!ctx || !n_out || (capacity > 0 && !out)) return fail(TDPM_ERR_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(ctx->mu);
    tdpm_status st = set_device(ctx);
    if (st) return st;
    Scores *sc = get_scores(ctx, scores_id);
    if (!sc) return fail(TDPM_ERR_STATE, "unknown scores id");
    const Plan &P = *sc->plan;
    cudaStream_t s = (cudaStream_t)stream;
    char *base = sc->arena.dev;
    const AsmJob *jobs = reinterpret_cast<const AsmJob *>(base + P.blob_off + P.asm_off);
    int *counts = reinterpret_cast<int *>(base + P.counts_off), *offsets = reinterpret_cast<int *>(base + P.offsets_off);
    long long *d_total = reinterpret_cast<long long *>(base + P.total_off);
    CUDA_TRY(cudaStreamWaitEvent(s, sc->done, 0));
    const float *d_job_tau = nullptr;
    if (tau_table) {
        // one threshold per assembly job, from the (image, component) table
        const Model *m = get_model(ctx, sc->model_id);
        if (!m) return fail(TDPM_ERR_STATE, "the scores' model was unloaded");
        const size_t nc = m->comps.size();
        std::vector<float> jt(std::max<size_t>(1, P.asms.size()));
        for (size_t k = 0; k < P.asms.size(); ++k) {
            jt[k] = tau_table[(size_t)P.asms[k].image * nc + P.asms[k].c];
            if (std::isnan(jt[k])) return fail(TDPM_ERR_ARG, "a threshold is NaN");
        }
        if (jt.size() > ctx->tau_cap) {
            if (ctx->d_job_tau) cudaFree(ctx->d_job_tau);
            ctx->d_job_tau = nullptr;
            ctx->tau_cap = 0;
            CUDA_TRY(cudaMalloc(&ctx->d_job_tau, sizeof(float) * jt.size() * 2));
            ctx->tau_cap = jt.size() * 2;
        }
        CUDA_TRY(cudaMemcpyAsync(ctx->d_job_tau, jt.data(), sizeof(float) * jt.size(), cudaMemcpyHostToDevice, s));
        d_job_tau = ctx->d_job_tau;
    }
    // count, scan and the ordered write of up to `want` records in one go, then ONE read-back: the count, the device
    // error flag and a prefix of the records as long as this plan's last count; a second copy only when more were
    // found (and a second write only when the device buffer was too short)
    Prof pr(ctx, s, "detect");
    CUDA_TRY(launch_detect_count(jobs, (int)P.asms.size(), P.total, tau, d_job_tau, counts, offsets, P.n_det_blocks,
                                 d_total, s));
    const size_t limit = std::min<size_t>((size_t)std::max<long long>(P.total, 0), capacity);
    auto grow = [&](size_t need) -> tdpm_status {
        if (need <= ctx->rec_cap) return TDPM_OK;
        const size_t cap = std::max(need, ctx->rec_cap * 2);
        if (ctx->d_records) {
            cudaStreamSynchronize(s);
            cudaFree(ctx->d_records);
            ctx->used -= std::min(ctx->used, ctx->rec_cap * sizeof(tdpm_detection));
            ctx->d_records = nullptr;
            ctx->rec_cap = 0;
        }
        if (ctx->budget && ctx->used + cap * sizeof(tdpm_detection) > ctx->budget)
            return fail(TDPM_ERR_OOM, "detection buffer exceeds the memory budget");
        CUDA_TRY(cudaMalloc(&ctx->d_records, cap * sizeof(tdpm_detection)));
        ctx->rec_cap = cap;
        ctx->used += cap * sizeof(tdpm_detection);
        return TDPM_OK;
    };
    auto hint = ctx->det_last.find(P.uid);
    const size_t last = hint == ctx->det_last.end() ? 4096 : hint->second;
    const size_t want = std::min(limit, std::max(ctx->rec_cap, last + last / 8 + 64));
    if ((st = grow(want))) return st;
    if (want)
        CUDA_TRY(launch_detect_write(jobs, (int)P.asms.size(), P.total, tau, d_job_tau, offsets, P.n_det_blocks,
                                     ctx->d_records, (long long)want, sc->model_id, s));
    CUDA_TRY(cudaMemcpyAsync(ctx->h_total, d_total, sizeof(long long), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(ctx->h_err, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    const size_t first = hint == ctx->det_last.end() ? 0 : std::min(want, last);
    if (first) CUDA_TRY(cudaMemcpyAsync(out, ctx->d_records, first * sizeof(tdpm_detection), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (*ctx->h_err) {
        cudaMemset(ctx->d_err, 0, sizeof(int));
        *ctx->h_err = 0;
        return fail(TDPM_ERR_TIMEOUT, "a bounded device wait expired; results of the last scoring are invalid");
    }
    const long long total = *ctx->h_total;
    const size_t n = std::min<size_t>((size_t)total, capacity);
    if (n > want) {
        // the device buffer was too short: write again into a larger one
        if ((st = grow(n))) return st;
        CUDA_TRY(launch_detect_write(jobs, (int)P.asms.size(), P.total, tau, d_job_tau, offsets, P.n_det_blocks,
                                     ctx->d_records, (long long)n, sc->model_id, s));
        CUDA_TRY(cudaMemcpyAsync(out, ctx->d_records, n * sizeof(tdpm_detection), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
    } else if (n > first) {
        CUDA_TRY(cudaMemcpyAsync(out + first, ctx->d_records + first, (n - first) * sizeof(tdpm_detection),
                                 cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
    }
    if (ctx->det_last.size() > 4096) ctx->det_last.clear();  // hints of plans long gone
    ctx->det_last[P.uid] = n;
    pr.end();
    CUDA_TRY(cudaEventRecord(sc->done, s));
    *n_out = (size_t)total;
    if ((size_t)total > capacity)
        return fail(TDPM_ERR_CAPACITY, "detections exceed capacity: " + std::to_string(total));
    return TDPM_OK;
}

}  // namespace tdpm

using namespace tdpm;

extern "C" {

tdpm_status tdpm_build_batch_scores(tdpm_ctx *ctx, int32_t model_id, const tdpm_pyramid *pyrs, int32_t n_images,
                                    int32_t form, int32_t precision, void *stream, int32_t *scores_id)
{
    return tdpm_build_batch_scores_subset(ctx, model_id, pyrs, n_images, nullptr, form, precision, stream, scores_id);
}

tdpm_status tdpm_build_batch_scores_subset(tdpm_ctx *ctx, int32_t model_id, const tdpm_pyramid *pyrs,
                                           int32_t n_images, const uint8_t *component_mask, int32_t form,
                                           int32_t precision, void *stream, int32_t *scores_id)
{
    const uint8_t *mask = component_mask;
    clear_error();
    if (!ctx || !pyrs || !scores_id) return fail(TDPM_ERR_ARG, "NULL argument");
    if (n_images < 1 || n_images > 4096) return fail(TDPM_ERR_ARG, "n_images must be in [1, 4096]");
    if (form != TDPM_FORM_FULL && form != TDPM_FORM_DECOMPOSED) return fail(TDPM_ERR_ARG, "bad form");
    if (!valid_precision(precision)) return fail(TDPM_ERR_ARG, "unsupported precision");
    std::vector<const tdpm_level *> lv;
    for (int i = 0; i < n_images; ++i) {
        const tdpm_pyramid &py = pyrs[i];
        if (py.n_levels <= 0 || !py.levels) return fail(TDPM_ERR_ARG, "empty pyramid");
        if (py.n_levels > 4096) return fail(TDPM_ERR_ARG, "too many levels");
        if (py.lambda < 1 || py.lambda > py.n_levels) return fail(TDPM_ERR_ARG, "lambda out of range");
        for (int j = 0; j < py.n_levels; ++j) {
            const tdpm_level &l = py.levels[j];
            if (l.H <= 0 || l.W <= 0 || !l.data) return fail(TDPM_ERR_ARG, "level with non-positive size or NULL data");
            if (l.H > 4096 || l.W > 4096) return fail(TDPM_ERR_ARG, "level side above 4096 cells");
            if (reinterpret_cast<uintptr_t>(l.data) % 16) return fail(TDPM_ERR_ARG, "level data not 16-byte aligned");
            lv.push_back(&l);
        }
    }
    std::lock_guard<std::mutex> lk(ctx->mu);
    tdpm_status st = set_device(ctx);
    if (st) return st;
    Model *m = get_model(ctx, model_id);
    if (!m) return fail(TDPM_ERR_STATE, "unknown model id");
    if (form == TDPM_FORM_DECOMPOSED && !m->decomposed)
        return fail(TDPM_ERR_STATE, "decomposed form requested before tdpm_decompose");
    cudaStream_t s = (cudaStream_t)stream;
    const std::string key = plan_key(model_id, *m, form, precision, pyrs, n_images, mask, ctx->fuse, ctx->zsep_form);
    std::shared_ptr<Plan> plan;
    auto pit = ctx->plans.find(key);
    if (pit != ctx->plans.end()) {
        plan = pit->second;
    } else {
        plan = make_plan(*m, model_id, pyrs, n_images, form, precision, mask, ctx->fuse, ctx->zsep_form);
        if (plan->max_W > kDtMaxSide || plan->max_H > kDtMaxSide)
            return fail(TDPM_ERR_ARG, "part score maps wider or taller than " + std::to_string(kDtMaxSide) +
                                          " cells are not supported");
        if (ctx->plans.size() > 256) ctx->plans.clear();
        ctx->plans[key] = plan;
    }
    auto sc = std::make_unique<Scores>();
    sc->model_id = model_id;
    sc->plan = plan;
    if ((st = arena_get(ctx, *plan, sc->arena))) return st;
    Arena &A = sc->arena;
    if (A.plan_uid != plan->uid) {
        if (A.graph) {
            cudaGraphExecDestroy(A.graph);
            A.graph = nullptr;
        }
        A.uses = 0;
        if ((st = fill_blob(*plan, *m, lv, A))) {
            arena_put(ctx, A);
            return st;
        }
        A.plan_uid = plan->uid;
        A.blob_on_device = false;
    } else {
        bool same = A.levels.size() == lv.size();
        for (size_t j = 0; same && j < lv.size(); ++j) same = A.levels[j] == lv[j]->data;
        if (!same) {
            for (const auto &pt : plan->patches)
                *reinterpret_cast<const float **>(A.host + pt.first) = lv[pt.second]->data;
            A.levels.assign(lv.size(), nullptr);
            for (size_t j = 0; j < lv.size(); ++j) A.levels[j] = lv[j]->data;
            A.blob_on_device = false;
        }
    }
    cudaError_t e = cudaSuccess;
    if (!plan->tuned) {
        if (ctx->autotune) e = autotune_plan(ctx, *plan, *m, A, s);
        else plan->tuned = true;
        if (e != cudaSuccess) {
            cudaStreamSynchronize(s);
            arena_put(ctx, A);
            return fail(TDPM_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
        }
    }
    // the job tables go to the device only when the host blob changed (new plan or new level pointers); a reused
    // arena keeps them, so repeated batches of the same shapes copy nothing but their own inputs
    if (!A.blob_on_device) {
        e = cudaMemcpyAsync(A.dev + plan->blob_off, A.host, plan->blob_bytes, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) {
            cudaStreamSynchronize(s);
            arena_put(ctx, A);
            return fail(TDPM_ERR_CUDA, std::string("job tables: ") + cudaGetErrorString(e));
        }
        A.blob_on_device = true;
    }
    const bool graphs = ctx->use_graphs && !ctx->prof;
    if (graphs && !A.graph && A.uses >= 1) {
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            int captured = 0;
            t_capture_launches = &captured;
            const cudaError_t eq = enqueue(ctx, *plan, *m, A, ctx->cap_stream);
            t_capture_launches = nullptr;
            A.graph_kernels = captured;
            e = cudaStreamEndCapture(ctx->cap_stream, &g);
            if (eq != cudaSuccess) e = eq;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&A.graph, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            cudaGetLastError();
            A.graph = nullptr;
            e = cudaSuccess;  // fall back to direct launches below
        }
    }
    if (graphs && A.graph) {
        e = cudaGraphLaunch(A.graph, s);
        if (e == cudaSuccess) note_launches(A.graph_kernels);
    } else {
        e = enqueue(ctx, *plan, *m, A, s);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sc->done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(sc->done, s);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(s);
        if (sc->done) cudaEventDestroy(sc->done);
        A.plan_uid = 0;
        arena_put(ctx, A);
        return fail(TDPM_ERR_CUDA, std::string("enqueue: ") + cudaGetErrorString(e));
    }
    A.uses++;
    const int id = ctx->next_id++;
    ctx->scores[id] = std::move(sc);
    *scores_id = id;
    return TDPM_OK;
}

tdpm_status tdpm_scores_bytes(tdpm_ctx *ctx, int32_t model_id, const tdpm_pyramid *pyrs, int32_t n_images,
                              int32_t form, int32_t precision, size_t *bytes)
{
    clear_error();
    if (!ctx || !pyrs || !bytes) return fail(TDPM_ERR_ARG, "NULL argument");
    if (n_images < 1 || n_images > 4096) return fail(TDPM_ERR_ARG, "n_images must be in [1, 4096]");
    if (form != TDPM_FORM_FULL && form != TDPM_FORM_DECOMPOSED) return fail(TDPM_ERR_ARG, "bad form");
    if (!valid_precision(precision)) return fail(TDPM_ERR_ARG, "unsupported precision");
    for (int i = 0; i < n_images; ++i) {
        const tdpm_pyramid &py = pyrs[i];
        if (py.n_levels <= 0 || py.n_levels > 4096 || !py.levels) return fail(TDPM_ERR_ARG, "empty pyramid");
        if (py.lambda < 1 || py.lambda > py.n_levels) return fail(TDPM_ERR_ARG, "lambda out of range");
        for (int j = 0; j < py.n_levels; ++j)
            if (py.levels[j].H <= 0 || py.levels[j].W <= 0 || py.levels[j].H > 4096 || py.levels[j].W > 4096)
                return fail(TDPM_ERR_ARG, "level with a bad size");
    }
    return batch_arena_bytes(ctx, model_id, pyrs, n_images, nullptr, form, precision, bytes);
}

tdpm_status tdpm_build_pyramid_scores(tdpm_ctx *ctx, int32_t model_id, const tdpm_pyramid *pyr, int32_t form,
                                      int32_t precision, void *stream, int32_t *scores_id)
{
    return tdpm_build_batch_scores(ctx, model_id, pyr, 1, form, precision, stream, scores_id);
}

tdpm_status tdpm_detect(tdpm_ctx *ctx, int32_t scores_id, float tau, tdpm_detection *out, size_t capacity,
                        size_t *n_out, void *stream)
{
    clear_error();
    if (std::isnan(tau)) return fail(TDPM_ERR_ARG, "tau is NaN");
    return detect_impl(ctx, scores_id, tau, nullptr, out, capacity, n_out, stream);
}

tdpm_status tdpm_detect_thresholds(tdpm_ctx *ctx, int32_t scores_id, const float *tau, tdpm_detection *out,
                                   size_t capacity, size_t *n_out, void *stream)
{
    clear_error();
    if (!tau) return fail(TDPM_ERR_ARG, "NULL thresholds");
    return detect_impl(ctx, scores_id, 0.f, tau, out, capacity, n_out, stream);
}

namespace {

size_t a256(size_t b) { return (b + 255) & ~(size_t)255; }

// The records of a scores set with score >= tau, written to the context's post-processing scratch (grow-only,
// shared by the calls below; they hold the context lock and finish before they return). Counts first (one
// synchronisation), then makes room for the records plus `extra(n)` bytes and writes them. *d_rec: the records,
// *d_extra: 256-aligned, right after them.
tdpm_status scratch_records(tdpm_ctx *ctx, Scores *sc, float tau, cudaStream_t s,
                            const std::function<size_t(long long)> &extra, long long &n, tdpm_detection *&d_rec,
                            char *&d_extra)
{
    const Plan &P = *sc->plan;
    char *base = sc->arena.dev;
    const AsmJob *jobs = reinterpret_cast<const AsmJob *>(base + P.blob_off + P.asm_off);
    int *counts = reinterpret_cast<int *>(base + P.counts_off), *offsets = reinterpret_cast<int *>(base + P.offsets_off);
    long long *d_total = reinterpret_cast<long long *>(base + P.total_off);
    CUDA_TRY(cudaStreamWaitEvent(s, sc->done, 0));
    CUDA_TRY(launch_detect_count(jobs, (int)P.asms.size(), P.total, tau, nullptr, counts, offsets, P.n_det_blocks,
                                 d_total, s));
    CUDA_TRY(cudaMemcpyAsync(ctx->h_total, d_total, sizeof(long long), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    tdpm_status st = check_device_flag(ctx);
    if (st) return st;
    n = *ctx->h_total;
    if (n > (1ll << 30)) return fail(TDPM_ERR_CAPACITY, "more than 2^30 detections above tau");
    const size_t rec_b = a256(sizeof(tdpm_detection) * (size_t)std::max<long long>(n, 1));
    const size_t need = rec_b + a256(extra(n)) + 256;
    if (need > ctx->nms_cap) {
        if (ctx->d_nms) {
            cudaFree(ctx->d_nms);
            ctx->used -= std::min(ctx->used, ctx->nms_cap);
            ctx->d_nms = nullptr;
            ctx->nms_cap = 0;
        }
        if (ctx->budget && ctx->used + need > ctx->budget)
            return fail(TDPM_ERR_OOM, "post-processing scratch exceeds the budget");
        CUDA_TRY(cudaMalloc(&ctx->d_nms, need));
        ctx->nms_cap = need;
        ctx->used += need;
    }
    d_rec = static_cast<tdpm_detection *>(ctx->d_nms);
    d_extra = static_cast<char *>(ctx->d_nms) + rec_b;
    if (n > 0)
        CUDA_TRY(launch_detect_write(jobs, (int)P.asms.size(), P.total, tau, nullptr, offsets, P.n_det_blocks, d_rec, n,
                                     sc->model_id, s));
    return TDPM_OK;
}

// Copies the kept records (count at d_n) back and records the set's use.
tdpm_status read_kept(tdpm_ctx *ctx, Scores *sc, const long long *d_n, const tdpm_detection *d_kept,
                      tdpm_detection *out, size_t capacity, size_t *n_out, cudaStream_t s)
{
    CUDA_TRY(cudaMemcpyAsync(ctx->h_total, d_n, sizeof(long long), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    const long long kept = *ctx->h_total;
    const size_t nk = std::min<size_t>((size_t)kept, capacity);
    if (nk) {
        CUDA_TRY(cudaMemcpyAsync(out, d_kept, nk * sizeof(tdpm_detection), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
    }
    CUDA_TRY(cudaEventRecord(sc->done, s));
    *n_out = (size_t)kept;
    if ((size_t)kept > capacity)
        return fail(TDPM_ERR_CAPACITY, "kept detections exceed capacity: " + std::to_string(kept));
    return TDPM_OK;
}

}  // namespace

tdpm_status tdpm_detect_nms(tdpm_ctx *ctx, int32_t scores_id, float tau, const int32_t *component_class,
                            double overlap, double cell0, tdpm_detection *out, size_t capacity, size_t *n_out,
                            void *stream)
{
    clear_error();
    if (!ctx || !n_out || (capacity > 0 && !out)) return fail(TDPM_ERR_ARG, "NULL argument");
    if (!(overlap >= 0.0 && overlap <= 1.0)) return fail(TDPM_ERR_ARG, "overlap must be in [0, 1]");
    if (!(cell0 > 0.0) || !std::isfinite(cell0)) return fail(TDPM_ERR_ARG, "cell0 must be finite and > 0");
    if (std::isnan(tau)) return fail(TDPM_ERR_ARG, "tau is NaN");
    std::lock_guard<std::mutex> lk(ctx->mu);
    tdpm_status st = set_device(ctx);
    if (st) return st;
    Scores *sc = get_scores(ctx, scores_id);
    if (!sc) return fail(TDPM_ERR_STATE, "unknown scores id");
    const Model *m = get_model(ctx, sc->model_id);
    if (!m) return fail(TDPM_ERR_STATE, "the scores' model was unloaded");
    const Plan &P = *sc->plan;
    const int nc = (int)m->comps.size();
    int n_classes = 1;
    if (component_class)
        for (int c = 0; c < nc; ++c) {
            if (component_class[c] < 0) return fail(TDPM_ERR_ARG, "negative class id");
            n_classes = std::max(n_classes, component_class[c] + 1);
        }
    cudaStream_t s = (cudaStream_t)stream;
    int max_levels = 1;
    for (int L : P.img_L) max_levels = std::max(max_levels, L);
    // after the records: the kept records, the NMS working set, the per-component and per-level tables
    const size_t cls_b = a256(4 * (size_t)nc * 3), cell_b = a256(8 * (size_t)P.n_images * max_levels);
    auto extra = [&](long long n) {
        return a256(sizeof(tdpm_detection) * (size_t)std::max<long long>(n, 1)) +
               a256(nms_scratch_bytes(n, P.n_images * n_classes)) + cls_b + cell_b + 256;
    };
    long long n = 0;
    tdpm_detection *d_rec = nullptr;
    char *q = nullptr;
    if ((st = scratch_records(ctx, sc, tau, s, extra, n, d_rec, q))) return st;
    const size_t work_b = nms_scratch_bytes(n, P.n_images * n_classes);
    auto *d_kept = reinterpret_cast<tdpm_detection *>(q);
    q += a256(sizeof(tdpm_detection) * (size_t)std::max<long long>(n, 1));
    void *d_work = q;
    char *tab = q + a256(work_b);
    auto *d_cls = reinterpret_cast<int32_t *>(tab);
    auto *d_rh = d_cls + nc, *d_rw = d_rh + nc;
    auto *d_cell = reinterpret_cast<double *>(tab + cls_b);
    auto *d_nk = reinterpret_cast<long long *>(tab + cls_b + cell_b);
    // the tables: classes, root filter sizes, and the cell size of every (image, level) in image pixels
    std::vector<int32_t> tabs((size_t)nc * 3);
    for (int c = 0; c < nc; ++c) {
        tabs[c] = component_class ? component_class[c] : 0;
        tabs[nc + c] = m->filters[m->comps[c].root_fid].h;
        tabs[2 * nc + c] = m->filters[m->comps[c].root_fid].w;
    }
    std::vector<double> cells((size_t)P.n_images * max_levels, 0.0);
    for (int im = 0; im < P.n_images; ++im)
        for (int j = 0; j < P.img_L[im]; ++j)
            cells[(size_t)im * max_levels + j] = cell0 * std::pow(2.0, (double)j / (double)P.img_lam[im]);
    CUDA_TRY(cudaMemcpyAsync(d_cls, tabs.data(), 4 * tabs.size(), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(d_cell, cells.data(), 8 * cells.size(), cudaMemcpyHostToDevice, s));
    CUDA_TRY(launch_nms(d_rec, n, component_class ? d_cls : nullptr, n_classes, P.n_images, d_rh, d_rw, d_cell,
                        max_levels, overlap, d_work, work_b, d_kept, d_nk, s));
    return read_kept(ctx, sc, d_nk, d_kept, out, capacity, n_out, s);
}

// ------------------------------------------------------------------------------ convolution shortening (Sec. 4)
namespace {

// Device tables of one cascade call, packed in one host blob and copied with one transfer: the filter slots of every
// component (root, then parts), each filter's term order (decreasing |lambda_r|, ties by index) and thresholds, and
// the caller's levels. Needs per-filter factors (Sec. 4); the pyramids must be those the scores set was built from.
struct CascSetup {
    std::vector<char> blob;
    size_t filt_off = 0, first_off = 0, count_off = 0, lev_off = 0, lam_off = 0;
    int max_levels = 1, max_slots = 1, max_terms = 1, n_comps = 0;
    std::vector<int> comp_slots;  // per component: filter slots (1 + parts)
    std::vector<int> slot_fid;    // per (component, slot) in order: the filter id
    std::vector<int> fid_terms;   // per filter: its number of terms
    CascArgs args;                // pointer fields relative to the device copy of the blob
};

tdpm_status casc_setup(const Model &m, const Plan &P, const Arena &A, const tdpm_pyramid *pyrs, int n_images,
                       const float *thr, int thr_stride, char *d_blob, CascSetup &C)
{
    if (!m.decomposed || m.decomp_mode != TDPM_DECOMP_PER_FILTER)
        return fail(TDPM_ERR_STATE, "the cascade needs the model decomposed per filter (Sec. 4)");
    if (!pyrs || n_images != P.n_images)
        return fail(TDPM_ERR_ARG, "pass the pyramids the scores set was built from");
    C.max_levels = 1;
    for (int L : P.img_L) C.max_levels = std::max(C.max_levels, L);
    std::vector<CascLevel> lv((size_t)n_images * C.max_levels, CascLevel{nullptr, 0, 0});
    for (int im = 0; im < n_images; ++im) {
        const tdpm_pyramid &py = pyrs[im];
        if (py.n_levels != P.img_L[im] || py.lambda != P.img_lam[im] || !py.levels)
            return fail(TDPM_ERR_ARG, "pyramid " + std::to_string(im) + " differs from the scored one");
        for (int j = 0; j < py.n_levels; ++j) {
            const tdpm_level &L = py.levels[j];
            const auto &sz = P.sizes[(size_t)P.img_base[im] + j];
            const size_t flat = (size_t)P.img_base[im] + j;
            if (!L.data || L.H != sz.first || L.W != sz.second || flat >= A.levels.size() || A.levels[flat] != L.data)
                return fail(TDPM_ERR_ARG, "pyramid " + std::to_string(im) + " level " + std::to_string(j) +
                                              " is not the level the scores set was built from");
            lv[(size_t)im * C.max_levels + j] = CascLevel{L.data, L.H, L.W};
        }
    }
    C.n_comps = (int)m.comps.size();
    C.fid_terms.assign(m.filters.size(), 0);
    std::vector<std::vector<int>> order(m.filters.size());
    for (size_t f = 0; f < m.filters.size(); ++f) {
        const FilterH &F = m.filters[f];
        const Group &g = m.groups[F.group];
        const int r0 = g.rank_off[F.gidx], r1 = g.rank_off[F.gidx + 1];
        for (int r = r0; r < r1; ++r) order[f].push_back(r);
        std::stable_sort(order[f].begin(), order[f].end(), [&](int a, int b) {
            return std::fabs(g.Lam[(size_t)F.gidx * g.R + a]) > std::fabs(g.Lam[(size_t)F.gidx * g.R + b]);
        });
        C.fid_terms[f] = r1 - r0;
        C.max_terms = std::max(C.max_terms, r1 - r0);
    }
    if (thr && thr_stride < C.max_terms)
        return fail(TDPM_ERR_ARG, "threshold stride below the largest rank " + std::to_string(C.max_terms));
    C.comp_slots.clear();
    C.slot_fid.clear();
    for (const CompH &c : m.comps) {
        C.comp_slots.push_back(1 + (int)c.parts.size());
        C.slot_fid.push_back(c.root_fid);
        for (const PartH &p : c.parts) C.slot_fid.push_back(p.fid);
        C.max_slots = std::max(C.max_slots, 1 + (int)c.parts.size());
    }
    // blob: CascFilter[slots] | first[nc] | count[nc] | levels | img_lam | per slot: order, thresholds
    const size_t n_slots = C.slot_fid.size();
    Bump b;
    C.filt_off = b.take(sizeof(CascFilter) * n_slots);
    C.first_off = b.take(4 * (size_t)C.n_comps);
    C.count_off = b.take(4 * (size_t)C.n_comps);
    C.lev_off = b.take(sizeof(CascLevel) * lv.size());
    C.lam_off = b.take(4 * (size_t)n_images);
    std::vector<size_t> ord_off(n_slots), thr_off(n_slots);
    for (size_t k = 0; k < n_slots; ++k) {
        ord_off[k] = b.take(4 * (size_t)std::max(1, C.fid_terms[C.slot_fid[k]]));
        thr_off[k] = b.take(4 * (size_t)std::max(1, C.fid_terms[C.slot_fid[k]]));
    }
    C.blob.assign(align256(b.off), 0);
    char *hb = C.blob.data();
    size_t k = 0;
    for (int ci = 0; ci < C.n_comps; ++ci) {
        const CompH &c = m.comps[ci];
        reinterpret_cast<int *>(hb + C.first_off)[ci] = (int)k;
        reinterpret_cast<int *>(hb + C.count_off)[ci] = C.comp_slots[ci];
        for (int sl = 0; sl < C.comp_slots[ci]; ++sl, ++k) {
            const int fid = C.slot_fid[k];
            const FilterH &F = m.filters[fid];
            const Group &g = m.groups[F.group];
            CascFilter cf{};
            cf.A = g.d_A;
            cf.B = g.d_B;
            cf.Ct = g.d_Ct;
            cf.lam = g.d_lam;
            cf.order = reinterpret_cast<const int *>(d_blob + ord_off[k]);
            cf.thr = reinterpret_cast<const float *>(d_blob + thr_off[k]);
            cf.R = g.R;
            cf.nterms = C.fid_terms[fid];
            cf.h = F.h;
            cf.w = F.w;
            cf.part = sl > 0;
            cf.vy = sl > 0 ? c.parts[sl - 1].vy : 0;
            cf.vx = sl > 0 ? c.parts[sl - 1].vx : 0;
            reinterpret_cast<CascFilter *>(hb + C.filt_off)[k] = cf;
            int *o = reinterpret_cast<int *>(hb + ord_off[k]);
            float *t = reinterpret_cast<float *>(hb + thr_off[k]);
            for (int q = 0; q < cf.nterms; ++q) {
                o[q] = order[fid][q];
                t[q] = thr ? thr[(size_t)fid * thr_stride + q] : -INFINITY;
                if (std::isnan(t[q])) return fail(TDPM_ERR_ARG, "a threshold is NaN");
            }
        }
    }
    std::memcpy(hb + C.lev_off, lv.data(), sizeof(CascLevel) * lv.size());
    std::memcpy(hb + C.lam_off, P.img_lam.data(), 4 * (size_t)n_images);
    C.args = CascArgs{};
    C.args.filt = reinterpret_cast<const CascFilter *>(d_blob + C.filt_off);
    C.args.comp_first = reinterpret_cast<const int *>(d_blob + C.first_off);
    C.args.comp_count = reinterpret_cast<const int *>(d_blob + C.count_off);
    C.args.levels = reinterpret_cast<const CascLevel *>(d_blob + C.lev_off);
    C.args.max_levels = C.max_levels;
    C.args.img_lam = reinterpret_cast<const int *>(d_blob + C.lam_off);
    return TDPM_OK;
}

// Size of the blob casc_setup will build (a dry run on a throwaway device base).
size_t casc_blob_bytes(const Model &m, const Plan &P, int n_images)
{
    size_t n_slots = 0, terms = 0;
    for (const CompH &c : m.comps) n_slots += 1 + c.parts.size();
    for (const CompH &c : m.comps) {
        auto add = [&](int fid) {
            const FilterH &F = m.filters[fid];
            const Group &g = m.groups[F.group];
            terms += (size_t)std::max(1, g.rank_off.empty() ? 0 : g.rank_off[F.gidx + 1] - g.rank_off[F.gidx]);
        };
        add(c.root_fid);
        for (const PartH &p : c.parts) add(p.fid);
    }
    int max_levels = 1;
    for (int L : P.img_L) max_levels = std::max(max_levels, L);
    return sizeof(CascFilter) * n_slots + 8 * m.comps.size() + sizeof(CascLevel) * (size_t)n_images * max_levels +
           4 * (size_t)n_images + 8 * terms + 256 * (6 + 2 * n_slots);
}

tdpm_status casc_begin(tdpm_ctx *ctx, int32_t scores_id, Scores *&sc, const Model *&m)
{
    tdpm_status st = set_device(ctx);
    if (st) return st;
    sc = get_scores(ctx, scores_id);
    if (!sc) return fail(TDPM_ERR_STATE, "unknown scores id");
    m = get_model(ctx, sc->model_id);
    if (!m) return fail(TDPM_ERR_STATE, "the scores' model was unloaded");
    if (!m->decomposed || m->decomp_mode != TDPM_DECOMP_PER_FILTER)
        return fail(TDPM_ERR_STATE, "the cascade needs the model decomposed per filter (Sec. 4)");
    return TDPM_OK;
}

// Partial sums at caller records (no exits): out [n][max_slots][max_terms] on the host, NaN where not evaluated.
tdpm_status casc_partials(tdpm_ctx *ctx, Scores *sc, const Model &m, const tdpm_pyramid *pyrs, int n_images,
                          const tdpm_detection *records, size_t n, std::vector<float> &out, CascSetup &C,
                          cudaStream_t s)
{
    const Plan &P = *sc->plan;
    const size_t blob_b = casc_blob_bytes(m, P, n_images);
    // validate the records on the host: component, image and level ranges (windows are checked on the device)
    for (size_t i = 0; i < n; ++i) {
        const tdpm_detection &d = records[i];
        if (d.image < 0 || d.image >= P.n_images || d.component < 0 || d.component >= (int)m.comps.size() ||
            d.level < 0 || d.level >= P.img_L[d.image])
            return fail(TDPM_ERR_ARG, "record " + std::to_string(i) + " is outside the scores set");
    }
    // size the partials with a dry setup first (max_slots, max_terms)
    tdpm_status st = casc_setup(m, P, sc->arena, pyrs, n_images, nullptr, 0, nullptr, C);
    if (st) return st;
    const size_t rec_b = a256(sizeof(tdpm_detection) * std::max<size_t>(n, 1));
    const size_t part_b = a256(4 * std::max<size_t>(n, 1) * C.max_slots * C.max_terms);
    const size_t need = rec_b + part_b + a256(blob_b) + a256(32) + 256;
    if (need > ctx->nms_cap) {
        if (ctx->d_nms) {
            cudaFree(ctx->d_nms);
            ctx->used -= std::min(ctx->used, ctx->nms_cap);
            ctx->d_nms = nullptr;
            ctx->nms_cap = 0;
        }
        if (ctx->budget && ctx->used + need > ctx->budget)
            return fail(TDPM_ERR_OOM, "post-processing scratch exceeds the budget");
        CUDA_TRY(cudaMalloc(&ctx->d_nms, need));
        ctx->nms_cap = need;
        ctx->used += need;
    }
    char *q = static_cast<char *>(ctx->d_nms);
    auto *d_rec = reinterpret_cast<tdpm_detection *>(q);
    auto *d_part = reinterpret_cast<float *>(q + rec_b);
    char *d_blob = q + rec_b + part_b;
    auto *d_stats = reinterpret_cast<unsigned long long *>(d_blob + a256(blob_b));
    if ((st = casc_setup(m, P, sc->arena, pyrs, n_images, nullptr, 0, d_blob, C))) return st;
    if (C.blob.size() > a256(blob_b)) return fail(TDPM_ERR_STATE, "cascade table larger than its estimate");
    out.assign(std::max<size_t>(n, 1) * C.max_slots * C.max_terms, NAN);
    CUDA_TRY(cudaStreamWaitEvent(s, sc->done, 0));
    if (n) {
        CUDA_TRY(cudaMemcpyAsync(d_rec, records, sizeof(tdpm_detection) * n, cudaMemcpyHostToDevice, s));
        CUDA_TRY(cudaMemcpyAsync(d_part, out.data(), 4 * out.size(), cudaMemcpyHostToDevice, s));
    }
    CUDA_TRY(cudaMemcpyAsync(d_blob, C.blob.data(), C.blob.size(), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemsetAsync(d_stats, 0, 32, s));
    CascArgs a = C.args;
    a.rec = d_rec;
    a.n = (long long)n;
    a.partials = d_part;
    a.max_slots = C.max_slots;
    a.max_terms = C.max_terms;
    a.stats = d_stats;
    CUDA_TRY(launch_cascade(a, s));
    unsigned long long h_stats[4] = {0, 0, 0, 0};
    if (n) CUDA_TRY(cudaMemcpyAsync(out.data(), d_part, 4 * out.size(), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(h_stats, d_stats, sizeof(h_stats), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    CUDA_TRY(cudaEventRecord(sc->done, s));
    if (h_stats[3]) return fail(TDPM_ERR_ARG, "a record's filter window lies outside its level");
    return TDPM_OK;
}

}  // namespace

tdpm_status tdpm_cascade_partials(tdpm_ctx *ctx, int32_t scores_id, const tdpm_pyramid *pyrs, int32_t n_images,
                                  const tdpm_detection *records, size_t n, float *out, int32_t max_slots,
                                  int32_t max_terms, void *stream)
{
    clear_error();
    if (!ctx || (n > 0 && (!records || !out))) return fail(TDPM_ERR_ARG, "NULL argument");
    if (n > (1u << 24)) return fail(TDPM_ERR_ARG, "at most 2^24 records");
    std::lock_guard<std::mutex> lk(ctx->mu);
    Scores *sc = nullptr;
    const Model *m = nullptr;
    tdpm_status st = casc_begin(ctx, scores_id, sc, m);
    if (st) return st;
    CascSetup C;
    std::vector<float> part;
    if ((st = casc_partials(ctx, sc, *m, pyrs, n_images, records, n, part, C, (cudaStream_t)stream))) return st;
    if (max_slots < C.max_slots || max_terms < C.max_terms)
        return fail(TDPM_ERR_CAPACITY, "partials need max_slots >= " + std::to_string(C.max_slots) +
                                           " and max_terms >= " + std::to_string(C.max_terms));
    for (size_t i = 0; i < n; ++i)
        for (int sl = 0; sl < max_slots; ++sl)
            for (int q = 0; q < max_terms; ++q)
                out[((size_t)i * max_slots + sl) * max_terms + q] =
                    sl < C.max_slots && q < C.max_terms ? part[((size_t)i * C.max_slots + sl) * C.max_terms + q] : NAN;
    return TDPM_OK;
}

tdpm_status tdpm_cascade_thresholds(tdpm_ctx *ctx, int32_t scores_id, const tdpm_pyramid *pyrs, int32_t n_images,
                                    const tdpm_detection *positives, size_t n, float *t, int32_t stride, void *stream)
{
    clear_error();
    if (!ctx || !t || (n > 0 && !positives)) return fail(TDPM_ERR_ARG, "NULL argument");
    if (n > (1u << 24)) return fail(TDPM_ERR_ARG, "at most 2^24 positives");
    std::lock_guard<std::mutex> lk(ctx->mu);
    Scores *sc = nullptr;
    const Model *m = nullptr;
    tdpm_status st = casc_begin(ctx, scores_id, sc, m);
    if (st) return st;
    CascSetup C;
    std::vector<float> part;
    if ((st = casc_partials(ctx, sc, *m, pyrs, n_images, positives, n, part, C, (cudaStream_t)stream))) return st;
    if (stride < C.max_terms) return fail(TDPM_ERR_ARG, "stride below the largest rank " + std::to_string(C.max_terms));
    // t[fid][q] = min over the positives of the filter's partial sum of its first q + 1 terms; -inf without positives
    const size_t nf = m->filters.size();
    for (size_t f = 0; f < nf; ++f)
        for (int q = 0; q < stride; ++q) t[f * stride + q] = -INFINITY;
    std::vector<char> seen(nf, 0);
    for (size_t i = 0; i < n; ++i) {
        const int ci = positives[i].component;
        int k = 0;
        for (int c = 0; c < ci; ++c) k += C.comp_slots[c];
        for (int sl = 0; sl < C.comp_slots[ci]; ++sl) {
            const int fid = C.slot_fid[(size_t)k + sl];
            float *tf = t + (size_t)fid * stride;
            for (int q = 0; q < C.fid_terms[fid]; ++q) {
                const float p = part[((size_t)i * C.max_slots + sl) * C.max_terms + q];
                tf[q] = seen[fid] ? std::min(tf[q], p) : p;
            }
            seen[fid] = 1;
        }
    }
    return TDPM_OK;
}

tdpm_status tdpm_detect_cascade(tdpm_ctx *ctx, int32_t scores_id, const tdpm_pyramid *pyrs, int32_t n_images,
                                const float *t, int32_t stride, float tau, tdpm_detection *out, size_t capacity,
                                size_t *n_out, tdpm_cascade_stats *stats, void *stream)
{
    clear_error();
    if (!ctx || !t || !n_out || (capacity > 0 && !out)) return fail(TDPM_ERR_ARG, "NULL argument");
    if (std::isnan(tau)) return fail(TDPM_ERR_ARG, "tau is NaN");
    std::lock_guard<std::mutex> lk(ctx->mu);
    Scores *sc = nullptr;
    const Model *m = nullptr;
    tdpm_status st = casc_begin(ctx, scores_id, sc, m);
    if (st) return st;
    const Plan &P = *sc->plan;
    cudaStream_t s = (cudaStream_t)stream;
    CascSetup C;
    if ((st = casc_setup(*m, P, sc->arena, pyrs, n_images, t, stride, nullptr, C))) return st;  // validation before any work
    const size_t blob_b = casc_blob_bytes(*m, P, n_images);
    // after the records: the kept records, the flags, the tables, the statistics, the compaction scratch
    auto extra = [&](long long n) {
        const size_t nn = (size_t)std::max<long long>(n, 1);
        return a256(sizeof(tdpm_detection) * nn) + a256(nn) + a256(blob_b) + a256(40) + compact_scratch_bytes(n);
    };
    long long n = 0;
    tdpm_detection *d_rec = nullptr;
    char *q = nullptr;
    if ((st = scratch_records(ctx, sc, tau, s, extra, n, d_rec, q))) return st;
    const size_t nn = (size_t)std::max<long long>(n, 1);
    auto *d_kept = reinterpret_cast<tdpm_detection *>(q);
    auto *d_alive = reinterpret_cast<uint8_t *>(q + a256(sizeof(tdpm_detection) * nn));
    char *d_blob = q + a256(sizeof(tdpm_detection) * nn) + a256(nn);
    auto *d_stats = reinterpret_cast<unsigned long long *>(d_blob + a256(blob_b));
    auto *d_nk = reinterpret_cast<long long *>(d_stats + 4);
    void *d_cs = d_blob + a256(blob_b) + a256(40);
    if ((st = casc_setup(*m, P, sc->arena, pyrs, n_images, t, stride, d_blob, C))) return st;
    if (C.blob.size() > a256(blob_b)) return fail(TDPM_ERR_STATE, "cascade table larger than its estimate");
    CUDA_TRY(cudaMemcpyAsync(d_blob, C.blob.data(), C.blob.size(), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemsetAsync(d_stats, 0, 40, s));
    CascArgs a = C.args;
    a.rec = d_rec;
    a.n = n;
    a.apply_thr = true;
    a.alive = d_alive;
    a.stats = d_stats;
    CUDA_TRY(launch_cascade(a, s));
    CUDA_TRY(launch_compact_records(d_rec, d_alive, n, d_cs, compact_scratch_bytes(n), d_kept, d_nk, s));
    unsigned long long h_stats[4] = {0, 0, 0, 0};
    CUDA_TRY(cudaMemcpyAsync(h_stats, d_stats, sizeof(h_stats), cudaMemcpyDeviceToHost, s));
    if ((st = read_kept(ctx, sc, d_nk, d_kept, out, capacity, n_out, s)) && st != TDPM_ERR_CAPACITY) return st;
    if (h_stats[3]) return fail(TDPM_ERR_STATE, "a record's filter window lies outside its level");
    if (stats) {
        stats->candidates = n;
        stats->pruned = (int64_t)h_stats[2];
        stats->terms_evaluated = (int64_t)h_stats[0];
        stats->terms_total = (int64_t)h_stats[1];
    }
    return st;
}

tdpm_status tdpm_get_maps(tdpm_ctx *ctx, int32_t scores_id, int32_t kind, int32_t image, int32_t index_a,
                          int32_t index_b, void *out_host, size_t capacity_bytes, int32_t *rows, int32_t *cols,
                          void *stream)
{
    clear_error();
    if (!ctx || !rows || !cols) return fail(TDPM_ERR_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(ctx->mu);
    tdpm_status st = set_device(ctx);
    if (st) return st;
    Scores *sc = get_scores(ctx, scores_id);
    if (!sc) return fail(TDPM_ERR_STATE, "unknown scores id");
    const Plan &P = *sc->plan;
    const std::map<std::pair<int, int>, MapRef> *mp = nullptr;
    switch (kind) {
    case TDPM_MAP_FILTER_SCORE: mp = &P.filter_maps; break;
    case TDPM_MAP_FINAL_SCORE: mp = &P.final_maps; break;
    case TDPM_MAP_PART_DT: mp = &P.dt_maps; break;
    case TDPM_MAP_PART_ARG: mp = &P.arg_maps; break;
    default: return fail(TDPM_ERR_ARG, "bad map kind");
    }
    if (image < 0 || image >= P.n_images) return fail(TDPM_ERR_ARG, "image out of range");
    if (index_b < 0 || index_b >= P.img_L[image]) return fail(TDPM_ERR_ARG, "level out of range");
    auto it = mp->find({index_a, P.img_base[image] + index_b});
    *rows = 0;
    *cols = 0;
    if (it == mp->end()) return TDPM_OK;
    *rows = it->second.rows;
    *cols = it->second.cols;
    const size_t bytes = (size_t)it->second.rows * it->second.cols * 4;
    if (bytes > capacity_bytes || !out_host)
        return fail(TDPM_ERR_CAPACITY, "map needs " + std::to_string(bytes) + " bytes");
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(cudaStreamWaitEvent(s, sc->done, 0));
    CUDA_TRY(cudaMemcpyAsync(out_host, sc->arena.dev + it->second.off, bytes, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return check_device_flag(ctx);
}

tdpm_status tdpm_release(tdpm_ctx *ctx, int32_t scores_id)
{
    clear_error();
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

// ------------------------------------------------------------------------------------------------ instrumentation
uint64_t tdpm_kernel_launches(void) { return g_launches.load(); }

tdpm_status tdpm_selftest_bounded_wait(tdpm_ctx *ctx)
{
    clear_error();
    if (!ctx) return fail(TDPM_ERR_ARG, "ctx is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    tdpm_status st = set_device(ctx);
    if (st) return st;
    cudaStream_t s = ctx->cap_stream;  // a stream of the context's own, idle outside graph capture
    CUDA_TRY(launch_bounded_wait_probe(ctx->d_err, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    st = check_device_flag(ctx);  // clears the flag it finds raised
    if (st == TDPM_OK) return fail(TDPM_ERR_STATE, "the bounded wait did not report its expiry");
    return st;
}

tdpm_status tdpm_set_fusion(tdpm_ctx *ctx, int32_t enable)
{
    clear_error();
    if (!ctx) return fail(TDPM_ERR_ARG, "ctx is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->fuse = enable != 0;
    return TDPM_OK;
}

tdpm_status tdpm_profile_enable(tdpm_ctx *ctx, int32_t enable)
{
    clear_error();
    if (!ctx) return fail(TDPM_ERR_ARG, "ctx is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->prof = enable != 0;
    return TDPM_OK;
}

tdpm_status tdpm_profile_read(tdpm_ctx *ctx, int32_t index, char *name, size_t name_cap, double *total_ms,
                              int64_t *launches, int32_t *n_stages)
{
    clear_error();
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

tdpm_status tdpm_autotune_read(tdpm_ctx *ctx, int32_t index, char *key, size_t key_cap, int32_t *tile_n,
                               int32_t *persistent, int32_t *n_entries)
{
    clear_error();
    if (!ctx || !n_entries) return fail(TDPM_ERR_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(ctx->mu);
    *n_entries = (int32_t)ctx->tune_cache.size();
    if (index < 0 || index >= *n_entries) return TDPM_OK;
    auto it = ctx->tune_cache.begin();
    std::advance(it, index);
    if (key && key_cap) {
        std::strncpy(key, it->first.c_str(), key_cap - 1);
        key[key_cap - 1] = 0;
    }
    if (tile_n) *tile_n = it->second & 0xffff;
    if (persistent) *persistent = (it->second & kTcPersistent) ? 1 : 0;
    return TDPM_OK;
}

tdpm_status tdpm_profile_reset(tdpm_ctx *ctx)
{
    clear_error();
    if (!ctx) return fail(TDPM_ERR_ARG, "ctx is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    prof_collect(ctx);
    ctx->stages.clear();
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
    clear_error();
    if (!S || !d || !D || !arg || !scratch) return fail(TDPM_ERR_ARG, "NULL argument");
    if (H <= 0 || W <= 0 || H > kDtMaxSide || W > kDtMaxSide)
        return fail(TDPM_ERR_ARG, "map sides must be in [1, " + std::to_string(kDtMaxSide) + "]");
    for (int k = 0; k < 4; ++k)
        if (!std::isfinite(d[k])) return fail(TDPM_ERR_ARG, "non-finite deformation coefficient");
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
    // the fused form (the scratch's V / IV areas stay unused; tdpm_dt_noalloc runs the two-pass form)
    CUDA_TRY(launch_dt_fused(reinterpret_cast<const DtJob *>(sb), 1, nullptr,
                             dt_job_strips(nx), W, H, s));
    return TDPM_OK;
}

tdpm_status tdpm_correlate(const float *feat, int32_t H, int32_t W, const float *filt_host, int32_t K, int32_t h,
                           int32_t w, int32_t precision, float *out, void *stream)
{
    clear_error();
    if (!feat || !filt_host || !out) return fail(TDPM_ERR_ARG, "NULL argument");
    if (H <= 0 || W <= 0 || K <= 0 || h <= 0 || w <= 0 || h > 16 || w > 16 || H > 4096 || W > 4096 || K > 4096)
        return fail(TDPM_ERR_ARG, "bad sizes");
    if (!valid_precision(precision)) return fail(TDPM_ERR_ARG, "unsupported precision");
    if (reinterpret_cast<uintptr_t>(feat) % 16) return fail(TDPM_ERR_ARG, "feat not 16-byte aligned");
    const int Ho = H - h + 1, Wo = W - w + 1;
    if (Ho <= 0 || Wo <= 0) return TDPM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int taps = h * w;
    std::vector<char> tmp;
    void *dmem = nullptr;
    cudaError_t e = cudaSuccess;
    if (precision == TDPM_PREC_FP32) {
        const int Kpad = (K + corr_f32_tile_k() - 1) / corr_f32_tile_k() * corr_f32_tile_k();
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
        const size_t fbytes = align256(sizeof(float) * ft.size());
        CUDA_TRY(cudaMalloc(&dmem, fbytes + sizeof(CorrJob)));
        char *db = reinterpret_cast<char *>(dmem);
        e = cudaMemcpyAsync(db, ft.data(), sizeof(float) * ft.size(), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(db + fbytes, &J, sizeof(J), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = launch_corr_f32(reinterpret_cast<const CorrJob *>(db + fbytes), 1, tiles, reinterpret_cast<float *>(db),
                                K, Kpad, h, w, s);
    } else {
        // tensor cores: BF16 filter bank(s) and planar BF16 copies of the level (split precision adds the lo
        // parts), or an E4M3 bank and an E4M3 planar copy with per-tensor scales
        const bool split = precision == TDPM_PREC_BF16X3, fp8 = precision == TDPM_PREC_FP8;
        const int Npad = corr_tc_bank_rows(K), NT = corr_tc_default_nt(K, taps);
        std::vector<uint16_t> fb, fl;
        std::vector<uint8_t> f8;
        float fscale = 1.f;
        if (fp8) {
            float mx = 0.f;
            for (size_t i = 0; i < (size_t)K * taps * FD; ++i) mx = std::max(mx, std::fabs(filt_host[i]));
            fscale = mx > 0.f ? 448.f / mx : 1.f;
            f8.assign((size_t)taps * 2 * Npad * 16, 0);
            for (int k = 0; k < K; ++k)
                for (int t = 0; t < taps; ++t)
                    for (int c = 0; c < FD; ++c)
                        f8[(((size_t)t * 2 + c / 16) * Npad + k) * 16 + (c % 16)] =
                            e4m3_bits(filt_host[((size_t)k * taps + t) * FD + c] * fscale);
        } else {
            fb.assign((size_t)taps * 4 * Npad * 8, 0);
            fl.assign(fb.size(), 0);
            for (int k = 0; k < K; ++k)
                for (int t = 0; t < taps; ++t)
                    for (int c = 0; c < FD; ++c) {
                        const float x = filt_host[((size_t)k * taps + t) * FD + c];
                        const size_t i = (((size_t)t * 4 + c / 8) * Npad + k) * 8 + (c % 8);
                        fb[i] = bf16_bits(x);
                        fl[i] = bf16_bits(x - bf16_round(x));
                    }
        }
        const long long cells = (long long)H * W;
        const size_t fbytes = align256(fp8 ? f8.size() : sizeof(uint16_t) * fb.size());
        const size_t pbytes = align256((fp8 ? 1 : sizeof(uint16_t)) * (size_t)cells * FD);
        const size_t parts = split ? 2 : 1;
        CUDA_TRY(cudaMalloc(&dmem, parts * (fbytes + pbytes) + align256(sizeof(ConvJob)) + sizeof(TcJob) + 256));
        char *db = reinterpret_cast<char *>(dmem);
        void *bank = db;
        void *bank_lo = split ? db + fbytes : nullptr;
        uint16_t *planar = reinterpret_cast<uint16_t *>(db + parts * fbytes);
        uint16_t *planar_lo = split ? reinterpret_cast<uint16_t *>(db + parts * fbytes + pbytes) : nullptr;
        char *cjd = db + parts * (fbytes + pbytes), *tjd = cjd + align256(sizeof(ConvJob));
        int *d_err = reinterpret_cast<int *>(tjd + align256(sizeof(TcJob)));
        ConvJob cj{feat, planar, planar_lo, cells, 0};
        TcJob tj{};
        const bool ok = fp8 ? encode_level_tmap_fp8(&tj.tmap, reinterpret_cast<const uint8_t *>(planar), cells)
                            : encode_level_tmap(&tj.tmap, planar, cells) &&
                                  (!split || encode_level_tmap(&tj.tmap_lo, planar_lo, cells));
        if (!ok) {
            cudaFree(dmem);
            return fail(TDPM_ERR_CUDA, "cuTensorMapEncodeTiled failed");
        }
        tj.out = out; tj.H = H; tj.W = W; tj.Ho = Ho; tj.Wo = Wo; tj.begin = 0;
        const long long span = (long long)(Ho - 1) * W + Wo;
        const int tiles = (int)((span + corr_tc_tile_m() - 1) / corr_tc_tile_m());
        if (fp8)
            e = cudaMemcpyAsync(bank, f8.data(), f8.size(), cudaMemcpyHostToDevice, s);
        else
            e = cudaMemcpyAsync(bank, fb.data(), sizeof(uint16_t) * fb.size(), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && split)
            e = cudaMemcpyAsync(bank_lo, fl.data(), sizeof(uint16_t) * fl.size(), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(cjd, &cj, sizeof(cj), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(tjd, &tj, sizeof(tj), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(d_err, 0, sizeof(int), s);
        if (e == cudaSuccess)
            e = fp8 ? launch_to_fp8_planar(reinterpret_cast<const ConvJob *>(cjd), 1, 2 * cells, kFp8FeatureScale, s)
                    : launch_to_bf16_planar(reinterpret_cast<const ConvJob *>(cjd), 1, 4 * cells, s);
        if (e == cudaSuccess)
            e = launch_corr_tc(reinterpret_cast<const TcJob *>(tjd), 1, tiles, bank, bank_lo, K, Npad, NT, h, w, 1,
                               d_err, s, fp8, fp8 ? 1.f / (fscale * kFp8FeatureScale) : 1.f,
                               corr_form_override() == 1);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(dmem);
    if (e != cudaSuccess) return fail(TDPM_ERR_CUDA, std::string("correlate: ") + cudaGetErrorString(e));
    return TDPM_OK;
}

}  // extern "C"
