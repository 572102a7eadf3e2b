"""GPU: the serving loop (continuous batching). Every request's detections are the same alone, in a mix with other
requests, under a memory budget that forces one image per batch, and through the direct scoring calls; failures stay
with the request that caused them."""
import time

import numpy as np
import pytest

from helpers import device_pyramid
from paper_1707_03268_gb300 import synth

pytestmark = pytest.mark.gpu

FIELDS = ("image", "model", "component", "level", "y", "x", "score", "n_parts", "part_y", "part_x")


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.fixture(scope="module")
def T(torch):
    from paper_1707_03268_gb300 import tdpm
    return tdpm


@pytest.fixture(scope="module")
def setup(torch, T):
    """Three class models, five images of different sizes, eight requests with different model subsets."""
    ctx = T.tdpm_create(0)
    models = [T.tdpm_load_model(ctx, synth.Model(synth.make_dpm_class(np.random.default_rng(100 + c))))
              for c in range(3)]
    rng = np.random.default_rng(7)
    sizes = [(120, 160), (150, 200), (200, 150), (240, 320), (96, 128)]
    pyrs = [device_pyramid(synth.make_pyramid(rng, synth.pyramid_sizes(h, w), synth.LAMBDA), torch)
            for (h, w) in sizes]
    subsets = [[0], [1, 2], [2], [0, 1, 2], [1], [2, 0], [0], [1]]
    reqs = []
    for i, sub in enumerate(subsets):
        img = i % len(pyrs)
        mids = [models[c] for c in sub]
        # threshold: the 97th percentile of this image's scores under its first model (direct call)
        sid = T.tdpm_build_pyramid_scores(ctx, mids[0], pyrs[img], T.FORM_FULL, T.PREC_BF16X3)
        allp = T.tdpm_detect(ctx, sid, -np.inf)
        T.tdpm_release(ctx, sid)
        reqs.append({"image": img, "models": mids, "tau": float(np.percentile(allp["score"], 97))})
    yield ctx, models, pyrs, reqs
    T.tdpm_destroy(ctx)


def _direct(T, ctx, pyrs, req, form, prec):
    out = []
    for mid in req["models"]:
        sid = T.tdpm_build_pyramid_scores(ctx, mid, pyrs[req["image"]], form, prec)
        out.append(T.tdpm_detect(ctx, sid, req["tau"]))
        T.tdpm_release(ctx, sid)
    return np.concatenate(out)


def _same(a, b):
    assert len(a) == len(b)
    for f in FIELDS:
        np.testing.assert_array_equal(a[f], b[f])


@pytest.mark.parametrize("form,prec", [("full", "bf16x3"), ("decomposed", "bf16x3")])
def test_alone_mix_and_budget_give_the_same_detections(T, setup, form, prec):
    ctx, models, pyrs, reqs = setup
    f = T.FORM_FULL if form == "full" else T.FORM_DECOMPOSED
    p = T.PREC_BF16X3
    if f == T.FORM_DECOMPOSED:
        for mid in models:
            T.tdpm_decompose(ctx, mid, 8, T.DECOMP_PER_FILTER, max_iters=40, seed=1)
    ref = [_direct(T, ctx, pyrs, r, f, p) for r in reqs]
    assert sum(len(r) for r in ref) > 0
    for r, d in zip(reqs, ref):
        assert np.all(d["model"] == np.repeat(r["models"], [np.sum(d["model"] == m) for m in r["models"]]))

    # alone: one request in the system at a time
    T.tdpm_server_start(ctx, max_batch_images=8, max_inflight=2, max_wait_us=0)
    alone = []
    for r in reqs:
        t = T.tdpm_submit(ctx, pyrs[r["image"]], r["models"], f, p, r["tau"])
        alone.append(T.tdpm_poll(ctx, t)[0])
    # mix: everything submitted at once, batched by model, two batches in flight
    tickets = [T.tdpm_submit(ctx, pyrs[r["image"]], r["models"], f, p, r["tau"]) for r in reqs]
    mixed = [T.tdpm_poll(ctx, t) for t in tickets]
    T.tdpm_server_stop(ctx)
    assert max(info["batch_images"] for _, info in mixed) > 1   # the mix really was batched
    for d_ref, d_alone, (d_mix, info) in zip(ref, alone, mixed):
        _same(d_alone, d_ref)
        _same(d_mix, d_ref)
        assert info["status"] == T.OK and info["n_detections"] == len(d_ref)
        assert info["t_submit_ns"] <= info["t_start_ns"] <= info["t_done_ns"]

    # memory budget that holds the largest single image's arena: batches are cut down (halved) to fit
    biggest = max(T.tdpm_scores_bytes(ctx, mid, [pyrs[r["image"]]], f, p) for r in reqs for mid in r["models"])
    assert T.tdpm_scores_bytes(ctx, models[0], pyrs, f, p) > biggest
    T.tdpm_server_start(ctx, max_batch_images=8, max_inflight=2, max_wait_us=0, mem_budget_bytes=biggest)
    tickets = [T.tdpm_submit(ctx, pyrs[r["image"]], r["models"], f, p, r["tau"]) for r in reqs]
    budgeted = [T.tdpm_poll(ctx, t) for t in tickets]
    T.tdpm_server_stop(ctx)
    for d_ref, (d, info) in zip(ref, budgeted):
        _same(d, d_ref)
        assert info["status"] == T.OK


def test_failures_stay_with_their_request(T, setup):
    ctx, models, pyrs, reqs = setup
    T.tdpm_server_start(ctx, max_batch_images=4, max_inflight=2, max_wait_us=100)
    good = T.tdpm_submit(ctx, pyrs[0], [models[0]], T.FORM_FULL, T.PREC_BF16X3, reqs[0]["tau"])
    bad = T.tdpm_submit(ctx, pyrs[1], [models[1], 987654], T.FORM_FULL, T.PREC_BF16X3, 0.0)  # unknown model
    good2 = T.tdpm_submit(ctx, pyrs[1], [models[1]], T.FORM_FULL, T.PREC_BF16X3, reqs[1]["tau"])
    with pytest.raises(T.TdpmError) as e:
        T.tdpm_poll(ctx, bad)
    assert e.value.status == T.ERR_STATE
    d, info = T.tdpm_poll(ctx, good)
    assert info["status"] == T.OK
    d2, info2 = T.tdpm_poll(ctx, good2)
    assert info2["status"] == T.OK
    with pytest.raises(T.TdpmError) as e:   # released after the first poll
        T.tdpm_poll(ctx, good)
    assert e.value.status == T.ERR_STATE
    with pytest.raises(T.TdpmError) as e:   # never issued
        T.tdpm_poll(ctx, 10 ** 12, timeout_ms=0)
    assert e.value.status == T.ERR_STATE
    # invalid requests are refused at submission
    with pytest.raises(T.TdpmError) as e:
        T.tdpm_submit(ctx, pyrs[0], [], T.FORM_FULL, T.PREC_BF16X3, 0.0)
    assert e.value.status == T.ERR_ARG
    with pytest.raises(T.TdpmError) as e:
        T.tdpm_submit(ctx, pyrs[0], [models[0], models[0]], T.FORM_FULL, T.PREC_BF16X3, 0.0)
    assert e.value.status == T.ERR_ARG
    T.tdpm_server_stop(ctx)
    # a budget below any single image: the request fails with ERR_OOM, the server keeps going
    T.tdpm_server_start(ctx, max_batch_images=4, max_inflight=1, max_wait_us=0, mem_budget_bytes=1)
    t = T.tdpm_submit(ctx, pyrs[4], [models[0]], T.FORM_FULL, T.PREC_BF16X3, 0.0)
    with pytest.raises(T.TdpmError) as e:
        T.tdpm_poll(ctx, t)
    assert e.value.status == T.ERR_OOM
    T.tdpm_server_stop(ctx)
    with pytest.raises(T.TdpmError) as e:   # stopped
        T.tdpm_submit(ctx, pyrs[0], [models[0]], T.FORM_FULL, T.PREC_BF16X3, 0.0)
    assert e.value.status == T.ERR_STATE


def test_poll_timeout_then_result(T, setup):
    ctx, models, pyrs, reqs = setup
    # a long wait for companions keeps the request pending for a while: a zero-timeout poll must say so
    T.tdpm_server_start(ctx, max_batch_images=64, max_inflight=1, max_wait_us=300000)
    t0 = time.monotonic()
    t = T.tdpm_submit(ctx, pyrs[3], [models[0]], T.FORM_FULL, T.PREC_BF16X3, reqs[3]["tau"])
    with pytest.raises(T.TdpmError) as e:
        T.tdpm_poll(ctx, t, timeout_ms=0)
    assert e.value.status == T.ERR_TIMEOUT or time.monotonic() - t0 > 0.25
    d, info = T.tdpm_poll(ctx, t, timeout_ms=20000)
    assert info["status"] == T.OK
    T.tdpm_server_stop(ctx)


def test_class_subsets_of_a_bank(T, torch):
    """Several classes loaded as one bank model; each request asks for some classes (component subsets). Alone, in
    the mix and scored directly with the full bank (then filtered), the detections are the same."""
    ctx = T.tdpm_create(0)
    comps = []
    for c in range(4):
        comps += synth.make_dpm_class(np.random.default_rng(200 + c))
    bank = T.tdpm_load_model(ctx, synth.Model(comps))
    rng = np.random.default_rng(11)
    pyrs = [device_pyramid(synth.make_pyramid(rng, synth.pyramid_sizes(h, w), synth.LAMBDA), torch)
            for (h, w) in [(120, 160), (180, 240), (150, 150)]]
    classes = [[0], [1, 3], [2], [0, 1, 2, 3], [3]]
    reqs = []
    for i, cl in enumerate(classes):
        img = i % len(pyrs)
        sid = T.tdpm_build_pyramid_scores(ctx, bank, pyrs[img], T.FORM_FULL, T.PREC_BF16X3)
        allp = T.tdpm_detect(ctx, sid, -np.inf)
        T.tdpm_release(ctx, sid)
        cs = [6 * c + k for c in cl for k in range(6)]
        tau = float(np.percentile(allp[np.isin(allp["component"], cs)]["score"], 96))
        ref = allp[np.isin(allp["component"], cs) & (allp["score"] >= tau)]
        reqs.append({"image": img, "components": cs, "tau": tau, "ref": ref})
    T.tdpm_server_start(ctx, max_batch_images=8, max_inflight=2, max_wait_us=0)
    alone = []
    for r in reqs:
        t = T.tdpm_submit(ctx, pyrs[r["image"]], [bank], T.FORM_FULL, T.PREC_BF16X3, r["tau"], r["components"])
        alone.append(T.tdpm_poll(ctx, t)[0])
    tickets = [T.tdpm_submit(ctx, pyrs[r["image"]], [bank], T.FORM_FULL, T.PREC_BF16X3, r["tau"], r["components"])
               for r in reqs]
    mixed = [T.tdpm_poll(ctx, t) for t in tickets]
    bad = T.tdpm_submit(ctx, pyrs[0], [bank], T.FORM_FULL, T.PREC_BF16X3, 0.0, [999])  # no such component
    with pytest.raises(T.TdpmError) as e:
        T.tdpm_poll(ctx, bad)
    assert e.value.status == T.ERR_ARG
    T.tdpm_server_stop(ctx)
    assert max(info["batch_images"] for _, info in mixed) > 1
    for r, a, (m, info) in zip(reqs, alone, mixed):
        assert len(r["ref"]) > 0
        _same(a, r["ref"])
        _same(m, r["ref"])
    T.tdpm_destroy(ctx)


def test_served_detections_match_the_oracle(torch, T):
    """Serving against the FP64 oracle (Algorithm 1's detection set D): a mix of requests with different image sizes,
    class subsets of one bank model and thresholds taken from the oracle's own scores, submitted together and batched
    by the server, each compared with the oracle's detections for the same image, components and threshold on the same
    per-filter factors (split BF16: >= 99.5% agreement; matched detections carry the oracle's part positions up to
    near-ties at the precision's tolerance, Sec. 2 argmax)."""
    from helpers import agreement, dt_value
    from oracle import oracle as orc

    ctx = T.tdpm_create(0)
    rng = np.random.default_rng(31)
    comps = []
    for _ in range(3):
        comps.extend(synth.make_dpm_class(rng))  # three classes of six components: one bank model
    bank = synth.Model(comps)
    mid = T.tdpm_load_model(ctx, bank)
    T.tdpm_decompose(ctx, mid, 8, T.DECOMP_PER_FILTER, max_iters=60, seed=5)
    n_f, n_groups = T.tdpm_model_info(ctx, mid)
    rebuilt = [None] * n_f
    for gi in range(n_groups):
        info = T.tdpm_group_info(ctx, mid, gi)
        A, B, C, Lam = T.tdpm_get_factors(ctx, mid, gi)
        F = orc.joint_reconstruct(Lam, A, B, C)
        for k, fid in enumerate(info["filter_ids"]):
            rebuilt[fid] = F[k]
    first_fid = np.cumsum([0] + [1 + len(c.parts) for c in comps])
    sizes = [(96, 128), (120, 160), (150, 200)]
    host = [synth.make_pyramid(rng, synth.pyramid_sizes(h, w), synth.LAMBDA) for (h, w) in sizes]
    dev = [device_pyramid(p, torch) for p in host]
    subsets = [[0], [1, 2], [2, 0], [0, 1, 2], [1]]  # classes per request
    reqs = []
    for i, classes in enumerate(subsets):
        img = i % len(sizes)
        cs = [6 * c + k for c in classes for k in range(6)]
        sub = synth.Model([comps[c] for c in cs])
        fs = [rebuilt[f] for c in cs for f in range(first_fid[c], first_fid[c + 1])]
        scored = orc.score_pyramid(sub, host[img], filters=fs)
        tau = float(np.percentile(orc.all_scores(scored), 98))
        ref = {(cs[d[0]],) + tuple(d[1:4]): d for d in orc.detect(scored, tau)}
        reqs.append({"image": img, "components": cs, "tau": tau, "ref": ref, "sub": sub, "fs": fs})
    T.tdpm_server_start(ctx, max_batch_images=8, max_inflight=2, max_wait_us=200)
    tickets = [T.tdpm_submit(ctx, dev[r["image"]], [mid], T.FORM_DECOMPOSED, T.PREC_BF16X3, r["tau"],
                             r["components"]) for r in reqs]
    served = [T.tdpm_poll(ctx, t) for t in tickets]
    T.tdpm_server_stop(ctx)
    assert max(info["batch_images"] for _, info in served) > 1  # the requests really were batched together
    n_parts_checked = 0
    for r, (d, info) in zip(reqs, served):
        assert info["status"] == T.OK
        got = {(int(x["component"]), int(x["level"]), int(x["y"]), int(x["x"])): x for x in d}
        assert set(k[0] for k in got) <= set(r["components"])
        assert agreement(set(got), set(r["ref"])) >= 0.995
        # part positions of the matched detections: equal, or a near-tie of the oracle's FP64 values within what split
        # BF16 moves a part score (1e-4 of the map's largest value, for each of the two placements)
        pyr = host[r["image"]]
        for key in set(got) & set(r["ref"]):
            c, j, y, x = key
            comp = comps[c]
            ref_d = r["ref"][key]
            lp = j - pyr.lam
            for i, part in enumerate(comp.parts):
                gy, gx = int(got[key]["part_y"][i]), int(got[key]["part_x"][i])
                oy, ox = ref_d[5][i], ref_d[6][i]
                if (gy, gx) == (oy, ox):
                    continue
                S = orc.correlate(pyr.levels[lp], rebuilt[first_fid[c] + 1 + i])
                py, px = 2 * y + part.anchor[0], 2 * x + part.anchor[1]
                d4 = list(part.deform)
                gap = dt_value(S, d4, oy, ox, py, px) - dt_value(S, d4, gy, gx, py, px)
                assert gap <= 2e-4 * float(np.max(np.abs(S)))
            n_parts_checked += 1
    assert n_parts_checked > 100
    T.tdpm_destroy(ctx)
