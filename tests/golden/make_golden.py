"""Write tests/golden/thresholds.json: detection thresholds tau for the seeded workloads, from the FP64 oracle only.

The paper gives no thresholds for synthetic data, so tau is set from the oracle's own full-form scores: the median of
all scored positions for the single-level case, the 99th percentile for the class model on a full pyramid, and the
99th percentile of each class's scores for the 20-class bank on the 1280x720 pyramid. Run:

    python tests/golden/make_golden.py
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as orc  # noqa: E402
from paper_1707_03268_gb300 import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "thresholds.json")


def main():
    res = {}
    for name, wl, q in [("c1", synth.config_c1(), 50.0), ("c2", synth.config_c2(), 99.0)]:
        t0 = time.time()
        scored = orc.score_pyramid(wl.model, wl.pyramids[0])
        scores = orc.all_scores(scored)
        tau = float(np.percentile(scores, q))
        n_det = len(orc.detect(scored, tau))
        res[name] = {"workload": wl.name, "percentile": q, "tau": tau, "n_positions": int(scores.size),
                     "n_detections": n_det}
        print(name, res[name], f"{time.time() - t0:.1f}s", flush=True)
    # the 20-class bank on one 1280x720 pyramid: one threshold per class (its six components), the 99th percentile of
    # the class's scores over every scored position of its components
    t0 = time.time()
    wl = synth.config_c3()
    scored = orc.score_pyramid(wl.model, wl.pyramids[0])
    n_classes = len(wl.model.components) // 6
    taus = []
    for c in range(n_classes):
        sc = orc.all_scores([s for s in scored if s["component"] // 6 == c])
        taus.append(float(np.percentile(sc, 99.0)))
    n_det = sum(int(np.sum(s["score"] >= taus[s["component"] // 6])) for s in scored)
    res["c3"] = {"workload": wl.name, "percentile": 99.0, "components_per_class": 6, "tau_per_class": taus,
                 "n_detections": n_det}
    print("c3", n_det, f"{time.time() - t0:.1f}s", flush=True)
    with open(OUT, "w") as f:
        json.dump(res, f, indent=1, sort_keys=True)
        f.write("\n")


if __name__ == "__main__":
    main()
