"""The autotuner's operation-count model (Sec. IV-B) from host-only plans: subimage samples
grow level by level (Eq. eq_smpratiosim2 gives about four per 4-way level asymptotically),
leaves trade leaf updates against interpolation as they shrink, and the ranking follows the
prediction.  CPU only."""
import numpy as np

import synth
from paper_2506_23568_gb300 import tune


def test_subimage_samples_grow_level_by_level():
    s = synth.large()
    import paper_2506_23568_gb300 as hh

    ex = hh.Plan(s.traj, s.freqs, s.grid, host_only=True, leaf_size=64, eta=1.6).export()
    ls = ex["level_start"]
    sizes = np.prod(ex["N"].astype(np.float64), axis=1)
    per_node = [sizes[ls[lv]:ls[lv + 1]].mean() for lv in range(len(ls) - 2)]
    # samples per node grow at every level (the lattices' fixed padding steps keep the lowest
    # ratios below the paper's asymptotic 4 per 4-way level, which ignores padding)
    assert all(a < b for a, b in zip(per_node, per_node[1:])), per_node
    assert per_node[-1] / per_node[-2] > 3.0, per_node


def test_leaf_and_interpolation_terms_trade_off():
    s = synth.mid()
    c = [tune.op_counts(s.traj, s.freqs, s.grid, leaf_size=l, eta=1.6) for l in (64, 128, 256, 512)]
    leaf = [x["leaf"] for x in c]
    interp = [x["interp"] for x in c]
    assert all(a < b for a, b in zip(leaf, leaf[1:])), leaf            # bigger leaves: more leaf updates
    assert interp[0] > interp[-1], interp                               # ... and fewer levels to merge
    assert c[0]["levels"] > c[-1]["levels"]
    assert c[0]["rc"] == len(s.traj) * len(s.freqs) * np.log2(len(s.freqs))


def test_ranking_follows_the_prediction():
    s = synth.tiny()
    cands = [dict(leaf_size=l, eta=e, taps=t) for l in (16, 64) for e in (1.5, 2.0) for t in (4, 6)]
    preds = [tune.predicted_ms(tune.op_counts(s.traj, s.freqs, s.grid, **c), c["taps"]) for c in cands]
    # denser lattices and more taps never predict less work
    for i, c in enumerate(cands):
        for j, d in enumerate(cands):
            if c["leaf_size"] == d["leaf_size"] and c["eta"] <= d["eta"] and c["taps"] <= d["taps"]:
                assert preds[i] <= preds[j] + 1e-12
