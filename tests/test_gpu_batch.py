"""Batched imaging (hhffbp_batch_*): several uneven scans, one plan each, imaged by one CUDA
graph launch, against the same plans' single-scan images (bit for bit: the graph replays the
same kernels on the same buffers); replay, re-capture on new buffers, and the autotuner's
choice meeting the accuracy bar."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hh():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2506_23568_gb300 as m

    m.lib()
    return m


def _scans():
    shapes = [(16, 16, 32, 24, 20, 6), (12, 20, 24, 17, 23, 5), (20, 12, 40, 31, 9, 7), (10, 10, 16, 8, 8, 3),
              (18, 22, 32, 26, 26, 4)]
    return [synth.small(n_lines=a, n_per_line=b, n_f=f, nx=x, ny=y, nz=z, seed=1200 + i)
            for i, (a, b, f, x, y, z) in enumerate(shapes)]


def test_batch_matches_single_scans_and_replays(hh):
    scans = _scans()
    echos = [synth.scene_echo(s, device="cuda") for s in scans]
    plans = [hh.Plan(s.traj, s.freqs, s.grid, leaf_size=8 + 4 * (i % 3)) for i, s in enumerate(scans)]
    single = [p.form_image(e).clone() for p, e in zip(plans, echos)]
    batch = hh.Batch(plans, n_streams=3)
    out = batch.form_images(echos)
    torch.cuda.synchronize()
    for a, b in zip(single, out):
        assert torch.equal(a, b)
    for o in out:
        o.fill_(float("nan"))
    out2 = batch.form_images(echos, out)  # the same buffers: the graph is replayed
    torch.cuda.synchronize()
    for a, b in zip(single, out2):
        assert torch.equal(a, b)
    fresh = [torch.empty_like(o) for o in out]  # new buffers: recorded again
    batch.form_images(echos, fresh)
    torch.cuda.synchronize()
    for a, b in zip(single, fresh):
        assert torch.equal(a, b)
    for p in plans:
        c = p.counters()
        assert c["errors"] == 0 and c["gate_miss"] == 0, c
    batch.close()


def test_batch_refuses_host_buffers(hh):
    s = _scans()[0]
    plan = hh.Plan(s.traj, s.freqs, s.grid, leaf_size=8)
    batch = hh.Batch([plan])
    with pytest.raises(ValueError):
        batch.form_images([synth.scene_echo(s, device="cpu")])
    batch.close()


def test_autotuner_choice_meets_the_bar(hh):
    from paper_2506_23568_gb300 import tune

    s = synth.tiny()
    e = synth.scene_echo(s, device="cuda")
    cands = [dict(leaf_size=l, eta=eta, taps=6) for l in (16, 32, 64) for eta in (1.25, 2.0)]
    res = tune.tune(s.traj, s.freqs, s.grid, e, target_db=-30.0, candidates=cands, top=4, every=4)
    assert res["accepted"], res
    chosen = [t for t in res["tried"] if all(t[k] == v for k, v in res["config"].items())][0]
    assert chosen["nrmse_db"] <= -30.0
    assert chosen["measured_ms"] == min(t["measured_ms"] for t in res["tried"] if t["accepted"])
