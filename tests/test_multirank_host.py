"""The benchmark's multi-rank path on the CPU: two gloo ranks, each with its own scan.

`bench.py --gpus N` runs one process per GPU; every rank images its own scan (weak
scaling, no collective on the data path) and the job's time is the maximum over ranks.
This covers that host logic without a GPU: per-rank scans differ, each rank's plan is
valid on its own, and the timing reduction takes the slowest rank.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, ws, port, out_dir):
    import sys

    if ROOT not in sys.path:  # spawned interpreters do not inherit the test's path setup
        sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    import paper_2506_23568_gb300 as hh

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=ws)
    try:
        s = bench._scene("tiny", rank)
        plan = hh.Plan(s.traj, s.freqs, s.grid, host_only=True, leaf_size=32)
        info = plan.info()
        # a made-up per-rank step time: the job's time must be the slowest rank's
        job_ms, hh_ms = bench.reduce_over_ranks(dist, [10.0 + rank, 5.0 + 2.0 * rank], "cpu")
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), traj=s.traj, perm=plan.export()["perm"],
                 n_levels=info["n_levels"], job_ms=job_ms, hh_ms=hh_ms,
                 per_volume=bench.per_volume_s(hh_ms, ws))
        plan.close()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_image_their_own_scans(tmp_path):
    ws = 2
    mp.spawn(_rank_main, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, join=True)
    r = [np.load(tmp_path / f"rank{k}.npz") for k in range(ws)]
    # independent scans: same recipe, different trajectories, each with a valid plan
    assert r[0]["traj"].shape == r[1]["traj"].shape
    assert not np.array_equal(r[0]["traj"], r[1]["traj"])
    for k in range(ws):
        assert sorted(r[k]["perm"].tolist()) == list(range(len(r[k]["traj"])))
        assert int(r[k]["n_levels"]) >= 2
    # the reduction gives every rank the maximum over ranks
    for k in range(ws):
        assert float(r[k]["job_ms"]) == 11.0 and float(r[k]["hh_ms"]) == 7.0
        assert float(r[k]["per_volume"]) == pytest.approx(7.0 / 1e3 / ws)
