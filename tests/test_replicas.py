"""Multi-rank (replica) host path on CPU: two gloo ranks, each detecting its round-robin share of the
frames, gathered on rank 0 must equal one process detecting every frame; the slowest rank's time wins.

The per-rank detector here is the CPU oracle (a stand-in for each rank's GPU handle): the test covers the
partition, the record gather and the timing reduction, which are the only multi-rank parts of the path.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_1807_02752_gb300 import replicas, scenes
from paper_1807_02752_gb300.ld import LANES_DTYPE

N_FRAMES = 5
CFG = scenes.with_size(scenes.SMALL_320x120, width=160, height=72, n_disp=32)


def _record(res: dict) -> np.ndarray:
    r = np.zeros((), LANES_DTYPE)
    n = res["n_lanes"]
    r["n_lanes"], r["flags"], r["v_top"] = n, res["flags"], res["v_top"]
    r["start_u"][:n] = res["start_u"]
    r["energy"][:n] = res["energy"]
    r["centre"], r["scale_exp"] = res["centre"], res["scale_exp"]
    r["rounds_y"], r["rounds_x"] = res["rounds_y"], res["rounds_x"]
    r["beta"], r["gamma"] = res["beta"], res["gamma"]
    return r


def _detect(frames):
    disp, img, _ = scenes.make_batch(CFG, N_FRAMES, first_frame=20)
    p = oracle.default_params(n_disp=CFG.n_disp)
    return np.array([_record(oracle.detect(disp[f], img[f], p, dumps=False)) for f in frames], LANES_DTYPE)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        frames = replicas.frames_of_rank(N_FRAMES, rank, world)
        got = replicas.gather_lanes(_detect(frames), frames, N_FRAMES)
        slowest = replicas.max_over_ranks(1.0 + rank)
        if rank == 0:
            np.save(os.path.join(out_dir, "gathered.npy"), got.view(np.uint8))
        else:
            assert got is None
        np.save(os.path.join(out_dir, f"max{rank}.npy"), np.array([slowest]))
    finally:
        dist.destroy_process_group()


def test_partition_is_round_robin_and_complete():
    parts = [replicas.frames_of_rank(10, r, 3) for r in range(3)]
    assert parts == [[0, 3, 6, 9], [1, 4, 7], [2, 5, 8]]
    assert sorted(sum(parts, [])) == list(range(10))
    with pytest.raises(ValueError):
        replicas.frames_of_rank(10, 3, 3)


def test_single_process_gather_checks_coverage():
    rec = np.zeros(3, LANES_DTYPE)
    rec["n_lanes"] = [1, 2, 3]
    out = replicas.gather_lanes(rec, [2, 0, 1], 3)
    assert out["n_lanes"].tolist() == [2, 3, 1]
    with pytest.raises(ValueError):
        replicas.gather_lanes(rec[:2], [0, 1], 3)
    assert replicas.max_over_ranks(2.5) == 2.5


def test_two_gloo_ranks_match_one_process(tmp_path):
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    gathered = np.load(tmp_path / "gathered.npy").view(LANES_DTYPE)
    single = _detect(list(range(N_FRAMES)))
    assert gathered.tobytes() == single.tobytes()
    assert any(r["n_lanes"] > 0 for r in single), "the scenes should hold lanes"
    for r in range(world):
        assert float(np.load(tmp_path / f"max{r}.npy")[0]) == 2.0
