"""Host logic of bench.py's CPU legs (no GPU): the oracle baseline splits the frames over the pool's
processes, one chunk per process, renders each process's frames before its timed section, and reports the
wall time of the oracle sections and the summed single-thread time per frame."""
import pytest


def test_oracle_baseline_times_the_oracle_alone(oracle_mod):
    import bench
    from paper_1807_02752_gb300 import scenes

    cfg, _ = scenes.WORKLOADS[bench.WORKLOAD]
    pdict = oracle_mod.default_params(n_disp=cfg.n_disp).as_dict()
    pool = bench.oracle_pool(2)
    try:
        frames = [0, 1, 2, 3]
        bench.run_oracle_frames(pool, [4, 5], pdict, 2)   # both processes up and warm, as in bench.py
        wall, cpu_s = bench.run_oracle_frames(pool, frames, pdict, 2)
        res = pool.map(bench._oracle_chunk, [(bench.WORKLOAD, [f], pdict) for f in frames[:2]], chunksize=1)
        with pytest.raises(ValueError):
            bench.run_oracle_frames(pool, [7], pdict, 2)   # a process without a frame would hold the barrier
    finally:
        pool.close()
        pool.join()
    # two processes with two frames each: the sections overlap, so the wall is below the summed time and
    # at least the longer process's share
    assert 0.0 < wall < cpu_s
    assert wall >= 0.4 * cpu_s
    assert res[0][0] != res[1][0]                      # one chunk per process
    for _, t_start, t_end, cpu in res:
        assert 0.0 < cpu <= t_end - t_start
