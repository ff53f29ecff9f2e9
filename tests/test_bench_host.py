"""Host logic of bench.py's CPU legs (no GPU): the oracle baseline splits the frames over the pool's
processes, renders each process's frames before its timed section, and reports the wall time of the
oracle sections and the summed single-thread time per frame."""
import multiprocessing as mp


def test_oracle_baseline_times_the_oracle_alone(oracle_mod):
    import bench
    from paper_1807_02752_gb300 import scenes

    cfg, _ = scenes.WORKLOADS[bench.WORKLOAD]
    pdict = oracle_mod.default_params(n_disp=cfg.n_disp).as_dict()
    pool = mp.get_context("spawn").Pool(2)
    try:
        frames = [0, 1, 2, 3]
        bench.run_oracle_frames(pool, [4, 5], pdict, 2)   # both processes up and warm, as in bench.py
        wall, cpu_s = bench.run_oracle_frames(pool, frames, pdict, 2)
        res = pool.map(bench._oracle_chunk, [(bench.WORKLOAD, [f], pdict) for f in frames], chunksize=1)
    finally:
        pool.close()
        pool.join()
    # two processes with two frames each: the sections overlap, so the wall is below the summed time and
    # at least the longer process's share
    assert 0.0 < wall < cpu_s
    assert wall >= 0.4 * cpu_s
    for t_start, t_end, cpu in res:
        assert 0.0 < cpu <= t_end - t_start
