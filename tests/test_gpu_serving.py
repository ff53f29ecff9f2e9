"""Serving: frames of two sizes from three camera streams through one server (continuous batching over
slots).  Every result must be the one the frame gets alone, byte for byte, and that result the oracle's;
results carry the caller's tag and per-stream sequence numbers; the device-kept stream state is each
stream's latest result.
"""
import numpy as np
import pytest

from paper_1807_02752_gb300 import ld, scenes
from gpu_util import compare_frame

pytestmark = pytest.mark.gpu

SIZES = [(320, 120), (256, 96)]
N_STREAMS, PER_STREAM = 3, 6


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1807_02752_gb300 import build
    build.build()
    return torch


def _frames():
    """(stream, frame index in stream, size class, disp, img) in an interleaved submission order."""
    out = []
    for k in range(PER_STREAM):
        for sid in range(N_STREAMS):
            w, h = SIZES[(sid + k) % len(SIZES)]
            cfg = scenes.with_size(scenes.SMALL_320x120, width=w, height=h, n_disp=48)
            d, i, _ = scenes.make_frame(cfg, 100 + 10 * sid + k)
            out.append((sid, k, (w, h), d, i))
    return out


def _alone(frames, p):
    dets = {wh: ld.Detector(wh[0], wh[1], 1, p) for wh in SIZES}
    res = []
    for sid, k, wh, d, i in frames:
        res.append(dets[wh].detect_host(d[None], i[None])[0])
    for det in dets.values():
        det.close()
    return res


def test_alone_results_match_oracle(torch_cuda):
    """The per-frame results the serving tests compare against are the oracle's (every frame of both sizes)."""
    p = ld.default_params(n_disp=48)
    frames = _frames()
    for tag, ((sid, k, wh, d, i), r) in enumerate(zip(frames, _alone(frames, p))):
        compare_frame(None, r, tag, d, i, p, stages=False)


def _serve(frames, p, **kw):
    srv = ld.Server(SIZES, p, n_streams=N_STREAMS, **kw)
    got = []
    for tag, (sid, k, wh, d, i) in enumerate(frames):
        while not srv.submit(sid, d, i, tag):
            got.extend(srv.poll(timeout_ms=100))
    srv.drain()
    while True:
        r = srv.poll()
        if len(r) == 0:
            break
        got.extend(r)
    return srv, got


@pytest.mark.parametrize("kw", [dict(slots_per_size=2, max_batch=4, max_wait_us=200),
                                dict(slots_per_size=1, max_batch=3, max_wait_us=100000),
                                dict(slots_per_size=3, max_batch=1, max_wait_us=0)])
def test_results_match_alone(torch_cuda, kw):
    p = ld.default_params(n_disp=48)
    frames = _frames()
    alone = _alone(frames, p)
    srv, got = _serve(frames, p, **kw)
    try:
        assert sorted(int(r["tag"]) for r in got) == list(range(len(frames)))
        for r in got:
            tag = int(r["tag"])
            sid, k, wh, _, _ = frames[tag]
            assert (int(r["stream_id"]), int(r["seq"]), int(r["w"]), int(r["h"])) == (sid, k, wh[0], wh[1])
            assert r["lanes"].tobytes() == alone[tag].tobytes(), f"frame {tag} differs from its result alone"
            assert r["latency_ms"] > 0
        for sid in range(N_STREAMS):
            last = max(t for t, f in enumerate(frames) if f[0] == sid)
            assert srv.stream_state(sid).tobytes() == alone[last].tobytes()
        st = srv.stats()
        assert st["submitted"] == st["completed"] == len(frames)
        assert st["batches"] >= len(frames) / kw["max_batch"]
        assert 0 < st["p50_ms"] <= st["p99_ms"]
    finally:
        srv.close()


def test_rejects_unknown_size_and_stream(torch_cuda):
    p = ld.default_params(n_disp=48)
    srv = ld.Server(SIZES, p, n_streams=2, slots_per_size=1, max_batch=2)
    try:
        d = np.zeros((50, 60), np.float32)
        i = np.zeros((50, 60), np.uint8)
        with pytest.raises(ld.LDError):
            srv.submit(0, d, i)
        d2 = np.zeros((120, 320), np.float32)
        i2 = np.zeros((120, 320), np.uint8)
        with pytest.raises(ld.LDError):
            srv.submit(5, d2, i2)
        with pytest.raises(ld.LDError):
            srv.stream_state(0)  # nothing completed yet
    finally:
        srv.close()


def test_concurrent_submitters(torch_cuda):
    """Three host threads submit their streams at once (the server is thread-safe); nothing is lost or
    mixed up, and each result is still the frame's result alone."""
    import threading

    p = ld.default_params(n_disp=48)
    frames = _frames()
    alone = _alone(frames, p)
    srv = ld.Server(SIZES, p, n_streams=N_STREAMS, slots_per_size=2, max_batch=3, max_wait_us=300)
    errors = []

    def producer(sid):
        try:
            for tag, f in enumerate(frames):
                if f[0] != sid:
                    continue
                while not srv.submit(sid, f[3], f[4], tag):
                    threading.Event().wait(0.0005)
        except Exception as e:  # reported below
            errors.append(e)

    try:
        ths = [threading.Thread(target=producer, args=(sid,)) for sid in range(N_STREAMS)]
        for t in ths:
            t.start()
        got = []
        while any(t.is_alive() for t in ths):
            got.extend(srv.poll(timeout_ms=5))
        for t in ths:
            t.join()
        srv.drain()
        while True:
            r = srv.poll()
            if len(r) == 0:
                break
            got.extend(r)
        assert not errors, errors
        assert sorted(int(r["tag"]) for r in got) == list(range(len(frames)))
        for r in got:
            tag = int(r["tag"])
            assert int(r["stream_id"]) == frames[tag][0] and int(r["seq"]) == frames[tag][1]
            assert r["lanes"].tobytes() == alone[tag].tobytes()
    finally:
        srv.close()


def test_learned_form_matches_alone(torch_cuda):
    """With the learned form switched on, every result is the frame's learned result alone (ld_detect_learned
    on a one-frame handle, the package's trained weights, the same top_k), byte for byte; switching it off
    again gives the plain results; switching while a frame waits in a slot is refused."""
    import os

    torch = torch_cuda
    p = ld.default_params(n_disp=48)
    w = np.load(os.path.join(os.path.dirname(ld.__file__), "proposal_weights.npy")).astype(np.float32)
    theta = torch.from_numpy(w).cuda()
    top_k = 16
    frames = _frames()
    dets = {wh: ld.Detector(wh[0], wh[1], 1, p) for wh in SIZES}
    nets = {wh: ld.Net(det) for wh, det in dets.items()}
    alone = []
    for net in nets.values():
        net.set_params(theta)
    for sid, k, wh, d, i in frames:
        out = nets[wh].detect(torch.from_numpy(d[None]).cuda(), torch.from_numpy(i[None]).cuda(), top_k=top_k)
        torch.cuda.synchronize()
        alone.append(ld.Detector.lanes(out)[0].copy())
    for wh in SIZES:
        nets[wh].close()
        dets[wh].close()
    plain = _alone(frames, p)

    srv = ld.Server(SIZES, p, n_streams=N_STREAMS, slots_per_size=2, max_batch=4, max_wait_us=200)
    try:
        srv.set_learned(theta, top_k)
        got = []
        for tag, (sid, k, wh, d, i) in enumerate(frames):
            while not srv.submit(sid, d, i, tag):
                got.extend(srv.poll(timeout_ms=100))
        srv.drain()
        while len(r := srv.poll()):
            got.extend(r)
        assert sorted(int(r["tag"]) for r in got) == list(range(len(frames)))
        for r in got:
            tag = int(r["tag"])
            assert r["lanes"].tobytes() == alone[tag].tobytes(), f"frame {tag} differs from its learned result alone"

        srv.set_learned(None, 0)
        got = []
        for tag, (sid, k, wh, d, i) in enumerate(frames):
            while not srv.submit(sid, d, i, tag):
                got.extend(srv.poll(timeout_ms=100))
        srv.drain()
        while len(r := srv.poll()):
            got.extend(r)
        for r in got:
            assert r["lanes"].tobytes() == plain[int(r["tag"])].tobytes()
    finally:
        srv.close()

    # a frame waiting in a filling slot (max_batch 3, ten-second wait): the form cannot change
    srv = ld.Server(SIZES, p, n_streams=N_STREAMS, slots_per_size=1, max_batch=3, max_wait_us=10_000_000)
    try:
        sid, k, wh, d, i = frames[0]
        assert srv.submit(sid, d, i, 0)
        with pytest.raises(ld.LDError) as e:
            srv.set_learned(theta, top_k)
        assert e.value.code == ld.E_STATE
        with pytest.raises(ld.LDError) as e:
            srv.set_learned(theta, ld.NET_TOPK_MAX + 1)
        assert e.value.code == ld.E_ARG
        srv.drain()
    finally:
        srv.close()
