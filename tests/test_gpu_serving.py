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


def _collect(srv, got):
    srv.drain()
    while len(r := srv.poll()):
        got.extend(r)
    return got


def _check(got, frames, alone, order=None):
    """Every frame came back once, with its stream's sequence number in submission order (order: the tags
    as submitted, by default the list order) and its result alone."""
    assert sorted(int(r["tag"]) for r in got) == list(range(len(frames)))
    order = list(range(len(frames))) if order is None else order
    seq, count = {}, {}
    for t in order:
        sid = frames[t][0]
        seq[t] = count.get(sid, 0)
        count[sid] = seq[t] + 1
    for r in got:
        tag = int(r["tag"])
        sid, _, wh, _, _ = frames[tag]
        assert (int(r["stream_id"]), int(r["seq"]), int(r["w"]), int(r["h"])) == (sid, seq[tag], wh[0], wh[1])
        assert r["lanes"].tobytes() == alone[tag].tobytes(), f"frame {tag} differs from its result alone"


def _runs(frames):
    """The frames split into runs of one size, in submission order: (tags, stream ids, disp, img)."""
    runs, cur = [], []
    for tag, f in enumerate(frames):
        if cur and frames[cur[-1]][2] != f[2]:
            runs.append(cur)
            cur = []
        cur.append(tag)
    runs.append(cur)
    return [(np.array(r, np.uint64), np.array([frames[t][0] for t in r], np.int32),
             np.stack([frames[t][3] for t in r]), np.stack([frames[t][4] for t in r])) for r in runs]


@pytest.mark.parametrize("mode", ["pinned", "batch", "batch_pinned"])
def test_pinned_and_batched_submits_match_alone(torch_cuda, mode):
    """Frames the device reads from the caller's page-locked memory (ld_server_submit_pinned) and frames handed
    over several at a time (ld_server_submit_batch, staged or pinned, with runs longer than a slot so that one
    call fills several slots): every result is the frame's result alone, with its stream's sequence number."""
    torch = torch_cuda
    p = ld.default_params(n_disp=48)
    frames = sorted(_frames(), key=lambda f: f[2])      # runs of one size, several streams within a run
    alone = _alone(frames, p)
    srv = ld.Server(SIZES, p, n_streams=N_STREAMS, slots_per_size=2, max_batch=4, max_wait_us=300)
    keep = []                                           # pinned frames stay untouched until polled
    got = []
    try:
        if mode == "pinned":
            for tag, (sid, k, wh, d, i) in enumerate(frames):
                dt, it = torch.from_numpy(d).pin_memory(), torch.from_numpy(i).pin_memory()
                keep.append((dt, it))
                while not srv.submit_pinned(sid, dt, it, tag):
                    got.extend(srv.poll(timeout_ms=100))
        else:
            pinned = mode == "batch_pinned"
            for tags, sids, d, i in _runs(frames):
                if pinned:
                    d, i = torch.from_numpy(d).pin_memory(), torch.from_numpy(i).pin_memory()
                    keep.append((d, i))
                at = 0
                while at < len(tags):
                    acc = srv.submit_batch(sids[at:], d[at:], i[at:], tags[at:], pinned=pinned)
                    assert 0 <= acc <= len(tags) - at
                    at += acc
                    if at < len(tags):
                        got.extend(srv.poll(timeout_ms=100))
        _check(_collect(srv, got), frames, alone)
        st = srv.stats()
        assert st["submitted"] == st["completed"] == len(frames)
        assert st["slots"] == 2 * len(SIZES)
    finally:
        srv.close()


def test_concurrent_batched_submitters(torch_cuda):
    """Three threads hand over runs of their streams' frames at once (copies outside the server's lock):
    nothing is lost or mixed up and every result is the frame's result alone."""
    import threading

    p = ld.default_params(n_disp=48)
    frames = _frames()
    alone = _alone(frames, p)
    srv = ld.Server(SIZES, p, n_streams=N_STREAMS, slots_per_size=2, max_batch=3, max_wait_us=300)
    errors = []

    def producer(sid):
        try:
            mine = [t for t, f in enumerate(frames) if f[0] == sid]
            for a in range(0, len(mine), 2):            # pairs of consecutive frames of one size
                run = [t for t in mine[a:a + 2] if frames[t][2] == frames[mine[a]][2]]
                tags = np.array(run, np.uint64)
                sids = np.full(len(run), sid, np.int32)
                d = np.stack([frames[t][3] for t in run])
                i = np.stack([frames[t][4] for t in run])
                at = 0
                while at < len(run):
                    at += srv.submit_batch(sids[at:], d[at:], i[at:], tags[at:])
                    if at < len(run):
                        threading.Event().wait(0.0005)
                for t in mine[a:a + 2]:
                    if t not in run:                    # the pair's second frame has the other size
                        while not srv.submit(sid, frames[t][3], frames[t][4], t):
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
        assert not errors, errors
        _check(_collect(srv, got), frames, alone)
    finally:
        srv.close()


def test_hbm_budget_adds_slots(torch_cuda):
    """Admission by device memory: with one initial slot per size, a run of frames handed over in one call
    fills a slot, finds it in flight and has the server add slots while their device bytes stay within the
    budget; every result is the frame's result alone, also in the learned form on a slot added after it was
    switched on.  A budget below the initial slots is refused at creation."""
    import os

    torch = torch_cuda
    p = ld.default_params(n_disp=48)
    frames = _frames()
    alone = _alone(frames, p)
    with pytest.raises(ld.LDError) as e:
        ld.Server(SIZES, p, n_streams=N_STREAMS, slots_per_size=1, max_batch=2, hbm_budget_bytes=1 << 16)
    assert e.value.code == ld.E_ARG
    probe = ld.Server(SIZES, p, n_streams=N_STREAMS, slots_per_size=1, max_batch=2)
    base = probe.stats()
    probe.close()
    probe = ld.Server(SIZES[:1], p, n_streams=N_STREAMS, slots_per_size=1, max_batch=2)
    slot_a = probe.stats()["device_bytes"]
    probe.close()
    assert base["slots"] == 2 and 0 < slot_a < base["device_bytes"]
    budget = base["device_bytes"] + 2 * slot_a + slot_a // 2     # room for two more slots of the first size
    run = [t for t, f in enumerate(frames) if f[2] == SIZES[0]][:8]
    rest = [t for t in range(len(frames)) if t not in run]
    tags = np.array(run, np.uint64)
    sids = np.array([frames[t][0] for t in run], np.int32)
    d = np.stack([frames[t][3] for t in run])
    i = np.stack([frames[t][4] for t in run])
    srv = ld.Server(SIZES, p, n_streams=N_STREAMS, slots_per_size=1, max_batch=2, max_wait_us=10_000_000,
                    hbm_budget_bytes=budget)
    try:
        got, at = [], 0
        while at < len(run):
            at += srv.submit_batch(sids[at:], d[at:], i[at:], tags[at:])
            if at < len(run):
                got.extend(srv.poll(timeout_ms=50))
        st = srv.stats()
        assert 3 <= st["slots"] <= 4, st                 # the second run of the call found the first in flight
        assert st["device_bytes"] == base["device_bytes"] + (st["slots"] - 2) * slot_a <= budget
        for t in rest:
            sid, k, wh, dd, ii = frames[t]
            while not srv.submit(sid, dd, ii, t):
                got.extend(srv.poll(timeout_ms=50))
        _check(_collect(srv, got), frames, alone, order=run + rest)
    finally:
        srv.close()

    # the learned form on a slot the budget adds after it was switched on
    w = np.load(os.path.join(os.path.dirname(ld.__file__), "proposal_weights.npy")).astype(np.float32)
    theta = torch.from_numpy(w).cuda()
    top_k = 16
    srv = ld.Server(SIZES, p, n_streams=N_STREAMS, slots_per_size=1, max_batch=2, max_wait_us=10_000_000,
                    hbm_budget_bytes=1 << 34)
    learned = {}
    try:
        srv.set_learned(theta, top_k)
        del theta
        at = 0
        while at < len(run):
            at += srv.submit_batch(sids[at:], d[at:], i[at:], tags[at:])
        assert srv.stats()["slots"] >= 3
        for r in _collect(srv, []):
            learned[int(r["tag"])] = r["lanes"].tobytes()
    finally:
        srv.close()
    det = ld.Detector(SIZES[0][0], SIZES[0][1], 1, p)
    net = ld.Net(det)
    net.set_params(torch.from_numpy(w).cuda())
    try:
        assert sorted(learned) == run
        for t in run:
            _, _, _, dd, ii = frames[t]
            out = net.detect(torch.from_numpy(dd[None]).cuda(), torch.from_numpy(ii[None]).cuda(), top_k=top_k)
            torch.cuda.synchronize()
            assert ld.Detector.lanes(out)[0].tobytes() == learned[t], f"frame {t}"
    finally:
        net.close()
        det.close()
