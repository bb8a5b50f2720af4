"""GPU test of the serving loop: sessions served concurrently in shared
batched launches give, session by session, exactly the results of serving
that session alone; launches of the two slots are on the device at the same
time; the first frame of every served session equals the oracle's."""
import numpy as np
import pytest

from paper_1911_10217_gb300 import scenes

pytestmark = pytest.mark.gpu


def _sessions():
    out = {}
    specs = [(64, 48, 8, 64, 16), (96, 64, 16, 128, 32), (40, 24, 4, 32, 64), (80, 60, 12, 64, 32)]
    for sid, (w, h, npatch, tpp, M) in enumerate(specs):
        out[sid] = scenes.frame_scene(seed=70 + sid, width=w, height=h, n_patches=npatch, tris_per_patch=tpp,
                                      n_boxes=32, table_size=1 << 12, cut_size=M, frames=1)
    return out


def _serve(torch, rll, sc, sids, arrivals, budget, timeline=False, max_items=8, cap=1 << 16):
    from paper_1911_10217_gb300 import serving
    dev = torch.device("cuda:0")
    ex = serving.GpuExecutor(torch, rll, dev, max_items=max_items, max_records=cap, max_cells=cap, keep_results=True,
                             timeline=timeline)
    sched = serving.Scheduler(budget, max_items, cap, cap)
    for sid in sids:
        s = sc[sid]
        sched.add_session(sid, serving.session_bytes(s.n_lights, s.n_points, s.grid.table_size, s.grid.cut_size),
                          s.n_points * s.spp, s.grid.table_size, len(arrivals[sid]))
    log = serving.serve(ex, sched, {k: sc[k] for k in sids}, {k: arrivals[k] for k in sids})
    assert all(st == 0 for st in ex.status())
    if timeline:
        return ex.results, log, ex.device_intervals()
    return ex.results, log


def test_alone_equals_in_the_mix():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1911_10217_gb300 import rll
    sc = _sessions()
    rng = np.random.default_rng(0)
    arrivals = {sid: np.cumsum(rng.exponential(0.002, size=6)) for sid in sc}
    big = 10**12
    mix, log = _serve(torch, rll, sc, list(sc), arrivals, big)
    assert len(log) == sum(len(a) for a in arrivals.values())
    # requests overlapped: some launch held more than one session
    starts = {}
    for r in log:
        starts.setdefault(r.start, set()).add(r.session)
    assert max(len(v) for v in starts.values()) > 1
    for sid in sc:
        alone, _ = _serve(torch, rll, sc, [sid], arrivals, big)
        a, b = alone[sid], mix[sid]
        assert np.array_equal(a["rgb"], b["rgb"])
        oa, ob = np.argsort(a["grid"]["keys"]), np.argsort(b["grid"]["keys"])
        for k in ("keys", "cut", "q", "c"):
            assert np.array_equal(a["grid"][k][oa], b["grid"][k][ob]), (sid, k)


def test_two_slots_overlap_on_the_device():
    """Continuous batching on the device: six sessions of 480 x 270 points
    whose frames are all requested at once, at most two sessions per launch;
    the second slot's launch is enqueued while the first slot's is still on
    the GPU, so their device intervals (CUDA events on the slots' streams)
    overlap, and the results equal those of each session served alone."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1911_10217_gb300 import rll
    sc = {sid: scenes.frame_scene(seed=90 + sid, width=480, height=270, n_patches=16, tris_per_patch=256,
                                  table_size=1 << 16, cut_size=32, frames=1) for sid in range(6)}
    arrivals = {sid: np.zeros(3) for sid in sc}
    cap = 1 << 20
    mix, log, spans = _serve(torch, rll, sc, list(sc), arrivals, 10**12, timeline=True, max_items=2, cap=cap)
    assert len(log) == 18
    overlaps = sum(1 for (s1, a1, b1) in spans for (s2, a2, b2) in spans if s1 < s2 and a1 < b2 and a2 < b1)
    assert overlaps >= 1, spans
    for sid in (0, 5):
        alone, _ = _serve(torch, rll, sc, [sid], arrivals, 10**12, max_items=2, cap=cap)
        assert np.array_equal(alone[sid]["rgb"], mix[sid]["rgb"])


def test_budget_admits_in_turn():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1911_10217_gb300 import rll, serving
    sc = _sessions()
    sizes = {sid: serving.session_bytes(s.n_lights, s.n_points, s.grid.table_size, s.grid.cut_size)
             for sid, s in sc.items()}
    arrivals = {sid: np.linspace(0.0, 0.01, 4) for sid in sc}
    budget = max(sizes.values()) + min(sizes.values())   # never all four at once
    res, log = _serve(torch, rll, sc, list(sc), arrivals, budget)
    assert len(log) == 16 and set(res) == set(sc)


def test_served_first_frames_equal_the_oracle():
    """Four sessions whose first frame is requested at once are served in
    shared launches; each session's estimate of that frame and its learned
    tables afterwards (Eq. 1, split-collapse, Eq. 2) equal the oracle's pass
    over that session alone: estimates and Q, C within 1e-4, cuts exact."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle import oracle as O
    from paper_1911_10217_gb300 import rll

    from .gpu_common import compare_tables, oracle_state
    sc = _sessions()
    arrivals = {sid: np.zeros(1) for sid in sc}
    res, log = _serve(torch, rll, sc, list(sc), arrivals, 10**12)
    assert len(log) == len(sc) and max(sum(1 for r in log if r.start == x.start) for x in log) > 1
    for sid, s in sc.items():
        ot = O.Tree(s.tris, s.emission)
        og = O.Grid.for_scene(ot, s)
        o = og.sample_frame(O.scene_arrays(s), s.seed, 0, s.spp)
        got = res[sid]["rgb"].astype(np.float64)
        assert np.allclose(got, o["rgb"], rtol=1e-4, atol=1e-7 * max(1.0, np.abs(o["rgb"]).max())), sid
        og.split_collapse(og.learn(o["slot"], o["s"], o["reward"]))
        compare_tables(res[sid]["grid"], oracle_state(og), og.m, 1e-4, check_cut=True)
