"""GPU test of the serving loop: sessions served concurrently in shared
batched launches give, session by session, exactly the results of serving
that session alone."""
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


def _serve(torch, rll, sc, sids, arrivals, budget):
    from paper_1911_10217_gb300 import serving
    dev = torch.device("cuda:0")
    ex = serving.GpuExecutor(torch, rll, dev, max_items=8, max_records=1 << 16, max_cells=1 << 16, keep_results=True)
    sched = serving.Scheduler(budget, 8, 1 << 16, 1 << 16)
    for sid in sids:
        s = sc[sid]
        sched.add_session(sid, serving.session_bytes(s.n_lights, s.n_points, s.grid.table_size, s.grid.cut_size),
                          s.n_points * s.spp, s.grid.table_size, len(arrivals[sid]))
    log = serving.serve(ex, sched, {k: sc[k] for k in sids}, {k: arrivals[k] for k in sids})
    assert all(st == 0 for st in ex.status())
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
