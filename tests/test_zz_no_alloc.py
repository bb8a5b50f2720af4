"""GPU test of rll_learn_update_noalloc, the learning step for callers that
cannot allocate device memory while they run (for example a host whose
device memory is all handed to its own pool): the same result as
rll_learn_update, on two consecutive passes (the second call runs on the
scratch contents the first one left), and a refusal above the size limit.

Runs alone in a fresh process or after the other tests: it builds its own
context, tree and grids.
"""
import ctypes

import numpy as np
import pytest

from paper_1911_10217_gb300 import scenes

from .gpu_common import RTOL, device_scene, params_for, run_sample

pytestmark = pytest.mark.gpu


def _state_rows(st, m):
    order = np.argsort(st["keys"])
    occ = st["keys"][order] != np.uint64(0xFFFFFFFFFFFFFFFF)
    idx = order[occ]
    return st["keys"][idx], st["cut"][idx, :m], st["q"][idx, :m], st["c"][idx, :m]


def test_noalloc_learning_matches_learn_update():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1911_10217_gb300 import rll
    dev = torch.device("cuda:0")
    ctx = rll.Context(0, torch.cuda.current_stream(dev))
    lib = rll.load()
    s = scenes.small_frame_scene()
    d = device_scene(s, dev)
    tree = rll.Tree(ctx, d["tri"], d["em"])
    ref = rll.Grid(ctx, tree, params_for(rll, s))
    alt = rll.Grid(ctx, tree, params_for(rll, s))
    for frame in range(2):
        out = run_sample(rll, ctx, ref, tree, d, s.seed, frame, s.spp)
        st = ref.export()
        alt.import_state(st["keys"], st["cut"], st["q"], st["c"])  # same state, same slots
        n = out["key"].shape[0]
        rll.learn_update(ctx, ref, out["key"], out["val"])
        rc = lib.rll_learn_update_noalloc(ctx.h, alt.h, out["key"].data_ptr(), out["val"].data_ptr(), n)
        assert rc == 0, lib.rll_last_error(ctx.h).decode()
        assert ctx.sync_status() == 0
        a = _state_rows(ref.export(), ref.m)
        b = _state_rows(alt.export(), alt.m)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
        assert np.allclose(a[2], b[2], rtol=RTOL["fp32"], atol=1e-12)
        assert np.allclose(a[3], b[3], rtol=RTOL["fp32"], atol=1e-12)
        rll.split_collapse(ctx, ref, tree)
    # above the limit: refused with a message, nothing launched
    big = (1 << 20) + 1
    rc = lib.rll_learn_update_noalloc(ctx.h, alt.h, ctypes.c_void_p(8), ctypes.c_void_p(8), big)
    assert rc == 1
    assert b"at most 1048576 records" in lib.rll_last_error(ctx.h)
    assert ctx.sync_status() == 0
