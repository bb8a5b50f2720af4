"""GPU test of rll_learn_update_noalloc, the learning step for callers that
cannot allocate device memory while they run (for example a host whose
device memory is all handed to its own pool): the same result as
rll_learn_update, on two consecutive passes (the second call runs on the
scratch contents the first one left), for every table precision; the
touched cells it records drive rll_split_collapse exactly as those of
rll_learn_update do; no device memory is taken by a call; and a refusal above
the size limit.

Runs alone in a fresh process or after the other tests: it builds its own
context, tree and grids.
"""
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


def _same(ref, alt, rtol):
    a = _state_rows(ref.export(), ref.m)
    b = _state_rows(alt.export(), alt.m)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert np.allclose(a[2], b[2], rtol=rtol, atol=1e-12)
    assert np.allclose(a[3], b[3], rtol=rtol, atol=1e-12)


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1911_10217_gb300 import rll
    dev = torch.device("cuda:0")
    ctx = rll.Context(0, torch.cuda.current_stream(dev))
    return dict(torch=torch, rll=rll, dev=dev, ctx=ctx, lib=rll.load())


@pytest.mark.parametrize("precision", ["fp32", "fp16", "bf16"])
def test_noalloc_learning_matches_learn_update(env, precision):
    torch, rll, ctx, lib = env["torch"], env["rll"], env["ctx"], env["lib"]
    ctx.sync_status()
    s = scenes.small_frame_scene()
    d = device_scene(s, env["dev"])
    tree = rll.Tree(ctx, d["tri"], d["em"])
    ref = rll.Grid(ctx, tree, params_for(rll, s, precision=precision))
    alt = rll.Grid(ctx, tree, params_for(rll, s, precision=precision))
    rtol = RTOL[precision]
    for frame in range(2):
        out = run_sample(rll, ctx, ref, tree, d, s.seed, frame, s.spp)
        st = ref.export()
        alt.import_state(st["keys"], st["cut"], st["q"], st["c"])  # same state, same slots
        n = out["key"].shape[0]
        rll.learn_update(ctx, ref, out["key"], out["val"])
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info(env["dev"])[0]
        rc = lib.rll_learn_update_noalloc(ctx.h, alt.h, out["key"].data_ptr(), out["val"].data_ptr(), n)
        assert rc == 0, lib.rll_last_error(ctx.h).decode()
        assert ctx.sync_status() == 0
        if frame > 0:  # after the first call's one-time set-up, a call takes no device memory
            assert torch.cuda.mem_get_info(env["dev"])[0] == free0
        assert alt.touched_cells() == ref.touched_cells()
        _same(ref, alt, rtol)
        # split-collapse reads the touched cells each learning call left behind
        rll.split_collapse(ctx, ref, tree)
        rll.split_collapse(ctx, alt, tree)
        assert ctx.sync_status() == 0
        _same(ref, alt, max(rtol, 1e-5))


def test_noalloc_refuses_more_than_its_limit(env):
    """Above the limit the call is refused with a message before anything is
    launched (real device buffers are passed, so a launch would still stay in
    bounds)."""
    torch, rll, ctx, lib = env["torch"], env["rll"], env["ctx"], env["lib"]
    ctx.sync_status()
    s = scenes.tiny_scene()
    d = device_scene(s, env["dev"])
    tree = rll.Tree(ctx, d["tri"], d["em"])
    grid = rll.Grid(ctx, tree, params_for(rll, s))
    big = (1 << 20) + 1
    key = torch.full((big,), -1, dtype=torch.int32, device=env["dev"])  # 0xFFFFFFFF: no cell
    val = torch.zeros(big, device=env["dev"])
    rc = lib.rll_learn_update_noalloc(ctx.h, grid.h, key.data_ptr(), val.data_ptr(), big)
    assert rc == 1
    assert b"at most 1048576 records" in lib.rll_last_error(ctx.h)
    assert ctx.sync_status() == 0
