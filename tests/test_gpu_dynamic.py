"""Parity at the dynamic-lighting size (marked gpu): 2^20 emissive triangles
(10 % blinking), a 3840 x 2160 G-buffer, cut size 64, 2^21 cells, in the
launch configuration the benchmark times (the whole frame in one call).
The tree is compared bit-exactly; sampled pixel ranges of the frame are
compared with the oracle sample by sample (light, cell, cluster exact;
estimates, rewards and pdfs within 1e-4), for binary32 and 16-bit tables,
with the frame's blinking radiance."""
import numpy as np
import pytest

from paper_1911_10217_gb300 import scenes

from .gpu_common import (RTOL, compare_samples, compare_tables, oracle_state, params_for, rows_by_key, run_sample,
                         split_margin, to_host)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dyn():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle import oracle as O
    from paper_1911_10217_gb300 import rll
    dev = torch.device("cuda:0")
    ctx = rll.Context(0, torch.cuda.current_stream(dev))
    s = scenes.dynamic_scene()
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    bound = s.emission_bound()
    d = dict(tri=T(s.tris.reshape(-1, 9)), boxes=T(s.boxes), pos=T(s.pos), nrm=T(s.nrm), alb=T(s.albedo))
    dt = rll.Tree(ctx, d["tri"], T(bound))
    ot = O.Tree(s.tris, bound)
    return dict(torch=torch, O=O, rll=rll, ctx=ctx, dev=dev, s=s, d=d, dt=dt, ot=ot, T=T)


def test_dynamic_tree_bit_exact(dyn):
    ex, ot = dyn["dt"].export(), dyn["ot"]
    assert np.array_equal(ex["perm"], ot.perm)
    assert np.array_equal(ex["left"], ot.left) and np.array_equal(ex["right"], ot.right)
    assert np.array_equal(ex["rec"].view(np.uint32), ot.rec.view(np.uint32))


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_dynamic_frame_slices_match_oracle(dyn, precision):
    O, rll, ctx, s, d = dyn["O"], dyn["rll"], dyn["ctx"], dyn["s"], dyn["d"]
    ctx.sync_status()
    frame = 7
    em = s.emission_at(frame)
    dyn["dt"].update_emission(dyn["T"](em))
    dg = rll.Grid(ctx, dyn["dt"], params_for(rll, s, precision=precision))
    g = to_host(run_sample(rll, ctx, dg, dyn["dt"], d, s.seed, frame, s.spp))
    keys = dg.export()["keys"]
    og = O.Grid.for_scene(dyn["ot"], s, precision=precision)
    A = O.scene_arrays(s)
    rng = np.random.default_rng(11)
    P = s.n_points
    for start in rng.integers(0, P - 4096, size=4):
        o = og.sample_frame(A, s.seed, frame, s.spp, first=int(start), count=4096, emission=em)
        sl = slice(int(start), int(start) + 4096)
        gsub = {k: (v[:, sl] if k == "rgb" else v[sl]) for k, v in g.items()}
        compare_samples(gsub, o, keys, og.keys, dg.M)
    assert ctx.sync_status() == 0
    dg.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_dynamic_learned_state_fused_step(dyn, precision):
    """The call the benchmark times at this size, from a learned state: the
    oracle runs two learning passes (sampling with each frame's blinking
    radiance, Eq. 1, Eq. 2, split-collapse) over the whole 3840 x 2160 frame
    on its own; its state is imported, pass 2 is compared sample by sample
    over the whole frame, then the device's fused rll_learn_update_split on
    its own records is compared with the oracle's learn + split-collapse on
    every touched cell (cut size 64; cells of more than 240 records take the
    two-warp and block teams): cuts exact, Q and C within the table
    tolerance (1e-4 for binary32, 2e-2 for bfloat16 tables). A split
    decision within the rounding of Eq. 1 in the oracle's own state may go the
    other way; every such cell is checked to be a near-tie (relative gap at
    most 1e-5, or two bfloat16 roundings) and left out. They are more frequent than at 1080p (here at
    most 2 %, measured 0.9 %): with 64-leaf cuts after two passes many leaves
    have seen the same few updates, so their Q values tie exactly in the
    oracle's double arithmetic (broken by range order) and differ only by
    binary32 rounding on the device."""
    O, rll, ctx, s, d, torch = dyn["O"], dyn["rll"], dyn["ctx"], dyn["s"], dyn["d"], dyn["torch"]
    ctx.sync_status()
    ot, dt = dyn["ot"], dyn["dt"]
    og = O.Grid.for_scene(ot, s, precision=precision)
    A = O.scene_arrays(s)
    K = 2
    for f in range(K):
        o = og.sample_frame(A, s.seed, f, s.spp, emission=s.emission_at(f))
        og.split_collapse(og.learn(o["slot"], o["s"], o["reward"]))
    em = s.emission_at(K)
    dt.update_emission(dyn["T"](em))
    dg = rll.Grid(ctx, dt, params_for(rll, s, precision=precision))
    dg.import_state(og.keys, og.cut, og.Q, og.C)
    g = to_host(run_sample(rll, ctx, dg, dt, d, s.seed, K, s.spp))
    o = og.sample_frame(A, s.seed, K, s.spp, emission=em)
    skip = compare_samples(g, o, dg.export()["keys"], og.keys, dg.M)
    rll.learn_update_split(ctx, dg, dt, torch.from_numpy(g["key"]).to(dyn["dev"]),
                           torch.from_numpy(g["val"]).to(dyn["dev"]))
    touched = og.learn(o["slot"], o["s"], o["reward"])
    m = og.m
    pre = {int(og.keys[sl]): (og.cut[sl, :m].copy(), og.Q[sl, :m].copy()) for sl in np.nonzero(touched)[0]}
    changed = og.split_collapse(touched)
    assert dg.touched_cells() == int(touched.sum())
    assert changed > 100
    st = dg.export()
    g_rows = rows_by_key(st["keys"], st["cut"])
    o_rows = rows_by_key(og.keys, og.cut)
    flipped = {k for k in o_rows if k in g_rows and not np.array_equal(g_rows[k][0][:m], o_rows[k][0][:m])}
    tol = {"fp32": 1e-5, "bf16": 2 * 2.0 ** -8}[precision]
    for k in flipped:
        assert k in pre and split_margin(*pre[k], ot.parent, ot.n, s.grid.threshold) <= tol, k
    assert len(flipped) <= max(2, len(pre) // 50), len(flipped)
    compare_tables(st, oracle_state(og), m, RTOL[precision], check_cut=True, skip=skip | flipped)
    assert ctx.sync_status() == 0
    dg.close()


@pytest.mark.parametrize("builder", ["saoh", "median"])
def test_dynamic_tree_other_builders_bit_exact(dyn, builder):
    """The surface-area-orientation and median-split builders at 2^20 lights:
    light order, topology and node records bit-exact with the oracle's."""
    O, rll, ctx, s = dyn["O"], dyn["rll"], dyn["ctx"], dyn["s"]
    bound = s.emission_bound()
    dt = rll.Tree(ctx, dyn["d"]["tri"], dyn["T"](bound), builder=builder)
    ot = O.Tree(s.tris, bound, builder=builder)
    ex = dt.export()
    assert np.array_equal(ex["perm"], ot.perm)
    assert np.array_equal(ex["left"], ot.left) and np.array_equal(ex["right"], ot.right)
    assert np.array_equal(ex["rec"].view(np.uint32), ot.rec.view(np.uint32))
    dt.close()
