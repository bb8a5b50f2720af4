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

from .gpu_common import compare_samples, params_for, run_sample, to_host

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
