"""Precision form against the FP64 oracle: after learning a dynamic
(blinking) scene with FP32, FP16 and BF16 tables, the device estimate at
sampled points is unbiased for the oracle's brute-force direct lighting,
and the 16-bit tables' per-sample variance stays close to FP32's.
Set RLL_REPORT_DIR to write the measured bias and variance as JSON."""
import json
import os

import numpy as np
import pytest

from paper_1911_10217_gb300 import scenes

from .gpu_common import device_scene, params_for

pytestmark = pytest.mark.gpu


def test_16bit_tables_unbiased_vs_oracle():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle import oracle as O
    from paper_1911_10217_gb300 import rll
    dev = torch.device("cuda:0")
    ctx = rll.Context(0, torch.cuda.current_stream(dev))
    s = scenes.dynamic_scene(seed=5, width=192, height=108, n_patches=64, tris_per_patch=64, table_size=1 << 14)
    d = device_scene(s, dev, emission=s.emission_bound())
    tree = rll.Tree(ctx, d["tri"], d["em"])
    frames = 24
    em_last = s.emission_at(frames - 1)
    rng = np.random.default_rng(3)
    pts = rng.choice(s.n_points, 6, replace=False)
    ref = [O.direct_bruteforce(s.pos[:, i], s.nrm[:, i], s.albedo[i], s.tris, em_last, s.boxes, level=3) for i in pts]
    R = 1 << 18
    report = {}
    var = {}
    for prec in ("fp32", "fp16", "bf16"):
        grid = rll.Grid(ctx, tree, params_for(rll, s, precision=prec))
        P = s.n_points
        rgb = torch.empty(3, P, device=dev)
        key = torch.empty(P, dtype=torch.int32, device=dev)
        val = torch.empty(P, device=dev)
        for f in range(frames):
            tree.update_emission(torch.from_numpy(s.emission_at(f)).to(dev))
            rll.sample_and_shade(ctx, grid, tree, d["pos"], d["nrm"], d["alb"], d["boxes"], s.seed, f, 1, rgb,
                                 key, val)
            rll.learn_update(ctx, grid, key, val)
            rll.split_collapse(ctx, grid, tree)
        rows = []
        for k, i in enumerate(pts):
            pos = d["pos"][:, i:i + 1].repeat(1, R).contiguous()
            nrm = d["nrm"][:, i:i + 1].repeat(1, R).contiguous()
            alb = d["alb"][i:i + 1].repeat(R).contiguous()
            out = torch.empty(3, R, device=dev)
            rll.sample_and_shade(ctx, grid, tree, pos, nrm, alb, d["boxes"], 77, 10**6, 1, out)
            lum = (torch.tensor([0.2126, 0.7152, 0.0722], device=dev, dtype=torch.float64) @ out.double())
            m, sd = float(lum.mean()), float(lum.std())
            r = float(np.dot([0.2126, 0.7152, 0.0722], ref[k]))
            assert abs(m - r) <= 5 * sd / np.sqrt(R) + 2e-3 * r + 1e-12, (prec, int(i), m, r, sd)
            rows.append(dict(point=int(i), oracle=r, mean=m, rel_bias=(m - r) / r if r > 0 else 0.0,
                             std_err=sd / np.sqrt(R), sample_var=sd * sd))
        var[prec] = np.array([x["sample_var"] for x in rows])
        report[prec] = rows
        grid.close()
    lit = var["fp32"] > 0
    for prec in ("fp16", "bf16"):
        ratio = var[prec][lit] / var["fp32"][lit]
        assert np.all(ratio < 4.0), (prec, ratio)
    assert ctx.sync_status() == 0
    out_dir = os.environ.get("RLL_REPORT_DIR")
    if out_dir:
        with open(os.path.join(out_dir, "precision_vs_oracle.json"), "w") as f:
            json.dump(report, f, indent=1)
