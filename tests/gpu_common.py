"""Shared helpers of the GPU tests: device copies of a scene, one pass through
the C ABI, comparisons against the oracle keyed by cell key."""
import numpy as np

# tolerance on learned values and cdfs per table precision: binary32 is the
# stated 1e-4 relative; a 16-bit table adds one rounding of its format
# (2^-11 for binary16, 2^-8 for bfloat16) on each side
RTOL = {"fp32": 1e-4, "fp16": 2.5e-3, "bf16": 2e-2}


def device_scene(scene, dev, emission=None):
    import torch
    t = lambda a, dt=None: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    d = dict(tri=t(scene.tris.reshape(-1, 9)), em=t(scene.emission if emission is None else emission),
             boxes=t(scene.boxes), pos=t(scene.pos), nrm=t(scene.nrm), alb=t(scene.albedo))
    if scene.footprint is not None:
        d["fp"] = t(scene.footprint)
    return d


def params_for(rll, scene, **kw):
    return rll.grid_params_for(scene.grid, **kw)


def run_sample(rll, ctx, grid, tree, d, seed, frame, spp):
    import torch
    dev = d["pos"].device
    P = d["alb"].shape[0]
    out = dict(rgb=torch.empty(3, P, device=dev),
               key=torch.empty(P * spp, dtype=torch.int32, device=dev),
               val=torch.empty(P * spp, device=dev),
               light=torch.empty(P * spp, dtype=torch.int32, device=dev),
               pcut=torch.empty(P * spp, device=dev), pin=torch.empty(P * spp, device=dev))
    rll.sample_and_shade(ctx, grid, tree, d["pos"], d["nrm"], d["alb"], d["boxes"], seed, frame, spp,
                         out["rgb"], out["key"], out["val"], dbg_light=out["light"],
                         dbg_pcut=out["pcut"], dbg_pin=out["pin"], footprint=d.get("fp"))
    return out


def to_host(out):
    return {k: v.cpu().numpy() for k, v in out.items()}


def compare_samples(gpu, orc, gpu_keys, orc_keys, M, rtol=1e-4):
    """Light index bit-exact except draws within 1e-6 of a threshold (at most
    1e-5 of the samples, rounded down: none below 10^5 samples); the same cell
    key and cluster; estimates and rewards within rtol. The estimate of every
    point whose samples all agree is compared. Returns the set of cell keys a
    mismatched sample fed on either side (empty when the light choices all
    agree): the cells whose learned rows may then legitimately differ."""
    light_g = gpu["light"].astype(np.int64)
    n = light_g.size
    mism = light_g != orc["light"]
    near = orc["margin"] < 1e-6
    assert not np.any(mism & ~near), f"{int(np.sum(mism & ~near))} light choices differ away from a boundary"
    assert mism.sum() <= int(1e-5 * n), f"{int(mism.sum())} boundary mismatches of {n}"
    ok = ~mism
    kg = gpu["key"].view(np.uint32).astype(np.int64)
    slot_g = np.where(kg == 0xFFFFFFFF, -1, kg // M)
    s_g = np.where(kg == 0xFFFFFFFF, -1, kg % M)
    cell_g = np.where(slot_g >= 0, gpu_keys[np.maximum(slot_g, 0)], np.uint64(0))
    cell_o = np.where(orc["slot"] >= 0, orc_keys[np.maximum(orc["slot"], 0)], np.uint64(0))
    assert np.array_equal(cell_g[ok], cell_o[ok]), "cell keys differ"
    assert np.array_equal(s_g[ok], orc["s"][ok]), "clusters differ"
    rv = gpu["val"].astype(np.float64)
    assert np.allclose(rv[ok], orc["reward"][ok], rtol=rtol, atol=1e-7 * max(1.0, np.abs(orc["reward"]).max())), \
        "rewards differ"
    pdf_g = gpu["pcut"].astype(np.float64) * gpu["pin"]
    pdf_o = orc["p_cut"] * orc["p_in"]
    assert np.allclose(pdf_g[ok], pdf_o[ok], rtol=rtol), "pdfs differ"
    P = gpu["rgb"].shape[1]
    spp = n // max(P, 1)
    pt_ok = ok.reshape(P, spp).all(axis=1) if P else np.zeros(0, bool)
    assert np.allclose(gpu["rgb"][:, pt_ok], orc["rgb"][:, pt_ok], rtol=rtol,
                       atol=1e-7 * max(1.0, np.abs(orc["rgb"]).max())), "estimates differ"
    skip = set()
    for i in np.nonzero(mism)[0]:
        for c in (cell_g[i], cell_o[i]):
            skip.add(int(c))
    return skip


def rows_by_key(keys, *tables, Hl=None):
    """Occupied rows by cell key (by (level, key) when Hl, the slots per
    resolution level, is given: keys of different levels may coincide)."""
    occ = np.nonzero(keys != np.uint64(0xFFFFFFFFFFFFFFFF))[0]
    if Hl is None:
        return {int(keys[i]): tuple(t[i] for t in tables) for i in occ}
    return {(int(i) // Hl, int(keys[i])): tuple(t[i] for t in tables) for i in occ}


def compare_tables(gstate, ostate, m, rtol, check_cut=True, only=None, Hl=None, skip=()):
    """Compare two grid states cell by cell (matched by key, or by level and
    key for a multi-resolution grid). Cells in `skip` (those fed by a
    boundary-mismatched sample) are left out; at most a handful, checked."""
    g = rows_by_key(gstate["keys"], gstate["cut"], gstate["q"], gstate["c"], Hl=Hl)
    o = rows_by_key(ostate["keys"], ostate["cut"], ostate["q"], ostate["c"], Hl=Hl)
    assert set(g) == set(o), f"cell sets differ: {len(set(g) ^ set(o))}"
    keys = o.keys() if only is None else only
    assert len(skip) <= max(2, len(o) // 100), f"{len(skip)} cells left out"
    for k in keys:
        if (k[1] if isinstance(k, tuple) else k) in skip:
            continue
        gc, gq, gcc = g[k]
        oc, oq, occ = o[k]
        if check_cut:
            assert np.array_equal(gc[:m], oc[:m]), f"cut differs in cell {k}"
        assert np.allclose(gq[:m], oq[:m], rtol=rtol, atol=1e-12), f"Q differs in cell {k}"
        assert np.allclose(gcc[:m], occ[:m], rtol=rtol, atol=1e-12), f"C differs in cell {k}"


def split_margin(cut, q, parent, n_lights, T):
    """Smallest relative gap among the decisions split-collapse takes on one
    row: the leaf of largest Q (not a single light) against the runner-up,
    the parent of two cut leaves with the smallest Q sum against the
    runner-up, and Q(l_max) against T Q(p_min). An exact tie is a gap of 0:
    values equal in the oracle may differ by an ulp on the device. When the
    smallest gap is within the rounding of Eq. 1 (binary32 on the device,
    double in the oracle), either outcome is correct."""
    q = np.asarray(q, np.float64)
    m = len(cut)
    gaps = [np.inf]
    cand = sorted((q[i] for i in range(m) if cut[i] < n_lights - 1), reverse=True)
    if len(cand) > 1 and cand[0] > 0:
        gaps.append((cand[0] - cand[1]) / cand[0])
    sums = sorted(float(np.float32(q[i]) + np.float32(q[i + 1])) for i in range(m - 1)
                  if parent[cut[i]] >= 0 and parent[cut[i]] == parent[cut[i + 1]])
    if len(sums) > 1 and sums[1] > 0:
        gaps.append((sums[1] - sums[0]) / sums[1])
    if cand and sums and cand[0] > 0:
        gaps.append(abs(cand[0] - T * sums[0]) / cand[0])
    return min(gaps)


def oracle_state(og):
    return dict(keys=og.keys.copy(), cut=og.cut.copy(), q=og.Q.copy(), c=og.C.copy())


def clone_oracle_grid(O, og):
    p = og.params
    g2 = O.Grid(og.tree, og.H, og.M, origin=p["origin"], cell_size=p["cell_size"],
                normal_bins=p["normal_bins"], jitter=p["jitter"], mode=p["mode"], reward=p["reward"],
                precision=p["precision"], alpha=p["alpha"], T=p["T"], eps=p["eps"], q_init=p["q_init"],
                split_iterations=p["split_iterations"])
    g2.copy_state_from(og.keys, og.cut, og.Q, og.C)
    return g2
