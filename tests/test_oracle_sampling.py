"""Pins of the oracle's estimator (Section 3 sampling, Section 4 baseline).

- the pdf over all lights sums to one and equals p_cut * p_in for every draw;
- sampled light frequencies follow that pdf (chi-square);
- cut = all lights, Q = power, uniform in-cluster choice reduces to the
  energy-based sampler of Section 4;
- the brute-force direct lighting (quadrature) agrees with Lambert's closed
  form for polygon irradiance when nothing is occluded;
- the estimator is unbiased for the brute-force value, fresh and learned;
- learning reduces the error at equal sample count (Section 4).
"""
import math

import numpy as np
import pytest
from scipy import stats

from paper_1911_10217_gb300 import scenes


def _repeat_point(scene, idx, count):
    """A G-buffer made of one shading point repeated `count` times."""
    pos = np.repeat(scene.pos[:, idx:idx + 1], count, axis=1)
    nrm = np.repeat(scene.nrm[:, idx:idx + 1], count, axis=1)
    alb = np.repeat(scene.albedo[idx:idx + 1], count)
    return pos, nrm, alb


def _arrays(scene, pos, nrm, alb):
    return (np.ascontiguousarray(scene.tris.reshape(-1, 9)), scene.emission,
            np.ascontiguousarray(scene.boxes), np.ascontiguousarray(pos), np.ascontiguousarray(nrm),
            np.ascontiguousarray(alb))


def _learned_grid(oracle_mod, scene, tree, iters=4, **kw):
    g = oracle_mod.Grid.for_scene(tree, scene, **kw)
    A = oracle_mod.scene_arrays(scene)
    for f in range(iters):
        out = g.sample_frame(A, scene.seed, f, scene.spp)
        touched = g.learn(out["slot"], out["s"], out["reward"])
        g.split_collapse(touched)
    return g


@pytest.fixture(scope="module")
def tiny(oracle_mod):
    s = scenes.tiny_scene()
    return s, oracle_mod.Tree(s.tris, s.emission)


@pytest.mark.parametrize("mode", ["descent", "uniform", "descent2"])
def test_pdf_sums_to_one(oracle_mod, tiny, mode):
    s, tree = tiny
    g = _learned_grid(oracle_mod, s, tree, iters=3, mode=mode)
    rng = np.random.default_rng(0)
    for idx in rng.integers(0, s.n_points, size=6):
        x, n = s.pos[:, idx], s.nrm[:, idx]
        slot = g.lookup_insert(g.cell_key(x, n))
        p = np.array([g.light_pdf(slot, x, n, l) for l in range(tree.n)])
        assert p.sum() == pytest.approx(1.0, abs=1e-9)
        assert np.all(p > 0)  # the floor keeps every light reachable


@pytest.mark.parametrize("mode", ["descent", "uniform", "descent2"])
def test_sample_pdf_is_cut_times_descent(oracle_mod, tiny, mode):
    s, tree = tiny
    g = _learned_grid(oracle_mod, s, tree, iters=2, mode=mode)
    A = oracle_mod.scene_arrays(s)
    out = g.sample_frame(A, 7, 99, 2, first=1000, count=300)
    for r in range(0, 600, 7):
        i = 1000 + r // 2
        x, n = s.pos[:, i], s.nrm[:, i]
        p = g.light_pdf(int(out["slot"][r]), x, n, int(out["light"][r]))
        assert out["p_cut"][r] * out["p_in"][r] == pytest.approx(p, rel=1e-12)


@pytest.mark.parametrize("mode", ["descent", "descent2"])
def test_light_frequencies_follow_pdf(oracle_mod, tiny, mode):
    s, tree = tiny
    g = _learned_grid(oracle_mod, s, tree, iters=3, mode=mode)
    idx = 64 * 20 + 17
    R = 200_000
    pos, nrm, alb = _repeat_point(s, idx, R)
    out = g.sample_frame(_arrays(s, pos, nrm, alb), 3, 0, 1)
    slot = int(out["slot"][0])
    assert np.all(out["slot"] == slot)
    x, n = s.pos[:, idx], s.nrm[:, idx]
    p = np.array([g.light_pdf(slot, x, n, l) for l in range(tree.n)])
    counts = np.bincount(out["light"], minlength=tree.n)
    exp = p * R
    keep = exp >= 5
    chi2 = np.sum((counts[keep] - exp[keep]) ** 2 / exp[keep]) + \
        (counts[~keep].sum() - exp[~keep].sum()) ** 2 / max(exp[~keep].sum(), 1e-9)
    dof = keep.sum()
    assert stats.chi2.sf(chi2, dof) > 1e-6, (chi2, dof)


def test_full_cut_with_power_is_energy_sampler(oracle_mod, tiny):
    """M = N, Q = power, eps = 0 and uniform in-cluster choice give the pdf
    phi_l / sum(phi) of the energy-based sampler (Section 4)."""
    s, tree = tiny
    g = oracle_mod.Grid.for_scene(tree, s, cut_size=256, mode="uniform", eps=0.0)
    assert g.m == tree.n
    x, n = s.pos[:, 100], s.nrm[:, 100]
    slot = g.lookup_insert(g.cell_key(x, n))
    phi = tree.phi64[tree.n - 1 + np.arange(tree.n)]
    cut_leaf = g.cut[slot, :g.m] - (tree.n - 1)
    g.Q[slot, :g.m] = phi[cut_leaf]
    g.C[slot, :g.m] = oracle_mod.cdf(g.Q[slot, :g.m], eps=0.0)
    p = np.array([g.light_pdf(slot, x, n, l) for l in range(tree.n)])
    # C is stored in binary32: C(s) - C(s-1) carries ulp(C(m-1)) / p of error
    assert np.allclose(p, phi / phi.sum(), rtol=1e-4)
    # and the power sampler's draws use the same pdf
    A = oracle_mod.scene_arrays(s)
    rgb, light = oracle_mod.sample_power(tree, A, 0, 0, 1, first=0, count=2000)
    assert light.min() >= 0 and light.max() < tree.n


def _lambert_irradiance(x, n, tri):
    """Lambert's formula: E/L = 1/2 sum_i theta_i (n . gamma_i) for a polygon
    above the tangent plane (textbook closed form)."""
    R = [np.asarray(v, np.float64) - x for v in tri]
    tot = 0.0
    for i in range(3):
        a, b = R[i], R[(i + 1) % 3]
        g = np.cross(a, b)
        g /= np.linalg.norm(g)
        th = math.acos(np.clip(a @ b / np.linalg.norm(a) / np.linalg.norm(b), -1, 1))
        tot += th * (n @ g)
    return abs(0.5 * tot)


def test_quadrature_matches_lambert(oracle_mod):
    rng = np.random.default_rng(1)
    x = np.array([0.4, 0.0, 0.6], np.float32)
    n = np.array([0, 1, 0], np.float32)
    for trial in range(6):
        c = rng.uniform([0.1, 0.3, 0.1], [0.9, 0.9, 0.9])
        tri = c + rng.uniform(-0.15, 0.15, size=(3, 3)) * [1, 0.2, 1]
        e = np.cross(tri[1] - tri[0], tri[2] - tri[0])
        if e[1] > 0:  # make it face down, towards the point
            tri = tri[[0, 2, 1]]
        tri = tri.astype(np.float32)
        le = np.array([[1.0, 2.0, 0.5]], np.float32)
        got = oracle_mod.direct_bruteforce(x, n, math.pi, tri[None], le, np.zeros((0, 6)), level=7)
        E = _lambert_irradiance(x.astype(np.float64), n.astype(np.float64), tri.astype(np.float64))
        assert got == pytest.approx(E * le[0], rel=2e-4)


def _mean_and_se(v):
    return v.mean(), v.std(ddof=1) / math.sqrt(v.size)


@pytest.mark.parametrize("variant", ["fresh", "learned", "uniform", "fp16", "jitter", "descent2"])
def test_estimator_unbiased(oracle_mod, variant):
    s = scenes.tiny_scene(jitter=(variant == "jitter"))
    tree = oracle_mod.Tree(s.tris, s.emission)
    kw = {}
    if variant in ("uniform", "descent2"):
        kw["mode"] = variant
    if variant == "fp16":
        kw["precision"] = "fp16"
    iters = 0 if variant == "fresh" else 4
    g = _learned_grid(oracle_mod, s, tree, iters=iters, **kw)
    R = 60_000
    for idx in (64 * 16 + 16, 64 * 40 + 50, 64 * 5 + 60):
        pos, nrm, alb = _repeat_point(s, idx, R)
        out = g.sample_frame(_arrays(s, pos, nrm, alb), 11, 1000, 1)
        ref = oracle_mod.direct_bruteforce(s.pos[:, idx], s.nrm[:, idx], s.albedo[idx],
                                           s.tris, s.emission, s.boxes, level=5)
        for k in range(3):
            m, se = _mean_and_se(out["rgb"][k])
            assert abs(m - ref[k]) < 5 * se + 2e-3 * ref[k] + 1e-9, (variant, idx, k, m, ref[k], se)


def _image_mse(oracle_mod, s, tree, g, ref, frame):
    out = g.sample_frame(oracle_mod.scene_arrays(s), s.seed, frame, s.spp)
    return float(np.mean((out["rgb"] - ref) ** 2)), out


def test_learning_reduces_error(oracle_mod):
    """At equal spp the learned distributions beat both the fresh cut and the
    energy-based sampler on the walled-cells scene (Section 4)."""
    s = scenes.tiny_scene()
    tree = oracle_mod.Tree(s.tris, s.emission)
    rng = np.random.default_rng(2)
    idx = rng.choice(s.n_points, size=256, replace=False)
    sub = scenes.Scene("sub", s.tris, s.emission, s.boxes, s.pos[:, idx].copy(), s.nrm[:, idx].copy(),
                       s.albedo[idx].copy(), s.grid, s.spp, s.frames, s.seed)
    ref = np.stack([oracle_mod.direct_bruteforce(sub.pos[:, i], sub.nrm[:, i], sub.albedo[i],
                                                 s.tris, s.emission, s.boxes, level=4)
                    for i in range(256)], axis=1)
    g = oracle_mod.Grid.for_scene(tree, s)
    A = oracle_mod.scene_arrays(s)
    mse0, _ = _image_mse(oracle_mod, sub, tree, g, ref, 500)
    for f in range(s.frames):
        out = g.sample_frame(A, s.seed, f, s.spp)
        touched = g.learn(out["slot"], out["s"], out["reward"])
        g.split_collapse(touched)
    mse_learned = np.mean([_image_mse(oracle_mod, sub, tree, g, ref, 600 + k)[0] for k in range(4)])
    rgb_p, _ = oracle_mod.sample_power(tree, oracle_mod.scene_arrays(sub), s.seed, 700, s.spp)
    mse_power = float(np.mean((rgb_p - ref) ** 2))
    assert mse_learned < 0.5 * mse0, (mse_learned, mse0)
    assert mse_learned < 0.5 * mse_power, (mse_learned, mse_power)


def test_estimator_unbiased_sky_dome(oracle_mod):
    """The sky-dome interior (far, large, inward-facing dome triangles and a
    small bright distant quad, light entering only through small openings):
    the learned estimator's mean equals brute-force direct lighting."""
    s = scenes.tiny_sky_scene()
    tree = oracle_mod.Tree(s.tris, s.emission)
    g = _learned_grid(oracle_mod, s, tree, iters=4)
    R = 100_000
    for idx in (64 * 10 + 10, 64 * 50 + 20):
        pos, nrm, alb = _repeat_point(s, idx, R)
        out = g.sample_frame(_arrays(s, pos, nrm, alb), 13, 1000, 1)
        ref = oracle_mod.direct_bruteforce(s.pos[:, idx], s.nrm[:, idx], s.albedo[idx],
                                           s.tris, s.emission, s.boxes, level=7)
        for k in range(3):
            m, se = _mean_and_se(out["rgb"][k])
            assert abs(m - ref[k]) < 5 * se + 3e-3 * ref[k] + 1e-9, (idx, k, m, ref[k], se)


def test_two_level_step_over_two_leaves_is_the_binary_step(oracle_mod):
    """When both children of a node are single lights the two-level step has
    the same two candidates as the binary step, with weights in the same
    ratio: the light pdfs of the two modes agree (to rounding)."""
    s = scenes.tiny_scene()
    tree = oracle_mod.Tree(s.tris, s.emission)
    n = tree.n
    # cut nodes whose two children are both leaves: the cut of n/2 nodes of the
    # balanced bottom level exists when cut_size = n / 2 covers it
    g1 = oracle_mod.Grid.for_scene(tree, s, cut_size=128, mode="descent")
    g2 = oracle_mod.Grid.for_scene(tree, s, cut_size=128, mode="descent2")
    cut = g1.def_cut
    pairs = [c for c in cut if c < n - 1 and tree.left[c] >= n - 1 and tree.right[c] >= n - 1]
    assert len(pairs) > 10
    rng = np.random.default_rng(2)
    for idx in rng.integers(0, s.n_points, size=4):
        x, nn = s.pos[:, idx], s.nrm[:, idx]
        s1 = g1.lookup_insert(g1.cell_key(x, nn))
        s2 = g2.lookup_insert(g2.cell_key(x, nn))
        for c in pairs[:20]:
            for leaf in (tree.left[c], tree.right[c]):
                l = leaf - (n - 1)
                assert g2.light_pdf(s2, x, nn, l) == pytest.approx(g1.light_pdf(s1, x, nn, l), rel=1e-6)
