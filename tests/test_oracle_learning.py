"""Pins of the oracle's learning step: Eq. 1, Eq. 2, table rounding and
split-collapse (Section 3, Fig. "TreeCuts", Section 3.1)."""
import json
import os

import numpy as np
import pytest
import torch

from paper_1911_10217_gb300 import scenes

from .test_oracle_tree import _grid_lights


def _single_cell_grid(oracle_mod, alpha=0.1, precision="fp32", eps=0.01, M=8):
    tris, em = _grid_lights(4)
    tree = oracle_mod.Tree(tris, em)
    g = oracle_mod.Grid(tree, table_size=16, cut_size=M, alpha=alpha, precision=precision, eps=eps)
    slot = g.lookup_insert(12345)
    assert slot >= 0
    return g, slot


def test_eq1_closed_form(oracle_mod):
    """After n updates with rewards c_1..c_n, Eq. 1 gives
    Q_n = (1-a)^n Q_0 + a sum_i (1-a)^(n-i) c_i."""
    rng = np.random.default_rng(0)
    a = 0.1
    g, slot = _single_cell_grid(oracle_mod, alpha=a)
    c = rng.exponential(size=37)
    q0 = g.Q[slot, 3]
    g.learn(np.full(37, slot), np.full(37, 3), c)
    n = len(c)
    expect = (1 - a) ** n * q0 + a * np.sum((1 - a) ** (n - np.arange(1, n + 1)) * c)
    assert g.Q[slot, 3] == pytest.approx(expect, rel=1e-7)
    # other leaves untouched
    assert g.Q[slot, 2] == q0


def test_eq1_interleaved_keys_follow_sample_order(oracle_mod):
    rng = np.random.default_rng(1)
    a = 0.25
    g, slot = _single_cell_grid(oracle_mod, alpha=a)
    s = rng.integers(0, 8, size=200)
    c = rng.uniform(0, 3, size=200)
    q0 = g.Q[slot].copy()
    g.learn(np.full(200, slot), s, c)
    for leaf in range(8):
        ci = c[s == leaf]
        n = len(ci)
        expect = (1 - a) ** n * q0[leaf] + a * np.sum((1 - a) ** (n - np.arange(1, n + 1)) * ci)
        assert g.Q[slot, leaf] == pytest.approx(expect, rel=1e-7)


def test_eq1_constant_reward_converges(oracle_mod):
    g, slot = _single_cell_grid(oracle_mod, alpha=0.3)
    g.learn(np.full(400, slot), np.zeros(400, np.int32), np.full(400, 2.5))
    assert g.Q[slot, 0] == pytest.approx(2.5, rel=1e-6)


def test_eq1_alpha_zero_freezes(oracle_mod):
    g, slot = _single_cell_grid(oracle_mod, alpha=0.0)
    q0 = g.Q[slot].copy()
    g.learn(np.full(10, slot), np.arange(10) % 8, np.arange(10, dtype=np.float64))
    assert np.array_equal(g.Q[slot], q0)


def test_records_without_cell_are_ignored(oracle_mod):
    g, slot = _single_cell_grid(oracle_mod)
    q0 = g.Q.copy()
    touched = g.learn(np.array([-1, -1]), np.array([0, 1]), np.array([5.0, 6.0]))
    assert not touched.any() and np.array_equal(g.Q, q0)


def test_eq2_prefix_sum(oracle_mod):
    rng = np.random.default_rng(2)
    q = rng.uniform(0, 2, size=32)
    c = oracle_mod.cdf(q, eps=0.0)
    assert np.allclose(c, np.cumsum(q).astype(np.float32).astype(np.float64), rtol=1e-7)
    c = oracle_mod.cdf(q, eps=0.05)
    qt = q + 0.05 * q.sum() / 32
    assert np.allclose(c, np.cumsum(qt), rtol=1e-6)
    # leaf probabilities sum to one
    p = np.diff(np.concatenate([[0.0], c])) / c[-1]
    assert p.sum() == pytest.approx(1.0, abs=1e-12) and np.all(p > 0)


def test_eq2_zero_cell_is_uniform(oracle_mod):
    c = oracle_mod.cdf(np.zeros(5), eps=0.01)
    assert c.tolist() == [1.0, 2.0, 3.0, 4.0, 5.0]


@pytest.mark.parametrize("precision", ["fp16", "bf16"])
def test_eq2_half_tables(oracle_mod, precision):
    rng = np.random.default_rng(3)
    for trial in range(50):
        m = int(rng.choice([16, 32, 64]))
        q = rng.exponential(size=m) * rng.choice([1e-6, 1.0, 1e4])
        q[rng.uniform(size=m) < 0.3] = 0.0
        c = oracle_mod.cdf(q, eps=float(rng.choice([0.0, 0.01])), precision=precision)
        assert c[-1] == 1.0
        assert np.all(np.diff(c) > 0) and c[0] > 0
        if precision == "fp16":
            assert np.array_equal(c.astype(np.float16).astype(np.float64), c)
        else:
            bits = c.astype(np.float32).view(np.uint32)
            assert np.all(bits & 0xFFFF == 0)


def test_storage_rounding_matches_library(oracle_mod):
    rng = np.random.default_rng(4)
    vals = np.concatenate([rng.exponential(size=2000) * 10.0 ** rng.uniform(-9, 6, 2000),
                           [1.0, 0.5, 65504.0, 1e6, 2.0 ** -24, 3 * 2.0 ** -25, 1.0 + 2 ** -11]])
    for v in vals:
        h = oracle_mod.round_storage(v, "fp16")
        with np.errstate(over="ignore"):
            ref = float(np.float64(v).astype(np.float16))
        if np.isinf(ref):
            ref = 65504.0  # the table saturates instead of overflowing
        assert h == ref, v
        b = oracle_mod.round_storage(v, "bf16")
        assert b == float(torch.tensor(v, dtype=torch.float64).to(torch.bfloat16).double()), v
        assert oracle_mod.round_storage(v, "fp32") == float(np.float32(v))


# ---------------------------------------------------------------- split-collapse

def _fig_treecuts(oracle_mod):
    """8 lights on a 2x2x2 grid: balanced tree, cut of 4 nodes at depth 2."""
    tris, em = _grid_lights(2)
    tree = oracle_mod.Tree(tris, em)
    cut = tree.initial_cut(4)
    assert [(int(tree.begin[c]), int(tree.end[c])) for c in cut] == [(0, 2), (2, 4), (4, 6), (6, 8)]
    return tree, cut


def test_split_collapse_figure_example(oracle_mod):
    """Fig. "TreeCuts": a balanced 4-leaf cut; the leaf of highest Q is split
    and the parent of lowest Q collapsed."""
    fig = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "fig_treecuts.json")))
    tree, cut = _fig_treecuts(oracle_mod)
    q = np.array(fig["q_before"])
    new_cut, new_q, c, changed = oracle_mod.split_collapse_cell(tree, cut, q, T=fig["T"], eps=0.0)
    assert changed
    A = cut[0]
    parent_cd = tree.parent[cut[2]]
    assert new_cut.tolist() == [tree.left[A], tree.right[A], cut[1], parent_cd]
    # Q of A split in proportion to its children's stored (binary32) power
    # (equal up to float32 rounding of the triangle areas); the collapsed
    # parent sums its leaves
    pa, pc = float(tree.rec[tree.left[A], 6]), float(tree.rec[tree.right[A], 6])
    assert new_q[0] == pytest.approx(10.0 * pa / (pa + pc), rel=1e-7)
    assert new_q[1] == pytest.approx(10.0 * pc / (pa + pc), rel=1e-7)
    assert new_q[0] == pytest.approx(5.0, rel=1e-5)
    assert new_q[2:].tolist() == fig["q_after_collapsed"]
    assert new_q.sum() == pytest.approx(fig["q_after_total"], rel=1e-7)
    assert c == pytest.approx(np.cumsum(new_q), rel=1e-7)


def test_split_collapse_threshold(oracle_mod):
    tree, cut = _fig_treecuts(oracle_mod)
    # Q(lmax) = 1.5 is not > T * Q(pmin) = 2 * 0.75: nothing changes
    q = np.array([1.5, 1.0, 0.5, 0.25])
    new_cut, new_q, _, changed = oracle_mod.split_collapse_cell(tree, cut, q, T=2.0)
    assert not changed and new_cut.tolist() == cut.tolist() and new_q.tolist() == q.tolist()
    # the same Q with T = 1.5 splits
    _, _, _, changed = oracle_mod.split_collapse_cell(tree, cut, q, T=1.9)
    assert changed


def test_split_collapse_skips_when_lmax_under_pmin(oracle_mod):
    tree, cut = _fig_treecuts(oracle_mod)
    # the largest leaf (position 0) is a child of the smallest parent (0, 1)
    q = np.array([1.0, 0.0, 0.6, 0.6])
    new_cut, _, _, changed = oracle_mod.split_collapse_cell(tree, cut, q, T=1.0)
    assert not changed and new_cut.tolist() == cut.tolist()


def test_split_never_picks_single_lights(oracle_mod):
    tris, em = _grid_lights(2)
    tree = oracle_mod.Tree(tris, em)
    cut = tree.initial_cut(8)  # all single lights
    q = np.arange(8, dtype=np.float64)
    _, _, _, changed = oracle_mod.split_collapse_cell(tree, cut, q, T=1.0)
    assert not changed


def test_split_collapse_invariants_random(oracle_mod):
    """Size, partition and total Q are preserved over many calls; the chosen
    parent has the smallest Q over all internal nodes of the cut."""
    rng = np.random.default_rng(6)
    s = scenes.small_frame_scene()
    tree = oracle_mod.Tree(s.tris, s.emission)
    for M in (8, 32):
        cut = tree.initial_cut(M)
        q = rng.exponential(size=len(cut))
        for it in range(60):
            # brute-force minimum over every internal node above the cut
            internal = {}
            for i, c in enumerate(cut):
                p = tree.parent[c]
                while p >= 0:
                    internal[p] = internal.get(p, 0.0) + np.float32(q[i])
                    p = tree.parent[p]
            new_cut, new_q, c, changed = oracle_mod.split_collapse_cell(tree, cut, q, T=1.2, eps=0.01)
            assert len(new_cut) == len(cut)
            b, e = tree.begin[new_cut], tree.end[new_cut]
            assert b[0] == 0 and e[-1] == tree.n and np.all(b[1:] == e[:-1])
            assert new_q.sum() == pytest.approx(q.sum(), rel=1e-6)
            if changed:
                gone = set(cut.tolist()) - set(new_cut.tolist())
                born = set(new_cut.tolist()) - set(cut.tolist())
                collapsed = [p for p in born if p < tree.n - 1 and tree.left[p] in gone]
                assert len(collapsed) == 1
                assert np.float32(internal[collapsed[0]]) <= min(internal.values()) * (1 + 1e-6)
            cut, q = new_cut, new_q * rng.uniform(0.5, 2.0, size=len(new_q))


def _line_lights():
    """16 equal lights on a 4 x 2 x 2 grid: a balanced tree of depth 4."""
    tris = []
    for x in (0.125, 0.375, 0.625, 0.875):
        for y in (0.25, 0.75):
            for z in (0.25, 0.75):
                c = np.array([x, y, z])
                tris.append([c + [-0.01, 0, -0.01], c + [0.02, 0, -0.01], c + [-0.01, 0, 0.02]])
    t = np.asarray(tris, np.float32)
    return t, np.ones((t.shape[0], 3), np.float32)


def test_split_collapse_iterated_by_hand(oracle_mod):
    """Repeating split-collapse until no pair is touched (Section 3). Cut
    [A1, A2, B, C, D1, D2] of a balanced 16-light tree (A1, A2, D1, D2: two
    lights; B, C: four), Q = [8, 8, 1, 0.3, 0.1, 0.1], T = 2, equal powers.
    Step 1: l_max = A1 (tie with A2, smaller begin), p_min = D (0.2); 8 > 0.4
    -> [a0, a1, A2, B, C, D] with Q [4, 4, 8, 1, 0.3, 0.2].
    Step 2: l_max = A2 (8), p_min = parent(C, D) (0.5); 8 > 1
    -> [a0, a1, a2, a3, B, parent(C, D)] with Q [4, 4, 4, 4, 1, 0.5].
    Step 3: l_max = B (1), p_min = A1 (8): 1 > 16 fails, a fixed point."""
    tris, em = _line_lights()
    tree = oracle_mod.Tree(tris, em)
    rng = lambda node: (int(tree.begin[node]), int(tree.end[node]))  # noqa: E731
    root = 0
    L, R = tree.left[root], tree.right[root]
    A, B = tree.left[L], tree.right[L]
    C, D = tree.left[R], tree.right[R]
    assert [rng(x) for x in (A, B, C, D)] == [(0, 4), (4, 8), (8, 12), (12, 16)]
    cut = np.array([tree.left[A], tree.right[A], B, C, tree.left[D], tree.right[D]], np.int32)
    q = np.array([8.0, 8.0, 1.0, 0.3, 0.1, 0.1])
    q = np.array([float(np.float32(v)) for v in q])  # table values are binary32
    c1, q1, _, steps = oracle_mod.split_collapse_cell(tree, cut, q, T=2.0, max_iter=1)
    assert steps == 1
    assert [rng(x) for x in c1] == [(0, 1), (1, 2), (2, 4), (4, 8), (8, 12), (12, 16)]
    assert q1 == pytest.approx([4, 4, 8, 1, 0.3, 0.2], rel=1e-6)
    c2, q2, c, steps = oracle_mod.split_collapse_cell(tree, cut, q, T=2.0, max_iter=8)
    assert steps == 2
    assert [rng(x) for x in c2] == [(0, 1), (1, 2), (2, 3), (3, 4), (4, 8), (8, 16)]
    assert q2 == pytest.approx([4, 4, 4, 4, 1, 0.5], rel=1e-6)
    assert q2.sum() == pytest.approx(q.sum(), rel=1e-7)
    # a fixed point stays put
    _, _, _, steps = oracle_mod.split_collapse_cell(tree, c2, q2, T=2.0, max_iter=8)
    assert steps == 0


def test_split_collapse_iterated_reaches_fixed_point(oracle_mod):
    """Repeated steps keep size, partition and total Q; the result is either
    a fixed point of one more step or the step limit was reached."""
    rng = np.random.default_rng(11)
    s = scenes.small_frame_scene()
    tree = oracle_mod.Tree(s.tris, s.emission)
    hit_fixed = 0
    for trial in range(40):
        cut = tree.initial_cut(16)
        q = rng.exponential(size=len(cut)) ** 3
        new_cut, new_q, c, steps = oracle_mod.split_collapse_cell(tree, cut, q, T=1.5, eps=0.01, max_iter=32)
        b, e = tree.begin[new_cut], tree.end[new_cut]
        assert len(new_cut) == len(cut)
        assert b[0] == 0 and e[-1] == tree.n and np.all(b[1:] == e[:-1])
        assert new_q.sum() == pytest.approx(q.sum(), rel=1e-6)
        _, _, _, more = oracle_mod.split_collapse_cell(tree, new_cut, new_q, T=1.5, max_iter=1)
        assert steps == 32 or more == 0
        hit_fixed += steps < 32
        # k single steps give the same cut as one call of k steps
        c1, q1 = cut, q
        for _ in range(steps):
            c1, q1, _, one = oracle_mod.split_collapse_cell(tree, c1, q1, T=1.5, max_iter=1)
            assert one == 1
        assert c1.tolist() == new_cut.tolist() and np.array_equal(q1, new_q)
    assert hit_fixed > 0
