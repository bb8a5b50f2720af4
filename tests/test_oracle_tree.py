"""Pins of the oracle's light tree and initial cut (Section 3, Section 3.1).

The tree is the binary radix tree over the sorted 64-bit keys
(Morton code << 32 | input index); it is unique given the keys, so checking
the defining property at every node pins the construction.
"""
import numpy as np
import pytest

from paper_1911_10217_gb300 import scenes


def _clz64(v):
    v = int(v)
    return 64 - v.bit_length()


def _grid_lights(k):
    """k^3 small triangles with centroids on a regular grid, facing down."""
    tris = []
    g = (np.arange(k) + 0.5) / k
    for x in g:
        for y in g:
            for z in g:
                c = np.array([x, y, z])
                tris.append([c + [-0.01, 0, -0.01], c + [0.02, 0, -0.01], c + [-0.01, 0, 0.02]])
    t = np.asarray(tris, np.float32)
    return t, np.ones((t.shape[0], 3), np.float32)


def _keys(tree):
    return [(int(tree.code[l]) << 32) | int(tree.perm[l]) for l in range(tree.n)]


def _check_radix(tree):
    n = tree.n
    keys = _keys(tree)
    assert keys == sorted(keys)
    assert sorted(tree.perm.tolist()) == list(range(n))
    seen_leaves = set()
    for i in range(n - 1):
        b, e = int(tree.begin[i]), int(tree.end[i])
        a, c = int(tree.left[i]), int(tree.right[i])
        assert tree.begin[a] == b and tree.end[c] == e and tree.end[a] == tree.begin[c]
        g = int(tree.end[a]) - 1
        node_prefix = _clz64(keys[b] ^ keys[e - 1])
        # split at the highest differing bit: both halves share a longer prefix
        assert _clz64(keys[g] ^ keys[g + 1]) == node_prefix
        assert _clz64(keys[b] ^ keys[g]) > node_prefix or g == b
        assert _clz64(keys[g + 1] ^ keys[e - 1]) > node_prefix or g + 1 == e - 1
        # numbering: a left child covering [b, g] is node g, a right child
        # covering [g+1, e-1] is node g+1; single lights are leaves n-1+l
        assert a == (n - 1 + g if g == b else g)
        assert c == (n - 1 + g + 1 if g + 1 == e - 1 else g + 1)
        assert tree.parent[a] == i and tree.parent[c] == i
        for ch in (a, c):
            if ch >= n - 1:
                seen_leaves.add(ch - (n - 1))
    assert tree.parent[0] == -1 and tree.begin[0] == 0 and tree.end[0] == n
    if n > 1:
        assert seen_leaves == set(range(n))


@pytest.mark.parametrize("maker", ["tiny", "small_frame", "grid4"])
def test_radix_tree_defining_property(oracle_mod, maker):
    if maker == "grid4":
        tris, em = _grid_lights(4)
    else:
        s = getattr(scenes, maker + "_scene")()
        tris, em = s.tris, s.emission
    tree = oracle_mod.Tree(tris, em)
    _check_radix(tree)


def test_duplicate_centroids_break_ties_by_index(oracle_mod):
    t = np.tile(np.array([[[0, 0, 0], [1, 0, 0], [0, 0, 1]]], np.float32), (7, 1, 1))
    tree = oracle_mod.Tree(t, np.ones((7, 3), np.float32))
    assert tree.perm.tolist() == list(range(7))
    _check_radix(tree)


def test_single_light(oracle_mod):
    t = np.array([[[0, 1, 0], [1, 1, 0], [0, 1, 1]]], np.float32)
    tree = oracle_mod.Tree(t, np.ones((1, 3), np.float32))
    assert tree.initial_cut(16).tolist() == [0]
    assert tree.begin[0] == 0 and tree.end[0] == 1


def test_node_bounds_contain_their_lights(oracle_mod):
    s = scenes.small_frame_scene()
    tree = oracle_mod.Tree(s.tris, s.emission)
    tris = s.tris.astype(np.float64)
    e1 = tris[:, 1] - tris[:, 0]
    e2 = tris[:, 2] - tris[:, 0]
    cr = np.cross(e1, e2)
    area = 0.5 * np.linalg.norm(cr, axis=1)
    nrm = cr / np.linalg.norm(cr, axis=1, keepdims=True)
    lum = s.emission.astype(np.float64) @ np.array([0.2126, 0.7152, 0.0722])
    phi_light = lum * area
    for node in range(2 * tree.n - 1):
        idx = tree.perm[tree.begin[node]:tree.end[node]]
        r = tree.rec[node]
        v = tris[idx].reshape(-1, 3)
        assert np.all(v >= r[0:3] - 0) and np.all(v <= r[3:6] + 0)
        assert tree.phi64[node] == pytest.approx(phi_light[idx].sum(), rel=1e-12)
        assert r[6] == pytest.approx(phi_light[idx].sum(), rel=1e-5)
        if r[10] > -1.0:
            axis = r[7:10].astype(np.float64)
            assert np.linalg.norm(axis) == pytest.approx(1.0, abs=1e-6)
            assert np.all(nrm[idx] @ axis >= r[10] - 1e-6)


def test_bfs_initial_cut_on_balanced_tree(oracle_mod):
    # 4x4x4 lights on a grid: 6-bit codes, a perfectly balanced tree of depth
    # 6; a breadth-first cut of M = 8 is the 8 nodes at depth 3 (octants).
    tris, em = _grid_lights(4)
    tree = oracle_mod.Tree(tris, em)
    cut = tree.initial_cut(8)
    ranges = [(int(tree.begin[c]), int(tree.end[c])) for c in cut]
    assert ranges == [(8 * i, 8 * i + 8) for i in range(8)]
    cut16 = tree.initial_cut(16)
    assert [(int(tree.begin[c]), int(tree.end[c])) for c in cut16] == [(4 * i, 4 * i + 4) for i in range(16)]
    assert tree.initial_cut(200).tolist() == [63 + l for l in range(64)]


def test_initial_cut_is_partition(oracle_mod):
    s = scenes.tiny_scene()
    tree = oracle_mod.Tree(s.tris, s.emission)
    for M in (1, 2, 3, 16, 100, 256, 300):
        cut = tree.initial_cut(M)
        assert len(cut) == min(M, tree.n)
        b = tree.begin[cut]
        e = tree.end[cut]
        assert b[0] == 0 and e[-1] == tree.n and np.all(b[1:] == e[:-1])


def test_importance_bounds_are_conservative(oracle_mod):
    """I * d^2 / phi bounds cos_x * cos_l for every point of every light below
    the node (the receiver and emitter bounds of the descent)."""
    rng = np.random.default_rng(5)
    s = scenes.small_frame_scene()
    tree = oracle_mod.Tree(s.tris, s.emission)
    tris = s.tris.astype(np.float64)
    cr = np.cross(tris[:, 1] - tris[:, 0], tris[:, 2] - tris[:, 0])
    nl = cr / np.linalg.norm(cr, axis=1, keepdims=True)
    checked = 0
    for trial in range(300):
        node = int(rng.integers(0, 2 * tree.n - 1))
        x = rng.uniform(0, 1, 3).astype(np.float32)
        nv = rng.normal(size=3)
        nv = (nv / np.linalg.norm(nv)).astype(np.float32)
        r = tree.rec[node].astype(np.float64)
        c = 0.5 * (r[0:3] + r[3:6])
        d = c - x
        d2 = d @ d
        r2 = 0.25 * np.sum((r[3:6] - r[0:3]) ** 2)
        if d2 <= r2 * 1.0001:
            continue
        I = oracle_mod.Tree.importance(tree, node, x, nv)
        idx = tree.perm[tree.begin[node]:tree.end[node]]
        # points: vertices and random interior points of every light
        bary = rng.dirichlet([1, 1, 1], size=8)
        pts = np.concatenate([tris[idx].reshape(-1, 3),
                              np.einsum("kj,ljd->lkd", bary, tris[idx]).reshape(-1, 3)])
        nrep = np.concatenate([np.repeat(nl[idx], 3, axis=0), np.repeat(nl[idx], 8, axis=0)])
        w = pts - x
        w /= np.linalg.norm(w, axis=1, keepdims=True)
        val = np.maximum(0, w @ nv) * np.maximum(0, -np.sum(nrep * w, axis=1))
        bound = I * d2 / r[6]
        assert val.max() <= bound * (1 + 1e-4) + 1e-6, (node, val.max(), bound)
        checked += 1
    assert checked > 100


# ---- surface-area-orientation split positions (Section 3.1 names such a
# hierarchy as future work); reading: Morton order kept, split positions by
# cost phi * SA(box) * (2 - |sum c| / sum |c|) among fixed candidates

def _line_lights(xs, up):
    """Small triangles at x positions along a line; facing +y (up) or -y."""
    tris = []
    for x, u in zip(xs, up):
        a, b, c = [x, 0.0, 0.0], [x + 0.01, 0.0, 0.0], [x, 0.0, 0.01]
        tris.append([a, c, b] if u else [a, b, c])   # winding normal +y or -y
    tris = np.asarray(tris, np.float32)
    return tris, np.ones((len(xs), 3), np.float32)


def test_saoh_tree_is_a_binary_tree_over_ranges(oracle_mod):
    for maker in ("tiny", "small_frame"):
        s = getattr(scenes, maker + "_scene")()
        a = oracle_mod.Tree(s.tris, s.emission)
        t = oracle_mod.Tree(s.tris, s.emission, builder="saoh")
        n = t.n
        assert np.array_equal(t.perm, a.perm)           # same light order
        assert t.parent[0] == -1 and t.begin[0] == 0 and t.end[0] == n
        seen = np.zeros(2 * n - 1, int)
        for i in range(n - 1):
            l, r = t.left[i], t.right[i]
            seen[l] += 1
            seen[r] += 1
            assert t.parent[l] == i and t.parent[r] == i
            assert t.begin[l] == t.begin[i] and t.end[l] == t.begin[r] and t.end[r] == t.end[i]
            # id rule: (split position - the root's) mod (n - 1)
            g_root = int(t.begin[t.right[0]]) - 1
            assert i == ((int(t.begin[r]) - 1) - g_root) % (n - 1)
        assert seen[0] == 0 and np.all(seen[1:] == 1)
        for l in range(n):
            assert t.begin[n - 1 + l] == l and t.end[n - 1 + l] == l + 1


def test_saoh_split_moves_toward_a_change_of_facing(oracle_mod):
    # 32 equal lights evenly spaced on a line. All facing up: the power-times-
    # area term alone is symmetric and least in the middle (k^2 + (32-k)^2),
    # so the root splits at 16. With the last 8 facing down, every split left
    # of the middle leaves more mixed facing on the right, so the root split
    # moves right of 16, but not past the change of facing at 24.
    xs = np.arange(32) / 31.0
    tris, em = _line_lights(xs, [True] * 32)
    assert oracle_mod.Tree(tris, em, builder="saoh").begin[
        oracle_mod.Tree(tris, em, builder="saoh").right[0]] == 16
    tris, em = _line_lights(xs, [True] * 24 + [False] * 8)
    t = oracle_mod.Tree(tris, em, builder="saoh")
    assert 16 < int(t.begin[t.right[0]]) <= 24


def test_saoh_separates_distant_clusters(oracle_mod):
    # 20 lights near x = 0 and 12 near x = 1: every candidate except the gap
    # leaves one child spanning the gap
    xs = np.concatenate([np.linspace(0.0, 0.1, 20), np.linspace(0.9, 1.0, 12)])
    tris, em = _line_lights(xs, [True] * 32)
    t = oracle_mod.Tree(tris, em, builder="saoh")
    assert t.begin[t.right[0]] == 20


# ---- median split positions (a balanced tree over the same light order)

def _ranges(t):
    """(begin, split, end) of every internal node."""
    return sorted((int(t.begin[i]), int(t.begin[t.right[i]]), int(t.end[i])) for i in range(t.n - 1))


@pytest.mark.parametrize("n", [2, 3, 5, 7, 8, 13, 17, 100])
def test_median_tree_is_balanced_over_ranges(oracle_mod, n):
    rng = np.random.default_rng(n)
    tris, em = _line_lights(rng.uniform(0.0, 1.0, n), [True] * n)
    a = oracle_mod.Tree(tris, em)
    t = oracle_mod.Tree(tris, em, builder="median")
    assert np.array_equal(t.perm, a.perm)               # same light order
    assert t.parent[0] == -1 and t.begin[0] == 0 and t.end[0] == n
    seen = np.zeros(2 * n - 1, int)
    depth = {0: 0}
    g_root = n // 2 - 1
    for i in range(n - 1):
        l, r = int(t.left[i]), int(t.right[i])
        seen[l] += 1
        seen[r] += 1
        assert t.parent[l] == i and t.parent[r] == i
        b, k, e = int(t.begin[i]), int(t.begin[r]), int(t.end[i])
        assert t.end[l] == k and t.begin[l] == b and t.end[r] == e
        assert k == b + (e - b) // 2                    # split at the middle
        assert i == ((k - 1) - g_root) % (n - 1)        # id rule
    assert seen[0] == 0 and np.all(seen[1:] == 1)
    stack = [0]
    while stack:
        v = stack.pop()
        if v < n - 1:
            for c in (int(t.left[v]), int(t.right[v])):
                depth[c] = depth[v] + 1
                stack.append(c)
    leaf = np.array([depth[n - 1 + l] for l in range(n)])
    lo, hi = int(np.floor(np.log2(n))), int(np.ceil(np.log2(n)))
    assert leaf.min() >= lo and leaf.max() <= hi


def test_median_tree_equals_radix_tree_on_a_complete_grid(oracle_mod):
    # 8 x 8 x 8 lights on a regular grid: the top 3 bits of each quantised
    # axis enumerate the 8 rows, so the 512 Morton codes differ first in 9
    # interleaved bits that take every value once; the radix tree of those
    # codes (Section 3.1) is the complete tree that halves every range.
    tris, em = _grid_lights(8)
    a = oracle_mod.Tree(tris, em)
    t = oracle_mod.Tree(tris, em, builder="median")
    assert _ranges(a) == _ranges(t)


# ---- compact descent-bound constants: binary16 cone rounded outward

def test_half_round_directed(oracle_mod):
    """Rounding to binary16 toward -inf / +inf against numpy's float16: both
    results are binary16 values, bracket x, and no binary16 value lies
    strictly between either result and x."""
    rng = np.random.default_rng(5)
    xs = np.concatenate([rng.uniform(-1.0, 1.0, 4000), rng.uniform(-1e-3, 1e-3, 500),
                         rng.uniform(-1e-6, 1e-6, 200),
                         [1.0, -1.0, 0.5, -0.5, 1.0 / 3.0, -1.0 / 3.0, 2.0 ** -14, -2.0 ** -14, 2.0 ** -20,
                          0.999999, -0.999999]]).astype(np.float32)
    inf16 = np.float16(np.inf)
    for x in xs:
        d, u = oracle_mod.half_round(x, False), oracle_mod.half_round(x, True)
        assert d <= x <= u
        assert float(np.float16(d)) == d and float(np.float16(u)) == u
        if d < x:
            assert float(np.nextafter(np.float16(d), inf16)) > x
        if u > x:
            assert float(np.nextafter(np.float16(u), -inf16)) < x
        if float(np.float16(x)) == float(x):
            assert d == u == x


def test_radius_rounded_up_keeps_r_squared():
    """The sphere constant of the descent bound: r = the binary32 square root
    of the squared half diagonal, one ulp up, and r^2 = fl(r r) is never below
    the squared half diagonal itself (binary32 throughout)."""
    rng = np.random.default_rng(9)
    rb2 = np.concatenate([rng.uniform(0.0, 1.0, 200000), 10.0 ** rng.uniform(-30, 10, 200000),
                          [0.0, 1.0, 2.0, 0.25, 1e-38, 3.4e38 / 4]]).astype(np.float32)
    r = np.nextafter(np.sqrt(rb2, dtype=np.float32), np.float32(np.inf))
    r2 = (r * r).astype(np.float32)
    assert r2.dtype == np.float32 and np.all(r2 >= rb2)
