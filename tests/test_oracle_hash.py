"""Pins of the oracle's 5-d cell key and table probing (Section 3: jittered
quantised position and normal). Without jitter a field is floor((p - o) / h)
biased by 2^15; the octahedral normal of the six axis directions lands in
known bins; probing is linear from the hash and stops at the 64th slot."""
import numpy as np
import pytest

from paper_1911_10217_gb300 import scenes


def _fields(key):
    key = int(key)
    return [(key >> s) & 0xFFFF for s in (0, 16, 32)] + [(key >> 48) & 0xFF, (key >> 56) & 0xFF]


@pytest.fixture(scope="module")
def grid(oracle_mod):
    s = scenes.tiny_scene()
    tree = oracle_mod.Tree(s.tris, s.emission)
    return oracle_mod.Grid(tree, 64, 4, origin=(-1.0, 0.5, 2.0), cell_size=0.3, normal_bins=4)


def test_position_fields_are_floor_of_cell_coordinates(grid):
    rng = np.random.default_rng(0)
    for _ in range(500):
        p = rng.uniform(-5, 5, size=3).astype(np.float32)
        t = (p.astype(np.float64) - np.array([-1.0, 0.5, 2.0])) / 0.3
        if np.any(np.abs(t - np.round(t)) < 1e-4):
            continue  # too close to a cell boundary for a float64 reference
        f = _fields(grid.cell_key(p, [0, 1, 0]))
        assert f[:3] == (np.floor(t).astype(int) + 32768).tolist()


def test_axis_normals_land_in_known_bins(grid):
    # octahedral map with y up: (a, b) = (nx, nz) / |n|_1, lower hemisphere
    # folded; bins of width 2/4 over [-1, 1], clamped to [0, 3]
    cases = {(0, 1, 0): (2, 2), (1, 0, 0): (3, 2), (-1, 0, 0): (0, 2), (0, 0, 1): (2, 3),
             (0, 0, -1): (2, 0), (0, -1, 0): (3, 3)}
    for n, (iu, iv) in cases.items():
        f = _fields(grid.cell_key([0.1, 0.7, 2.1], n))
        assert (f[3], f[4]) == (iu, iv), n


def test_jitter_moves_at_most_one_cell(oracle_mod):
    s = scenes.tiny_scene()
    tree = oracle_mod.Tree(s.tris, s.emission)
    g0 = oracle_mod.Grid(tree, 64, 4, cell_size=0.1, normal_bins=8)
    g1 = oracle_mod.Grid(tree, 64, 4, cell_size=0.1, normal_bins=8, jitter=True)
    rng = np.random.default_rng(1)
    for _ in range(300):
        p = rng.uniform(0, 1, 3)
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        j = rng.uniform(0, 1, 5)
        a, b = np.array(_fields(g0.cell_key(p, n))), np.array(_fields(g1.cell_key(p, n, j)))
        assert np.all(np.abs(a - b) <= 1)
    # a jitter of exactly 1/2 leaves the key unchanged (u - 1/2 = 0)
    assert g1.cell_key([0.33, 0.2, 0.9], [0, 1, 0], [0.5] * 5) == g0.cell_key([0.33, 0.2, 0.9], [0, 1, 0])


def test_probing_and_probe_limit(oracle_mod):
    s = scenes.tiny_scene()
    tree = oracle_mod.Tree(s.tris, s.emission)
    g = oracle_mod.Grid(tree, 128, 4)
    slots = [g.lookup_insert(k) for k in range(1, 101)]
    assert len(set(slots)) == 100 and min(slots) >= 0
    assert [g.lookup_insert(k) for k in range(1, 101)] == slots  # found again
    for sl, k in zip(slots, range(1, 101)):
        assert int(g.keys[sl]) == k
        assert g.cut[sl, :g.m].tolist() == g.def_cut.tolist()  # copied on first access
    lib = oracle_mod.lib()
    # a key sits at most (64 - 1) slots after its hash position
    for sl, k in zip(slots, range(1, 101)):
        h = lib.orc_fmix64(k) % 128
        assert (sl - h) % 128 < 64
    small = oracle_mod.Grid(tree, 16, 4)
    got = [small.lookup_insert(k) for k in range(1, 40)]
    assert sum(x >= 0 for x in got) == 16 and got.count(-1) == 23
