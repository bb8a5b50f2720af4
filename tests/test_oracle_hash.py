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


# ---- footprint-sized cells (Section 3: cell sizes from the ray footprint of
# each path vertex, coarser on later bounces); reading: levels of cell size
# h * 2^l, l = ceil(log2(f / h)) clamped to [0, levels - 1]

def _level_reference(f, h, levels):
    r = np.float32(np.float32(f) / np.float32(h))  # the binary32 quotient
    if not (r > 1.0):
        return 0
    return min(int(np.ceil(np.log2(np.float64(r)))), levels - 1)


def test_footprint_level_rule(oracle_mod):
    h = np.float32(1.0 / 64.0)
    for k in range(8):
        exact = np.float32(h * np.float32(2.0 ** k))
        assert oracle_mod.footprint_level(exact, h, 16) == k             # cell exactly as wide
        above = np.nextafter(exact, np.float32(np.inf))
        assert oracle_mod.footprint_level(above, h, 16) == k + 1          # one ulp wider: next level
    for f in (0.0, -1.0, float("nan"), float(h) / 3):
        assert oracle_mod.footprint_level(f, h, 16) == 0
    assert oracle_mod.footprint_level(float("inf"), h, 6) == 5
    rng = np.random.default_rng(3)
    for f in np.exp(rng.uniform(np.log(1e-4), np.log(50.0), 2000)).astype(np.float32):
        for levels in (1, 4, 8):
            assert oracle_mod.footprint_level(f, h, levels) == _level_reference(f, h, levels)


def test_level_keys_quantise_with_the_level_cell(grid):
    rng = np.random.default_rng(4)
    o = np.array([-1.0, 0.5, 2.0])
    for level in (0, 1, 3, 6):
        hl = 0.3 * 2.0 ** level
        for _ in range(200):
            p = rng.uniform(-5, 5, size=3).astype(np.float32)
            t = (p.astype(np.float64) - o) / np.float64(np.float32(np.float32(0.3) * np.float32(2.0 ** level)))
            if np.any(np.abs(t - np.round(t)) < 1e-4):
                continue
            f = _fields(grid.cell_key_level(level, p, [0, 1, 0]))
            assert f[:3] == (np.floor(t).astype(int) + 32768).tolist(), (level, hl)


def test_levels_use_their_own_slot_ranges(oracle_mod):
    s = scenes.tiny_scene()
    tree = oracle_mod.Tree(s.tris, s.emission)
    g = oracle_mod.Grid.for_scene(tree, s, levels=4)
    assert g.H == 4 * s.grid.table_size
    rng = np.random.default_rng(5)
    P = s.n_points
    fp = (s.grid.cell_size * 2.0 ** rng.uniform(-1, 4, P)).astype(np.float32)
    out = g.sample_frame(oracle_mod.scene_arrays(s), s.seed, 0, 1, footprint=fp)
    lv = np.array([oracle_mod.footprint_level(f, s.grid.cell_size, 4) for f in fp])
    assert set(np.unique(lv)) == {0, 1, 2, 3}
    Hl = s.grid.table_size
    assert np.all(out["slot"] // Hl == lv)
    # a level-l cell holds only points whose level-l key is its key
    keys = g.keys[out["slot"]]
    for i in rng.choice(P, 200, replace=False):
        x, n = s.pos[:, i], s.nrm[:, i]
        assert keys[i] == g.cell_key_level(lv[i], x, n)
