"""Pins of the descent bound (the in-cluster choice of Section 3 descends by
unoccluded bounds, as the bound-based many-light samplers of Section 2 do).

The oracle evaluates the bound in binary32 in a rearranged form (cosines
carried multiplied by |d|, bounds compared without a division), because its
value decides which child a descent step takes. These tests tie that form to
things outside it:

* the node constants it reads (centre, radius rounded up, cone rounded
  outward to binary16) against numpy's own rounding;
* a plain double-precision statement of the bound, with unit vectors and
  sines and cosines of the half angles, over 10^5 random configurations,
  including points just outside the bounding sphere and cones of width 0 and
  a full sphere;
* the receiver and emitter factors against brute-force suprema over the cone
  of directions to the sphere and the cone of normals;
* tightness: a tiny light far away gets cos_x * cos_l, and a node of lights
  whose normals span a cone gets the exact largest emitter cosine.
"""
import numpy as np
import pytest

from paper_1911_10217_gb300 import scenes


def _unit(v):
    v = np.asarray(v, np.float64)
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def _i32(oracle_mod, rec, x, n):
    """The oracle's binary32 bound num / den as a double."""
    import ctypes
    num, den = ctypes.c_float(), ctypes.c_float()
    oracle_mod.lib().orc_importance32(oracle_mod._p(np.ascontiguousarray(rec, np.float32)),
                                      oracle_mod._p(np.ascontiguousarray(x, np.float32)),
                                      oracle_mod._p(np.ascontiguousarray(n, np.float32)),
                                      ctypes.byref(num), ctypes.byref(den))
    return float(num.value) / float(den.value)


def _i64(oracle_mod, rec, x, n):
    k = oracle_mod.node_consts(rec)
    return oracle_mod.bound64(k[0:3], k[3], k[5], k[6], rec[7:10], rec[6], x, n), k


def _random_unit(rng, size=None):
    return _unit(rng.normal(size=(3,) if size is None else (size, 3)))


# ---- node constants ------------------------------------------------------------

def test_node_constants(oracle_mod):
    """Centre = binary32 midpoint of the box; r r not below the squared half
    diagonal and r at most two binary32 ulps above its square root; the cone
    as v = 1 - cos theta rounded up to the nearest binary16 value (so the
    cone is at least as wide), and the sine of the cone 1 - v rounded up to
    binary16."""
    s = scenes.small_frame_scene()
    tree = oracle_mod.Tree(s.tris, s.emission)
    inf16 = np.float16(np.inf)
    checked = 0
    for node in range(0, 2 * tree.n - 1, 7):
        rec = tree.rec[node]
        k = oracle_mod.node_consts(rec)
        lo, hi = rec[0:3], rec[3:6]
        assert np.array_equal(k[0:3], ((lo + hi) * np.float32(0.5)).astype(np.float32))
        half2 = 0.25 * np.sum((hi.astype(np.float64) - lo.astype(np.float64)) ** 2)
        assert float(k[3]) ** 2 >= half2 * (1 - 1e-7)
        assert float(k[4]) >= float(np.float32(0.25) * np.float32(np.sum((hi - lo) ** 2)) * (1 - 1e-6))
        assert float(k[3]) <= np.sqrt(half2) * (1 + 4 * 2.0 ** -24) + 1e-30
        ct, st = float(k[5]), float(k[6])
        v, v_exact = 1.0 - ct, 1.0 - float(rec[10])
        assert float(np.float16(v)) == v and float(np.float16(st)) == st
        assert v >= v_exact and (v == 0.0 or float(np.nextafter(np.float16(v), -inf16)) < v_exact)
        s_exact = np.sqrt(v * (2.0 - v))
        assert st >= s_exact and (st == 0.0 or float(np.nextafter(np.float16(st), -inf16)) < s_exact)
        checked += 1
    assert checked > 100
    # narrow cones stay narrow: a cone of half angle 1e-3 keeps a half angle within 1e-6 of it
    for th in (1e-3, 1e-2, 0.3, 1.5, 2.5):
        rec = tree.rec[0].copy()
        rec[10] = np.float32(np.cos(th))
        k = oracle_mod.node_consts(rec)
        assert np.arccos(float(k[5])) >= np.arccos(float(rec[10]))
        assert np.arccos(float(k[5])) - th <= max(2e-6, th * 2.0 ** -10 + 1e-6), th


# ---- binary32 form against the plain double statement ------------------------------

def _compare(oracle_mod, rec, x, n, stats):
    i32 = _i32(oracle_mod, rec, x, n)
    i64, k = _i64(oracle_mod, rec, x, n)
    d = k[0:3].astype(np.float64) - np.asarray(x, np.float64)
    d2 = float(d @ d)
    r2 = float(k[3]) ** 2
    if abs(d2 - r2) <= 1e-5 * r2:
        stats["band"] += 1  # the inside/outside decision itself is within rounding of its threshold
        return
    scale = float(rec[6]) / max(d2, r2)  # the bound with both angular factors at 1
    # condition number of the half angle beta: |d| cos(beta) = sqrt(d^2 - r^2) loses the relative
    # precision d^2 / (d^2 - r^2) * 2^-24 in binary32 just outside the sphere
    kappa = d2 / (d2 - r2) if d2 > r2 else 1.0
    eps = 2.0 ** -24
    err = abs(i32 - i64)
    assert err <= 8 * eps * kappa * scale + 1e-6 * i64, (rec.tolist(), list(x), list(n), i32, i64, kappa)
    if i64 >= 0.1 * scale and kappa < 2:
        assert err <= 1e-5 * i64, (rec.tolist(), list(x), list(n), i32, i64, kappa)
        stats["rel"] += 1
    stats["n"] += 1


def test_binary32_bound_equals_plain_double(oracle_mod):
    """The rearranged binary32 bound equals the plain statement in double.
    Measured in units of phi / d^2 (the bound with both angular factors at
    1), the error is at most 8 binary32 unit roundoffs times kappa =
    d^2 / (d^2 - r^2), the condition number of the half angle beta, which
    grows just outside the bounding sphere; where the point is not that
    close (kappa < 2) and the factors' product is at least 0.1, the relative
    error is at most 1e-5. (Near 0 the factors are cosines at their clamp,
    where a relative comparison has no meaning.)"""
    rng = np.random.default_rng(20240611)
    s = scenes.small_frame_scene()
    tree = oracle_mod.Tree(s.tris, s.emission)
    recs = tree.rec
    stats = {"n": 0, "rel": 0, "band": 0}
    # random nodes, points and normals in and around the room
    for _ in range(60000):
        rec = recs[rng.integers(0, recs.shape[0])]
        x = rng.uniform(-0.2, 1.2, 3).astype(np.float32)
        n = _random_unit(rng).astype(np.float32)
        _compare(oracle_mod, rec, x, n, stats)
    # points just outside the bounding sphere, at relative distances 1e-5 .. 1e-1
    for _ in range(25000):
        rec = recs[rng.integers(0, recs.shape[0])]
        k = oracle_mod.node_consts(rec)
        u = _random_unit(rng)
        x = (k[0:3] + float(k[3]) * (1 + 10 ** rng.uniform(-5, -1)) * u).astype(np.float32)
        n = _random_unit(rng).astype(np.float32)
        _compare(oracle_mod, rec, x, n, stats)
    # cones of width 0, a full sphere, and nearly so, in either direction
    for ct in (1.0, -1.0, 0.99999, -0.99999, 0.0):
        for _ in range(3000):
            rec = recs[rng.integers(0, recs.shape[0])].copy()
            rec[7:10] = _random_unit(rng)
            rec[10] = ct
            x = rng.uniform(-0.2, 1.2, 3).astype(np.float32)
            n = _random_unit(rng).astype(np.float32)
            _compare(oracle_mod, rec, x, n, stats)
    assert stats["n"] > 95000 and stats["rel"] > 20000 and stats["band"] < 100, stats


# ---- the angular factors are the suprema they stand for ---------------------------------

def _frame(a, b):
    """Unit u orthogonal to a in the plane of a and b (any if parallel)."""
    u = b - (b @ a) * a
    if np.linalg.norm(u) < 1e-9:
        u = np.cross(a, [1.0, 0.0, 0.0] if abs(a[0]) < 0.9 else [0.0, 1.0, 0.0])
    return _unit(u)


def _cone_samples(rng, axis, half, k):
    """k directions uniformly spread over the spherical cap of half angle
    `half` around `axis`."""
    u = _frame(axis, _random_unit(rng))
    v = np.cross(axis, u)
    cz = rng.uniform(np.cos(half), 1.0, k)
    sz = np.sqrt(np.maximum(0.0, 1 - cz * cz))
    ph = rng.uniform(0, 2 * np.pi, k)
    return cz[:, None] * axis + sz[:, None] * (np.cos(ph)[:, None] * u + np.sin(ph)[:, None] * v)


def test_receiver_factor_is_the_supremum(oracle_mod):
    """With a full cone of normals (emitter factor 1), I d^2 / phi equals the
    largest max(0, n . omega) over the directions omega within beta of the
    direction to the centre: brute force over the plane of n and that
    direction (where the maximum lies) to 1e-6, and no direction of the cap
    off that plane exceeds it."""
    rng = np.random.default_rng(3)
    for _ in range(300):
        c = rng.uniform(-1, 1, 3)
        dist = 10 ** rng.uniform(-0.5, 1)
        w = _random_unit(rng)
        x = c - dist * w
        r = dist * rng.uniform(0.01, 0.99)
        n = _random_unit(rng)
        got = oracle_mod.bound64(c, r, -1.0, 0.0, [0.0, 0.0, 1.0], 1.0, x, n) * dist * dist
        beta = np.arcsin(r / dist)
        u = _frame(w, n)
        phis = np.linspace(-beta, beta, 20001)
        om = np.cos(phis)[:, None] * w + np.sin(phis)[:, None] * u
        want = max(0.0, float(np.max(om @ n)))
        assert got == pytest.approx(want, abs=1e-6), (got, want)
        off = _cone_samples(rng, w, beta, 4000)
        assert float(np.max(np.maximum(0.0, off @ n))) <= got + 1e-9


def test_emitter_factor_is_the_supremum(oracle_mod):
    """With the receiver normal facing the centre (receiver factor 1),
    I d^2 / phi equals the largest max(0, -n_l . omega) over normals n_l
    within theta of the cone axis and directions omega within beta of the
    direction to the centre: brute force over their common plane to 1e-5,
    and random pairs off that plane never exceed it."""
    rng = np.random.default_rng(4)
    for _ in range(200):
        c = rng.uniform(-1, 1, 3)
        dist = 10 ** rng.uniform(-0.5, 1)
        w = _random_unit(rng)
        x = c - dist * w
        r = dist * rng.uniform(0.0, 0.9)
        theta = rng.uniform(0, np.pi)
        a = _random_unit(rng)
        got = oracle_mod.bound64(c, r, np.cos(theta), np.sin(theta), a, 1.0, x, w) * dist * dist
        beta = np.arcsin(r / dist)
        # in-plane: omega turned from w, n_l turned from a, in the plane of w and a
        u = _frame(w, -a)
        e = _frame(a, -w) if abs(a @ w) < 1 - 1e-12 else u
        phis = np.linspace(-beta, beta, 1201)
        taus = np.linspace(-theta, theta, 1201)
        om = np.cos(phis)[:, None] * w + np.sin(phis)[:, None] * u
        nl = np.cos(taus)[:, None] * a + np.sin(taus)[:, None] * e
        want = max(0.0, float(np.max(-(nl @ om.T))))
        assert got == pytest.approx(want, abs=1e-5), (got, want, theta, beta)
        om2 = _cone_samples(rng, w, beta, 3000)
        nl2 = _cone_samples(rng, a, theta, 3000)
        assert float(np.max(np.maximum(0.0, -(nl2 @ om2.T)))) <= got + 1e-9


# ---- tightness on actual lights ----------------------------------------------------

def _tri_facing(centre, normal, size):
    """A small triangle at `centre` whose winding normal is `normal`."""
    normal = _unit(normal)
    u = _frame(normal, _random_unit(np.random.default_rng(0)))
    v = np.cross(normal, u)
    return np.array([centre, centre + size * u, centre + size * v])


def test_tiny_far_light_gets_the_exact_cosines(oracle_mod):
    """One tiny light seen from a distance d of 10^3 to 10^5 r: its cone is
    as narrow as the binary32 cone cosine of one normal allows (half angle
    theta' under 1e-3), and the binary32 bound I d^2 / phi is cos_x cos_l of
    the light's centre, never below it and above it by no more than the
    widening of the two angles: to first order beta sin(gamma) + (beta +
    theta') sin(psi), with beta = r / d the half angle of the sphere."""
    rng = np.random.default_rng(11)
    for _ in range(400):
        nl = _random_unit(rng)
        t = _tri_facing(rng.uniform(-1, 1, 3), nl, 1e-3).astype(np.float32)
        t64 = t.astype(np.float64)
        nl = _unit(np.cross(t64[1] - t64[0], t64[2] - t64[0]))  # of the binary32 vertices
        tree = oracle_mod.Tree(t[None], np.ones((1, 3), np.float32))
        rec = tree.rec[0]
        k = oracle_mod.node_consts(rec)
        theta = float(np.arccos(np.float64(k[5])))
        assert theta < 1e-3
        centre = k[0:3].astype(np.float64)
        rr = float(k[3])
        dist = rr * 10 ** rng.uniform(3, 5)
        # x in the half space the light faces, normal random in the hemisphere facing the light
        wl = _random_unit(rng)
        if wl @ nl < 0:
            wl = -wl
        x = (centre + dist * wl).astype(np.float32)
        n = _random_unit(rng)
        if n @ (centre - x) < 0:
            n = -n
        n = n.astype(np.float32)
        d = centre - x.astype(np.float64)
        dd = float(np.sqrt(d @ d))
        cos_x = max(0.0, float(n.astype(np.float64) @ d) / dd)
        cos_l = max(0.0, float(-(nl @ d)) / dd)
        got = _i32(oracle_mod, rec, x, n) * dd * dd / float(rec[6])
        beta = rr / dd
        sin_x, sin_l = np.sqrt(1 - cos_x ** 2), np.sqrt(1 - cos_l ** 2)
        assert got >= cos_x * cos_l * (1 - 1e-5) - 1e-7
        widen = beta * sin_x + (beta + theta) * sin_l
        assert got <= cos_x * cos_l + 1.05 * widen + (beta + theta) ** 2 + 1e-5, (got, cos_x * cos_l, beta, theta)


def test_emitter_bound_is_the_largest_cosine_of_a_cone_of_lights(oracle_mod):
    """A node of tiny lights whose normals lie on a cone of half angle theta
    (16 azimuths, one of them in the plane of the axis and the viewing
    direction) seen from far away at angle psi > theta from the axis, with the
    receiver facing it: I d^2 / phi is the largest cos_l over the lights,
    cos(psi - theta), to within the widening of the cone by beta and by the
    binary16 rounding of its cosine and sine (first order: the widening
    angle times sin(psi - theta), and the lengthening of the rounded
    (cos, sin) pair times cos(psi - theta))."""
    rng = np.random.default_rng(12)
    for _ in range(60):
        a = _random_unit(rng)
        theta = rng.uniform(0.05, 1.2)
        psi = rng.uniform(theta + 0.05, min(np.pi, theta + np.pi / 2 - 0.05))
        view = _unit(np.cos(psi) * a + np.sin(psi) * _frame(a, _random_unit(rng)))  # from node to x
        e1 = _frame(a, view)
        e2 = np.cross(a, e1)
        centre = rng.uniform(-0.01, 0.01, 3)  # small coordinates: the binary32 normals stay on the cone
        tris = []
        for j in range(16):
            ph = 2 * np.pi * j / 16
            nj = np.cos(theta) * a + np.sin(theta) * (np.cos(ph) * e1 + np.sin(ph) * e2)
            tris.append(_tri_facing(centre + 1e-3 * rng.normal(size=3), nj, 1e-2))
        tris = np.asarray(tris, np.float32)
        nrm = _unit(np.cross(tris[:, 1].astype(np.float64) - tris[:, 0], tris[:, 2].astype(np.float64) - tris[:, 0]))
        tree = oracle_mod.Tree(tris, np.ones((16, 3), np.float32))
        rec = tree.rec[0]
        k = oracle_mod.node_consts(rec)
        dist = 200.0
        x = (k[0:3].astype(np.float64) + dist * view).astype(np.float32)
        n = (-view).astype(np.float32)
        d = k[0:3].astype(np.float64) - x.astype(np.float64)
        dd = float(np.sqrt(d @ d))
        exact = float(np.max(-(nrm @ d) / dd))
        assert exact == pytest.approx(np.cos(psi - theta), abs=2e-4)
        got = _i32(oracle_mod, rec, x, n) * dd * dd / float(rec[6])
        beta = float(k[3]) / dd
        ct, st = float(k[5]), float(k[6])
        cone_slack = np.arccos(ct) - np.arccos(float(rec[10]))   # 1 - cos rounded up to binary16
        # sin rounded up to binary16 by ds: (ct, st) is the direction of angle theta' + ds ct,
        # lengthened by ds st
        ds = st - np.sqrt(1.0 - ct * ct)
        slack = beta + cone_slack + ds * ct
        assert got >= exact * (1 - 1e-5)
        assert got <= exact + 1.01 * (slack * np.sin(psi - theta) + ds * st * np.cos(psi - theta)) + slack ** 2 + 1e-6, \
            (got, exact, slack, ds)
