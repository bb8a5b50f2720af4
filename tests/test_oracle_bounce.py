"""Pins of the oracle's path vertices (Section 3, first ingredient: cells sized
from the ray footprint of each path vertex, derived from its area pdf): one
cosine-weighted bounce from each shading point, traced to the nearest box
face or room wall, with footprint (N_t p_A)^(-1/2).

* the directions follow the cosine density (cos^2 theta uniform, azimuth
  uniform), by chi-square over 2 * 10^5 bounces of one point;
* on a plane the footprint has a closed form: a floor point at height H
  below a ceiling reaches it at distance H / cos theta with both cosines
  equal, so p_A = cos^4 theta / (pi H^2);
* every vertex lies on the face it reports, that face is turned toward the
  point, and the open segment to it crosses no box (float64 slab test);
  only paths from points outside the room escape.
"""
import numpy as np
import pytest

from paper_1911_10217_gb300 import scenes

ROOM = np.array([0, 0, 0, 1, 1, 1], np.float32)


def _chi2_uniform(u, bins=20):
    h, _ = np.histogram(u, bins=bins, range=(0.0, 1.0))
    e = len(u) / bins
    return float(np.sum((h - e) ** 2 / e))


def test_directions_are_cosine_weighted(oracle_mod):
    P = 200000
    pos = np.tile(np.array([[0.5], [0.0], [0.5]], np.float32), (1, P))
    nrm = np.tile(np.array([[0.0], [1.0], [0.0]], np.float32), (1, P))
    y, ny, fp = oracle_mod.bounce_vertices(pos, nrm, np.zeros((0, 6)), ROOM, 3, 0, 1.0)
    o = pos.astype(np.float64) + 1e-4 * nrm
    d = y.astype(np.float64) - o
    d /= np.linalg.norm(d, axis=0)
    cos_t = d[1]
    assert np.all(cos_t > 0)
    # chi-square with 19 degrees of freedom: 99.99 % quantile 52.6
    assert _chi2_uniform(cos_t ** 2) < 52.6
    phi = (np.arctan2(d[2], d[0]) / (2 * np.pi)) % 1.0
    assert _chi2_uniform(phi) < 52.6
    # and not uniform in cos theta (a uniform-hemisphere sampler would pass the azimuth test)
    assert _chi2_uniform(cos_t) > 1000


def test_footprint_closed_form_on_a_plane(oracle_mod):
    rng = np.random.default_rng(2)
    P = 50000
    pos = np.stack([rng.uniform(0.2, 0.8, P), np.zeros(P), rng.uniform(0.2, 0.8, P)]).astype(np.float32)
    nrm = np.tile(np.array([[0.0], [1.0], [0.0]], np.float32), (1, P))
    for n_t in (1.0, 100.0):
        y, ny, fp = oracle_mod.bounce_vertices(pos, nrm, np.zeros((0, 6)), ROOM, 5, 1, n_t)
        ceil = ny[1] == -1.0
        assert ceil.sum() > P // 8
        o = pos.astype(np.float64) + 1e-4 * nrm.astype(np.float64)
        H = 1.0 - o[1][ceil]
        dist = np.linalg.norm(y[:, ceil].astype(np.float64) - o[:, ceil], axis=0)
        cos_t = H / dist
        want = np.sqrt(np.pi * H ** 2 / (n_t * cos_t ** 4))
        assert np.allclose(fp[ceil], want, rtol=2e-5), np.max(np.abs(fp[ceil] / want - 1))
        assert np.allclose(y[1][ceil], 1.0, atol=1e-6)


def _segment_hits_box(o, y, boxes, shrink=1e-4):
    """Float64 slab test of the open segment o + t (y - o), t in (shrink,
    1 - shrink), against every box; True where some box is crossed."""
    d = y - o
    hit = np.zeros(o.shape[1], bool)
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / d
        for b in boxes.astype(np.float64):
            t1 = (b[:3, None] - o) * inv
            t2 = (b[3:, None] - o) * inv
            tn = np.nanmax(np.minimum(t1, t2), axis=0)
            tf = np.nanmin(np.maximum(t1, t2), axis=0)
            hit |= (np.maximum(tn, shrink) < np.minimum(tf, 1 - shrink))
    return hit


def test_vertices_lie_on_the_nearest_face(oracle_mod):
    s = scenes.small_frame_scene()
    y, ny, fp = oracle_mod.bounce_vertices(s.pos, s.nrm, s.boxes, ROOM, 7, 0, 100.0)
    o = s.pos.astype(np.float64) + 1e-4 * s.nrm.astype(np.float64)
    # paths escape only from points outside the room (some tilted G-buffer planes leave it)
    esc = ~np.isfinite(fp)
    outside = np.any((s.pos < 0) | (s.pos > 1), axis=0)
    assert np.all(outside[esc]) and np.all(ny[:, esc] == 0) and esc.sum() < s.n_points // 100
    y, ny, fp, o = y[:, ~esc], ny[:, ~esc], fp[~esc], o[:, ~esc]
    P = fp.size
    y64 = y.astype(np.float64)
    # unit axis normals turned toward the point
    assert np.all(np.sum(np.abs(ny), axis=0) == 1.0) and np.all(np.sum(ny != 0, axis=0) == 1)
    assert np.all(np.sum(ny * (o - y64), axis=0) > 0)
    # on a face: a room wall or a face of some box (the plane of the reported normal's axis)
    axis = np.argmax(np.abs(ny), axis=0)
    coord = y64[axis, np.arange(P)]
    on = np.isclose(coord, 0.0, atol=1e-5) | np.isclose(coord, 1.0, atol=1e-5)
    for b in s.boxes.astype(np.float64):
        inside = np.all((y64 >= b[:3, None] - 1e-5) & (y64 <= b[3:, None] + 1e-5), axis=0)
        on |= inside & (np.isclose(coord, b[axis], atol=1e-5) | np.isclose(coord, b[3 + axis], atol=1e-5))
    assert np.all(on), int((~on).sum())
    # nothing in between (a point inside a box leaves that box unseen: it is not a surface point)
    in_box = np.zeros(P, bool)
    for b in s.boxes.astype(np.float64):
        in_box |= np.all((o > b[:3, None]) & (o < b[3:, None]), axis=0)
    assert not np.any(_segment_hits_box(o, y64, s.boxes) & ~in_box)
    in_room = ~outside[~esc]
    assert np.all((y64[:, in_room] >= -1e-5) & (y64[:, in_room] <= 1 + 1e-5))
    assert np.all(np.isfinite(fp)) and np.all(fp > 0)
