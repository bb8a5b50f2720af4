"""Input generators (not the method): the sky-dome interior is built as
documented -- every emitter faces the room, no triangle is degenerate, the
walls are closed except at the openings."""
import numpy as np

from paper_1911_10217_gb300 import scenes


def _segment_blocked(o, y, boxes):
    d = y - o
    for b in boxes:
        with np.errstate(divide="ignore", invalid="ignore"):
            t0 = (b[:3] - o) / d
            t1 = (b[3:] - o) / d
        lo = np.nanmax(np.minimum(t0, t1))
        hi = np.nanmin(np.maximum(t0, t1))
        if max(lo, 0.0) < min(hi, 1.0):
            return True
    return False


def test_sky_scene_geometry():
    s = scenes.sky_scene(width=64, height=36, sun=True)
    assert s.n_lights == 2 * 32 * 32 + 2
    assert scenes.sky_scene(width=8, height=8).n_lights == 2 * 32 * 32
    t = s.tris.astype(np.float64)
    n = np.cross(t[:, 1] - t[:, 0], t[:, 2] - t[:, 0])
    assert np.all(np.linalg.norm(n, axis=1) > 1e-3)
    centroid = t.mean(axis=1)
    assert np.all(np.einsum("ij,ij->i", n, np.array([0.5, 0.0, 0.5]) - centroid) > 0)
    boxes = s.boxes.astype(np.float64)
    # straight up from the room centre hits the ceiling; through a skylight it does not
    assert _segment_blocked(np.array([0.5, 0.1, 0.5]), np.array([0.5, 5.0, 0.5]), boxes)
    assert not _segment_blocked(np.array([0.31, 0.6, 0.36]), np.array([0.31, 5.0, 0.36]), boxes)
    # every horizontal ray from the centre at window height is blocked except through windows
    hits = [_segment_blocked(np.array([0.5, 0.45, 0.5]),
                             np.array([0.5 + 3 * np.cos(a), 0.45, 0.5 + 3 * np.sin(a)]), boxes)
            for a in np.linspace(0, 2 * np.pi, 720, endpoint=False)]
    assert 0.5 < np.mean(hits) < 1.0
