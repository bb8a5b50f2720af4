"""Pins of the oracle's binary32 shadow test (the visibility V of the
contribution, Section 3): segment from o = x + 1e-4 n to the light point y,
t in (0, 0.9999), slab test against every box with open intervals. It is
checked against the double test of the brute-force reference, which treats a
segment parallel to an axis by containment (b_min < o < b_max on that axis):

* hand cases: a segment lying in the plane x = 0.5 is blocked by a box whose
  x range contains 0.5 and by no box beside that plane, whatever its y and z
  ranges;
* segments exactly parallel to one axis (y_k = o_k) next to boxes that do not
  reach that coordinate are never blocked (1/d_k would be infinite: the
  planes of that axis are undefined unless the component is handled);
* random segments in the room against the frame workload's 64 boxes, a third
  of them made exactly parallel to a random axis: both tests agree on all
  but grazing segments (at most 1 in 10^4).
"""
import numpy as np

from paper_1911_10217_gb300 import scenes


def test_parallel_segment_hand_cases(oracle_mod):
    o = np.array([0.5, 0.1, 0.1], np.float32)
    y = np.array([0.5, 0.9, 0.9], np.float32)  # d_x = 0 exactly
    beside = np.array([[0.6, 0.0, 0.0, 0.8, 1.0, 1.0]], np.float32)
    across = np.array([[0.4, 0.4, 0.4, 0.6, 0.6, 0.6]], np.float32)
    below = np.array([[-0.2, 0.0, 0.0, 0.4999, 1.0, 1.0]], np.float32)
    for boxes, blocked in ((beside, False), (across, True), (below, False)):
        assert oracle_mod.occluded32(o, y, boxes) is blocked
        assert oracle_mod.occluded64(o, y, boxes) is blocked
    # the same along y and z
    for axis in (1, 2):
        perm = [axis, (axis + 1) % 3, (axis + 2) % 3]
        inv = np.argsort(perm)
        bx = np.concatenate([beside[0, :3][inv], beside[0, 3:][inv]])[None]
        ax = np.concatenate([across[0, :3][inv], across[0, 3:][inv]])[None]
        assert not oracle_mod.occluded32(o[inv], y[inv], bx)
        assert oracle_mod.occluded32(o[inv], y[inv], ax)


def test_parallel_segments_beside_boxes_are_never_blocked(oracle_mod):
    rng = np.random.default_rng(5)
    boxes = np.array([[0.6, 0.0, 0.0, 0.8, 1.0, 1.0],
                      [0.1, 0.2, 0.3, 0.45, 0.7, 0.9],
                      [0.55, 0.05, 0.5, 0.95, 0.35, 0.95]], np.float32)
    for _ in range(2000):
        o = rng.uniform(0.0, 1.0, 3).astype(np.float32)
        y = rng.uniform(0.0, 1.0, 3).astype(np.float32)
        o[0] = y[0] = np.float32(rng.choice([0.5, 0.47, 0.52]))  # between the boxes' x ranges
        assert not oracle_mod.occluded32(o, y, boxes)
        assert not oracle_mod.occluded64(o, y, boxes)


def test_shadow_test_agrees_with_the_double_test(oracle_mod):
    s = scenes.frame_scene()
    boxes = s.boxes.astype(np.float32)
    rng = np.random.default_rng(9)
    n = 20000
    diff = 0
    n_par = 0
    for i in range(n):
        o = rng.uniform(0.0, 1.0, 3).astype(np.float32)
        y = rng.uniform(0.0, 1.0, 3).astype(np.float32)
        if i % 3 == 0:
            k = int(rng.integers(3))
            y[k] = o[k]
            n_par += 1
        a = oracle_mod.occluded32(o, y, boxes)
        b = oracle_mod.occluded64(o.astype(np.float64), y.astype(np.float64), boxes)
        diff += a != b
    assert n_par > n // 4
    assert diff <= n // 10000, diff
