"""CPU tests of the serving policy (no GPU): admission by memory budget,
one frame in flight per session, oldest request first, per-launch capacity,
release of finished sessions."""
import pytest

from paper_1911_10217_gb300.serving import Request, Scheduler, poisson_arrivals, session_bytes


def _sched(budget=100, items=4, records=1000, cells=1000):
    return Scheduler(budget, items, records, cells)


def test_admission_respects_budget_and_order():
    s = _sched(budget=100)
    s.add_session(0, 60, 10, 10, 1)
    s.add_session(1, 50, 10, 10, 1)
    s.add_session(2, 30, 10, 10, 1)
    assert s.admit() == [0]          # 1 does not fit; 2 waits behind it (no overtaking)
    assert s.used == 60
    s.arrive(Request(0, 0, 0.0))
    b = s.form_batch()
    assert [r.session for r in b] == [0]
    assert s.complete(b, 1.0) == [0] and s.used == 0
    assert s.admit() == [1, 2] and s.used == 80


def test_one_frame_in_flight_per_session_and_fifo():
    s = _sched()
    for sid in range(3):
        s.add_session(sid, 1, 10, 10, 5)
    s.admit()
    s.arrive(Request(1, 0, 0.5))
    s.arrive(Request(0, 0, 0.1))
    s.arrive(Request(0, 1, 0.2))
    s.arrive(Request(2, 0, 0.9))
    b1 = s.form_batch()
    assert [(r.session, r.frame) for r in b1] == [(0, 0), (1, 0), (2, 0)]
    assert s.form_batch() == []       # every session busy
    s.complete(b1, 1.0)
    b2 = s.form_batch()
    assert [(r.session, r.frame) for r in b2] == [(0, 1)]
    assert s.sessions[0].next_frame == 1


def test_launch_capacity():
    s = _sched(items=2, records=25, cells=1000)
    for sid in range(4):
        s.add_session(sid, 1, 10, 10, 1)
        s.arrive(Request(sid, 0, float(sid)))
    s.admit()
    assert [r.session for r in s.form_batch()] == [0, 1]
    s2 = _sched(items=8, records=25, cells=15)
    for sid in range(3):
        s2.add_session(sid, 1, 10, 10, 1)
        s2.arrive(Request(sid, 0, float(sid)))
    s2.admit()
    assert [r.session for r in s2.form_batch()] == [0]   # cells: 10 + 10 > 15
    with pytest.raises(ValueError):
        s2.add_session(9, 1, 100, 1, 1)


def test_all_sessions_finish():
    s = _sched(budget=3)
    for sid in range(6):
        s.add_session(sid, 1, 1, 1, 2)
    t = 0.0
    for sid in range(6):
        for f in range(2):
            s.arrive(Request(sid, f, t))
            t += 0.01
    steps = 0
    while not s.idle():
        s.admit()
        b = s.form_batch()
        assert len({r.session for r in b}) == len(b)
        s.complete(b, t)
        steps += 1
        assert steps < 100
    assert len(s.log) == 12 and s.used == 0


def test_helpers():
    import numpy as np
    a = poisson_arrivals(np.random.default_rng(0), 20000, 50.0)
    assert np.all(np.diff(a) > 0)
    assert np.mean(np.diff(a)) == pytest.approx(1 / 50.0, rel=0.05)
    assert session_bytes(1 << 20, 3840 * 2160, 1 << 21, 64, "bf16") == pytest.approx(1.7e9, rel=0.1)
