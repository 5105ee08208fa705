"""Host logic of the serving loop (no GPU): admission by volume memory and the
Poisson frame schedule."""
import math

import numpy as np

from paper_2608_08287_gb300 import serving


def _check(plans, budget, window, fps):
    admitted = [p for p in plans if not math.isnan(p.admit)]
    # memory in use never exceeds the budget
    ev = []
    for p in admitted:
        b = serving.volume_bytes(p.res)
        ev += [(p.admit, 1, b), (p.admit + p.duration, 0, -b)]
    used = 0
    for _, _, b in sorted(ev):
        used += b
        assert used <= budget + 1
    # first come, first served: admission order follows request order
    by_req = sorted(admitted, key=lambda p: (p.request, p.sid))
    assert all(a.admit <= b.admit + 1e-12 for a, b in zip(by_req, by_req[1:]))
    for p in admitted:
        assert p.admit >= p.request
        a = p.arrivals
        assert np.all(np.diff(a) > 0)
        if len(a):
            assert a[0] >= p.admit and a[-1] < min(p.admit + p.duration, window)
    return admitted


def test_admission_respects_budget_and_order():
    budget = 60e9
    plans = serving.plan_sessions(96, budget_bytes=budget, window=4.0, min_dur=1.0, max_dur=3.0)
    admitted = _check(plans, budget, 4.0, 30.0)
    waits = [p.admit - p.request for p in admitted]
    assert max(waits) > 0          # the budget actually made sessions wait


def test_unlimited_budget_admits_at_request():
    plans = serving.plan_sessions(40, window=3.0, min_dur=1.0, max_dur=2.0)
    for p in plans:
        assert p.admit == p.request


def test_poisson_rate():
    plans = serving.plan_sessions(64, window=10.0, min_dur=9.0, max_dur=9.5)
    n = sum(len(p.arrivals) for p in plans)
    span = sum(min(p.admit + p.duration, 10.0) - p.admit for p in plans)
    rate = n / span
    assert abs(rate - 30.0) < 1.5    # mean of 30 fps exponential gaps
