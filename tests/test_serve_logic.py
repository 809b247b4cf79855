"""Scheduling logic of the continuous-batching loop, driven by a fake backend on the CPU."""
import itertools

import pytest

import synthmedia
from paper_2006_11945_gb300.serve import NoMemory, Request, serve


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 1e-4
        return self.t


class FakeBackend:
    """Holds solves in a fixed 'memory' budget; one evolve chunk advances time."""

    def __init__(self, budget_cells, clock):
        self.budget = budget_cells
        self.used = 0
        self.clock = clock
        self.log = []

    def admit(self, req):
        if self.used + req.problem.cells > self.budget:
            raise NoMemory()
        self.used += req.problem.cells
        self.log.append(('admit', req.rid))

    def evolve(self, reqs, steps, cfl):
        assert len(reqs) == len(steps) and all(s > 0 for s in steps)
        self.log.append(('evolve', tuple(r.rid for r in reqs), tuple(steps)))
        self.clock.t += 0.01

    def finish(self, req):
        self.used -= req.problem.cells
        self.log.append(('finish', req.rid))
        return req.rid


def _reqs(n, steps, arrivals):
    out = []
    for i, t in zip(range(n), arrivals):
        p = synthmedia.vti_homogeneous(n=16, n_theta=16, steps=steps[i % len(steps)])
        out.append(Request(i, t, p))
    return out


def test_all_requests_complete_and_memory_bounds_admission():
    clock = FakeClock()
    reqs = _reqs(10, [7, 30, 61], [0.001 * i for i in range(10)])
    cells = reqs[0].problem.cells
    be = FakeBackend(budget_cells=3 * cells, clock=clock)
    st = serve(reqs, be, chunk_steps=10, clock=clock)
    assert sorted(r.rid for r in st.completed) == list(range(10))
    assert st.max_active <= 3
    assert st.refused_admissions > 0
    assert be.used == 0
    for r in st.completed:
        assert r.finished >= r.admitted >= r.arrival
        assert r.steps_left == 0


def test_steps_are_exact_per_request():
    clock = FakeClock()
    reqs = _reqs(4, [7, 30, 61, 1], [0.0] * 4)
    be = FakeBackend(budget_cells=10 ** 9, clock=clock)
    serve(reqs, be, chunk_steps=10, clock=clock)
    taken = {r.rid: 0 for r in reqs}
    for e in be.log:
        if e[0] == 'evolve':
            for rid, s in zip(e[1], e[2]):
                taken[rid] += s
    assert taken == {0: 7, 1: 30, 2: 61, 3: 1}


def test_late_arrivals_join_running_batch():
    clock = FakeClock()
    reqs = _reqs(2, [100], [0.0, 0.015])
    be = FakeBackend(budget_cells=10 ** 9, clock=clock)
    serve(reqs, be, chunk_steps=10, clock=clock)
    evolves = [e for e in be.log if e[0] == 'evolve']
    assert any(e[1] == (0, 1) for e in evolves), evolves
    assert evolves[0][1] == (0,)


def test_time_limit_stops_admission():
    clock = FakeClock()
    reqs = _reqs(5, [10], [0.0, 0.0, 0.5, 0.6, 0.7])
    be = FakeBackend(budget_cells=10 ** 9, clock=clock)
    st = serve(reqs, be, chunk_steps=10, clock=clock, time_limit=0.2)
    assert sorted(r.rid for r in st.completed) == [0, 1]
