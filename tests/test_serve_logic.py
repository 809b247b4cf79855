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

    def cancel(self, req):
        self.used -= req.problem.cells
        self.log.append(('cancel', req.rid))


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
    # the requests still queued when admission closed are counted, so every offered one is accounted for
    assert sorted(r.rid for r in st.not_admitted) == [2, 3, 4]
    s = st.summary(5)
    assert s['completed'] + s['cancelled'] + s['unfinished'] + s['not_admitted'] == 5


def test_request_cancelled_between_chunks_is_released_and_frees_its_memory():
    """A client cancels request 0 while it is on the device: the loop releases its solve at the next
    chunk boundary (no superposition), the waiting request takes its memory, the others complete."""
    clock = FakeClock()
    reqs = _reqs(3, [100, 20, 20], [0.0, 0.0, 0.0])
    cells = reqs[0].problem.cells
    be = FakeBackend(budget_cells=2 * cells, clock=clock)
    orig = be.evolve

    def evolve(active, steps, cfl):
        orig(active, steps, cfl)
        if sum(1 for e in be.log if e[0] == 'evolve') == 1:
            reqs[0].cancel()
    be.evolve = evolve
    st = serve(reqs, be, chunk_steps=10, clock=clock)
    assert [r.rid for r in st.cancelled] == [0]
    assert sorted(r.rid for r in st.completed) == [1, 2]
    assert reqs[0].result is None and reqs[0].finished is None
    assert be.used == 0
    log = [e[:2] for e in be.log if e[0] in ('admit', 'cancel', 'finish')]
    # request 2 waits for memory and is admitted right after the cancellation frees it
    assert log.index(('cancel', 0)) < log.index(('admit', 2))
    assert not any(e[0] == 'evolve' and 0 in e[1] for e in be.log[be.log.index(('cancel', 0)):])
    assert st.summary(3)['cancelled'] == 1


def test_request_cancelled_before_admission_never_reaches_the_device():
    clock = FakeClock()
    reqs = _reqs(3, [30], [0.0, 0.0, 0.0])
    cells = reqs[0].problem.cells
    be = FakeBackend(budget_cells=cells, clock=clock)
    reqs[2].cancel()
    st = serve(reqs, be, chunk_steps=10, clock=clock)
    assert [r.rid for r in st.cancelled] == [2]
    assert sorted(r.rid for r in st.completed) == [0, 1]
    assert ('admit', 2) not in be.log


def test_wall_limit_releases_unfinished_requests():
    clock = FakeClock()
    reqs = _reqs(3, [1000], [0.0, 0.0, 0.0])
    be = FakeBackend(budget_cells=10 ** 9, clock=clock)
    st = serve(reqs, be, chunk_steps=10, clock=clock, wall_limit=0.05)
    assert not st.completed and sorted(r.rid for r in st.unfinished) == [0, 1, 2]
    assert be.used == 0 and st.summary(3)['unfinished'] == 3 and not st.not_admitted


def test_work_budgeted_chunks_finish_small_requests_first():
    """With a per-request work budget a small request finishes in its first chunk, and with a cap
    on a chunk's work the waiting small requests are admitted ahead of large ones."""
    clock = FakeClock()
    small = [Request(i, 0.0, synthmedia.vti_homogeneous(n=16, n_theta=16, steps=40)) for i in range(3)]
    large = [Request(10 + i, 0.0, synthmedia.vti_homogeneous(n=32, n_theta=32, steps=400)) for i in range(3)]
    cs, cl = small[0].problem.cells, large[0].problem.cells
    be = FakeBackend(budget_cells=10 ** 12, clock=clock)
    st = serve(large + small, be, chunk_steps=10, clock=clock, chunk_work=40 * cs,
               max_chunk_work=10 * cl + 3 * 40 * cs)
    evolves = [e for e in be.log if e[0] == 'evolve']
    first = dict(zip(evolves[0][1], evolves[0][2]))
    assert all(first[r.rid] == 40 for r in small)           # whole small solves in the first chunk
    assert sum(1 for rid in first if rid >= 10) == 1        # the cap admits one large request
    done_small = max(r.finished for r in st.completed if r.rid < 10)
    assert done_small < min(r.finished for r in st.completed if r.rid >= 10)
    assert sorted(r.rid for r in st.completed) == [0, 1, 2, 10, 11, 12]
