"""Host-side logic of the serving scheduler (no GPU): admission by memory budget and slots,
exact step counts, latency accounting."""
import numpy as np

from paper_1910_13515_gb300 import inputs
from paper_1910_13515_gb300.serve import Scheduler


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += dt


class FakeBackend:
    """Each run of n steps costs n * cells * 1e-6 s of fake time."""

    def __init__(self, clock):
        self.clock = clock
        self.needs_set = True
        self.resident = []
        self.steps_done = {}
        self.max_bytes_seen = 0
        self.live = {}

    def bytes_for(self, setup):
        return setup.ncells * 100

    def admit(self, setup):
        h = object()
        self.live[h] = setup
        self.steps_done[h] = 0
        self.max_bytes_seen = max(self.max_bytes_seen,
                                  sum(self.bytes_for(s) for s in self.live.values()))
        return h

    def set_resident(self, handles, steps):
        self.resident = list(zip(handles, steps))
        self.needs_set = False

    def run(self, n):
        cells = 0
        for h, target in self.resident:
            k = min(n, target - self.steps_done[h])
            self.steps_done[h] += k
            cells += self.live[h].ncells * k
        self.clock.t += cells * 1e-6 + 1e-6

    def read(self, h):
        return self.steps_done[h]

    def release(self, h):
        del self.live[h]


def make_requests(n=12, seed=4):
    rng = np.random.default_rng(seed)
    reqs = []
    t = 0.0
    for rid in range(n):
        t += rng.exponential(0.01)
        L = int(rng.choice([8, 16, 32]))
        s = inputs.shear_layer(L, 1.0, steps=int(rng.integers(5, 40)))
        reqs.append(inputs.Request(rid, t, s))
    return reqs


def test_every_request_gets_exactly_its_steps_within_budget():
    clock = FakeClock()
    be = FakeBackend(clock)
    reqs = make_requests()
    budget = 3 * 32 * 32 * 100
    rep = Scheduler(be, budget, max_resident=4, chunk_steps=7, clock=clock,
                    sleep=clock.sleep).run(reqs)
    assert sorted(rep.results) == [r.rid for r in reqs]
    for r in reqs:
        assert rep.results[r.rid] == r.setup.steps
    assert be.max_bytes_seen <= budget
    assert 1 <= rep.max_resident <= 4
    assert all(lat > 0 for lat in rep.latencies_s)
    assert rep.cell_steps == sum(r.setup.ncells * r.setup.steps for r in reqs)


def test_requests_overlap_when_budget_allows():
    clock = FakeClock()
    be = FakeBackend(clock)
    reqs = make_requests(8, seed=1)
    rep = Scheduler(be, 10 ** 12, max_resident=64, chunk_steps=1000, clock=clock,
                    sleep=clock.sleep).run(reqs)
    assert rep.max_resident >= 2


def test_oversized_request_is_rejected():
    clock = FakeClock()
    be = FakeBackend(clock)
    reqs = make_requests(2)
    try:
        Scheduler(be, 10, max_resident=2, clock=clock, sleep=clock.sleep).run(reqs)
    except ValueError:
        return
    raise AssertionError("expected ValueError")


def test_withdrawn_requests_are_dropped_or_released_between_steps():
    """A waiting request withdrawn by its client is never admitted; a resident one is released
    at the next run boundary and reported with the steps it completed; the memory it held goes
    to the next request; the others still get exactly their steps."""
    clock = FakeClock()
    be = FakeBackend(clock)
    big = inputs.shear_layer(32, 1.0, steps=400)
    reqs = [inputs.Request(0, 0.0, big, cancel_s=0.05),        # resident, withdrawn mid-run
            inputs.Request(1, 0.0, big),                        # waits for 0's memory
            inputs.Request(2, 0.001, big, cancel_s=0.002),      # withdrawn while waiting
            inputs.Request(3, 0.0, inputs.shear_layer(8, 1.0, steps=30), cancel_s=10.0)]
    budget = be.bytes_for(big) + be.bytes_for(reqs[3].setup)   # room for one big job at a time
    rep = Scheduler(be, budget_bytes=budget, max_resident=4, chunk_steps=16, clock=clock,
                    sleep=clock.sleep).run(reqs)
    # request 0 runs alone (1 waits for memory, 3 queues behind 1) in rounds of 16 steps of
    # 16 * 1024 us of fake time; its withdrawal at 0.05 s falls in the fourth round, so it is
    # released at that round's end with 64 steps done
    assert rep.cancelled[0] == 64
    assert rep.cancelled[2] == 0
    assert sorted(rep.results) == [1, 3]                       # 3 finished before its cancel time
    assert rep.results[1] == 400 and rep.results[3] == 30
    assert be.max_bytes_seen <= budget and not be.live        # everything released


def test_no_withdrawal_changes_nothing():
    reqs = make_requests()
    runs = []
    for cancel in (None, 1e9):
        clock = FakeClock()
        be = FakeBackend(clock)
        rs = [inputs.Request(r.rid, r.arrival_s, r.setup, cancel_s=cancel) for r in reqs]
        rep = Scheduler(be, budget_bytes=10 ** 6, max_resident=4, chunk_steps=8, clock=clock,
                        sleep=clock.sleep).run(rs)
        runs.append((rep.results, rep.latencies_s, rep.rounds, rep.cancelled))
    assert runs[0] == runs[1] and runs[0][3] == {}


class FakeAsyncBackend(FakeBackend):
    """run() only enqueues: the run occupies the fake GPU until its end time; busy() reports
    that, and steps are credited when the run ends.  Admissions while busy are recorded."""

    def __init__(self, clock):
        super().__init__(clock)
        self.end = 0.0
        self.admitted_while_busy = 0
        self.pending_run = None

    def admit(self, setup):
        if self.busy():
            self.admitted_while_busy += 1
        return super().admit(setup)

    def run(self, n):
        assert not self.busy()
        self.pending_run = n
        cells = sum(self.live[h].ncells * min(n, t - self.steps_done[h])
                    for h, t in self.resident)
        self.end = self.clock.t + cells * 1e-6 + 1e-6

    def busy(self):
        return self.clock.t < self.end

    def wait(self):
        if self.clock.t < self.end:
            self.clock.t = self.end
        if self.pending_run is not None:
            n, self.pending_run = self.pending_run, None
            for h, target in self.resident:
                self.steps_done[h] += min(n, target - self.steps_done[h])

    def set_resident(self, handles, steps):
        assert not self.busy()
        super().set_resident(handles, steps)

    def read(self, h):
        assert not self.busy()
        return super().read(h)

    def release(self, h):
        assert not self.busy()
        super().release(h)


def test_arrivals_during_a_run_are_set_up_meanwhile_and_join_the_next_run():
    """With an asynchronous backend the scheduler admits requests that arrive while a run is on
    the GPU (their set-up overlaps it), never changes the resident set, reads or releases while
    a run is in flight, and still gives every request exactly its steps within the budget."""
    clock = FakeClock()
    be = FakeAsyncBackend(clock)
    reqs = make_requests(16, seed=3)
    budget = 6 * 32 * 32 * 100
    rep = Scheduler(be, budget, max_resident=6, chunk_steps=8, clock=clock,
                    sleep=clock.sleep, poll_s=1e-4).run(reqs)
    assert sorted(rep.results) == [r.rid for r in reqs]
    for r in reqs:
        assert rep.results[r.rid] == r.setup.steps
    assert be.max_bytes_seen <= budget and not be.live
    assert be.admitted_while_busy > 0
    assert rep.cell_steps == sum(r.setup.ncells * r.setup.steps for r in reqs)


class FailingBackend(FakeBackend):
    """A backend whose lattice for one request reports fallback cell-steps."""

    def __init__(self, clock, failing_cells):
        super().__init__(clock)
        self.failing_cells = failing_cells

    def failed(self, h):
        return 17 if self.live[h].ncells == self.failing_cells else 0


def test_newton_failures_are_reported_per_request_and_do_not_stop_the_stream():
    clock = FakeClock()
    reqs = make_requests()
    odd = reqs[3].setup.ncells
    be = FailingBackend(clock, odd)
    rep = Scheduler(be, 3 * 32 * 32 * 100, max_resident=4, chunk_steps=7, clock=clock,
                    sleep=clock.sleep).run(reqs)
    assert sorted(rep.results) == [r.rid for r in reqs]
    assert rep.failed == {r.rid: 17 for r in reqs if r.setup.ncells == odd}
    assert rep.failed
