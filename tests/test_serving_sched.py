"""Host logic of the serving loop (no GPU): admission by HBM footprint,
slicing of the targets, retirement."""
import numpy as np
import pytest

from paper_2105_09644_gb300.serving import Request, Scheduler, footprint_bytes, percentile


def fake(rid, N, t):
    return Request(rid, t, N, 1.0, np.zeros((1, 1, 1)), np.zeros((0, 3)), np.zeros(0))


def drive(sched, reqs, rng):
    now = 0.0
    pending = sorted(reqs, key=lambda r: r.arrival)
    seen = {r.rid: [] for r in reqs}
    peak = 0
    while pending or not sched.idle():
        while pending and pending[0].arrival <= now:
            sched.submit(pending.pop(0))
        sched.admit(now)
        assert sched.in_use <= sched.budget
        assert sched.in_use == sum(r.footprint for r in sched.active)
        peak = max(peak, sched.in_use)
        slices = sched.plan()
        for r, f, c in slices:
            seen[r.rid].append((f, c))
        now += 1.0
        sched.complete(slices, now)
    return seen, peak


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_admission_and_coverage(seed):
    rng = np.random.default_rng(seed)
    reqs = [fake(k, int(rng.choice([8, 16, 32, 64])), float(rng.uniform(0, 20))) for k in range(40)]
    budget = 3 * footprint_bytes(64, 1)
    sched = Scheduler(budget, tick_targets=50000, precision=1)
    seen, peak = drive(sched, reqs, rng)
    assert len(sched.finished) == len(reqs) and peak <= budget
    for r in reqs:
        parts = seen[r.rid]
        # Morton ranges cover the targets once, in order
        pos = 0
        for f, c in parts:
            assert f == pos and c > 0
            pos += c
        assert pos == r.N ** 3
        assert r.done >= r.arrival and r.latency >= 0


def test_small_requests_go_first():
    sched = Scheduler(10 ** 12, tick_targets=10000, precision=1)
    big, small = fake(0, 64, 0.0), fake(1, 8, 0.0)
    sched.submit(big)
    sched.submit(small)
    sched.admit(0.0)
    plan = sched.plan()
    assert plan[0][0] is small and plan[0][2] == 512
    assert sum(c for _, _, c in plan) <= 10000 + 4096


def test_oversized_request_is_refused():
    sched = Scheduler(footprint_bytes(32, 1), tick_targets=1000)
    sched.submit(fake(0, 128, 0.0))
    with pytest.raises(ValueError):
        sched.admit(0.0)


def test_percentile():
    xs = list(range(1, 101))
    assert percentile(xs, 50) == 50 and percentile(xs, 99) == 99 and percentile([], 50) is None


def test_lazy_stream_is_filled_in_order_and_released():
    """Requests with lazy data get their density when the server asks for
    it, the same values as an eager stream, and the host copy is dropped
    once the request is on the device (no GPU: the device work is stubbed)."""
    from paper_2105_09644_gb300.serving import Server, poisson_stream

    class HostOnly(Server):
        def __init__(self, *a, **kw):
            super().__init__(*a, **kw)
            self.seen = []

        def _start(self, req):
            assert req.n_H is not None and req.n_H.shape == (req.N,) * 3
            self.seen.append((req.rid, float(req.n_H.sum())))
            if req.make is not None:
                req.n_H = None

        def tick(self):
            for req in self.sched.admit(self.now()):
                self._start(req)
            slices = self.sched.plan()
            if not slices:
                return 0
            for req in self.sched.complete(slices, self.now()):
                req.result = {}
            return sum(c for _, _, c in slices)

    eager = poisson_stream(12, 500.0, seed=7, sizes=(8, 16), nsides=(2,), max_sources=10)
    lazy = poisson_stream(12, 500.0, seed=7, sizes=(8, 16), nsides=(2,), max_sources=10, lazy=True)
    assert all(r.n_H is None for r in lazy)
    srv = HostOnly(budget_bytes=1 << 30, tick_targets=1 << 12, keep_results=False)
    done = srv.run(lazy, prefetch=2)
    assert len(done) == 12 and all(r.n_H is None for r in done)
    sums = dict(srv.seen)
    for r in eager:
        assert sums[r.rid] == float(r.n_H.sum())
