"""Host logic of the continuous-batching scheduler, driven by a fake executor
and a fake clock (no GPU)."""
import numpy as np

from paper_1904_02033_b300.serve import Request, Scheduler, run_open_loop


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 1e-5   # time advances with every look at the clock
        return self.t


class FakeExecutor:
    def __init__(self, clock, service=lambda n: 1e-3 + 1e-5 * n, per_query_bytes=100):
        self.clock = clock
        self.service = service
        self.per_query_bytes = per_query_bytes
        self.launched = []
        self.active_bytes = 0
        self.max_active_bytes = 0

    def bytes_for(self, db, n):
        return n * self.per_query_bytes

    def launch(self, db, reqs, slot):
        end = self.clock.t + self.service(len(reqs))
        self.launched.append((db, [r.rid for r in reqs], slot))
        self.active_bytes += self.bytes_for(db, len(reqs))
        self.max_active_bytes = max(self.max_active_bytes, self.active_bytes)
        return (end, len(reqs), db)

    def ready(self, h):
        return self.clock.t >= h[0]

    def finish(self, h, reqs):
        self.active_bytes -= self.bytes_for(h[2], h[1])
        for r in reqs:
            r.result = ("done", r.rid)


def _arrivals(n, rate, seed, dbs=("A", "B")):
    rnd = np.random.default_rng(seed)
    t = np.cumsum(rnd.exponential(1.0 / rate, size=n))
    return [Request(rid=i, db=dbs[int(rnd.integers(0, len(dbs)))], arrival=float(t[i]))
            for i in range(n)]


def test_every_request_served_once_with_batches_bounded():
    clk = FakeClock()
    ex = FakeExecutor(clk)
    s = Scheduler(ex, max_batch=16, slots=3, clock=clk)
    reqs = _arrivals(500, 20000.0, 1)
    stats = run_open_loop(s, reqs)
    served = sorted(rid for _, ids, _ in ex.launched for rid in ids)
    assert served == list(range(500))
    assert all(len(ids) <= 16 for _, ids, _ in ex.launched)
    assert all(r.result == ("done", r.rid) for r in reqs)
    assert len(stats.latencies) == 500 and min(stats.latencies) > 0
    # a batch only ever holds requests of one database, in arrival order
    by_rid = {r.rid: r for r in reqs}
    for db, ids, _ in ex.launched:
        assert all(by_rid[i].db == db for i in ids)
        arr = [by_rid[i].arrival for i in ids]
        assert arr == sorted(arr)


def test_requests_arriving_during_a_batch_join_the_next_one():
    clk = FakeClock()
    ex = FakeExecutor(clk, service=lambda n: 5e-3)
    s = Scheduler(ex, max_batch=128, slots=1, clock=clk)
    # one request, then 10 more while the first batch runs
    reqs = [Request(rid=0, db="A", arrival=0.0)] + \
           [Request(rid=i, db="A", arrival=1e-3 + i * 1e-5) for i in range(1, 11)]
    run_open_loop(s, reqs)
    assert [ids for _, ids, _ in ex.launched] == [[0], list(range(1, 11))]


def test_memory_admission_defers_instead_of_dropping():
    clk = FakeClock()
    ex = FakeExecutor(clk, per_query_bytes=100)
    s = Scheduler(ex, max_batch=64, slots=4, mem_budget=1000, clock=clk)
    reqs = _arrivals(300, 1e6, 2, dbs=("A",))
    run_open_loop(s, reqs)
    assert ex.max_active_bytes <= 1000
    assert all(len(ids) <= 10 for _, ids, _ in ex.launched)
    assert sorted(r for _, ids, _ in ex.launched for r in ids) == list(range(300))


def test_oldest_request_picks_the_database():
    clk = FakeClock()
    ex = FakeExecutor(clk)
    s = Scheduler(ex, max_batch=8, slots=1, clock=clk)
    s.submit(Request(rid=0, db="B", arrival=1.0))
    s.submit(Request(rid=1, db="A", arrival=2.0))
    s.submit(Request(rid=2, db="B", arrival=3.0))
    s.poll()
    assert ex.launched[0][0] == "B" and ex.launched[0][1] == [0, 2]


def test_request_larger_than_the_budget_is_rejected_not_held():
    # a request that alone exceeds the budget can never be admitted: it is
    # rejected at once instead of holding up the queue; the others are served
    clock = FakeClock()

    class PerDb(FakeExecutor):
        def bytes_for(self, db, n):
            return n * (100 if db == "A" else 1000)

    ex = PerDb(clock)
    sched = Scheduler(ex, max_batch=8, slots=2, mem_budget=500, clock=clock)
    reqs = _arrivals(60, 2000.0, 5)
    stats = run_open_loop(sched, reqs, clock=clock)
    big = [r for r in reqs if r.db == "B"]
    small = [r for r in reqs if r.db == "A"]
    assert big and small
    assert all(r.error and r.result is None for r in big)
    assert all(r.error is None and r.result == ("done", r.rid) for r in small)
    assert stats.rejected == len(big) and len(stats.latencies) == len(small)
    assert sched.idle() and ex.max_active_bytes <= 500


from hypothesis import given, settings, strategies as st  # noqa: E402


@settings(max_examples=60, deadline=None)
@given(n=st.integers(1, 80), rate=st.floats(100.0, 1e6), seed=st.integers(0, 2 ** 16),
       slots=st.integers(1, 4), max_batch=st.integers(1, 32), budget=st.integers(50, 5000),
       bytes_a=st.integers(1, 400), bytes_b=st.integers(1, 6000))
def test_scheduler_invariants(n, rate, seed, slots, max_batch, budget, bytes_a, bytes_b):
    # whatever the arrivals, sizes and budget: every request ends served or
    # rejected (rejected exactly when it alone exceeds the budget), the bytes
    # in flight never exceed the budget, batches stay within max_batch and one
    # database, and each database's requests start in arrival order
    clock = FakeClock()
    per = {"A": bytes_a, "B": bytes_b}

    class PerDb(FakeExecutor):
        def bytes_for(self, db, k):
            return k * per[db]

    ex = PerDb(clock)
    sched = Scheduler(ex, max_batch=max_batch, slots=slots, mem_budget=budget, clock=clock)
    reqs = _arrivals(n, rate, seed)
    stats = run_open_loop(sched, reqs, clock=clock)
    assert sched.idle()
    for r in reqs:
        if per[r.db] > budget:
            assert r.error and r.result is None
        else:
            assert r.error is None and r.result == ("done", r.rid)
    assert stats.rejected == sum(per[r.db] > budget for r in reqs)
    assert ex.max_active_bytes <= budget
    by_rid = {r.rid: r for r in reqs}
    for db, ids, _ in ex.launched:
        assert 1 <= len(ids) <= max_batch and all(by_rid[i].db == db for i in ids)
    for db in per:
        starts = [(by_rid[i].arrival, by_rid[i].start) for _, ids, _ in ex.launched for i in ids
                  if by_rid[i].db == db]
        assert [a for a, _ in starts] == sorted(a for a, _ in starts)


def test_batching_window_holds_a_queue_until_full_or_waited_out():
    # with a window, a database's queue is admitted only once it holds
    # max_batch requests or its oldest request has waited the window: batches
    # grow, and no request waits much longer than the window plus service
    clk = FakeClock()
    ex = FakeExecutor(clk)
    window = 2e-3
    s = Scheduler(ex, max_batch=16, slots=3, clock=clk, batch_window=window)
    reqs = _arrivals(400, 4000.0, 7)
    stats = run_open_loop(s, reqs, clock=clk)
    served = sorted(rid for _, ids, _ in ex.launched for rid in ids)
    assert served == list(range(400))
    sizes = [len(ids) for _, ids, _ in ex.launched]
    assert max(sizes) <= 16 and np.mean(sizes) > 3
    # every launched batch was full or its oldest member had waited the window
    by_rid = {r.rid: r for r in reqs}
    for (db, ids, _), (_, n, t) in zip(ex.launched, stats.batches):
        oldest = min(by_rid[i].arrival for i in ids)
        assert n == 16 or t - oldest >= window - 1e-9
    # without the window the same arrivals are admitted at once, in smaller batches
    clk2 = FakeClock()
    ex2 = FakeExecutor(clk2)
    run_open_loop(Scheduler(ex2, max_batch=16, slots=3, clock=clk2), _arrivals(400, 4000.0, 7), clock=clk2)
    assert np.mean([len(ids) for _, ids, _ in ex2.launched]) < np.mean(sizes)


def test_interpolated_service_times():
    from paper_1904_02033_b300.serve import interpolate_ms
    t = [(4, 2.5), (1, 0.75), (2, 1.3)]                 # any order
    assert interpolate_ms(t, 1) == 0.75 and interpolate_ms(t, 4) == 2.5
    assert abs(interpolate_ms(t, 3) - 1.9) < 1e-12       # between the measured sizes
    assert abs(interpolate_ms(t, 8) - 4.9) < 1e-12       # beyond: the last segment's slope
    assert interpolate_ms([(8, 4.0)], 16) == 8.0         # one point: proportional


def test_calibrated_route_takes_the_faster_path():
    from paper_1904_02033_b300.serve import tensor_path_is_faster
    per_query = [(1, 0.75), (2, 1.3), (4, 2.5)]           # about 0.6 ms a query
    big_db = [(8, 3.9), (32, 12.8), (128, 48.0)]         # expansion amortised: 0.4 ms a query
    small_db = [(8, 1.5), (32, 4.8), (128, 18.0)]
    small_pq = [(1, 0.14), (2, 0.23), (4, 0.42)]         # about 0.1 ms a query
    assert all(tensor_path_is_faster(per_query, big_db, n) for n in (8, 16, 64, 128))
    assert not any(tensor_path_is_faster(small_pq, small_db, n) for n in (8, 16, 64, 128))
    assert not tensor_path_is_faster(per_query, [(1, float("inf"))], 64)
