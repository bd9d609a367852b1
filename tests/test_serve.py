"""Host logic of the serving loop (no GPU): arena allocation and the
continuous-batching scheduler on a simulated device."""
import random

import pytest

from paper_2309_04909_gb300.serve import Arena, Engine, FakeExecutor, ServeRequest, ServeStats


def test_arena_first_fit_and_coalescing():
    a = Arena(1 << 20)
    x = a.alloc(1000)
    y = a.alloc(5000)
    z = a.alloc(256)
    assert x == 0 and y == 1024 and z == 1024 + 5120
    assert a.alloc(1 << 20) is None
    a.free(y, 5000)
    assert a.alloc(4000) == 1024          # first fit reuses the hole
    a.free(1024, 4000)
    a.free(x, 1000)
    a.free(z, 256)
    assert a.used == 0 and a.free_blocks == 1
    rng = random.Random(1)
    live = []
    for _ in range(2000):
        if live and rng.random() < 0.45:
            off, sz = live.pop(rng.randrange(len(live)))
            a.free(off, sz)
        else:
            sz = rng.randrange(1, 20000)
            off = a.alloc(sz)
            if off is not None:
                live.append((off, sz))
        spans = sorted((o, (s + 255) // 256 * 256) for o, s in live)
        assert all(s0 + l0 <= s1 for (s0, l0), (s1, _) in zip(spans, spans[1:]))
        assert a.used <= a.capacity
    for off, sz in live:
        a.free(off, sz)
    assert a.free_blocks == 1 and a.used == 0


def _trace(n, rate, seed=0, max_elems=5_000_000):
    rng = random.Random(seed)
    t, out = 0.0, []
    for i in range(n):
        t += rng.expovariate(rate)
        out.append(ServeRequest(i, t, rng.randrange(1000, max_elems)))
    return out


def test_engine_completes_every_request_in_budget():
    reqs = _trace(300, rate=2000.0)
    ex = FakeExecutor(rate_elems_per_s=8e9)
    budget = 4 << 30
    st = Engine(ex, budget, max_iter_elems=1 << 23).run(reqs)
    assert st.completed == len(reqs) and st.rejected == 0
    assert st.peak_bytes <= budget
    assert st.elements == sum(r.elements for r in reqs)
    for r in reqs:
        # no result before its own work could have run
        assert r.finished_s >= r.arrival_s + r.elements / 8e9 - 1e-12
        assert r.admitted_s >= r.arrival_s
    # every request's elements were launched exactly once, in order
    seen = {}
    for it in ex.launched:
        for rid, start, count in it:
            assert seen.get(rid, 0) == start
            seen[rid] = start + count
    assert all(seen[r.rid] == r.elements for r in reqs)


def test_engine_overlaps_requests_in_one_iteration():
    """Continuous batching: requests that arrive while others run share the
    next iteration instead of waiting for the device to drain."""
    reqs = [ServeRequest(0, 0.0, 4_000_000)] + [ServeRequest(i, 1e-4 * i, 10_000) for i in range(1, 6)]
    ex = FakeExecutor(rate_elems_per_s=1e9)
    Engine(ex, 1 << 30, max_iter_elems=1 << 20).run(reqs)
    mixed = [it for it in ex.launched if len({rid for rid, _, _ in it}) > 1]
    assert mixed, "no iteration mixed requests"
    small_done = max(r.finished_s for r in reqs[1:])
    assert small_done < reqs[0].finished_s     # the small requests did not wait for the big one


def test_engine_memory_budget_blocks_and_rejects():
    reqs = [ServeRequest(i, 0.0, 1_000_000) for i in range(10)] + [ServeRequest(99, 0.0, 10 ** 9)]
    ex = FakeExecutor(rate_elems_per_s=1e9)
    budget = 3 * 1_000_000 * 32 + 1000          # three requests at a time
    st = Engine(ex, budget, max_iter_elems=1 << 22).run(reqs)
    assert st.rejected == 1 and reqs[-1].rejected
    assert st.completed == 10
    assert st.peak_bytes <= budget
    # admissions were spaced by completions
    adm = sorted(r.admitted_s for r in reqs[:10])
    assert adm[3] > 0.0


def test_summary_percentiles():
    reqs = _trace(50, rate=100.0, max_elems=100_000)
    st = Engine(FakeExecutor(1e9), 1 << 30).run(reqs)
    s = st.summary()
    assert s["p50_ms"] <= s["p99_ms"] <= s["max_ms"]
    assert s["completed"] == 50


def test_engine_cancellation_and_deadlines():
    """Requests cancelled by the client or past their deadline are dropped:
    queued ones at once, admitted ones once their chunks in flight retire;
    their memory returns to the arena and every other request completes."""
    rng = random.Random(3)
    reqs = []
    for i in range(200):
        r = ServeRequest(i, 1e-4 * i, rng.randrange(500_000, 3_000_000))
        if i % 10 == 3:
            r.cancel_at_s = r.arrival_s + 2e-4
        if i % 10 == 7:
            r.deadline_s = r.arrival_s + 1e-3
        reqs.append(r)
    ex = FakeExecutor(rate_elems_per_s=2e9)          # overloaded: deadlines bite
    eng = Engine(ex, 2 << 30, max_iter_elems=1 << 22)
    st = eng.run(reqs)
    assert eng.arena.used == 0
    dropped = [r for r in reqs if r.dropped and r.finished_s is None]
    assert st.cancelled + st.expired == len(dropped) > 0
    assert st.completed + len(dropped) == len(reqs)
    assert all(r.finished_s is not None for r in reqs if r.dropped is None)
    for r in reqs:
        if r.dropped == "expired" and r.finished_s is None:
            assert r.deadline_s is not None
    # no chunk of a dropped request was launched after it was dropped
    assert all(r.done <= r.elements for r in reqs)


def test_engine_under_load_simulated():
    """The serving trace on a simulated device of the measured batched
    capacity: below capacity every request finishes within a few of its own
    service times and throughput follows the offered load; above it the
    device stays saturated and the queue grows."""
    from paper_2309_04909_gb300 import workloads as W
    per = {"vgg16": sum(W.VGG16_32_LAYERS), "lenet": sum(W.LENET_28_LAYERS)}
    cap = 7.7e9
    mean = 0.5 * 32.5 * (per["vgg16"] + per["lenet"])
    out = {}
    for frac in (0.5, 1.2):
        trace = W.serving_trace(frac * cap / mean, 1.0, seed=4)
        reqs = [ServeRequest(r.rid, r.arrival_s, r.images * per[r.net], r.net, r.images)
                for r in trace]
        st = Engine(FakeExecutor(cap), 40 << 30).run(reqs)
        assert st.completed == len(reqs)
        out[frac] = st.summary()
    half, over = out[0.5], out[1.2]
    largest = 64 * per["vgg16"] / cap * 1e3                 # ms of the largest request alone
    assert half["p99_ms"] < 4 * largest and half["max_waiting"] < 20
    assert abs(half["elems_per_s"] / (0.5 * cap) - 1) < 0.15
    assert over["elems_per_s"] > 0.95 * cap                   # saturated
    assert over["p50_ms"] > 20 * half["p50_ms"] and over["max_waiting"] > 100
    # the queue at the last arrival: it grows at about the excess arrival
    # rate above capacity, and finishing it takes a while; below capacity it
    # stays a handful of requests and drains at once
    excess = (1.2 - 1.0) * cap / mean                        # requests per second
    assert 0.5 * excess < over["queue_growth_per_s"] < 1.5 * excess
    assert over["drain_s"] > 0.1 and over["elems_per_s_during_arrivals"] > 0.95 * cap
    assert half["backlog_at_arrival_end"] < 20 and half["drain_s"] < 0.05


def test_latency_histogram():
    st = ServeStats(5, 5, 10, 1.0, [0.0005, 0.0015, 0.003, 0.003, 2.0], 1, 0, 0)
    h = st.summary()["latency_histogram_ms"]
    assert h == {"<=1": 1, "<=2": 1, "<=4": 2, ">1024": 1}
    assert sum(h.values()) == 5


def test_ideal_latencies_by_hand():
    """The ideal-server yardstick on cases worked by hand."""
    from paper_2309_04909_gb300.serve import ideal_latencies
    arr, work = [0.0, 1.0, 1.5], [2.0, 1.0, 0.25]
    # first come: finishes at 2, 3, 3.25
    assert ideal_latencies(arr, work, "fcfs") == pytest.approx([2.0, 2.0, 1.75])
    # shortest remaining first: 0 runs to 1 (1 left), 1 arrives (1 left) and
    # ties go to the lower index, so 0 runs to 1.5 (0.5 left); 2 (0.25) runs
    # to 1.75, then 0 to 2.25, then 1 to 3.25
    assert ideal_latencies(arr, work, "srpt") == pytest.approx([2.25, 2.25, 0.25])
    # processor sharing: two equal jobs arriving together both finish at 2 x work
    assert ideal_latencies([0.0, 0.0], [1.0, 1.0], "ps") == pytest.approx([2.0, 2.0])
    # a lone job is served at full rate, and order of the inputs does not matter
    assert ideal_latencies([5.0], [0.5], "ps") == pytest.approx([0.5])
    assert ideal_latencies([1.0, 0.0], [1.0, 2.0], "fcfs") == pytest.approx([2.0, 2.0])
    with pytest.raises(ValueError):
        ideal_latencies(arr, work, "lifo")
