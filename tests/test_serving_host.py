"""Host logic of the serving loop, on CPU: the native arena and the admission
scheduler driven by a fake executor (no GPU)."""

import math
import time

import numpy as np
import pytest

from paper_1607_04245_gb300 import build as fem_build


@pytest.fixture(scope="module")
def serving():
    fem_build.build()
    from paper_1607_04245_gb300 import serving

    return serving


def test_arena_first_fit_and_coalescing(serving):
    a = serving.Arena(4096, 256)
    assert a.capacity == 4096 and a.free_bytes == 4096
    x = a.alloc(100)  # rounded to 256
    y = a.alloc(1000)  # 1024
    z = a.alloc(256)
    assert (x, y, z) == (0, 256, 1280)
    assert a.free_bytes == 4096 - 256 - 1024 - 256
    assert a.alloc(4096) is None  # no room
    a.free(y)
    assert a.alloc(768) == 256  # first fit reuses the hole
    a.free(256)
    a.free(x)
    a.free(z)
    assert a.free_bytes == 4096 and a.largest_free == 4096  # fully merged
    with pytest.raises(Exception):
        a.free(12345)
    assert a.alloc(0) == 0  # zero-byte requests still get a distinct offset


def test_arena_random_ops_never_overlap(serving):
    rng = np.random.default_rng(0)
    a = serving.Arena(1 << 20, 256)
    live = {}
    for _ in range(2000):
        if live and rng.random() < 0.45:
            off = list(live)[int(rng.integers(0, len(live)))]
            a.free(off)
            del live[off]
        else:
            n = int(rng.integers(1, 50000))
            off = a.alloc(n)
            if off is not None:
                sz = (n + 255) // 256 * 256
                for o, s in live.items():
                    assert off + sz <= o or o + s <= off
                assert off + sz <= a.capacity
                live[off] = sz
        assert a.free_bytes == a.capacity - sum(live.values())


class FakeRequest:
    def __init__(self, rid, n_cells, mem, arrival):
        self.rid, self.n_cells, self.mem, self.arrival = rid, n_cells, mem, arrival
        self.status, self.error = "pending", ""
        self.t_arrive = self.t_admit = self.t_done = math.nan

    @property
    def latency(self):
        return self.t_done - self.t_arrive


class FakeExecutor:
    """Slots and a memory budget; a request 'runs' for 1e-8 s per cell of wall time."""

    def __init__(self, capacity, n_slots):
        self.capacity, self.n_slots = capacity, n_slots
        self.used, self.inflight, self.order, self.peak = 0, {}, [], 0

    def fits_ever(self, r):
        return r.mem <= self.capacity

    def try_admit(self, r):
        if len(self.inflight) >= self.n_slots or self.used + r.mem > self.capacity:
            return None
        return True

    def launch(self, r, adm):
        self.used += r.mem
        self.peak = max(self.peak, self.used)
        self.inflight[r.rid] = (r, time.perf_counter() + 1e-8 * r.n_cells)
        self.order.append(r.rid)

    def poll(self):
        now, done = time.perf_counter(), []
        for rid, (r, t) in list(self.inflight.items()):
            if now >= t:
                self.used -= r.mem
                del self.inflight[rid]
                done.append(r)
        return done

    def busy(self):
        return bool(self.inflight)


def test_scheduler_admission_by_memory_and_slots(serving):
    rng = np.random.default_rng(3)
    reqs = [FakeRequest(i, int(rng.integers(1000, 200000)), int(rng.integers(1, 40)), 0.0005 * i) for i in range(60)]
    reqs.append(FakeRequest(60, 1000, 1000, 0.001))  # can never fit: rejected
    ex = FakeExecutor(capacity=100, n_slots=4)
    st = serving.Scheduler(ex, backfill=False).run(reqs)
    assert st.n_done == 60 and st.n_rejected == 1
    assert ex.peak <= 100
    assert st.max_inflight <= 4
    # without backfill admission follows arrival order
    assert ex.order == sorted(ex.order)
    assert all(r.t_done >= r.t_admit >= r.t_arrive for r in reqs if r.status == "done")
    assert st.p99_ms >= st.p50_ms > 0


def test_scheduler_backfill_lets_small_requests_pass(serving):
    big = FakeRequest(0, 300000, 90, 0.0)
    blocked = FakeRequest(1, 1000, 50, 0.0001)  # cannot fit while `big` runs
    small = FakeRequest(2, 1000, 5, 0.0002)  # fits next to `big`
    ex = FakeExecutor(capacity=100, n_slots=4)
    serving.Scheduler(ex, backfill=True).run([big, blocked, small])
    assert ex.order.index(2) < ex.order.index(1)
    ex2 = FakeExecutor(capacity=100, n_slots=4)
    serving.Scheduler(ex2, backfill=False).run([FakeRequest(0, 300000, 90, 0.0), FakeRequest(1, 1000, 50, 0.0001),
                                                FakeRequest(2, 1000, 5, 0.0002)])
    assert ex2.order == [0, 1, 2]


def test_poisson_arrivals(serving):
    t = serving.poisson_arrivals(20000, rate=500.0, seed=1)
    assert np.all(np.diff(t) >= 0)
    assert t[-1] / 20000 == pytest.approx(1 / 500.0, rel=0.03)


def test_serving_specs_mix():
    import workloads

    specs = workloads.cases.serving_specs(500, seed=0)
    C = np.array([s["n_cells"] for s in specs])
    assert C.min() >= 1000 and C.max() <= 1_000_000
    assert {(s["physics"], s["dim"]) for s in specs} == set(workloads.cases.SERVING_PHYSICS)
    assert all(s["kind"] == "residual" for s in specs if s["physics"] == "elasticity")
    assert any(s["kind"] == "adjoint" for s in specs)
    # log-uniform: the median is near the geometric mean of the bounds
    assert 10 ** 4.2 < np.median(C) < 10 ** 4.8
    c = workloads.cases.serving_case(specs[0])
    assert c.n_cells == specs[0]["n_cells"]


def test_request_log_save_and_replay(serving, tmp_path):
    """A served stream's log (arrival, admission, completion, status) can be saved and its
    arrivals replayed: the second run admits in the same order."""
    rng = np.random.default_rng(7)
    reqs = [FakeRequest(i, int(rng.integers(1000, 50000)), int(rng.integers(1, 30)), 0.0003 * i) for i in range(30)]
    ex = FakeExecutor(capacity=100, n_slots=3)
    serving.Scheduler(ex, backfill=False).run(reqs)
    log = serving.request_log(reqs)
    assert len(log) == 30 and all(rec["status"] == "done" for rec in log)
    assert all(rec["t_done"] >= rec["t_admit"] >= rec["t_arrive"] >= 0 for rec in log)
    path = str(tmp_path / "log.json")
    serving.save_request_log(path, reqs)
    again = [FakeRequest(i, r.n_cells, r.mem, 99.0) for i, r in enumerate(reqs)]
    serving.replay_arrivals(path, again)
    assert [r.arrival for r in again] == [r.arrival for r in reqs]
    ex2 = FakeExecutor(capacity=100, n_slots=3)
    serving.Scheduler(ex2, backfill=False).run(again)
    assert ex2.order == ex.order
