"""Host logic of continuous-batching serving, on a fake backend with a virtual clock (no GPU):
admission by free slots and device memory, per-session step order, overlap of arrivals with work
in flight, session residency, the serial baseline, replica sharding over gloo ranks, and host-side
failure injection."""
import math
import os

import numpy as np
import pytest

from paper_1207_0486_gb300.serve import Scheduler, shard
from workloads import request_stream


class Stats:
    def __init__(self, iters, status=0):
        self.iters = iters
        self.status = status
        self.rel_residual_true = 1e-9


class FakeBackend:
    """Virtual clock. A quantum costs `t_launch + t_row * rows of the active systems`; a system
    needs iters(key) iterations; a serial solve costs its iterations x (t_iter_serial)."""

    def __init__(self, sessions, slots, total_bytes=1 << 40, t_launch=2e-4, t_row=2e-10, t_iter_serial=4e-5,
                 fail_at_quantum=None, bad_keys=(), oom_opens=0):
        self.sessions = sessions
        self.slots = slots
        self.t = 0.0
        self.total = total_bytes
        self.open = {}
        self.active = {}
        self.next_slot = 0
        self.t_launch, self.t_row, self.t_iter_serial = t_launch, t_row, t_iter_serial
        self.max_active = 0
        self.quanta = 0
        self.fail_at = fail_at_quantum
        self.bad = set(bad_keys)     # systems whose solve ends in breakdown (e.g. a NaN right-hand side)
        self.admitted = []
        self.oom_opens = oom_opens   # the first session openings fail with MemoryError (injected)
        self.closed = []
        self.peak_used = 0

    @staticmethod
    def iters(key):
        ri, j = key
        return 20 + (ri * 7 + j * 13) % 60 + (200 if j == 3 else 0)

    def rows(self, s):
        return s.side * s.side * s.nz

    def now(self):
        return self.t

    def sleep(self, s):
        self.t += max(s, 1e-6)

    def session_bytes(self, s):
        return self.rows(s) * 600

    def free_bytes(self):
        return self.total - sum(self.session_bytes(self.sessions[h]) for h in self.open.values())

    def open_session(self, sid, s):
        if self.oom_opens > 0:
            self.oom_opens -= 1
            raise MemoryError("device allocation failed (injected)")
        h = len(self.open) + 1000 * (1 + len(self.closed))
        self.open[h] = sid
        self.peak_used = max(self.peak_used, self.total - self.free_bytes())
        self.t += 1e-4
        return h

    def close_session(self, h):
        self.closed.append(self.open.pop(h))

    def admit(self, h, j, seed, key):
        if len(self.active) >= self.slots:
            return None
        free = [s for s in range(self.slots) if s not in self.active]
        s = free[0]
        self.admitted.append(key)
        self.active[s] = [key, self.iters(key), self.rows(self.sessions[self.open[h]])]
        self.max_active = max(self.max_active, len(self.active))
        return s

    def run(self, quantum):
        self.quanta += 1
        if self.fail_at is not None and self.quanta >= self.fail_at:
            from paper_1207_0486_gb300.api import PMError, PM_TIMEOUT
            raise PMError(PM_TIMEOUT, "server_run: device wait timed out (injected)")
        rows = sum(v[2] for v in self.active.values() if v[1] > 0)
        self.t += self.t_launch + self.t_row * rows * quantum
        for v in self.active.values():
            v[1] = max(0, v[1] - quantum)
        return sum(1 for v in self.active.values() if v[1] > 0)

    def poll(self):
        out = [(s, Stats(self.iters(v[0]), status=5 if v[0] in self.bad else 0))
               for s, v in self.active.items() if v[1] == 0]
        for s, _ in out:
            del self.active[s]
        return out

    def solve_now(self, h, j, seed, key):
        self.admitted.append(key)
        it = self.iters(key)
        self.t += it * self.t_iter_serial
        return Stats(it)


def stream(n=300, rate=200.0, sessions=8, steps=20, seed=5):
    return request_stream(seed=seed, rate=rate, n_requests=n, concurrent_sessions=sessions, steps_per_session=steps,
                          median_nodes=2e4, sigma=0.8, max_nodes=2e5)


def test_all_requests_complete_in_session_order_within_slots():
    sess, reqs = stream()
    be = FakeBackend(sess, slots=16)
    rep = Scheduler(be, sess, reqs, slots=16, quantum=8).run()
    assert all(not math.isnan(r.t_done) for r in rep.records)
    assert be.max_active <= 16
    by_session = {}
    for r in rep.records:
        by_session.setdefault(r.session, []).append(r)
    for rs in by_session.values():
        rs.sort(key=lambda r: r.step)
        assert [r.step for r in rs] == list(range(len(rs)))
        for a, b in zip(rs, rs[1:]):
            assert a.t_done <= b.t_admit  # step k+1 starts after step k finished
    # every session closed after its last step; iterations recorded per right-hand side
    assert sorted(be.closed) == sorted(by_session)
    assert all(len(r.iters) == r.nrhs and all(i == FakeBackend.iters((r.index, j)) for j, i in enumerate(r.iters))
               for r in rep.records)
    s = rep.summary()
    assert s["solves"] == sum(r.nrhs for r in reqs)
    assert s["p50_ms"] <= s["p99_ms"] <= s["max_ms"]


def test_arrivals_join_while_others_are_in_flight():
    """Continuous batching: a request is admitted while an earlier-admitted one is still running."""
    sess, reqs = stream(n=120)
    rep = Scheduler(FakeBackend(sess, slots=32), sess, reqs, slots=32, quantum=8).run()
    recs = sorted(rep.records, key=lambda r: r.t_admit)
    overlaps = sum(1 for a, b in zip(recs, recs[1:]) if b.t_admit < a.t_done)
    assert overlaps >= len(recs) // 4
    assert rep.summary()["quanta"] > 0


def test_admission_waits_for_device_memory():
    sess, reqs = stream(n=200, sessions=8, steps=10)
    rows = [s.side * s.side * s.nz for s in sess]
    cap = sorted(rows)[-1] * 600 * 2 + (1 << 20)  # room for about two of the largest sessions
    be = FakeBackend(sess, slots=32, total_bytes=cap)
    rep = Scheduler(be, sess, reqs, slots=32, quantum=8, reserve_bytes=0).run()
    assert all(not math.isnan(r.t_done) for r in rep.records)
    assert be.peak_used <= cap
    assert rep.deferred_for_memory > 0
    assert rep.peak_resident_sessions < 8


def test_too_few_slots_for_a_request_is_reported():
    sess, reqs = stream(n=20)
    big = max(r.nrhs for r in reqs)
    with pytest.raises(RuntimeError):
        Scheduler(FakeBackend(sess, slots=big - 1), sess, reqs, slots=big - 1, quantum=8).run()


def test_continuous_beats_serial_on_a_batching_backend():
    sess, reqs = stream(n=300)
    cont = Scheduler(FakeBackend(sess, slots=64), sess, reqs, slots=64, quantum=8).run().summary()
    ser = Scheduler(FakeBackend(sess, slots=64), sess, reqs, slots=64, mode="serial").run().summary()
    assert ser["solves"] == cont["solves"]
    assert cont["p99_ms"] < ser["p99_ms"]
    assert cont["solves_per_s"] >= ser["solves_per_s"]


def test_injected_device_timeout_propagates():
    from paper_1207_0486_gb300.api import PMError, PM_TIMEOUT
    sess, reqs = stream(n=40)
    with pytest.raises(PMError) as ei:
        Scheduler(FakeBackend(sess, slots=16, fail_at_quantum=5), sess, reqs, slots=16, quantum=8).run()
    assert ei.value.status == PM_TIMEOUT


def test_shard_partitions_sessions():
    sess, reqs = stream(n=200)
    parts = [set(shard(sess, reqs, r, 3)) for r in range(3)]
    assert set().union(*parts) == set(range(len(reqs)))
    assert sum(len(p) for p in parts) == len(reqs)
    for p in parts:
        assert len({reqs[i].session % 3 for i in p}) <= 1


def _replica_rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import torch
    sess, reqs = stream(n=160)
    mine = shard(sess, reqs, rank, world)
    sub = [reqs[i] for i in mine]
    rep = Scheduler(FakeBackend(sess, slots=32), sess, sub, slots=32, quantum=8).run()
    done = torch.zeros(len(reqs), dtype=torch.int64)
    for i, r in zip(mine, rep.records):
        done[i] += 0 if math.isnan(r.t_done) else 1
    dist.all_reduce(done)
    span = torch.tensor([rep.makespan], dtype=torch.float64)
    dist.all_reduce(span, op=dist.ReduceOp.MAX)
    if rank == 0:
        q.put((done.tolist(), float(span.item()), rep.makespan))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_over_gloo_cover_every_request_once():
    import multiprocessing as mp
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_replica_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    done, span_max, span0 = q.get(timeout=120)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert done == [1] * len(done)
    assert span_max >= span0


def test_empty_stream():
    sess, _ = stream(n=10)
    rep = Scheduler(FakeBackend(sess, slots=8), sess, [], slots=8).run()
    s = rep.summary()
    assert s["requests"] == 0 and s["solves"] == 0 and s["p99_ms"] is None


@pytest.mark.parametrize("mode", ["continuous", "serial"])
def test_memory_too_small_for_any_session_is_reported(mode):
    sess, reqs = stream(n=20)
    be = FakeBackend(sess, slots=16, total_bytes=1024)
    with pytest.raises(RuntimeError):
        Scheduler(be, sess, reqs, slots=16, quantum=8, reserve_bytes=0, mode=mode).run()


def test_a_request_needing_every_slot_is_served():
    from workloads.basins import Request, Session
    sess = [Session(side=8, nz=8, seed=1), Session(side=10, nz=8, seed=2)]
    reqs = [Request(t_arrival=0.001 * k, session=k % 2, step=k // 2, nrhs=4, rhs_seed=k) for k in range(6)]
    be = FakeBackend(sess, slots=4)
    rep = Scheduler(be, sess, reqs, slots=4, quantum=8).run()
    assert all(not math.isnan(r.t_done) for r in rep.records)
    assert be.max_active == 4
    # with four slots and four right-hand sides per request, requests never overlap
    recs = sorted(rep.records, key=lambda r: r.t_admit)
    assert all(b.t_admit >= a.t_done for a, b in zip(recs, recs[1:]))


def test_request_stream_right_hand_side_counts():
    """max_rhs = 7 (the consistent-mass correction's seven systems per step) draws 1..7 right-hand
    sides per request; the default keeps 1..4. Only the counts depend on max_rhs: arrivals and
    sessions are the same seeded stream."""
    _, reqs4 = stream(n=400)
    _, reqs7 = request_stream(seed=5, rate=200.0, n_requests=400, concurrent_sessions=8, steps_per_session=20,
                              median_nodes=2e4, sigma=0.8, max_nodes=2e5, max_rhs=7)
    n4 = [r.nrhs for r in reqs4]
    n7 = [r.nrhs for r in reqs7]
    assert set(n4) == {1, 2, 3, 4} and set(n7) == set(range(1, 8))
    assert [(r.t_arrival, r.session, r.step) for r in reqs4] == [(r.t_arrival, r.session, r.step) for r in reqs7]


def test_scheduler_serves_seven_system_requests():
    """Requests of up to seven systems go through the same loop: every system admitted once, a
    request completes when all its systems have."""
    sess, reqs = request_stream(seed=9, rate=200.0, n_requests=120, concurrent_sessions=6, steps_per_session=20,
                                median_nodes=2e4, sigma=0.8, max_nodes=2e5, max_rhs=7)
    be = FakeBackend(sess, slots=16)
    rep = Scheduler(be, sess, reqs, slots=16, quantum=8).run()
    assert all(not math.isnan(r.t_done) for r in rep.records)
    assert be.max_active <= 16
    assert sum(r.nrhs for r in rep.records) == rep.solves


def test_a_failed_system_fails_only_its_request():
    """A system that ends in breakdown (a NaN right-hand side, injected on the host) marks its own
    request's status and nothing else: every other request completes with PM_OK, and the report
    counts one failed solve."""
    sess, reqs = stream(n=120)
    bad = (7, 0)
    be = FakeBackend(sess, slots=16, bad_keys=[bad])
    rep = Scheduler(be, sess, reqs, slots=16, quantum=8).run()
    assert all(not math.isnan(r.t_done) for r in rep.records)
    for r in rep.records:
        want = [5 if (r.index, j) == bad else 0 for j in range(r.nrhs)]
        assert r.status == want, (r.index, r.status)
    assert rep.summary()["failed_solves"] == 1


@pytest.mark.parametrize("mode", ["continuous", "serial"])
def test_cancelled_requests_are_dropped_before_admission(mode):
    """Clients withdraw every fifth request just after it arrives. On a congested backend (few
    slots) those still queued are dropped: none of their systems is admitted or solved, their
    records say cancelled, every other request completes, and every opened session is closed
    (a session whose last step was cancelled included). A request already admitted when its
    client cancels runs to completion."""
    sess, reqs = stream(n=160, rate=2000.0)
    cancel = {i: reqs[i].t_arrival + 1e-6 for i in range(0, len(reqs), 5)}
    be = FakeBackend(sess, slots=6)
    rep = Scheduler(be, sess, reqs, slots=6, quantum=8, mode=mode, cancel=cancel).run()
    dropped = [r.index for r in rep.records if r.cancelled]
    assert dropped, "the backend was not congested enough for any cancellation to land"
    assert set(dropped) <= set(cancel)
    for r in rep.records:
        if r.cancelled:
            assert math.isnan(r.t_done) and not r.iters
            assert not any(k[0] == r.index for k in be.admitted)
        else:
            assert not math.isnan(r.t_done) and len(r.iters) == r.nrhs
    # cancellations that came after admission did not stop those requests
    assert any(i in cancel and not rep.records[i].cancelled for i in range(len(reqs)))
    assert not be.open, "a session stayed open"
    assert rep.summary()["cancelled_requests"] == len(dropped)
    assert rep.solves == sum(r.nrhs for r in rep.records if not r.cancelled)


def test_an_allocation_failure_when_opening_a_session_defers_it():
    """Three session openings fail with an out-of-memory error although the estimate said they fit
    (injected on the host): the requests wait as for memory and are served once an opening
    succeeds; nothing is lost and every session is closed at the end."""
    sess, reqs = stream(n=80)
    be = FakeBackend(sess, slots=16, oom_opens=3)
    rep = Scheduler(be, sess, reqs, slots=16, quantum=8).run()
    assert be.oom_opens == 0
    assert all(not math.isnan(r.t_done) for r in rep.records)
    assert rep.summary()["deferred_for_memory"] >= 1
    assert not be.open
