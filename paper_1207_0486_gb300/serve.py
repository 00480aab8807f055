"""Continuous-batching solve serving over the resident server (pm_server).

A stream of solve requests (each: one basin session, one time step, 1-4 right-hand sides) is
served by one loop:
  * arrivals join a queue; a queued request is admitted when its session has no step in flight,
    enough slots are free for its right-hand sides, and, for a session not yet resident, the
    device has room for its operators and Krylov state (free HBM minus a reserve);
  * admitted systems join the resident persistent kernel at its next quantum, next to the ones
    already iterating (no drain between batches);
  * finished systems are retired between quanta; a request completes when all its systems have;
    a session's operators, vectors and workspace stay resident across its consecutive steps and
    are released after its last one.
Right-hand side j of a request is the system of the projection step it stands for: the three
velocity components (j = 0, 1, 2; Eq. fofa_velo_pred_h) and the pressure increment (j = 3;
Eq. fofa_q_cor_h). With the consistent-mass velocity correction (Eq. fofa_velo_cor_h solved with
M rather than its lumped diagonal) a step has three more systems, M u_c = rhs_c (j = 4, 5, 6),
served with IC0 next to the others in the same persistent kernel.

The loop talks to a backend (the GPU one below, or a host fake in tests), so the scheduling logic
is the same code whichever runs the solves. `serial` mode is the plain baseline: requests in
arrival order, each right-hand side solved alone by the single-system FP64 path.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence

import numpy as np

RHS_WHICH = (0, 1, 2, 3)  # OP_VEL_U1, OP_VEL_U2, OP_VEL_U3, OP_PRESSURE
RHS_WHICH_CONSISTENT = RHS_WHICH + (4, 4, 4)  # and OP_MASS for each velocity component


@dataclass
class RequestRecord:
    index: int
    session: int
    step: int
    nrhs: int
    t_arrival: float
    t_admit: float = math.nan
    t_done: float = math.nan
    iters: List[int] = field(default_factory=list)
    status: List[int] = field(default_factory=list)
    rel_residual: List[float] = field(default_factory=list)
    cancelled: bool = False      # withdrawn by its client before it was admitted

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival


@dataclass
class ServeReport:
    mode: str
    records: List[RequestRecord]
    makespan: float
    sessions_opened: int
    peak_resident_sessions: int
    quanta: int
    deferred_for_memory: int
    host: Dict = field(default_factory=dict)

    @property
    def solves(self) -> int:
        return sum(r.nrhs for r in self.records if not math.isnan(r.t_done))

    def latencies_ms(self) -> np.ndarray:
        return np.array([r.latency * 1e3 for r in self.records if not math.isnan(r.t_done)])

    def summary(self) -> Dict:
        lat = self.latencies_ms()
        bad = sum(1 for r in self.records for s in r.status if s != 0)
        its = [i for r in self.records for i in r.iters]
        return {
            "mode": self.mode,
            "requests": len(self.records),
            "solves": self.solves,
            "solves_per_s": self.solves / self.makespan if self.makespan > 0 else 0.0,
            "p50_ms": float(np.percentile(lat, 50)) if lat.size else None,
            "p99_ms": float(np.percentile(lat, 99)) if lat.size else None,
            "max_ms": float(lat.max()) if lat.size else None,
            "makespan_s": self.makespan,
            "failed_solves": bad,
            "cancelled_requests": sum(1 for r in self.records if r.cancelled),
            "mean_iters": float(np.mean(its)) if its else 0.0,
            "sessions": self.sessions_opened,
            "peak_resident_sessions": self.peak_resident_sessions,
            "quanta": self.quanta,
            "deferred_for_memory": self.deferred_for_memory,
            "host_seconds": {k: round(v, 4) for k, v in self.host.items()},
        }


class Scheduler:
    """The request loop. backend: object with
        now() -> seconds;  sleep(seconds)
        free_bytes() -> int;  session_bytes(session) -> int
        open_session(session_id, session) -> handle (raises MemoryError when the device cannot hold
            the session now);  close_session(handle)
        admit(handle, j, rhs_seed, key) -> slot or None (no free slot)
        run(quantum) -> systems still active;  poll() -> [(slot, stats)]
        solve_now(handle, j, rhs_seed, key) -> stats          (serial mode)
    stats: objects with .iters, .status, .rel_residual_true.
    cancel: optional {request index: time} at which the request's client withdraws it (on the
    requests' clock). A request still queued then is dropped (record.cancelled); one already
    admitted runs to completion, since its systems are already on the GPU. A session closes once
    none of its requests is outstanding.
    """

    def __init__(self, backend, sessions: Sequence, requests: Sequence, slots: int = 64, quantum: int = 16,
                 reserve_bytes: int = 1 << 30, mode: str = "continuous", cancel: Optional[Dict[int, float]] = None):
        if mode not in ("continuous", "serial"):
            raise ValueError("mode must be 'continuous' or 'serial'")
        self.be = backend
        self.sessions = list(sessions)
        self.requests = list(requests)
        self.slots = slots
        self.quantum = quantum
        self.reserve = reserve_bytes
        self.mode = mode
        self.cancel = dict(cancel or {})

    def run(self) -> ServeReport:
        be = self.be
        recs = [RequestRecord(i, r.session, r.step, r.nrhs, r.t_arrival) for i, r in enumerate(self.requests)]
        order = sorted(range(len(recs)), key=lambda i: recs[i].t_arrival)
        queue: List[int] = []
        nxt = 0
        open_h: Dict[int, object] = {}
        busy: Dict[int, int] = {}          # session -> request in flight
        slot_of: Dict[int, tuple] = {}     # slot -> (request, j)
        remaining: Dict[int, int] = {}     # request -> systems not finished
        done = 0
        opened = peak = quanta = 0
        deferred = set()                   # requests that waited for device memory at least once
        need_of: Dict[int, int] = {}       # session -> device bytes it needs when opened
        t0 = be.now()
        first_arrival = recs[order[0]].t_arrival if recs else 0.0
        outstanding: Dict[int, int] = {}   # session -> requests neither finished nor cancelled
        for r in recs:
            outstanding[r.session] = outstanding.get(r.session, 0) + 1

        def resolve(rec):
            outstanding[rec.session] -= 1
            if outstanding[rec.session] == 0 and rec.session in open_h and rec.session not in busy:
                be.close_session(open_h.pop(rec.session))

        def finish(ri, t):
            nonlocal done
            rec = recs[ri]
            rec.t_done = t
            done += 1
            del busy[rec.session]
            resolve(rec)

        def drop_cancelled(t):
            nonlocal done
            for ri in [i for i in queue if self.cancel.get(i, math.inf) <= t]:
                queue.remove(ri)
                recs[ri].cancelled = True
                done += 1
                resolve(recs[ri])

        def ensure_open(rec) -> bool:
            nonlocal opened, peak
            if rec.session in open_h:
                return True
            if rec.session not in need_of:
                need_of[rec.session] = be.session_bytes(self.sessions[rec.session])
            if be.free_bytes() - need_of[rec.session] < self.reserve:
                deferred.add(rec.index)
                return False
            try:
                open_h[rec.session] = be.open_session(rec.session, self.sessions[rec.session])
            except MemoryError:
                # the estimate said it fits, the allocation said no: wait as for memory, and ask
                # for more headroom next time
                need_of[rec.session] *= 2
                deferred.add(rec.index)
                return False
            opened += 1
            peak = max(peak, len(open_h))
            return True

        while done < len(recs):
            t = be.now() - t0
            while nxt < len(order) and recs[order[nxt]].t_arrival <= t:
                queue.append(order[nxt])
                nxt += 1
            drop_cancelled(t)
            if self.mode == "serial":
                if not queue:
                    be.sleep(max(0.0, recs[order[nxt]].t_arrival - (be.now() - t0)))
                    continue
                ri = queue.pop(0)
                rec = recs[ri]
                if not ensure_open(rec):
                    raise RuntimeError(f"session {rec.session} does not fit in device memory")
                busy[rec.session] = ri
                rec.t_admit = be.now() - t0
                for j in range(rec.nrhs):
                    st = be.solve_now(open_h[rec.session], j, self.requests[ri].rhs_seed + j, (ri, j))
                    rec.iters.append(int(st.iters))
                    rec.status.append(int(st.status))
                    rec.rel_residual.append(float(st.rel_residual_true))
                finish(ri, be.now() - t0)
                continue
            # continuous: admit whatever is eligible, in arrival order
            free = self.slots - len(slot_of)
            for ri in list(queue):
                rec = recs[ri]
                if rec.session in busy or rec.nrhs > free:
                    continue
                if not ensure_open(rec):
                    continue
                h = open_h[rec.session]
                got = []
                for j in range(rec.nrhs):
                    s = be.admit(h, j, self.requests[ri].rhs_seed + j, (ri, j))
                    if s is None:
                        raise RuntimeError("server refused a slot the scheduler counted as free")
                    got.append(s)
                for j, s in enumerate(got):
                    slot_of[s] = (ri, j)
                remaining[ri] = rec.nrhs
                busy[rec.session] = ri
                rec.t_admit = be.now() - t0
                rec.iters = [0] * rec.nrhs
                rec.status = [0] * rec.nrhs
                rec.rel_residual = [0.0] * rec.nrhs
                free -= rec.nrhs
                queue.remove(ri)
            if slot_of:
                be.run(self.quantum)
                quanta += 1
                tq = be.now() - t0
                for s, st in be.poll():
                    ri, j = slot_of.pop(s)
                    rec = recs[ri]
                    rec.iters[j] = int(st.iters)
                    rec.status[j] = int(st.status)
                    rec.rel_residual[j] = float(st.rel_residual_true)
                    remaining[ri] -= 1
                    if remaining[ri] == 0:
                        del remaining[ri]
                        finish(ri, tq)
            elif nxt < len(order):
                be.sleep(max(0.0, recs[order[nxt]].t_arrival - (be.now() - t0)))
            elif queue and any(i in self.cancel for i in queue):
                be.sleep(max(0.0, min(self.cancel[i] for i in queue if i in self.cancel) - (be.now() - t0)))
            elif queue:
                raise RuntimeError("queued requests can never be admitted (slots or memory too small)")
        last = max((r.t_done for r in recs), default=0.0)
        host = dict(getattr(be, "timers", {}))
        return ServeReport(self.mode, recs, last - first_arrival, opened, peak, quanta, len(deferred), host)


def shard(sessions: Sequence, requests: Sequence, rank: int, world: int):
    """Replica sharding: whole sessions (basins) to ranks, session id mod world; requests follow
    their session. Returns the request indices of this rank."""
    return [i for i, r in enumerate(requests) if r.session % world == rank]


class GpuBackend:
    """Backend on the resident server (continuous) or on the single-system solver (serial)."""

    def __init__(self, opts=None, slots: int = 64, nz_cap: int = 64, tile_cols: int = 64, block: int = 128,
                 blocks_per_sm: int = 0, serial_opts=None, rhs: str = "device", keep=None,
                 correction: str = "lumped"):
        import dataclasses

        import torch

        from . import api
        if correction not in ("lumped", "consistent"):
            raise ValueError("correction must be 'lumped' or 'consistent'")
        self.torch = torch
        self.api = api
        self.which = RHS_WHICH if correction == "lumped" else RHS_WHICH_CONSISTENT
        # the mass systems take IC0; the others the server's (and the serial path's) preconditioner
        self.prec = [None if w != api.OP_MASS else api.PREC_IC0 for w in self.which]
        self._replace = dataclasses.replace
        # FP32 inner solves restarted from the FP64 residual every four orders of magnitude
        self.opts = opts or api.Options(prec=api.PREC_LINE, precision=api.FP32_REFINE, rtol=1e-8, inner_rtol=1e-4,
                                        max_iter=200000)
        self.serial_opts = serial_opts or api.Options(prec=api.PREC_LINE, precision=api.FP64, rtol=1e-8,
                                                      max_iter=200000, max_restarts=5)
        self.server = None
        self.server_args = (slots, nz_cap, tile_cols, block, blocks_per_sm)
        self.rhs = rhs
        self.keep = set(keep or ())
        self.kept: Dict = {}
        self._slot_key: Dict[int, tuple] = {}
        self.gen = torch.Generator(device="cuda")
        self.timers = {k: 0.0 for k in ("open", "rhs", "admit", "run", "poll", "solve", "sleep")}
        self.active_sum = 0
        self.runs = 0

    def _t(self, key, t0):
        self.timers[key] += time.perf_counter() - t0

    def _srv(self):
        if self.server is None:
            s, nzc, tc, blk, bps = self.server_args
            self.server = self.api.Server(s, nzc, self.opts, tc, blk, bps)
        return self.server

    def now(self):
        return time.perf_counter()

    def sleep(self, s):
        if s > 0:
            t0 = time.perf_counter()
            time.sleep(s)
            self._t("sleep", t0)

    def free_bytes(self):
        return int(self.torch.cuda.mem_get_info()[0])

    @staticmethod
    def _basin(session):
        from workloads import box_basin
        return box_basin(nh=session.side, nz=session.nz, seed=session.seed)

    def session_bytes(self, session):
        n = session.side * session.side * session.nz
        # operators + one (x, b, workspace) per system + low-precision copies, line and IC0 factors
        return self.api.operator_bytes(self._basin(session)) + n * (len(self.which) * (8 + 8 + 40) + 320 +
                                                                    (180 if len(self.which) > 4 else 0))

    def open_session(self, sid, session):
        t0 = time.perf_counter()
        h = self._open(sid, session)
        self._t("open", t0)
        return h

    def _open(self, sid, session):
        """Operators and per-system vectors of one session; MemoryError (nothing kept) when the
        device runs out during assembly or allocation."""
        torch = self.torch
        try:
            op = self.api.assemble_operator(self._basin(session))
        except self.api.PMError as ex:
            if ex.status == self.api.PM_ENOMEM:
                raise MemoryError(str(ex)) from ex
            raise
        n = op.n
        try:
            ws = int(self.api.load().pm_server_workspace_bytes(self.api._handle(op.handle), self.opts.precision))
            h = {"sid": sid, "op": op,
                 "x": [torch.zeros(n, dtype=torch.float64, device="cuda") for _ in self.which],
                 "b": [torch.empty(n, dtype=torch.float64, device="cuda") for _ in self.which],
                 "work": [torch.empty(ws, dtype=torch.uint8, device="cuda") for _ in self.which]}
        except torch.cuda.OutOfMemoryError as ex:
            op.close()
            raise MemoryError(str(ex)) from ex
        return h

    def close_session(self, h):
        h["op"].close()
        h.clear()

    def _fill_rhs(self, h, j, seed):
        t0 = time.perf_counter()
        b = self._rhs(h, j, seed)
        self._t("rhs", t0)
        return b

    def _rhs(self, h, j, seed):
        b = h["b"][j]
        if self.rhs == "device":
            self.gen.manual_seed(seed)
            b.normal_(generator=self.gen)
        else:
            from workloads import random_vector
            b.copy_(self.torch.from_numpy(random_vector(b.numel(), seed)))
        return b

    def admit(self, h, j, seed, key):
        b = self._fill_rhs(h, j, seed)
        t0 = time.perf_counter()
        s = self._srv().admit(h["op"], self.which[j], b, h["x"][j], h["work"][j], prec=self.prec[j])
        if s is not None:
            self._slot_key[s] = (key, h, j)
        self._t("admit", t0)
        return s

    def run(self, quantum):
        t0 = time.perf_counter()
        self.active_sum += len(self._slot_key)
        self.runs += 1
        a = self._srv().run(quantum)
        self._t("run", t0)
        return a

    def poll(self):
        t0 = time.perf_counter()
        out = self._srv().poll()
        for s, _ in out:
            key, h, j = self._slot_key.pop(s)
            if key in self.keep:
                self.kept[key] = h["x"][j].cpu().numpy().copy()
        self._t("poll", t0)
        return out

    def solve_now(self, h, j, seed, key):
        b = self._fill_rhs(h, j, seed)
        x = h["x"][j]
        t0 = time.perf_counter()
        opts = self.serial_opts if self.prec[j] is None else self._replace(self.serial_opts, prec=self.prec[j])
        st = h["op"].solve(self.which[j], b, x, opts, allow_not_converged=True)
        self._t("solve", t0)
        if key in self.keep:
            self.kept[key] = x.cpu().numpy().copy()
        return st

    def close(self):
        if self.server is not None:
            self.server.close()
            self.server = None
