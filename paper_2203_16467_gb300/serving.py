"""Continuous-batching server for whole crack-path simulations.

Requests (a grid size, a model variant, a microstructure seed) arrive over
time.  Simulations of one grid size form a lane: one batch (pff_create_batch),
one CUDA stream and one worker thread, which advances all of the lane's
simulations by one load step per pff_batch_step call (simulations of equal size
and precision share every kernel launch) and, between two of its own steps,
admits the simulations handed to it and retires those that broke
(C-bar < C_broken) or reached their step cap.  Lanes run independently, so a
request never waits for a load step of another grid size: a 128^2 request that
arrives during a 1024^2 step starts within one 128^2 step.  The request loop
admits arrived requests while the HBM budget (the sum of pff_problem_bytes of
the admitted simulations) and the slot count allow; a request that does not
fit waits for a retirement.  All simulation state (E, phi, eps*, solver
vectors) stays resident on the device between load steps.

Latencies: per load step (the step that advanced a simulation), start
(arrival to the start of the simulation's first step) and per simulation
(arrival to retirement), reported as p50 / p99, overall and per grid size.
"""
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import pff
from .inputs import eps_M, modulus_field


@dataclass
class Request:
    rid: int
    n: int
    fracture: str = "AT1"
    split: str = "SPECTRAL"
    irreversibility: str = "CRACK_SET"
    seed: int = 0
    lc: float = 8.0
    ell: float = 2.0
    precision: int = pff.MIXED
    max_steps: int = 5000
    preload: float = 0.0          # initial eps_bar_yy in units of eps_M
    arrival: float = 0.0          # seconds after the server started
    tol: float = 1e-8


@dataclass
class Sim:
    req: Request
    E: object                     # host modulus field (the lane creates the problem on its stream)
    bytes: int
    problem: object = None
    slot: int = -1
    steps: int = 0
    started: float = None
    reports: list = field(default_factory=list)


def _new_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.Stream()
    except ImportError:
        pass
    return None


def _pct(a, q):
    return float(np.percentile(a, q)) if len(a) else None


class Lane:
    """The simulations of one grid size: a batch on its own stream, stepped by a worker thread."""

    def __init__(self, server, key):
        self.server = server
        self.key = key
        # one stream for everything of this lane (the problems' uploads and read-backs, the batch's
        # steps and graph captures): only the lane's thread touches it
        self.cuda_stream = _new_stream()
        self.stream_ptr = self.cuda_stream.cuda_stream if self.cuda_stream is not None else None
        self.batch = pff.create_batch(server.max_slots, 1 << 62, self.stream_ptr)   # the server keeps the budget
        self.pending = []
        self.admitting = 0            # taken off pending, not yet in sims
        self.sims = {}
        self.steps_log = []           # (t_start, t_end) of every batch step of the lane
        self.cv = threading.Condition()
        self.stop = False
        self.error = None
        self.thread = threading.Thread(target=self._work, daemon=True)
        self.thread.start()

    def hand(self, sim):
        with self.cv:
            self.pending.append(sim)
            self.cv.notify()

    def busy(self):
        with self.cv:
            return bool(self.pending or self.sims or self.admitting)

    def _work(self):
        srv = self.server
        try:
            while True:
                with self.cv:
                    while not (self.pending or self.sims or self.stop):
                        self.cv.wait()
                    if self.stop:
                        return
                    new, self.pending = self.pending, []
                    self.admitting = len(new)
                for sim in new:   # between two steps of this lane, on the lane's stream
                    sim.problem = srv.make_problem(sim.req, sim.E, self.stream_ptr)
                    sim.E = None
                    slot = pff.batch_admit(self.batch, sim.problem.h)
                    with self.cv:
                        sim.slot = slot
                        self.sims[slot] = sim
                        self.admitting -= 1
                t0 = srv.now()
                out = pff.batch_step(self.batch, srv.max_slots, 1)
                t1 = srv.now()
                self.steps_log.append((t0, t1))
                finished = []
                for slot, sim in self.sims.items():
                    reps = out[slot]
                    if not reps:
                        continue
                    if sim.started is None:
                        sim.started = t0
                    sim.steps += 1
                    sim.reports.append(reps[0])
                    srv.record_step(self.key, t1 - t0)
                    if reps[0]["broken"] or sim.steps >= sim.req.max_steps:
                        finished.append(slot)
                for slot in finished:
                    pff.batch_release(self.batch, slot)
                    srv.retire(self.sims[slot], self.key)
                    with self.cv:
                        self.sims.pop(slot)
        except Exception as e:   # reported by the request loop
            self.error = e
            with self.cv:
                for sim in self.pending:
                    srv.release_budget(sim)
                self.pending = []
                self.admitting = 0
            srv.wake()

    def close(self):
        """Stop after the current step; simulations still running are retired as they are."""
        with self.cv:
            self.stop = True
            self.cv.notify()
        self.thread.join()
        for slot, sim in list(self.sims.items()):
            pff.batch_release(self.batch, slot)
            self.server.retire(sim, self.key)
        self.sims = {}
        for sim in self.pending:
            self.server.release_budget(sim)
        self.pending = []
        pff.destroy_batch(self.batch)


class Server:
    def __init__(self, hbm_budget, max_slots=64, stream=None, keep_fields=False):
        self.budget = int(hbm_budget)
        self.max_slots = max_slots
        self.stream = stream          # kept for compatibility: lanes and problems use their own streams
        self.keep_fields = keep_fields
        self.queue = []
        self.lanes = {}
        self.done = {}
        self.used = 0
        self.active = 0
        self.peak_active = 0
        self.load_steps = 0
        self.step_lat = {}
        self.start_lat = {}
        self.sim_lat = {}
        self.mu = threading.Lock()
        self.wake_cv = threading.Condition(self.mu)
        self.t0 = None

    # ---- time base and bookkeeping (called from the lanes' threads too)
    def now(self):
        return time.perf_counter() - self.t0

    def wake(self):
        with self.wake_cv:
            self.wake_cv.notify_all()

    def record_step(self, key, dt):
        with self.mu:
            self.step_lat.setdefault(key, []).append(dt)
            self.load_steps += 1

    def release_budget(self, sim):
        with self.mu:
            self.used -= sim.bytes
            self.active -= 1

    def retire(self, sim, key):
        res = {"steps": sim.steps, "broken": bool(sim.reports[-1]["broken"]) if sim.reports else False,
               "reports": sim.reports, "latency": self.now() - sim.req.arrival,
               "start_latency": (sim.started - sim.req.arrival) if sim.started is not None else None, "n": key}
        if self.keep_fields:
            res["phi"] = sim.problem.get_fields(pff.FIELD_PHI)
        sim.problem.close()
        with self.wake_cv:
            self.used -= sim.bytes
            self.active -= 1
            self.sim_lat.setdefault(key, []).append(res["latency"])
            if res["start_latency"] is not None:
                self.start_lat.setdefault(key, []).append(res["start_latency"])
            self.done[sim.req.rid] = res
            self.wake_cv.notify_all()

    # ---- requests
    def submit(self, req):
        """Queue a request (thread-safe; it is admitted once its arrival time has passed)."""
        with self.wake_cv:
            self.queue.append(req)
            self.wake_cv.notify_all()

    @staticmethod
    def make_problem(r, E, stream):
        """The device state of request r (called by its lane's thread, on the lane's stream)."""
        em = eps_M(1.0, 0.2, 1.0, r.ell)
        p = pff.Problem(r.n, r.n, r.precision, stream=stream, E=E, model=(r.fracture, r.split, r.irreversibility),
                        params=dict(nu=0.2, ell=r.ell, mech_tol=r.tol, pf_tol=r.tol, d_eps_bar=(0.0, em / 20, 0.0)))
        if r.preload:
            p.set_strain(None, (0.0, r.preload * em, 0.0))
        return p

    def _admit(self):
        """Hand every arrived request that fits the budget and the slots to its lane."""
        now = self.now()
        waiting = []
        with self.mu:
            queued, self.queue = self.queue, []
        for r in sorted(queued, key=lambda q: q.arrival):
            nb = pff.problem_bytes(r.n, r.n, r.precision)
            with self.mu:
                fits = r.arrival <= now and self.active < self.max_slots and self.used + nb <= self.budget
                if fits:
                    self.used += nb
                    self.active += 1
                    self.peak_active = max(self.peak_active, self.active)
            if not fits:
                waiting.append(r)
                continue
            key = (r.n, r.precision)
            if key not in self.lanes:
                self.lanes[key] = Lane(self, key)
            self.lanes[key].hand(Sim(r, modulus_field(r.n, r.n, r.lc, r.seed), nb))
        with self.mu:
            self.queue = waiting + self.queue   # (requests submitted meanwhile stay queued)

    def run(self, poll_s=0.0005):
        """Serve until every submitted request is done; returns stats()."""
        if self.t0 is None:
            self.t0 = time.perf_counter()
        while True:
            for lane in self.lanes.values():
                if lane.error is not None:
                    raise lane.error
            self._admit()
            with self.mu:
                queued = bool(self.queue)
            if not queued and not any(lane.busy() for lane in self.lanes.values()):
                break
            with self.wake_cv:
                nxt = min((r.arrival for r in self.queue), default=None)
                wait = poll_s if nxt is None else max(0.0, min(poll_s, nxt - self.now()))
                self.wake_cv.wait(timeout=max(wait, 1e-4))
        return self.stats()

    def stats(self):
        el = self.now() if self.t0 is not None else 0.0
        allv = (lambda d: [x for v in d.values() for x in v])
        per = {}
        for key in sorted(set(self.step_lat) | set(self.sim_lat)):
            n = key[0]
            per[f"{n}x{n}" + ("" if key[1] == pff.MIXED else "_fp64")] = {
                "requests": len(self.sim_lat.get(key, [])),
                "step_latency_s": {"p50": _pct(self.step_lat.get(key, []), 50), "p99": _pct(self.step_lat.get(key, []), 99)},
                "start_latency_s": {"p50": _pct(self.start_lat.get(key, []), 50),
                                    "p99": _pct(self.start_lat.get(key, []), 99)},
                "sim_latency_s": {"p50": _pct(self.sim_lat.get(key, []), 50), "p99": _pct(self.sim_lat.get(key, []), 99)}}
        return {"load_steps": self.load_steps, "seconds": el,
                "load_steps_per_s": self.load_steps / el if el > 0 else None,
                "step_latency_s": {"p50": _pct(allv(self.step_lat), 50), "p99": _pct(allv(self.step_lat), 99)},
                "start_latency_s": {"p50": _pct(allv(self.start_lat), 50), "p99": _pct(allv(self.start_lat), 99)},
                "sim_latency_s": {"p50": _pct(allv(self.sim_lat), 50), "p99": _pct(allv(self.sim_lat), 99)},
                "per_size": per, "completed": len(self.done), "peak_active": self.peak_active}

    def close(self):
        for lane in self.lanes.values():
            lane.close()
        self.lanes = {}


def poisson_requests(n_requests, rate_per_s, sizes=(128, 256, 512, 1024), seed=0, max_steps=200, **kw):
    """Seeded Poisson arrivals; grid size uniform over sizes, variant uniform over
    {AT1, AT2} x {ISOTROPIC, SPECTRAL} (crack-set irreversibility)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n_requests):
        t += rng.exponential(1.0 / rate_per_s)
        out.append(Request(rid=i, n=int(rng.choice(sizes)), fracture=str(rng.choice(["AT1", "AT2"])),
                           split=str(rng.choice(["ISOTROPIC", "SPECTRAL"])), seed=int(rng.integers(1 << 30)),
                           arrival=t, max_steps=max_steps, **kw))
    return out
