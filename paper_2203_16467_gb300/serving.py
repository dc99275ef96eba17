"""Continuous-batching server for whole crack-path simulations.

Requests (a grid size, a model variant, a microstructure seed) arrive over
time.  Each tick the server admits queued requests while batch slots and the
HBM budget allow (pff_batch_admit fails with OOM otherwise and the request
waits), advances every admitted simulation by one load step with one
pff_batch_step call (simulations of equal size and precision share every
kernel launch; different sizes run concurrently on their own streams), and
retires simulations that broke (C-bar < C_broken) or reached their step cap,
freeing their slot and memory.  All simulation state (E, phi, eps*, solver
vectors) stays resident on the device between ticks.

Latencies: per load step (the tick that advanced a simulation) and per
simulation (arrival to retirement), reported as p50 / p99.
"""
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
    problem: object
    slot: int
    admitted: float
    steps: int = 0
    reports: list = field(default_factory=list)


class Server:
    def __init__(self, hbm_budget, max_slots=64, stream=None, keep_fields=False):
        self.max_slots = max_slots
        self.batch = pff.create_batch(max_slots, int(hbm_budget), stream)
        self.stream = stream
        self.queue = []
        self.active = {}
        self.done = {}
        self.step_latencies = []
        self.sim_latencies = []
        self.load_steps = 0
        self.keep_fields = keep_fields
        self.t0 = None

    def submit(self, req):
        self.queue.append(req)

    def _make(self, r):
        em = eps_M(1.0, 0.2, 1.0, r.ell)
        E = modulus_field(r.n, r.n, r.lc, r.seed)
        p = pff.Problem(r.n, r.n, r.precision, stream=self.stream, E=E,
                        model=(r.fracture, r.split, r.irreversibility),
                        params=dict(nu=0.2, ell=r.ell, mech_tol=r.tol, pf_tol=r.tol,
                                    d_eps_bar=(0.0, em / 20, 0.0)))
        if r.preload:
            p.set_strain(None, (0.0, r.preload * em, 0.0))
        return p

    def _now(self):
        return time.perf_counter() - self.t0

    def _admit(self):
        now = self._now()
        waiting = []
        for r in self.queue:
            if r.arrival > now or len(self.active) >= self.max_slots:
                waiting.append(r)
                continue
            p = self._make(r)
            slot = pff.batch_admit(self.batch, p.h)
            if slot is None:          # does not fit the HBM budget now
                p.close()
                waiting.append(r)
                continue
            self.active[slot] = Sim(r, p, slot, now)
        self.queue = waiting

    def tick(self):
        """Admit, advance every active simulation by one load step, retire finished ones.
        Returns the number of simulations advanced."""
        if self.t0 is None:
            self.t0 = time.perf_counter()
        self._admit()
        if not self.active:
            return 0
        t = time.perf_counter()
        out = pff.batch_step(self.batch, self.max_slots, 1)
        dt = time.perf_counter() - t
        n = 0
        for slot, sim in list(self.active.items()):
            reps = out[slot]
            if not reps:
                continue
            n += 1
            sim.steps += 1
            sim.reports.append(reps[0])
            self.step_latencies.append(dt)
            if reps[0]["broken"] or sim.steps >= sim.req.max_steps:
                self._retire(slot)
        self.load_steps += n
        return n

    def _retire(self, slot):
        sim = self.active.pop(slot)
        pff.batch_release(self.batch, slot)
        res = {"steps": sim.steps, "broken": bool(sim.reports[-1]["broken"]), "reports": sim.reports,
               "latency": self._now() - sim.req.arrival}
        if self.keep_fields:
            res["phi"] = sim.problem.get_fields(pff.FIELD_PHI)
        self.sim_latencies.append(res["latency"])
        sim.problem.close()
        self.done[sim.req.rid] = res

    def run(self, max_ticks=10 ** 9):
        if self.t0 is None:
            self.t0 = time.perf_counter()
        ticks = 0
        while (self.queue or self.active) and ticks < max_ticks:
            if not self.active and self.queue:
                wait = min(r.arrival for r in self.queue) - self._now()
                if wait > 0:
                    time.sleep(wait)
            self.tick()
            ticks += 1
        return self.stats()

    def stats(self):
        el = self._now() if self.t0 is not None else 0.0
        pct = (lambda a, q: float(np.percentile(a, q)) if len(a) else None)
        return {"load_steps": self.load_steps, "seconds": el,
                "load_steps_per_s": self.load_steps / el if el > 0 else None,
                "step_latency_s": {"p50": pct(self.step_latencies, 50), "p99": pct(self.step_latencies, 99)},
                "sim_latency_s": {"p50": pct(self.sim_latencies, 50), "p99": pct(self.sim_latencies, 99)},
                "completed": len(self.done)}

    def close(self):
        for slot in list(self.active):
            self._retire(slot)
        pff.destroy_batch(self.batch)


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
