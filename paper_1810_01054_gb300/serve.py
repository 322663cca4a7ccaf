"""Request loop serving rollout and gradient requests with continuous batching.

Requests (a scene, a horizon, forward-only or forward+gradient) arrive over time.  The server
admits a request as soon as its batch has a slot and device memory for its checkpoints, keeps
its state resident on the GPU, and advances every admitted request step-synchronously in the
same launches (one batch per dimension and tile edge, libgbmpm mpm_batch_*).  Requests that arrive while others
run join at the next tick; finished ones leave and free their memory.  Latency is measured on the
host from arrival to the moment the result (final state, and gradients when asked) is ready.

    server = Server(device=0)
    rid = server.submit(spec, want_grad=True)          # or submit(..., arrival=t)
    server.run()                                       # until every request is done
    server.results[rid]  -> dict(status, x, v, C, F, grads, latency_s); a request that failed on
                            the device (status < 0, e.g. a particle left the grid) carries
                            status and error instead of a state, and the others are unaffected
    server.latency_percentiles()                       -> (p50, p99) in seconds
"""
from __future__ import annotations

import collections
import dataclasses
import time
from typing import Optional

import numpy as np

from . import mpm


@dataclasses.dataclass
class Request:
    rid: int
    spec: object
    want_grad: bool
    arrival: float
    n_steps: int
    scene: Optional[object] = None
    slot: int = -1
    dim: int = 2
    key: tuple = ()  # (dimension, tile edge): the batch that runs it
    admitted: float = 0.0
    done: float = 0.0


class Server:
    """Continuous-batching server on one GPU.

    mem_fraction: share of the device memory free at start-up that admitted requests may hold
    (scene buffers + rollout checkpoints); tick_steps: simulation steps per tick between
    admissions and completions."""

    def __init__(self, device: int = 0, mem_fraction: float = 0.5, tick_steps: int = 8, stream=None,
                 keep_results: bool = True):
        import torch
        self.torch = torch
        self.device = device
        self.ctx = mpm.Context(device, stream=stream)
        free, _total = torch.cuda.mem_get_info(device)
        self.budget = int(free * mem_fraction)
        # one batch per (dimension, tile edge), made when its first request arrives
        self.batches = {}
        self.tick_steps = tick_steps
        self.pending = collections.deque()
        self.active = {}
        self.results = {}
        self.keep_results = keep_results
        self._next = 0
        self.t0 = time.perf_counter()
        self.particle_steps = 0

    def now(self) -> float:
        return time.perf_counter() - self.t0

    def submit(self, spec, want_grad: bool, n_steps: Optional[int] = None, arrival: Optional[float] = None) -> int:
        rid = self._next
        self._next += 1
        req = Request(rid, spec, bool(want_grad), self.now() if arrival is None else arrival,
                      int(n_steps if n_steps is not None else spec.n_steps), dim=int(spec.dim))
        self.pending.append(req)
        return rid

    def _admit(self):
        now = self.now()
        waiting = collections.deque()
        while self.pending:
            req = self.pending.popleft()
            if req.arrival > now:
                waiting.append(req)
                continue
            if req.scene is None:
                req.scene = mpm.Scene(self.ctx, req.spec)
                req.key = (req.dim, req.scene.tile_edge)
            if req.key not in self.batches:
                self.batches[req.key] = mpm.Batch(self.ctx, req.dim, self.budget)
            slot = self.batches[req.key].admit(req.scene, req.n_steps, req.want_grad)
            if slot < 0:  # no memory for it now; it waits for a finished request to leave
                waiting.append(req)
                continue
            req.slot = slot
            req.admitted = now
            self.active[(req.key, slot)] = req
        self.pending = waiting

    def _complete(self):
        for key in list(self.active):
            req = self.active[key]
            batch = self.batches[req.key]
            if not batch.poll(req.slot):
                continue
            status = batch.status(req.slot)
            if status == mpm.MPM_OK:
                x, v, Cm, F = req.scene.get_state()
                res = {"status": status, "x": x, "v": v, "C": Cm, "F": F}
                if req.want_grad:
                    res["grads"] = req.scene.gradients()
            else:  # the request failed on the device (e.g. a particle left the grid); others go on
                res = {"status": status, "error": mpm.STATUS.get(status, "unknown")}
            req.done = self.now()
            res["latency_s"] = req.done - req.arrival
            res["queued_s"] = req.admitted - req.arrival
            if status == mpm.MPM_OK:
                self.particle_steps += req.scene.N * req.n_steps
            batch.release(req.slot)
            req.scene.close()
            req.scene = None
            del self.active[key]
            self.results[req.rid] = res if self.keep_results else {"status": status, "latency_s": res["latency_s"]}

    def step(self):
        """One scheduling round: admit arrived requests, advance every batch, collect results."""
        self._admit()
        for key, batch in self.batches.items():
            if any(k[0] == key for k in self.active):
                batch.tick(self.tick_steps)
        self._complete()

    def run(self, idle_sleep: float = 1e-4):
        while self.pending or self.active:
            if not self.active and self.pending and min(r.arrival for r in self.pending) > self.now():
                time.sleep(idle_sleep)
            self.step()

    def latency_percentiles(self):
        lat = np.array([r["latency_s"] for r in self.results.values()])
        if lat.size == 0:
            return float("nan"), float("nan")
        return float(np.percentile(lat, 50)), float(np.percentile(lat, 99))

    def close(self):
        for b in self.batches.values():
            b.close()
        self.ctx.close()
