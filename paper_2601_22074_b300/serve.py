"""Continuous-batching rollout server over one heterogeneous batch of slots.

Rollout requests (morphology, world count, horizon in env steps, seed) arrive at
any time. The server keeps a pool of world slots per morphology in one batch (the
pool sizes follow from an HBM budget: the bytes b3p_batch_plan charges per world),
and every tick
  1. admits queued requests in arrival order wherever their worlds fit (first fit;
     a request that can never fit is refused at submit with B3P_ERR_BUSY semantics),
     resetting its slots from the request seed with rng ids 0..n-1,
  2. draws every active world's PD targets from its own seed (b3p_sample_targets),
  3. advances every active slot by one environment step in ONE persistent launch
     (idle slots are skipped by the kernel),
  4. retires requests whose horizon is reached: their final qpos/qvel rows are
     gathered on the device and copied to pinned host memory behind a CUDA event,
     and their slots return to the free lists for the next tick.
Requests that arrive while others are running are admitted as soon as slots free up,
and their work shares the same launches; a request's result depends only on its
seed, model and horizon, not on its slots or its neighbours.
"""
from __future__ import annotations

import collections
import ctypes as C
import dataclasses
import math
import time
from typing import Dict, List, Optional, Sequence

import numpy as np
import torch

from . import _lib as L
from . import inputs as I
from .batch import Batch, Model


@dataclasses.dataclass
class Request:
    rid: int
    group: int          # index of the morphology in the server's model list
    nworld: int
    horizon: int        # env steps
    seed: int
    arrival: float = 0.0


@dataclasses.dataclass
class Result:
    rid: int
    qpos: np.ndarray    # [nworld, nq]
    qvel: np.ndarray    # [nworld, nv]
    arrival: float
    admitted: float
    done: float         # wall time the host saw the result in pinned memory


class ServerBusy(RuntimeError):
    """The request can never be admitted (larger than its morphology's slot pool)."""


def bytes_per_world(model: Model) -> float:
    import ctypes
    lib = L.load()
    s = L.Sizes()
    mh = (ctypes.c_void_p * 1)(model._h.value)
    nw = (ctypes.c_int32 * 1)(1024)
    L.check(lib.b3p_batch_plan(mh, nw, 1, None, ctypes.byref(s)), "b3p_batch_plan")
    return s.total_bytes / 1024.0


class RolloutServer:
    def __init__(self, specs: Sequence[I.ModelSpec], hbm_budget_bytes: float, decimation: int = 4,
                 sigma: Optional[Sequence[float]] = None, max_worlds_per_group: int = 32768,
                 max_inflight_ticks: int = 2):
        self.specs = list(specs)
        self.models = [Model(s) for s in self.specs]
        share = hbm_budget_bytes / len(self.models)
        self.capacity = [max(0, min(max_worlds_per_group, int(share // bytes_per_world(m))))
                         for m in self.models]
        if sum(self.capacity) == 0:
            raise ServerBusy("the HBM budget holds no world at all")
        # at least one slot per group keeps the batch layout valid
        caps = [max(c, 1) for c in self.capacity]
        self.batch = Batch(self.models, caps, schedule=1)
        self.decimation = decimation
        self.stream = torch.cuda.Stream()
        dev = self.batch.device
        sig = sigma if sigma is not None else [I.CTRL_SIGMA.get(s.name, 0.3) for s in self.specs]
        self.sigma = torch.tensor(sig, dtype=torch.float32, device=dev)
        self.ctrl = torch.zeros(max(self.batch.ctrl_size(), 1), dtype=torch.float32, device=dev)
        self.free: List[List[int]] = [list(range(c)) for c in self.capacity]
        self.queue: collections.deque = collections.deque()
        self.active: Dict[int, dict] = {}
        self.pending: List[dict] = []
        self.tick_events: collections.deque = collections.deque()
        self.max_inflight = max_inflight_ticks
        self.ticks = 0
        self.world_steps = 0
        self._lib = L.load()
        with torch.cuda.stream(self.stream):
            self.batch.reset(0)
            L.check(self._lib.b3p_set_idle(self.batch._h, None, 0, 1, self.stream.cuda_stream),
                    "b3p_set_idle")
        self.stream.synchronize()

    # ------------------------------------------------------------------ client API
    def submit(self, req: Request) -> None:
        if req.nworld > self.capacity[req.group]:
            raise ServerBusy(f"request {req.rid}: {req.nworld} worlds never fit the "
                             f"{self.capacity[req.group]}-slot pool of group {req.group}")
        self.queue.append(req)

    def idle(self) -> bool:
        return not self.queue and not self.active and not self.pending

    def poll(self) -> List[Result]:
        out, keep = [], []
        for p in self.pending:
            if p["event"].query():
                n = p["req"].nworld
                nq, nv = self.models[p["req"].group].nq, self.models[p["req"].group].nv
                host = p["host"].numpy()
                out.append(Result(p["req"].rid, host[: n * nq].reshape(n, nq).copy(),
                                  host[n * nq: n * (nq + nv)].reshape(n, nv).copy(),
                                  p["req"].arrival, p["admitted"], time.perf_counter()))
            else:
                keep.append(p)
        self.pending = keep
        return out

    # ------------------------------------------------------------------ server loop
    def _admit(self, now: float) -> None:
        s = self.stream.cuda_stream
        left = collections.deque()
        while self.queue:
            req = self.queue.popleft()
            fl = self.free[req.group]
            if len(fl) < req.nworld:
                left.append(req)
                continue
            fl.sort()
            slots, self.free[req.group] = fl[: req.nworld], fl[req.nworld:]
            start = self.batch.world_start[req.group]
            ids = torch.tensor([start + x for x in slots], dtype=torch.int32, device=self.batch.device)
            rng = torch.arange(req.nworld, dtype=torch.int32, device=self.batch.device)
            L.check(self._lib.b3p_reset(self.batch._h, C.c_uint64(req.seed), ids.data_ptr(),
                                        rng.data_ptr(), req.nworld, s), "b3p_reset")
            self.active[req.rid] = dict(req=req, slots=slots, ids=ids, rng=rng, steps=0, admitted=now)
        self.queue = left

    def tick(self) -> int:
        """Admit, step every active slot once, retire finished requests. Returns the
        number of active worlds advanced."""
        while len(self.tick_events) >= self.max_inflight:
            self.tick_events.popleft().synchronize()
        now = time.perf_counter()
        s = self.stream.cuda_stream
        with torch.cuda.stream(self.stream):
            self._admit(now)
            nact = sum(a["req"].nworld for a in self.active.values())
            if nact:
                L.check(self._lib.b3p_sample_targets(self.batch._h, self.sigma.data_ptr(),
                                                     self.ctrl.data_ptr(), s), "b3p_sample_targets")
                L.check(self._lib.b3p_step(self.batch._h, self.ctrl.data_ptr(), self.decimation, s),
                        "b3p_step")
                self.world_steps += nact
            done = []
            for rid, a in self.active.items():
                a["steps"] += 1
                if a["steps"] >= a["req"].horizon:
                    done.append(rid)
            for rid in done:
                a = self.active.pop(rid)
                req = a["req"]
                m = self.models[req.group]
                local = torch.tensor(a["slots"], dtype=torch.int32, device=self.batch.device)
                dev = torch.empty(req.nworld * (m.nq + m.nv), dtype=torch.float32, device=self.batch.device)
                L.check(self._lib.b3p_gather_state(self.batch._h, req.group, L.FIELD["qpos"],
                                                   local.data_ptr(), req.nworld, dev.data_ptr(), s),
                        "b3p_gather_state")
                L.check(self._lib.b3p_gather_state(self.batch._h, req.group, L.FIELD["qvel"],
                                                   local.data_ptr(), req.nworld,
                                                   dev[req.nworld * m.nq:].data_ptr(), s),
                        "b3p_gather_state")
                host = torch.empty(dev.numel(), dtype=torch.float32, pin_memory=True)
                host.copy_(dev, non_blocking=True)
                L.check(self._lib.b3p_set_idle(self.batch._h, a["ids"].data_ptr(), req.nworld, 1, s),
                        "b3p_set_idle")
                ev = torch.cuda.Event()
                ev.record(self.stream)
                self.pending.append(dict(req=req, host=host, dev=dev, local=local, event=ev,
                                         admitted=a["admitted"]))
                self.free[req.group].extend(a["slots"])
            ev = torch.cuda.Event()
            ev.record(self.stream)
            self.tick_events.append(ev)
        self.ticks += 1
        return nact


# ---------------------------------------------------------------------- load generator
def poisson_requests(n: int, rate: float, ngroup: int, seed: int, max_worlds: int = 1024,
                     horizon=(50, 500)) -> List[Request]:
    """Poisson arrivals; morphology uniform; worlds floor(exp(U[0, ln(max+1)))) (log-uniform
    in [1, max]); horizon uniform in [lo, hi]; a seed per request."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    g = rng.integers(0, ngroup, size=n)
    w = np.floor(np.exp(rng.uniform(0.0, math.log(max_worlds + 1), size=n))).astype(int)
    w = np.clip(w, 1, max_worlds)
    h = rng.integers(horizon[0], horizon[1] + 1, size=n)
    s = rng.integers(1, 2 ** 62, size=n)
    return [Request(i, int(g[i]), int(w[i]), int(h[i]), int(s[i]), float(t[i])) for i in range(n)]


def run_load(server: RolloutServer, reqs: List[Request], warmup_s: float = 1.0,
             time_limit_s: float = 600.0) -> dict:
    """Replay the arrival times in real time against the server; latency = time the
    result is in pinned host memory minus the request's arrival time."""
    t0 = time.perf_counter()
    nxt, results = 0, []
    busy = 0
    while True:
        now = time.perf_counter() - t0
        while nxt < len(reqs) and reqs[nxt].arrival <= now:
            r = reqs[nxt]
            r.arrival = t0 + r.arrival
            try:
                server.submit(r)
            except ServerBusy:
                busy += 1
            nxt += 1
        if server.active or server.queue:
            server.tick()
        elif nxt < len(reqs):
            time.sleep(min(0.001, max(0.0, reqs[nxt].arrival - now)))
        results.extend(server.poll())
        if nxt >= len(reqs) and server.idle():
            break
        if now > time_limit_s:
            break
    elapsed = time.perf_counter() - t0
    measured = [r for r in results if r.arrival - t0 >= warmup_s]
    lat = np.array([r.done - r.arrival for r in measured]) if measured else np.zeros(1)
    return {
        "requests": len(reqs), "completed": len(results), "measured": len(measured), "busy": busy,
        "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
        "mean_queue_ms": float(np.mean([r.admitted - r.arrival for r in measured]) * 1e3) if measured else 0.0,
        "env_steps_per_s": server.world_steps / elapsed, "elapsed_s": elapsed, "ticks": server.ticks,
        "capacity": server.capacity,
    }
