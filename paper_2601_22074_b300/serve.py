"""Rollout serving: Python handle on the native rollout server of the C ABI.

The server (b3p_server_* in include/b3phys.h, csrc/b3p_server.cpp) keeps one pool of
world slots per morphology in one batch (pool sizes from an HBM budget: the bytes
b3p_batch_plan charges per world), and every tick
  1. admits queued requests in arrival order wherever their worlds fit (first fit,
     lowest free slots; a request that can never fit is refused at submit with
     B3P_ERR_BUSY), resetting its slots from the request seed with rng ids 0..n-1,
  2. draws every active world's PD targets from its own seed (b3p_sample_targets),
  3. advances every active slot by one environment step in one step call (idle
     slots are skipped by the kernels),
  4. retires requests whose horizon is reached: their final qpos/qvel rows are
     gathered on the device and copied to pinned host memory behind a CUDA event,
     and their slots return to the free lists for the next tick.
Ticks run on a native server thread (run_thread=True) or when the caller calls
tick(). A request's result depends only on its seed, morphology and horizon, never
on its slots or its neighbours. This module only marshals requests and results.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import math
import time
from typing import Dict, List, Optional, Sequence

import numpy as np
import torch

from . import _lib as L
from . import inputs as I
from .batch import Model


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
    submitted: float    # server clock, seconds
    admitted: float
    done: float         # when a poll saw the result in pinned host memory


class ServerBusy(RuntimeError):
    """The request can never be admitted (larger than its morphology's slot pool)."""


def bytes_per_world(model: Model, options: Optional[dict] = None) -> float:
    lib = L.load()
    s = L.Sizes()
    mh = (C.c_void_p * 1)(model._h.value)
    nw = (C.c_int32 * 1)(1024)
    opt = L.Options(**(options or {}))
    L.check(lib.b3p_batch_plan(mh, nw, 1, C.byref(opt), C.byref(s)), "b3p_batch_plan")
    return s.total_bytes / 1024.0


class RolloutServer:
    def __init__(self, specs: Sequence[I.ModelSpec], hbm_budget_bytes: float, decimation: int = 4,
                 sigma: Optional[Sequence[float]] = None, max_worlds_per_group: int = 32768,
                 max_inflight_ticks: int = 2, options: Optional[dict] = None,
                 run_thread: bool = False, device: Optional[int] = None):
        self._lib = L.load()
        self.specs = list(specs)
        self.models = [Model(s) for s in self.specs]
        # grouped staged placement by default: idle slots leave each launch after one status read
        opts = options if options is not None else dict(working_set=3)
        sig = sigma if sigma is not None else [I.CTRL_SIGMA.get(s.name, 0.3) for s in self.specs]
        G = len(self.models)
        self._mh = (C.c_void_p * G)(*[m._h.value for m in self.models])
        self._sig = (C.c_float * G)(*sig)
        cfg = L.ServerCfg()
        cfg.nmodels = G
        cfg.models = C.cast(self._mh, C.POINTER(C.c_void_p))
        cfg.hbm_budget_bytes = float(hbm_budget_bytes)
        cfg.max_worlds_per_model = int(max_worlds_per_group)
        cfg.decimation = int(decimation)
        cfg.sigma_host = C.cast(self._sig, C.POINTER(C.c_float))
        cfg.options = L.Options(**opts)
        cfg.max_inflight_ticks = int(max_inflight_ticks)
        cfg.run_thread = 1 if run_thread else 0
        cfg.device = torch.cuda.current_device() if device is None else int(device)
        h = C.c_void_p()
        code = self._lib.b3p_server_create(C.byref(cfg), C.byref(h))
        if code == -7:
            raise ServerBusy(self._lib.b3p_last_error().decode())
        L.check(code, "b3p_server_create")
        self._h = h
        self.run_thread = run_thread
        cap = (C.c_int32 * G)()
        L.check(self._lib.b3p_server_capacity(h, cap, G), "b3p_server_capacity")
        self.capacity = list(cap)
        self._req: Dict[int, Request] = {}
        self._res = (L.Result * 64)()

    def __del__(self):
        try:
            self._lib.b3p_server_destroy(self._h)
        except Exception:
            pass

    # ------------------------------------------------------------------ client API
    def now(self) -> float:
        return float(self._lib.b3p_server_now(self._h))

    def submit(self, req: Request) -> None:
        r = L.Request(req.group, req.nworld, req.horizon, req.seed & ((1 << 64) - 1))
        nid = C.c_int64()
        code = self._lib.b3p_server_submit(self._h, C.byref(r), C.byref(nid))
        if code == -7:
            raise ServerBusy(self._lib.b3p_last_error().decode())
        L.check(code, "b3p_server_submit")
        self._req[nid.value] = req

    def tick(self) -> int:
        """Admit, step every active slot once, retire finished requests (caller-ticked
        servers only). Returns the number of active worlds advanced."""
        n = C.c_int32()
        L.check(self._lib.b3p_server_tick(self._h, C.byref(n)), "b3p_server_tick")
        return n.value

    def poll(self) -> List[Result]:
        out = []
        while True:
            n = C.c_int32()
            L.check(self._lib.b3p_server_poll(self._h, self._res, len(self._res), C.byref(n)),
                    "b3p_server_poll")
            for k in range(n.value):
                r = self._res[k]
                req = self._req.pop(r.id)
                nq, nv = self.models[r.model].nq, self.models[r.model].nv
                q = np.ctypeslib.as_array(r.qpos, shape=(r.nworld * nq,)).reshape(r.nworld, nq).copy()
                v = np.ctypeslib.as_array(r.qvel, shape=(r.nworld * nv,)).reshape(r.nworld, nv).copy()
                L.check(self._lib.b3p_server_release(self._h, r.id), "b3p_server_release")
                out.append(Result(req.rid, q, v, r.t_submit, r.t_admit, r.t_done))
            if n.value < len(self._res):
                return out

    def stats(self) -> dict:
        s = L.ServerStats()
        L.check(self._lib.b3p_server_get_stats(self._h, C.byref(s)), "b3p_server_get_stats")
        return {f: getattr(s, f) for f, _ in L.ServerStats._fields_ if f != "reserved"}

    def idle(self) -> bool:
        s = self.stats()
        return s["queued"] == 0 and s["active"] == 0 and s["pending"] == 0

    @property
    def ticks(self) -> int:
        return self.stats()["ticks"]

    @property
    def world_steps(self) -> int:
        return self.stats()["world_steps"]


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


def peak_rate(trace, window_s: float) -> float:
    """Highest served world-env-steps/s over any window of at least window_s seconds of a
    (seconds, cumulative world-env-steps) trace."""
    best = 0.0
    j = 0
    for i in range(len(trace)):
        while j < len(trace) and trace[j][0] - trace[i][0] < window_s:
            j += 1
        if j < len(trace):
            best = max(best, (trace[j][1] - trace[i][1]) / (trace[j][0] - trace[i][0]))
    return best


def run_load(server: RolloutServer, reqs: List[Request], warmup_s: float = 1.0,
             time_limit_s: float = 600.0) -> dict:
    """Replay the arrival times in real time against the server (on the server's clock);
    latency = the time a poll saw the result in pinned host memory minus the request's
    scheduled arrival."""
    t0 = server.now()
    steps0 = server.world_steps
    nxt, results, busy = 0, [], 0
    arrival = {}
    trace = [(0.0, 0)]          # (seconds, world-env-steps served) every >= 50 ms
    while True:
        now = server.now() - t0
        if now - trace[-1][0] >= 0.05:
            trace.append((now, server.world_steps - steps0))
        while nxt < len(reqs) and reqs[nxt].arrival <= now:
            r = reqs[nxt]
            arrival[r.rid] = t0 + r.arrival
            try:
                server.submit(r)
            except ServerBusy:
                busy += 1
            nxt += 1
        st = server.stats()
        if not server.run_thread and (st["queued"] or st["active"]):
            server.tick()
        results.extend(server.poll())
        if nxt >= len(reqs) and len(results) + busy >= len(reqs):
            break
        if now > time_limit_s:
            break
        if server.run_thread or not (st["queued"] or st["active"]):
            wait = reqs[nxt].arrival - now if nxt < len(reqs) else 1e9
            time.sleep(max(0.0, min(0.0005, wait)))
    elapsed = server.now() - t0
    measured = [r for r in results if arrival[r.rid] - t0 >= warmup_s]
    lat = np.array([r.done - arrival[r.rid] for r in measured]) if measured else np.zeros(1)
    # stability: median latency of the later half of the measured arrivals over the earlier
    # half (a queue that grows while requests arrive shows as a ratio well above 1)
    by_arrival = sorted(measured, key=lambda r: arrival[r.rid])
    half = len(by_arrival) // 2
    if half >= 4:
        early = np.median([r.done - arrival[r.rid] for r in by_arrival[:half]])
        late = np.median([r.done - arrival[r.rid] for r in by_arrival[half:]])
        growth = float(late / max(early, 1e-9))
    else:
        growth = 1.0
    return {
        "requests": len(reqs), "completed": len(results), "measured": len(measured), "busy": busy,
        "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
        "mean_queue_ms": float(np.mean([r.admitted - arrival[r.rid] for r in measured]) * 1e3)
        if measured else 0.0,
        "env_steps_per_s": (server.world_steps - steps0) / elapsed, "elapsed_s": elapsed,
        "latency_growth": growth,
        "peak_env_steps_per_s": peak_rate(trace, 1.0),
        "ticks": server.ticks, "capacity": server.capacity,
    }
