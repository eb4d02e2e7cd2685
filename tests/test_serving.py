"""Serving: continuous batching of rollout requests (GPU), plus the load generator (CPU)."""
import numpy as np
import pytest
import torch

from paper_2601_22074_b300 import inputs as I

SPECS = [I.pendulum(3), I.quadruped(), I.humanoid(), I.manipulation()]


def test_poisson_load_generator_statistics():
    from paper_2601_22074_b300.serve import poisson_requests
    reqs = poisson_requests(20000, rate=200.0, ngroup=4, seed=0)
    gaps = np.diff([r.arrival for r in reqs])
    assert abs(gaps.mean() - 1 / 200) < 2e-4
    w = np.array([r.nworld for r in reqs])
    assert w.min() >= 1 and w.max() <= 1024
    assert abs(w.mean() - 1024 / np.log(1025)) < 8        # log-uniform mean ~147.6
    h = np.array([r.horizon for r in reqs])
    assert h.min() >= 50 and h.max() <= 500 and abs(h.mean() - 275) < 5
    assert set(r.group for r in reqs) == {0, 1, 2, 3}


def _drain(srv, results=None):
    results = {} if results is None else results
    while not srv.idle():
        st = srv.stats()
        if st["queued"] or st["active"]:
            srv.tick()
        for r in srv.poll():
            results[r.rid] = r
    return results


def _run_alone(req, budget=1 << 28):
    from paper_2601_22074_b300.serve import RolloutServer, Request
    srv = RolloutServer(SPECS, budget, max_worlds_per_group=2048)
    srv.submit(Request(req.rid, req.group, req.nworld, req.horizon, req.seed))
    return _drain(srv)[req.rid]


@pytest.mark.gpu
def test_each_result_is_the_same_alone_and_in_the_mix():
    from paper_2601_22074_b300.serve import RolloutServer, Request
    rng = np.random.default_rng(1)
    reqs = [Request(i, int(rng.integers(0, 4)), int(rng.integers(1, 40)), int(rng.integers(3, 12)),
                    int(rng.integers(1, 1 << 40))) for i in range(24)]
    srv = RolloutServer(SPECS, 1 << 28, max_worlds_per_group=96)   # small pools: requests queue
    results = {}
    pending = list(reqs)
    while pending or not srv.idle():
        # staggered arrivals: two requests join per tick while others are on the GPU
        for _ in range(2):
            if pending:
                srv.submit(pending.pop(0))
        st = srv.stats()
        if st["queued"] or st["active"]:
            srv.tick()
        for r in srv.poll():
            results[r.rid] = r
    assert len(results) == len(reqs)
    assert srv.ticks < sum(r.horizon for r in reqs)          # work overlapped across requests
    for req in reqs[::3]:
        alone = _run_alone(req)
        mix = results[req.rid]
        assert np.array_equal(alone.qpos, mix.qpos), req
        assert np.array_equal(alone.qvel, mix.qvel), req
        assert np.isfinite(mix.qpos).all()


@pytest.mark.gpu
def test_admission_waits_for_free_slots_and_refuses_oversize():
    from paper_2601_22074_b300.serve import RolloutServer, Request, ServerBusy, bytes_per_world
    from paper_2601_22074_b300.batch import Model
    per = max(bytes_per_world(Model(s), dict(working_set=2)) for s in SPECS)
    srv = RolloutServer(SPECS, 4 * 64 * per, max_worlds_per_group=64)
    assert all(c <= 64 for c in srv.capacity)
    cap = srv.capacity[2]
    with pytest.raises(ServerBusy):
        srv.submit(Request(0, 2, cap + 1, 5, 1))
    srv.submit(Request(1, 2, cap, 5, 2))
    srv.submit(Request(2, 2, 1, 5, 3))      # must wait: the pool is full
    srv.tick()
    st = srv.stats()
    assert st["active"] == 1 and st["queued"] == 1
    done = _drain(srv)
    assert sorted(done) == [1, 2]
    assert srv.ticks >= 10                   # request 2 ran after request 1 retired
    assert done[2].admitted >= done[1].admitted


@pytest.mark.gpu
def test_bad_requests_and_thread_ownership_are_reported():
    from paper_2601_22074_b300.serve import RolloutServer, Request
    srv = RolloutServer(SPECS, 1 << 26, max_worlds_per_group=16, run_thread=True)
    with pytest.raises(RuntimeError, match="INVALID_ARG"):
        srv.submit(Request(0, 7, 1, 5, 1))
    with pytest.raises(RuntimeError, match="INVALID_ARG"):
        srv.submit(Request(0, 1, 1, 0, 1))
    with pytest.raises(RuntimeError, match="UNSUPPORTED"):
        srv.tick()


@pytest.mark.gpu
def test_poisson_load_reports_latency_percentiles():
    from paper_2601_22074_b300.serve import RolloutServer, poisson_requests, run_load
    srv = RolloutServer(SPECS, 1 << 30, max_worlds_per_group=4096)
    reqs = poisson_requests(60, rate=200.0, ngroup=4, seed=3, max_worlds=64, horizon=(5, 20))
    rep = run_load(srv, reqs, warmup_s=0.0)
    assert rep["completed"] == 60 and rep["busy"] == 0
    assert 0 < rep["p50_ms"] <= rep["p99_ms"]
    assert rep["env_steps_per_s"] > 0


@pytest.mark.gpu
def test_server_thread_serves_the_same_results():
    """The native server thread ticks on its own; every result equals the caller-ticked
    server's for the same request."""
    from paper_2601_22074_b300.serve import RolloutServer, poisson_requests, run_load, Request
    reqs = poisson_requests(40, rate=400.0, ngroup=4, seed=5, max_worlds=48, horizon=(4, 16))
    srv = RolloutServer(SPECS, 1 << 30, max_worlds_per_group=512, run_thread=True)
    got = {}
    for r in reqs:
        srv.submit(Request(r.rid, r.group, r.nworld, r.horizon, r.seed))
    import time
    t0 = time.time()
    while len(got) < len(reqs) and time.time() - t0 < 120:
        for x in srv.poll():
            got[x.rid] = x
        time.sleep(0.001)
    assert len(got) == len(reqs)
    ref = RolloutServer(SPECS, 1 << 30, max_worlds_per_group=512)
    for r in reqs[::4]:
        ref.submit(Request(r.rid, r.group, r.nworld, r.horizon, r.seed))
    want = _drain(ref)
    for rid, x in want.items():
        assert np.array_equal(x.qpos, got[rid].qpos) and np.array_equal(x.qvel, got[rid].qvel)
    rep = run_load(RolloutServer(SPECS, 1 << 30, max_worlds_per_group=512, run_thread=True),
                   reqs, warmup_s=0.0)
    assert rep["completed"] == len(reqs) and rep["p50_ms"] <= rep["p99_ms"]


@pytest.mark.gpu
def test_served_targets_match_the_oracle_draw():
    """b3p_sample_targets (the server's per-world PD targets, drawn on the device from
    each world's seed, rng id and step count) against the oracle's restatement of the
    draw, for every world of a two-morphology batch over several env steps."""
    import ctypes as C
    from oracle.actuation import served_targets
    from paper_2601_22074_b300 import _lib as L
    from paper_2601_22074_b300.batch import Batch, Model
    specs = [I.quadruped(), I.humanoid()]
    Ws = [24, 16]
    seed = 987654321123                       # both key words non-zero
    b = Batch([Model(s) for s in specs], Ws)
    b.reset(seed)
    sig = [0.5, 0.3]
    sigma = torch.tensor(sig, dtype=torch.float32, device="cuda")
    ctrl = torch.zeros(b.ctrl_size(), dtype=torch.float32, device="cuda")
    lib = L.load()
    stream = torch.cuda.current_stream().cuda_stream
    worst = 0.0
    for t in range(4):
        L.check(lib.b3p_sample_targets(b._h, C.c_void_p(sigma.data_ptr()), C.c_void_p(ctrl.data_ptr()),
                                       C.c_void_p(stream)), "b3p_sample_targets")
        torch.cuda.synchronize()
        got = ctrl.double().cpu().numpy()
        sc = b.get("step_count").cpu().numpy()
        off = 0
        for g, (spec, W) in enumerate(zip(specs, Ws)):
            for w in range(W):
                ref = served_targets(spec, seed, w, int(sc[b.world_start[g] + w]), sig[g])
                row = got[off + w * spec.nu: off + (w + 1) * spec.nu]
                worst = max(worst, float(np.abs(row - ref).max()))
            off += W * spec.nu
        assert sc.min() == t
        b.step(ctrl, 4)
    print("served targets: max |gpu - oracle| =", worst)
    assert worst <= 2e-5


@pytest.mark.gpu
def test_served_request_steps_match_the_oracle():
    """Teacher-forced through the server: a request of horizon h returns the state after h
    env steps; the oracle steps the state of the horizon h - 1 request (horizon 1: the
    oracle's own seeded reset) once with the oracle's target draw and must land on the
    horizon-h result within the contact tolerance. Results depend only on (morphology,
    seed, horizon), so each horizon is its own request."""
    from oracle import Oracle
    from oracle.actuation import served_targets
    from paper_2601_22074_b300.serve import RolloutServer, Request
    srv = RolloutServer(SPECS, 1 << 28, max_worlds_per_group=64)
    seed, n, H = 424242, 6, 4
    for group in (1, 2):
        spec = SPECS[group]
        reqs = [Request(10 * group + h, group, n, h, seed) for h in range(1, H + 1)]
        for r in reqs:
            srv.submit(r)
        res = _drain(srv)
        o = Oracle(spec)
        sigma = I.CTRL_SIGMA[spec.name]
        f32 = lambda x: np.asarray(x, dtype=np.float32).astype(np.float64)   # noqa: E731
        worst = {"qpos": 0.0, "qvel": 0.0}
        for h in range(1, H + 1):
            out = res[10 * group + h]
            for w in range(n):
                if h == 1:
                    q0, v0 = (f32(x) for x in o.reset(seed, w))
                else:
                    prev = res[10 * group + h - 1]
                    q0, v0 = prev.qpos[w].astype(np.float64), prev.qvel[w].astype(np.float64)
                ctrl = f32(served_targets(spec, seed, w, h - 1, sigma))
                r = o.step(q0, v0, np.zeros(spec.nv), ctrl, nsub=4, kp=f32(spec.act_kp), kd=f32(spec.act_kd),
                           step_count=h - 1, seed=seed, world=w)
                for f, x in (("qpos", out.qpos[w]), ("qvel", out.qvel[w])):
                    e = np.abs(x - r[f]).max() / max(np.abs(r[f]).max(), 1.0)
                    worst[f] = max(worst[f], float(e))
        print(spec.name, "served vs oracle:", worst)
        assert max(worst.values()) <= 1e-3, (spec.name, worst)
