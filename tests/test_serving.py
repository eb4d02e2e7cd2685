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
