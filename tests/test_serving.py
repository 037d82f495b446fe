"""Continuous-batching request loop: results in the mix equal results alone.

Requests of mixed dimension, boundary condition and tolerance arrive while
others are on the GPU; the loop admits them by device-memory footprint and
overlaps their work on separate streams.  Each result must match the same
request transformed alone, within the request's tolerance.
"""
import time

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
F = pytest.importorskip("paper_2305_07165_gb300")
S = pytest.importorskip("paper_2305_07165_gb300.serving")

pytestmark = pytest.mark.gpu


def _requests(n, seed=0):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        d = int(rng.choice([2, 3]))
        per = bool(rng.integers(2))
        tol = float(rng.choice([1e-6, 1e-10]))
        delta = float(10 ** rng.uniform(-3.5, -1.5))
        k = 6 if d == 2 else 4
        tr = W.random_balanced_tree(d, int(rng.integers(1 << 30)), max_level=5 if d == 2 else 3,
                                    min_level=1, split_prob=0.4, periodic=per)
        sig = W.random_sigma(tr, k, int(rng.integers(1 << 30)))
        reqs.append(S.Request(d=d, k=k, delta=delta, tol=tol, level=tr.level, coord=tr.coord, sigma=sig,
                              bc=int(per)))
    return reqs


def _alone(r):
    plan = F.Plan(r.d, r.k, r.delta, r.tol, r.level, r.coord, bc=r.bc, prec=r.prec)
    u = plan(torch.from_numpy(r.sigma).cuda()).cpu().numpy()
    plan.close()
    return u


def test_results_in_the_mix_equal_results_alone():
    reqs = _requests(16)
    srv = S.Server(hbm_budget_bytes=2 << 30, max_inflight=6).start()
    futs = []
    for i, r in enumerate(reqs):
        futs.append(srv.submit(r))
        if i % 3 == 2:
            time.sleep(0.002)  # arrivals spread over time, some while others run
    outs = [f.result(timeout=120) for f in futs]
    srv.shutdown()
    st = srv.stats()
    assert st["requests"] == len(reqs) and st["p99_ms"] >= st["p50_ms"] > 0
    for r, u in zip(reqs, outs):
        ua = _alone(r)
        scale = np.abs(ua).max()
        assert np.abs(u - ua).max() <= 10 * r.tol * scale


def test_admission_refuses_requests_larger_than_the_budget():
    r = _requests(1, seed=3)[0]
    srv = S.Server(hbm_budget_bytes=1024, max_inflight=2).start()
    f = srv.submit(r)
    with pytest.raises(MemoryError):
        f.result(timeout=10)
    srv.shutdown()


def test_plan_cache_reuses_resident_plans():
    """Requests on geometries seen before run on the idle resident plan (no host planning) and
    still equal the request transformed alone."""
    base = _requests(3, seed=7)
    rng = np.random.default_rng(1)
    srv = S.Server(hbm_budget_bytes=2 << 30, max_inflight=4).start()
    outs, reqs = [], []
    for rnd in range(3):
        batch = [S.Request(d=b.d, k=b.k, delta=b.delta, tol=b.tol, level=b.level, coord=b.coord,
                           sigma=rng.uniform(-1, 1, size=b.sigma.shape), bc=b.bc) for b in base]
        futs = [srv.submit(r) for r in batch]
        outs += [f.result(timeout=120) for f in futs]   # the round's plans go back to the cache
        reqs += batch
    srv.shutdown()
    assert srv.stats()["plan_cache_hits"] >= 2 * len(base)
    for r, u in zip(reqs, outs):
        ua = _alone(r)
        assert np.abs(u - ua).max() <= 10 * r.tol * np.abs(ua).max()


def test_large_request_in_the_mix_and_resident_bytes_within_budget():
    """A 2.09M-point request (the 3D adaptive workload, split precision) arrives among small ones
    under a budget that cannot hold every plan at once: each result equals the request alone,
    idle cached plans were evicted to admit requests, and the bytes held on the device (in
    flight + idle cached) never exceeded the budget."""
    w = W.config_3d_free_adaptive(seed=0, p=8, delta=1e-3)
    big = S.Request(d=3, k=w.p, delta=w.delta, tol=1e-6, level=w.tree.level, coord=w.tree.coord,
                    sigma=w.sigma, bc=0)
    small = _requests(10, seed=11)
    big_bytes = F.analyze(3, w.p, w.delta, 1e-6, w.tree.level, w.tree.coord, prec=F.PREC_SPLIT)["device_bytes"]
    budget = int(big_bytes + 2 * 8 * w.n_points) + (96 << 20)
    srv = S.Server(hbm_budget_bytes=budget, max_inflight=4, plan_cache_bytes=4 << 30).start()
    reqs = small[:5] + [big] + small[5:]
    futs = []
    for i, r in enumerate(reqs):
        futs.append(srv.submit(r))
        if i % 2:
            time.sleep(0.002)
    outs = [f.result(timeout=300) for f in futs]
    again = srv.submit(S.Request(d=3, k=w.p, delta=w.delta, tol=1e-6, level=w.tree.level, coord=w.tree.coord,
                                 sigma=w.sigma, bc=0)).result(timeout=300)
    srv.shutdown()
    st = srv.stats()
    assert st["peak_resident_bytes"] <= budget
    assert big.n_points >= 2_000_000
    for r, u in zip(reqs, outs):
        ua = _alone(r)
        assert np.abs(u - ua).max() <= 10 * r.tol * np.abs(ua).max()
    # the same request again, on the cached plan (split precision: atomics make it reproducible
    # to rounding, not bit for bit)
    assert np.abs(again - outs[5]).max() <= 10 * big.tol * np.abs(outs[5]).max()
