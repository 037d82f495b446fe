"""Continuous-batching request loop for box Gauss transforms on one GPU.

Requests (a tree, a density, delta, tol, boundary condition) arrive at any
time.  The loop admits them while their device footprint fits a budget
(``fgt_plan_analyze`` reports a plan's bytes before anything is allocated),
builds plans on a host thread pool while the GPU works, and launches every
admitted, planned request as soon as it is ready -- each on its own CUDA stream
so that transforms overlap on the device -- without waiting for earlier
launches to finish.  Completed requests free their memory, which admits the
next ones.  Trees, tables and expansions stay resident on the device for the
life of a request; results come back to pinned host memory.

Plans outlive their requests in a cache keyed by the request's geometry and
parameters (tree, k, delta, tol, boundary condition, precision): a request on a
geometry seen before reuses an idle resident plan -- its tables, lists and
expansion workspace stay on the device -- and skips host planning.  Idle plans
count against the same device-memory budget as the requests in flight: a
request that does not fit next to them evicts idle plans, least recently used
first, before it waits; the cache also has a cap of its own.

Reports per-request latency (arrival -> result on the host) and the points/s
achieved over the run.
"""
from __future__ import annotations

import hashlib
import queue
import threading
import time
from collections import OrderedDict
from concurrent.futures import Future, ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

from . import BC_FREE, PREC_FP64, PREC_SPLIT, Plan, analyze


@dataclass
class Request:
    d: int
    k: int
    delta: float
    tol: float
    level: np.ndarray
    coord: np.ndarray
    sigma: np.ndarray               # float64 [n_leaves, k**d] (host)
    bc: int = BC_FREE
    prec: int | None = None         # default: split when tol >= 1e-7, else FP64
    rid: int = -1
    t_arrival: float = 0.0
    t_done: float = 0.0
    footprint: int = 0
    cached: object = None           # an idle resident plan for this geometry, when one was free
    future: Future = field(default_factory=Future)

    @property
    def n_points(self):
        return int(self.sigma.size)

    def key(self):
        """Geometry and parameters that determine the plan (not the density)."""
        h = hashlib.blake2b(digest_size=16)
        h.update(np.ascontiguousarray(self.level, dtype=np.int32).tobytes())
        h.update(np.ascontiguousarray(self.coord, dtype=np.int32).tobytes())
        return (self.d, self.k, float(self.delta), float(self.tol), int(self.bc), int(self.prec), h.hexdigest())


class Server:
    """Admission by device-memory footprint, host-side planning overlapped with GPU work,
    one stream per in-flight request, completion by CUDA events."""

    def __init__(self, hbm_budget_bytes: int, max_inflight: int = 32, planner_threads: int = 4,
                 device: int = 0, plan_cache_bytes: int = 4 << 30):
        import torch
        self.torch = torch
        self.device = device
        self.budget = int(hbm_budget_bytes)
        self.used = 0
        self.cache_budget = int(plan_cache_bytes)
        self.cache: "OrderedDict[tuple, list]" = OrderedDict()   # key -> idle plans (LRU order)
        self.cache_bytes = 0
        self.cache_hits = 0
        self.peak_resident = 0      # largest in-flight + idle-cached footprint seen (bytes)
        self.held = 0               # resident plans taken from the cache by requests not yet admitted
        self.max_inflight = max_inflight
        self.pending: "queue.Queue[Request]" = queue.Queue()
        self.pool = ThreadPoolExecutor(max_workers=planner_threads)
        self.streams = [torch.cuda.Stream(device=device) for _ in range(max_inflight)]
        self.free_streams = list(range(max_inflight))
        self.lock = threading.Lock()
        self.stop = False
        self.completed: list[Request] = []
        self.thread = threading.Thread(target=self._loop, daemon=True)
        self.next_id = 0

    # ---------------------------------------------------------------- client side
    def submit(self, req: Request) -> Future:
        req.t_arrival = time.perf_counter()
        with self.lock:
            req.rid = self.next_id
            self.next_id += 1
        if req.prec is None:
            req.prec = PREC_SPLIT if req.tol >= 1e-7 else PREC_FP64
        with self.lock:
            req.cached = self._cache_take(req.key())
            if req.cached is not None:
                self.held += int(req.cached.device_bytes())
        if req.cached is not None:
            # the plan is resident already: it now counts as in flight (taken out of the cache's
            # bytes), with sigma and u to place beside it
            req.footprint = int(req.cached.device_bytes()) + 2 * 8 * req.n_points
        else:
            info = analyze(req.d, req.k, req.delta, req.tol, req.level, req.coord, bc=req.bc, prec=req.prec)
            req.footprint = int(info["device_bytes"]) + 2 * 8 * req.n_points
        if req.footprint > self.budget:
            if req.cached is not None:
                with self.lock:
                    self.held -= int(req.cached.device_bytes())
                    self._cache_put(req.key(), req.cached)
                req.cached = None
            req.future.set_exception(MemoryError(f"request needs {req.footprint} bytes, budget {self.budget}"))
            return req.future
        self.pending.put(req)
        return req.future

    def start(self):
        self.thread.start()
        return self

    def shutdown(self):
        self.stop = True
        self.thread.join()
        self.pool.shutdown()
        with self.lock:
            for plans in self.cache.values():
                for p in plans:
                    p.close()
            self.cache.clear()
            self.cache_bytes = 0

    # ---------------------------------------------------------------- plan cache
    def _cache_take(self, key):
        plans = self.cache.get(key)
        if not plans:
            return None
        plan = plans.pop()
        if not plans:
            del self.cache[key]
        self.cache_bytes -= plan.device_bytes()
        self.cache_hits += 1
        return plan

    def _resident(self):
        """Device bytes held by requests in flight, idle cached plans and plans held for pending
        requests."""
        return self.used + self.cache_bytes + self.held

    def _cache_evict_one(self):
        old_key, plans = next(iter(self.cache.items()))     # least recently used
        victim = plans.pop(0)
        if not plans:
            del self.cache[old_key]
        self.cache_bytes -= victim.device_bytes()
        victim.close()

    def _cache_put(self, key, plan):
        """Keep an idle plan resident when it fits both the cache's cap and, next to the requests
        in flight, the device-memory budget (evicting older idle plans first); else release it."""
        nb = plan.device_bytes()
        if nb > min(self.cache_budget, self.budget - self.used - self.held):
            plan.close()
            return
        while (self.cache_bytes + nb > self.cache_budget or self._resident() + nb > self.budget) and self.cache:
            self._cache_evict_one()
        self.cache.setdefault(key, []).append(plan)
        self.cache.move_to_end(key)
        self.cache_bytes += nb

    # ---------------------------------------------------------------- loop
    def _plan(self, req: Request):
        torch = self.torch
        torch.cuda.set_device(self.device)
        plan = req.cached
        if plan is None:
            plan = Plan(req.d, req.k, req.delta, req.tol, req.level, req.coord, bc=req.bc, prec=req.prec)
        sig_h = torch.from_numpy(np.ascontiguousarray(req.sigma)).pin_memory()
        out_h = torch.empty_like(sig_h).pin_memory()
        return plan, sig_h, out_h

    def _loop(self):
        torch = self.torch
        torch.cuda.set_device(self.device)
        waiting: list[Request] = []          # admitted, not yet planned
        planning: list[tuple[Request, Future]] = []
        inflight: list[tuple] = []
        while True:
            # admit by footprint
            while True:
                if not waiting:
                    try:
                        waiting.append(self.pending.get_nowait())
                    except queue.Empty:
                        break
                r = waiting[0]
                if len(planning) + len(inflight) >= self.max_inflight:
                    break
                with self.lock:
                    # a plan this request took from the cache is already resident (counted as held)
                    own = int(r.cached.device_bytes()) if r.cached is not None else 0
                    # idle resident plans give way to requests, least recently used first
                    while self._resident() - own + r.footprint > self.budget and self.cache:
                        self._cache_evict_one()
                    fits = self._resident() - own + r.footprint <= self.budget
                    if fits:
                        self.held -= own
                        self.used += r.footprint
                        self.peak_resident = max(self.peak_resident, self._resident())
                if not fits:
                    break
                waiting.pop(0)
                planning.append((r, self.pool.submit(self._plan, r)))
            # launch everything that finished planning
            still = []
            for r, f in planning:
                if f.done() and self.free_streams:
                    try:
                        plan, sig_h, out_h = f.result()
                    except Exception as e:  # planning failed: report and release
                        self.used -= r.footprint
                        r.future.set_exception(e)
                        continue
                    si = self.free_streams.pop()
                    st = self.streams[si]
                    with torch.cuda.stream(st):
                        sig_d = sig_h.to(f"cuda:{self.device}", non_blocking=True)
                        u_d = torch.empty_like(sig_d)
                        plan.execute(sig_d, out=u_d, stream=st)
                        out_h.copy_(u_d, non_blocking=True)
                        ev = torch.cuda.Event()
                        ev.record(st)
                    inflight.append((r, plan, sig_d, u_d, out_h, ev, si))
                else:
                    still.append((r, f))
            planning = still
            # complete
            rest = []
            for item in inflight:
                r, plan, sig_d, u_d, out_h, ev, si = item
                if ev.query():
                    r.t_done = time.perf_counter()
                    r.future.set_result(out_h.numpy().reshape(r.sigma.shape))
                    self.free_streams.append(si)
                    with self.lock:
                        self.used -= r.footprint   # sigma, u and the plan leave the in-flight count ...
                        self._cache_put(r.key(), plan)   # ... and the plan stays resident if it fits
                        self.peak_resident = max(self.peak_resident, self._resident())
                    r.cached = None
                    self.completed.append(r)
                else:
                    rest.append(item)
            inflight = rest
            if self.stop and not waiting and not planning and not inflight and self.pending.empty():
                break
            if not (planning or inflight):
                time.sleep(1e-4)

    # ---------------------------------------------------------------- statistics
    def stats(self, t0=None, t1=None):
        done = self.completed
        if not done:
            return {}
        lat = np.array([r.t_done - r.t_arrival for r in done]) * 1e3
        t0 = min(r.t_arrival for r in done) if t0 is None else t0
        t1 = max(r.t_done for r in done) if t1 is None else t1
        pts = sum(r.n_points for r in done)
        return {"requests": len(done), "points": pts, "points_per_s": pts / max(t1 - t0, 1e-9),
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(lat.mean()), "plan_cache_hits": self.cache_hits,
                "peak_resident_bytes": int(self.peak_resident)}
