"""Serving randomized IDs with continuous batching.

Requests (a device-resident complex matrix A, rank k, l, a seed) arrive at
any time.  A request is admitted when a slot is free and its device
footprint (rid_plan_footprint: Omega, its split forms and all workspace, plus
the outputs Y, perm, T) fits in the HBM budget next to the requests already
running; otherwise it waits, first come first served.  Each slot is a worker
thread with its own CUDA stream, so admitted requests run concurrently on the
device; a request's whole ID runs on its slot's stream, its memory is freed
when it completes and the next request is admitted at once.  By default a
request's pivoted QR runs as one launch per step rather than one cooperative
launch, so it never holds the whole GPU while the other slots wait (the
results are the same bits).

Latency is measured from submit() to the moment the result (J, T, the error
estimate) is available on the host side of the worker.  A request's matrix A
is on the device when it is submitted (the caller owns it); no host-device
copy of A is part of the latency.

Plans are reused: a finished request's plan stays, idle, in a pool keyed by
its shape (m, n, k, l, dtype, mode, probes), and the next request of that
shape takes it, moves it to its own stream and redraws its test matrix for
its own seed in place (rid_plan_reseed); the result is bit for bit that of a
new plan with that seed.  Idle plans count against the HBM budget and are
destroyed, least recently used first, when an admission needs their memory.
The plan's share of the work is reported per request (plan_host_ms,
plan_dev_ms beside id_dev_ms; reused says whether the plan came from the
pool).
"""
from __future__ import annotations

import collections
import ctypes
import threading
import time

import torch

from . import Plan, _native, colmajor_empty, MODES, _DTYPES
from ._native import check


ROW_PROBE_MODES = ("fp64", "fp64_emulated")   # modes whose sketch can carry the row probes


def footprint(m, n, k, l, dtype=torch.complex128, mode="fp64_emulated", nprobe=8):
    """Device bytes one request of this shape holds while it runs: the plan
    (with its sketch widened by the row probes, where the mode takes them),
    the probe rows and X = G A, and the outputs Y, perm, T."""
    lib = _native.load()
    b = ctypes.c_size_t()
    rows = l + (nprobe if mode in ROW_PROBE_MODES else 0)
    check(lib.rid_plan_footprint(int(m), int(n), int(k), int(rows), _DTYPES[dtype], MODES[mode], ctypes.byref(b)),
          "rid_plan_footprint")
    probes = 0
    if mode in ROW_PROBE_MODES:
        ldo = (m + 15) // 16 * 16
        probes = 16 * rows * ldo + 16 * nprobe * n + (1 << 16)
    outputs = 16 * l * n + 4 * n + 16 * k * max(0, n - k)
    return int(b.value) + probes + outputs


class Request:
    __slots__ = ("rid", "A", "k", "l", "seed", "nprobe", "probe_seed", "bytes", "t_submit", "t_admit", "t_done",
                 "result", "error")

    def __init__(self, rid, A, k, l, seed, nprobe, probe_seed, nbytes):
        self.rid, self.A, self.k, self.l, self.seed = rid, A, int(k), int(l), int(seed)
        self.nprobe, self.probe_seed, self.bytes = nprobe, probe_seed, nbytes
        self.t_submit = time.perf_counter()
        self.t_admit = self.t_done = None
        self.result = self.error = None

    @property
    def latency(self):
        return None if self.t_done is None else self.t_done - self.t_submit


def output_bytes(n, k, l):
    """Device bytes of one request's outputs Y, perm and T."""
    return 16 * l * n + 4 * n + 16 * k * max(0, n - k)


class Server:
    """slots concurrent IDs, admitted by an HBM budget (bytes); reuse_plans
    keeps finished requests' plans for later requests of the same shape."""

    def __init__(self, slots=8, hbm_budget=None, mode="fp64_emulated", device=None, select_ctas=0,
                 reuse_plans=True):
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        if hbm_budget is None:
            free, _ = torch.cuda.mem_get_info(self.device)
            hbm_budget = int(0.8 * free)
        self.budget = int(hbm_budget)
        self.mode = mode
        # launch shape of each request's select (None: the plan's default).  One
        # launch per step (0) lets the other requests' kernels share the GPU
        # with a select; a cooperative launch holds every SM it spans for all
        # k steps.  The results are the same either way.
        self.select_ctas = select_ctas
        # plan reuse (the modes whose test matrix can be redrawn in place)
        self.reuse = bool(reuse_plans) and mode in ROW_PROBE_MODES
        self.idle = collections.OrderedDict()     # shape key -> [(plan, bytes)], least recently used first
        self.idle_bytes = 0
        self.reused = 0
        self.used = 0
        self.peak_used = 0
        self.running = 0
        self.peak_running = 0
        self.queue = collections.deque()
        self.done = []
        self.cv = threading.Condition()
        self.stop = False
        self.workers = [threading.Thread(target=self._worker, args=(i,), daemon=True) for i in range(slots)]
        for w in self.workers:
            w.start()

    # -- client side ---------------------------------------------------------------
    def submit(self, rid, A, k, l, seed, nprobe=8, probe_seed=1):
        m, n = A.shape
        nbytes = footprint(m, n, k, l, A.dtype, self.mode, nprobe)
        if nbytes > self.budget:
            raise ValueError(f"request {rid} needs {nbytes} bytes, above the server's budget {self.budget}")
        req = Request(rid, A, k, l, seed, nprobe, probe_seed, nbytes)
        with self.cv:
            self.queue.append(req)
            self.cv.notify_all()
        return req

    def drain(self, timeout=None):
        """Wait until every submitted request is done; returns them in completion order."""
        t_end = None if timeout is None else time.perf_counter() + timeout
        with self.cv:
            while self.queue or self.running:
                left = None if t_end is None else t_end - time.perf_counter()
                if left is not None and left <= 0:
                    raise TimeoutError("requests still running")
                self.cv.wait(timeout=left)
            return list(self.done)

    def close(self):
        with self.cv:
            self.stop = True
            self.cv.notify_all()
        for w in self.workers:
            w.join()
        with self.cv:
            idle = [p for plans in self.idle.values() for p, _ in plans]
            self.idle.clear()
            self.used -= self.idle_bytes
            self.idle_bytes = 0
        for p in idle:
            p.close()

    # -- the pool of idle plans (called with self.cv held) ---------------------------
    @staticmethod
    def _key(req, mode):
        m, n = req.A.shape
        return (int(m), int(n), req.k, req.l, req.A.dtype, mode, req.nprobe)

    def _evict_for(self, need, keep_key=None):
        """Take idle plans off the pool, least recently used first (never the
        plans of keep_key), until `need` more bytes fit in the budget; returns
        them (destroyed by the caller outside the lock)."""
        out = []
        for key in [k for k in self.idle if k != keep_key]:
            plans = self.idle[key]
            while plans and self.used + need > self.budget:
                plan, nbytes = plans.pop(0)
                self.idle_bytes -= nbytes
                self.used -= nbytes
                out.append(plan)
            if not plans:
                del self.idle[key]
            if self.used + need <= self.budget:
                break
        return out

    def _checkout(self, key):
        plans = self.idle.get(key)
        if not plans:
            return None
        plan, nbytes = plans.pop()
        if not plans:
            del self.idle[key]
        self.idle_bytes -= nbytes
        self.used -= nbytes                  # the request's own bytes already count the plan
        self.reused += 1
        return plan

    # -- workers -----------------------------------------------------------------------
    def _admit(self):
        """Pop the head request once it fits (first come, first served), with
        an idle plan of its shape if the pool has one."""
        while True:
            victims = []
            with self.cv:
                if self.stop and not self.queue:
                    return None, None
                if self.queue:
                    head = self.queue[0]
                    key = self._key(head, self.mode) if self.reuse else None
                    # an idle plan of its shape passes its bytes on to the request
                    avail = self.idle[key][-1][1] if key in self.idle else 0
                    need = head.bytes - avail
                    if self.used + need > self.budget:
                        victims = self._evict_for(need, keep_key=key)
                    if not victims and self.used + need <= self.budget:
                        req = self.queue.popleft()
                        plan = self._checkout(key) if avail else None
                        self.used += req.bytes
                        self.running += 1
                        self.peak_used = max(self.peak_used, self.used)
                        self.peak_running = max(self.peak_running, self.running)
                        req.t_admit = time.perf_counter()
                        return req, plan
                if not victims:
                    self.cv.wait()
            for p in victims:                     # outside the lock: destroying a plan waits for its stream
                p.close()

    def _worker(self, slot):
        torch.cuda.set_device(self.device)
        stream = torch.cuda.Stream(self.device)
        while True:
            req, plan = self._admit()
            if req is None:
                return
            kept = None
            try:
                with torch.cuda.stream(stream):
                    req.result = run_one(req.A, req.k, req.l, req.seed, req.nprobe, req.probe_seed, self.mode, stream,
                                         self.select_ctas, plan=plan, keep=self.reuse)
                kept = req.result.pop("plan", None)
            except Exception as exc:        # reported with the request, the server keeps running
                req.error = exc
                if plan is not None:
                    plan.close()
            req.t_done = time.perf_counter()
            with self.cv:
                self.used -= req.bytes
                if kept is not None:        # back to the pool: its bytes stay counted
                    m, n = req.A.shape
                    nbytes = max(0, req.bytes - output_bytes(n, req.k, req.l))
                    self.idle.setdefault(self._key(req, self.mode), []).append((kept, nbytes))
                    self.idle.move_to_end(self._key(req, self.mode))
                    self.idle_bytes += nbytes
                    self.used += nbytes
                self.running -= 1
                self.done.append(req)
                self.cv.notify_all()


def run_one(A, k, l, seed, nprobe=8, probe_seed=1, mode="fp64_emulated", stream=None, select_ctas=None, plan=None,
            keep=False):
    """One whole ID on `stream`; returns host copies of J, T and the estimate.
    In the FP64 modes the error comes from row probes that the sketch
    multiplies in its one pass over A; the mixed mode takes column probes.
    select_ctas (None: the plan's default) sets the select's launch shape;
    the results do not depend on it.  plan: an idle plan of this shape to
    reuse (moved to `stream` and reseeded); keep: return the plan in the
    result ("plan") instead of destroying it."""
    m, n = A.shape
    stream = stream or torch.cuda.current_stream(A.device)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    t0 = time.perf_counter()
    ev[0].record(stream)
    rows = mode in ROW_PROBE_MODES
    reused = plan is not None
    if reused:
        plan.set_stream(stream)
        plan.reseed(seed, probe_seed)
    else:
        plan = Plan(m, n, k, l, seed=seed, dtype=A.dtype, mode=mode, stream=stream, nprobe=nprobe if rows else 0,
                    probe_seed=probe_seed)
    try:
        if select_ctas is not None:
            plan.set_select_grid(select_ctas)
        with torch.cuda.stream(stream):
            Y = colmajor_empty(l, n, device=A.device)
            perm = torch.empty(n, dtype=torch.int32, device=A.device)
            T = colmajor_empty(k, n - k, device=A.device)
        ev[1].record(stream)
        plan_host_ms = 1e3 * (time.perf_counter() - t0)
        plan.sketch(A, Y)
        plan.select(Y, perm)
        plan.solve(Y, T)
        if rows:
            est, upper = plan.error_sketched(perm, T)                # synchronizes the stream
        else:
            est, upper = plan.error(A, perm, T, nprobe, probe_seed)
        ev[2].record(stream)
        plan.sync_status()
        out = {"perm": perm.cpu(), "T": T.cpu(), "est": est, "upper": upper, "plan_host_ms": plan_host_ms,
               "plan_dev_ms": ev[0].elapsed_time(ev[1]), "id_dev_ms": ev[1].elapsed_time(ev[2]), "reused": reused}
    except BaseException:
        plan.close()                         # a plan that failed does not go back to the pool
        raise
    if keep:
        out["plan"] = plan
    else:
        plan.close()
    return out


def latency_stats(reqs):
    lat = sorted(r.latency for r in reqs if r.latency is not None)
    if not lat:
        return {}

    def pct(p):
        return lat[min(len(lat) - 1, int(round(p / 100.0 * (len(lat) - 1))))]

    out = {"p50_ms": 1e3 * pct(50), "p99_ms": 1e3 * pct(99), "max_ms": 1e3 * lat[-1], "count": len(lat)}
    parts = [r.result for r in reqs if isinstance(getattr(r, "result", None), dict) and "plan_dev_ms" in r.result]
    if parts:
        for key in ("plan_host_ms", "plan_dev_ms", "id_dev_ms"):
            vals = sorted(p[key] for p in parts)
            out[key.replace("_ms", "_p50_ms")] = vals[len(vals) // 2]
        out["plans_reused"] = sum(1 for p in parts if p.get("reused"))
    return out
