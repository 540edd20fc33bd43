"""A serving loop with continuous batching over the fused runtime.

Requests (CG and BiCGSTAB solves on resident Poisson operators, and
Black-Scholes option batches) arrive over time.  The loop runs in ticks:

  1. admit, in arrival order, the requests that have arrived while the
     device-memory budget and the per-kind slot limit allow it (an idle
     operator is evicted, least recently used first, when the budget is
     short); a Black-Scholes batch is priced at once and completes in the tick
     that admits it; new solves have their data uploaded and are set up as one
     batched window per kind (b = A x*, the solver's start state) after the
     tick's iterations are launched, so that host work overlaps GPU work;
  2. advance every active solve by `iters_per_tick` iterations: all solves of
     one kind form the instances of one batched launch (their uneven sizes
     share one persistent kernel), repeated with dfs_batch_repeat while the
     set of solves does not change;
  3. read every active solve's r.r and b.b with one gather, and retire the
     solves that reached ||r|| <= tol ||b|| (or max_iters): copy x back to the
     host, free its stores, release its budget.

Results are delivered into page-locked host buffers taken at set-up time
(while the GPU iterates) from a pool keyed by dtype and power-of-two
capacity; when the caller does not keep outputs, a buffer returns to the pool
once its result has been handed over, so a steady stream pins little new
host memory.

Requests that arrive while others are on the GPU join the next tick's batches,
so their work shares launches with the solves already running.  A solve's
iterations, its convergence test (always after a multiple of iters_per_tick
of its own iterations) and its arithmetic (batched instances are bit-identical
to solo runs with the same tiles) do not depend on what else is in the mix, so
each result is the same alone and in the mix.

The admission policy is a plain function (`admit`) so that it can be tested
without a device.
"""
from __future__ import annotations

import math
import time
from collections import OrderedDict
from dataclasses import dataclass, field

import numpy as np

from . import arrays as A
from . import workloads as W
from .binding import DfsError

SOLVERS = ("cg", "bicgstab")
KINDS = SOLVERS + ("bs",)


def request_bytes(kind: str, size: int, dtype_bytes: int = 8) -> int:
    """Device bytes a request holds while active (operators not included):
    CG keeps x, r, p, q; BiCGSTAB x, r, rhat, p, v, s, t; both hold x* during
    set-up.  A Black-Scholes batch holds S, K, T, call and put (FP32)."""
    if kind == "bs":
        return 5 * 4 * size
    n = size ** 3
    vectors = 5 if kind == "cg" else 8
    return vectors * dtype_bytes * n + 64


def operator_bytes(m: int) -> int:
    """CSR of the 3-D 7-point Poisson matrix: int32 row pointers and columns,
    FP64 values."""
    n = m ** 3
    nnz = 7 * n - 6 * m * m
    return 4 * (n + 1) + 12 * nnz


def admit(queue, now: float, used: int, budget: int, active: dict, max_active: int, need, evictable: int = 0):
    """Requests to admit now, in arrival order: a prefix of the arrived part
    of `queue` (FIFO, no overtaking) whose bytes fit the budget, counting
    `evictable` bytes that idle operators could give back, and whose kinds
    have a free slot.  need(req) -> bytes the request adds (its state plus an
    operator not yet resident).  Returns (requests, bytes)."""
    out, add = [], 0
    slots = dict(active)
    for req in queue:
        if req["arrival"] > now:
            break
        k = req["kind"]
        if k in SOLVERS and slots.get(k, 0) >= max_active:
            break
        b = need(req, out)
        if used + add + b > budget + evictable:
            break
        out.append(req)
        add += b
        if k in SOLVERS:
            slots[k] = slots.get(k, 0) + 1
    return out, add


@dataclass
class Result:
    rid: int
    kind: str
    size: int
    arrival: float
    admitted: float = 0.0
    done: float = 0.0
    iterations: int = 0
    converged: bool = True
    rel_residual: float = 0.0
    output: object = None

    @property
    def latency(self) -> float:
        return self.done - self.arrival


@dataclass
class _Solve:
    req: dict
    res: Result
    m: int
    Am: A.CSR
    st: object
    bb: A.Array
    it: int = 0
    nbytes: int = 0
    out: object = None      # page-locked host buffer the solution is delivered into


@dataclass
class Stats:
    ticks: int = 0
    batched_launches: int = 0
    repeats: int = 0
    max_active: dict = field(default_factory=dict)
    peak_bytes: int = 0
    evictions: int = 0
    # host seconds per part of a tick: admission, option pricing (launch and
    # wait), launching the iterations, set-up of new solves, the convergence
    # read (mostly waiting for the tick's GPU work) and retirement
    host_s: dict = field(default_factory=dict)

    def add(self, part: str, t0: float) -> float:
        t = time.perf_counter()
        self.host_s[part] = self.host_s.get(part, 0.0) + (t - t0)
        return t


class Server:
    """Continuous-batching request loop over one runtime context.

    rt: the Runtime (its tile is every request's tile, so results do not
    depend on the mix); budget_bytes: device bytes for operators plus request
    state; tol: ||r|| <= tol ||b||; iters_per_tick: solver iterations between
    admissions and convergence tests; max_active: active solves per kind;
    operator(m): host CSR arrays (rowptr, col, val) of the m^3 Poisson matrix;
    clock: None for wall-clock arrivals, else a callable giving the time in
    seconds (a virtual clock: when idle the loop jumps to the next arrival);
    bs_rate, bs_sigma: the market's r and sigma for option batches; overlap:
    set new solves up after the tick's iterations are launched, so the
    uploads and set-up overlap GPU work (they start iterating a tick later).
    """

    def __init__(self, rt: A.Runtime, operator, *, budget_bytes: int = 120 * 10 ** 9, tol: float = 1e-8,
                 iters_per_tick: int = 8, max_iters: int = 20000, max_active: int = 64, clock=None,
                 keep_outputs: bool = True, bs_rate: float = 0.02, bs_sigma: float = 0.3, overlap: bool = True):
        self.rt = rt
        self.operator_fn = operator
        self.budget = int(budget_bytes)
        self.tol = tol
        self.C = int(iters_per_tick)
        self.max_iters = max_iters
        self.max_active = max_active
        self.clock = clock
        self.keep = keep_outputs
        self.bs_rate, self.bs_sigma = bs_rate, bs_sigma
        self.overlap = overlap
        self.ops: OrderedDict[int, A.CSR] = OrderedDict()   # resident operators, LRU order
        self.op_users: dict[int, int] = {}
        self.used = 0
        self.stats = Stats()
        self._inflight = []   # host buffers read by work not yet synchronised
        # page-locked result buffers, reused once their results are handed
        # over when outputs are not kept (pinning host memory takes tens of
        # milliseconds per 100 MB, which the GPU would otherwise wait out)
        self._pool: dict[tuple, list] = {}
        self.stats_pool = {"allocated": 0, "reused": 0}

    # ----------------------------------------------------------- operators
    def _need(self, req, admitted_now) -> int:
        b = request_bytes(req["kind"], req["size"])
        if req["kind"] in SOLVERS:
            m = req["size"]
            if m not in self.ops and all(r["size"] != m or r["kind"] == "bs" for r in admitted_now):
                b += operator_bytes(m)
        return b

    def _evictable(self) -> int:
        return sum(operator_bytes(m) for m in self.ops if self.op_users.get(m, 0) == 0)

    def _evict_for(self, nbytes: int) -> None:
        for m in list(self.ops):
            if self.used + nbytes <= self.budget:
                return
            if self.op_users.get(m, 0) == 0:
                del self.ops[m]          # its stores are released with the last reference
                self.used -= operator_bytes(m)
                self.stats.evictions += 1

    def _operator(self, m: int) -> A.CSR:
        if m in self.ops:
            self.ops.move_to_end(m)
            return self.ops[m]
        rp, col, val = self.operator_fn(m)
        Am = A.CSR(self.rt, rp, col, val)
        self.ops[m] = Am
        self.used += operator_bytes(m)
        return Am

    # ----------------------------------------------------- result buffers
    def _out_buffer(self, n: int, dtype):
        """A 1-D page-locked buffer of at least n elements: its capacity is
        the next power of two, so requests of similar sizes share buffers.
        Callers use buf[:n]."""
        cap = 1 << max(0, int(n) - 1).bit_length()
        key = (cap, np.dtype(dtype).str)
        free = self._pool.get(key)
        if free:
            self.stats_pool["reused"] += 1
            return free.pop()
        self.stats_pool["allocated"] += 1
        return A.Runtime.host_empty((cap,), dtype)

    def _recycle(self, buf) -> None:
        """Back to the pool once its result has been handed over (only when
        results are not kept, so no caller holds it)."""
        if not self.keep and buf is not None:
            self._pool.setdefault((len(buf), buf.dtype.str), []).append(buf)

    # ---------------------------------------------------------------- ticks
    def _now(self, t0: float) -> float:
        return (self.clock() if self.clock else time.perf_counter()) - t0

    def _inputs(self, hosts):
        """Stores over the requests' host arrays: read in place when every one
        lives in mapped page-locked memory (zero-copy), else uploaded."""
        rt = self.rt
        try:
            return [rt.wrap_host(h) for h in hosts], True
        except DfsError:
            return [rt.array(np.ascontiguousarray(h)) for h in hosts], False

    def _setup_solves(self, kind, reqs, payloads, now):
        rt = self.rt
        ops = []
        for req in reqs:
            m = req["size"]
            ops.append(self._operator(m))
            self.op_users[m] = self.op_users.get(m, 0) + 1
        xs_all, in_place = self._inputs([payloads(req) for req in reqs])
        items = list(zip(reqs, ops, xs_all))
        sols = []
        rt.batch_begin()
        for req, Am, xin in items:
            # in place: x* streamed from host memory once into a device copy,
            # which the SpMV gathers from
            xs = A.copy(xin) if in_place else xin
            b = Am @ xs
            del xs                      # the same liveness in every instance
            st = W.cg_start_inplace(b) if kind == "cg" else W.bicgstab_start_inplace(b)
            bb = A.dot(b, b)
            del b                       # a temporary of the set-up window
            res = Result(req["rid"], kind, req["size"], req["arrival"], admitted=now)
            sols.append(_Solve(req, res, req["size"], Am, st, bb,
                               nbytes=request_bytes(kind, req["size"]),
                               out=self._out_buffer(st.x.shape[0], st.x.dtype)))
            rt.batch_next()
        rt.batch_end()
        # the set-up runs asynchronously: keep the host data it reads (and
        # their stores) until the next synchronisation of the stream
        self._inflight.append((items, xs_all))
        return sols

    def _iterate(self, kind, sols) -> None:
        """iters_per_tick iterations of every solve of one kind."""
        rt = self.rt
        step = W.cg_iteration_inplace if kind == "cg" else W.bicgstab_iteration_inplace
        done = 0
        while done < self.C:
            rt.batch_begin()
            for s in sols:
                step(s.Am, s.st)
                rt.batch_next()
            rt.batch_end()
            self.stats.batched_launches += 1
            done += 1
            if done < self.C:
                try:
                    rt.batch_repeat(self.C - done)
                    self.stats.repeats += self.C - done
                    done = self.C
                except DfsError:
                    pass               # not steady yet (a store got its first value): issue again

    def _price(self, reqs, payloads, now):
        rt = self.rt
        hosts = [payloads(req) for req in reqs]
        arrs, _ = self._inputs([h for trio in hosts for h in trio])
        data = [(req, *arrs[3 * i:3 * i + 3]) for i, req in enumerate(reqs)]
        # one batched launch; the prices go straight from the kernel into
        # mapped page-locked host buffers (call and put become temporaries)
        results, hold = [], []
        rt.batch_begin()
        for req, S, K, T in data:
            bc = self._out_buffer(req["size"], np.float32)
            bp = self._out_buffer(req["size"], np.float32)
            hc, hp = bc[:req["size"]], bp[:req["size"]]
            wc, wp = rt.wrap_host(hc), rt.wrap_host(hp)
            call, put = W.black_scholes(S, K, T, self.bs_rate, self.bs_sigma)
            wc[...] = call
            wp[...] = put
            del call, put
            hold.append((wc, wp, bc, bp))
            res = Result(req["rid"], "bs", req["size"], req["arrival"], admitted=now)
            res.output = (hc, hp) if self.keep else None
            results.append(res)
            rt.batch_next()
        rt.batch_end()
        rt.sync()
        for _, _, bc, bp in hold:
            self._recycle(bc)
            self._recycle(bp)
        return results

    # ------------------------------------------------------------------ run
    def run(self, requests, payloads):
        """Serve `requests` (dicts with rid, arrival, kind, size, seed, in
        arrival order); payloads(req) gives the request's host data.  Returns
        the Results in completion order."""
        queue = list(requests)
        qi = 0
        active: dict[str, list[_Solve]] = {k: [] for k in SOLVERS}
        finished: list[Result] = []
        t0 = self.clock() if self.clock else time.perf_counter()
        st = self.stats
        while qi < len(queue) or any(active.values()):
            now = self._now(t0)
            tp = time.perf_counter()
            counts = {k: len(v) for k, v in active.items()}
            adm, add = admit(queue[qi:], now, self.used, self.budget, counts, self.max_active, self._need,
                             self._evictable())
            if not adm and not any(active.values()):
                if queue[qi]["arrival"] > now:
                    if self.clock is None:
                        time.sleep(max(0.0, min(queue[qi]["arrival"] - now, 0.01)))
                    else:
                        self._advance(queue[qi]["arrival"] - now)
                    continue
                raise RuntimeError(f"request {queue[qi]['rid']} does not fit the device-memory budget")
            qi += len(adm)
            if add:
                self._evict_for(add)
            tp = st.add("admit", tp)

            def setup_new():
                for kind in SOLVERS:
                    reqs = [r for r in adm if r["kind"] == kind]
                    if reqs:
                        sols = self._setup_solves(kind, reqs, payloads, now)
                        for s in sols:
                            self.used += s.nbytes
                        active[kind].extend(sols)
            # admission: set-up windows of new solves (now, or after this
            # tick's iterations are launched) and pricing of option batches
            if not self.overlap:
                setup_new()
                tp = st.add("setup", tp)
            bs = [r for r in adm if r["kind"] == "bs"]
            if bs:
                self.used += sum(request_bytes("bs", r["size"]) for r in bs)
                self.stats.peak_bytes = max(self.stats.peak_bytes, self.used)
                done = self._price(bs, payloads, now)
                t = self._now(t0)
                for res in done:
                    res.done = t
                finished.extend(done)
                self.used -= sum(request_bytes("bs", r["size"]) for r in bs)
                tp = st.add("price", tp)
            self.stats.peak_bytes = max(self.stats.peak_bytes, self.used)
            # one tick of every active solve
            for kind in SOLVERS:
                if active[kind]:
                    self.stats.max_active[kind] = max(self.stats.max_active.get(kind, 0), len(active[kind]))
                    self._iterate(kind, active[kind])
                    for s in active[kind]:
                        s.it += self.C
            tp = st.add("iterate", tp)
            if self.overlap:
                setup_new()                      # host work while the GPU iterates; they join next tick
                tp = st.add("setup", tp)
            self.stats.ticks += 1
            self._advance(0.0)
            # convergence test of every solve that iterated, one gather
            sols = [s for s in active["cg"] + active["bicgstab"] if s.it > 0]
            if sols:
                arrs = []
                for s in sols:
                    arrs += [s.bb, s.st.rho if s.res.kind == "cg" else s.st.rr]
                vals = self.rt.read_scalars(arrs)  # synchronises the stream
                tp = st.add("read_scalars", tp)
                self._inflight.clear()
                retire = []
                for i, s in enumerate(sols):
                    bb, rr = vals[2 * i], vals[2 * i + 1]
                    rel = math.sqrt(max(rr, 0.0) / bb) if bb > 0 else 0.0
                    if rel <= self.tol or s.it >= self.max_iters or not math.isfinite(rel):
                        s.res.rel_residual = rel
                        s.res.converged = rel <= self.tol
                        retire.append(s)
                # solutions go from one batched copy kernel straight into
                # mapped page-locked host buffers, one sync for all of them
                hold = []
                if retire:
                    self.rt.batch_begin()
                for s in retire:
                    hx = s.out[:s.st.x.shape[0]]
                    w = self.rt.wrap_host(hx)
                    w[...] = s.st.x
                    hold.append(w)
                    self.rt.batch_next()
                    s.res.iterations = s.it
                    s.res.output = hx if self.keep else None
                    active[s.res.kind].remove(s)
                    self.used -= s.nbytes
                    self.op_users[s.m] -= 1
                    s.st = s.bb = None
                if retire:
                    self.rt.batch_end()
                    self.rt.sync()
                    t = self._now(t0)
                    for s in retire:
                        s.res.done = t
                        finished.append(s.res)
                del hold
                for s in retire:
                    self._recycle(s.out)
                    s.out = None
                st.add("retire", tp)
        self.rt.sync()
        self._inflight.clear()
        return finished

    def _advance(self, dt: float) -> None:
        """Virtual clocks move on by one tick (plus dt when idle)."""
        adv = getattr(self.clock, "advance", None)
        if adv is not None:
            adv(dt)


class TickClock:
    """A virtual clock for deterministic runs: every tick takes `tick_s`."""

    def __init__(self, tick_s: float = 1e-3):
        self.t = 0.0
        self.tick_s = tick_s

    def __call__(self) -> float:
        return self.t

    def advance(self, dt: float) -> None:
        self.t += dt if dt > 0 else self.tick_s


def summarize(results, wall_s: float) -> dict:
    """p50/p99 latency (overall and per kind) and sustained throughput."""
    lat = np.array([r.latency for r in results]) if results else np.zeros(1)
    out = {"requests": len(results), "wall_s": wall_s, "sustained_rps": len(results) / wall_s if wall_s > 0 else 0.0,
           "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
           "mean_ms": float(lat.mean() * 1e3)}
    for k in KINDS:
        lk = np.array([r.latency for r in results if r.kind == k])
        if lk.size:
            out[k] = {"count": int(lk.size), "p50_ms": float(np.percentile(lk, 50) * 1e3),
                      "p99_ms": float(np.percentile(lk, 99) * 1e3)}
    its = [r.iterations for r in results if r.kind in SOLVERS]
    if its:
        out["solver_iterations"] = {"mean": float(np.mean(its)), "max": int(np.max(its))}
    out["unconverged"] = sum(1 for r in results if not r.converged)
    return out

