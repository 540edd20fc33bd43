"""A serving loop with continuous batching over the fused runtime.

Requests (CG and BiCGSTAB solves on resident Poisson operators, and
Black-Scholes option batches) arrive over time.  Active solves form two
groups that take turns on one CUDA stream; a turn of group g:

  1. wait for g's last convergence read (an asynchronous gather of every
     solve's r.r and b.b, dfs_read_scalars_async) -- the other group's
     iterations were issued after it, so the GPU keeps working while the
     host goes on -- and retire the solves that reached ||r|| <= tol ||b||
     (or max_iters): one batched kernel copies their x to the host, their
     stores are freed and their budget released;
  2. admit, in arrival order, the requests that have arrived while the
     device-memory budget and the per-kind slot limit allow it (an idle
     operator is evicted, least recently used first, when the budget is
     short): new solves are set up in g (b = A x*, the start state, b.b) as
     one batched window per kind; option batches are priced by one batched
     launch whose kernel writes the prices to the host;
  3. issue iters_per_tick iterations of every solve of g -- all solves of
     one kind form the instances of one batched launch (their uneven sizes
     share one persistent kernel), repeated with dfs_batch_repeat -- and the
     asynchronous read of their residuals.  An instance's iteration window is
     recorded once per kind and operator size and replayed over each solve's
     stores (dfs_template_replay): one call per instance, not one per task.

A result is complete when its copy to the host has finished (a completion
ticket, dfs_record); with the real clock its completion time is the device
time of that point.

Results are delivered into page-locked host buffers taken at set-up time
(while the GPU works on the other group) from a pool keyed by dtype and
power-of-two
capacity; when the caller does not keep outputs, a buffer returns to the pool
once its result has been handed over, so a steady stream pins little new
host memory.

Requests that arrive while others are on the GPU join the next turn's
batches, so their work shares launches with the solves already running.  A solve's
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
                 keep_outputs: bool = True, bs_rate: float = 0.02, bs_sigma: float = 0.3, overlap: bool = True,
                 templates: bool = True):
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
        # recorded iteration windows per (kind, operator size), replayed for
        # every other solve of that size (dfs_template_*): one call per
        # instance instead of one per task
        self.use_templates = templates
        self._templates: dict[tuple, object] = {}
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
        # the set-up runs asynchronously: the caller keeps the host data it
        # reads (and their stores) until work issued after it has completed
        self._inflight.append((items, xs_all))
        return sols

    @staticmethod
    def _stores_of(s) -> list:
        """The stores one iteration of solve s reads and writes."""
        st = s.st
        vec = ([st.x, st.r, st.p, st.q, st.rho] if s.res.kind == "cg" else
               [st.x, st.r, st.rhat, st.p, st.v, st.s, st.t, st.rho, st.alpha, st.omega, st.rr])
        return [s.Am.rowptr, s.Am.col, s.Am.val] + vec

    def _issue_iteration(self, kind, s) -> None:
        """One iteration of solve s as a batch instance: the recorded window
        of its kind and size replayed over its stores, else issued task by
        task (and recorded, the first time)."""
        step = W.cg_iteration_inplace if kind == "cg" else W.bicgstab_iteration_inplace
        key = (kind, s.m)
        ent = self._templates.get(key) if self.use_templates else False
        if ent:
            tpl, src = ent
            tpl.replay(src, [a.handle for a in self._stores_of(s)])
            return
        if ent is None:
            tpl = self.rt.record_template(step, s.Am, s.st)
            src = [a.handle for a in self._stores_of(s)]
            if set(tpl.inputs) <= set(src):
                self._templates[key] = (tpl, src)
            else:
                tpl.free()
                self._templates[key] = False
            return
        step(s.Am, s.st)

    def _iterate(self, kind, sols) -> None:
        """iters_per_tick iterations of every solve of one kind."""
        rt = self.rt
        done = 0
        while done < self.C:
            rt.batch_begin()
            for s in sols:
                self._issue_iteration(kind, s)
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
        """One batched launch pricing every option batch of `reqs`; the
        prices go straight from the kernel into page-locked host buffers.
        Returns (results, buffers, holds): the results are complete once work
        issued after this call has finished; holds keep the host data and
        stores the launch reads or writes alive until then."""
        rt = self.rt
        hosts = [payloads(req) for req in reqs]
        arrs, _ = self._inputs([h for trio in hosts for h in trio])
        data = [(req, *arrs[3 * i:3 * i + 3]) for i, req in enumerate(reqs)]
        # call and put become temporaries: the kernel stores into host memory
        results, bufs, hold = [], [], [hosts, arrs]
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
            hold.append((wc, wp))
            bufs += [bc, bp]
            res = Result(req["rid"], "bs", req["size"], req["arrival"], admitted=now)
            res.output = (hc, hp) if self.keep else None
            results.append(res)
            rt.batch_next()
        rt.batch_end()
        return results, bufs, hold

    # ------------------------------------------------------------------ run
    def _retire(self, group, sols, vals):
        """Convergence test of the solves of one read; the converged ones (or
        those at max_iters) copy x into their host buffers with one batched
        kernel and leave.  Returns a delivery (results, buffers, holds), or
        None."""
        retire = []
        for i, s in enumerate(sols):
            bb, rr = vals[2 * i], vals[2 * i + 1]
            rel = math.sqrt(max(rr, 0.0) / bb) if bb > 0 else 0.0
            if rel <= self.tol or s.it >= self.max_iters or not math.isfinite(rel):
                s.res.rel_residual = rel
                s.res.converged = rel <= self.tol
                retire.append(s)
        if not retire:
            return None
        hold = []
        self.rt.batch_begin()
        for s in retire:
            hx = s.out[:s.st.x.shape[0]]
            w = self.rt.wrap_host(hx)
            w[...] = s.st.x
            hold.append(w)
            self.rt.batch_next()
            s.res.iterations = s.it
            s.res.output = hx if self.keep else None
            group[s.res.kind].remove(s)
            self.used -= s.nbytes
            self.op_users[s.m] -= 1
            s.st = s.bb = None
        self.rt.batch_end()
        bufs = [s.out for s in retire]
        for s in retire:
            s.out = None
        return [s.res for s in retire], bufs, hold

    def run(self, requests, payloads):
        """Serve `requests` (dicts with rid, arrival, kind, size, seed, in
        arrival order); payloads(req) gives the request's host data.  Returns
        the Results in completion order.

        Active solves form two groups that take turns (one group without
        overlap).  A turn of group g: wait for g's last convergence read (the
        other group's iterations, issued after it, keep the GPU busy
        meanwhile), retire g's converged solves, admit arrived requests (new
        solves join g, option batches are priced), issue g's next
        iters_per_tick iterations and an asynchronous read of its residuals.
        Every solve still iterates iters_per_tick at a time and is tested
        after each block, so its iterations and result do not depend on the
        groups or the mix.  A result is complete when its copy to the host
        has finished: with the real clock its completion time is the device
        time of that point (CUDA events), else the clock when it is seen."""
        queue = list(requests)
        qi = 0
        G = 2 if self.overlap else 1
        groups = [{k: [] for k in SOLVERS} for _ in range(G)]
        pend = [None] * G          # (ScalarRead, solves, holds) in flight per group
        gbuf = [(None, None)] * G  # reusable page-locked gather buffers per group
        deliveries = []            # (ticket, results, buffers, holds, device bytes) in flight
        finished: list[Result] = []
        st = self.stats
        rt = self.rt
        t0 = self.clock() if self.clock else time.perf_counter()
        real = self.clock is None
        t_ref, host_ref = None, 0.0
        if real:
            rt.sync()                               # the device-time origin is this moment
            t_ref, host_ref = rt.record(), self._now(t0)

        def n_active():
            return sum(len(v) for grp in groups for v in grp.values())

        def complete(block: bool) -> None:
            keep = []
            for d in deliveries:
                ticket, results, bufs, hold, nbytes = d
                if block:
                    rt.wait(ticket)
                elif not rt.poll(ticket):
                    keep.append(d)
                    continue
                t = host_ref + rt.elapsed_ms(t_ref, ticket) / 1e3 if real else self._now(t0)
                rt.release_ticket(ticket)
                for r in results:
                    r.done = t
                    finished.append(r)
                for b in bufs:
                    self._recycle(b)
                self.used -= nbytes
            deliveries[:] = keep

        g = 0
        try:
            while qi < len(queue) or n_active() or any(p is not None for p in pend) or deliveries:
                tp = time.perf_counter()
                # 1. the group's convergence read, then retirement
                if pend[g] is not None:
                    rd, sols, _holds = pend[g]
                    vals = rd.values()
                    pend[g] = None
                    tp = st.add("wait", tp)
                    dl = self._retire(groups[g], sols, vals)
                    if dl is not None:
                        deliveries.append((rt.record(), *dl, 0))
                    tp = st.add("retire", tp)
                complete(block=False)
                # 2. admission into this group
                now = self._now(t0)
                counts = {k: sum(len(grp[k]) for grp in groups) for k in SOLVERS}
                adm, add = admit(queue[qi:], now, self.used, self.budget, counts, self.max_active, self._need,
                                 self._evictable())
                if not adm and not n_active() and all(p is None for p in pend):
                    if deliveries:
                        complete(block=True)
                        continue
                    if qi < len(queue) and queue[qi]["arrival"] > now:
                        if self.clock is None:
                            time.sleep(max(0.0, min(queue[qi]["arrival"] - now, 0.01)))
                        else:
                            self._advance(queue[qi]["arrival"] - now)
                        continue
                    if qi < len(queue):
                        raise RuntimeError(f"request {queue[qi]['rid']} does not fit the device-memory budget")
                    break
                qi += len(adm)
                if add:
                    self._evict_for(add)
                tp = st.add("admit", tp)
                holds = []
                for kind in SOLVERS:
                    reqs = [r for r in adm if r["kind"] == kind]
                    if reqs:
                        sols = self._setup_solves(kind, reqs, payloads, now)
                        holds.append(self._inflight.pop())
                        for s in sols:
                            self.used += s.nbytes
                        groups[g][kind].extend(sols)
                tp = st.add("setup", tp)
                bs = [r for r in adm if r["kind"] == "bs"]
                if bs:
                    nb = sum(request_bytes("bs", r["size"]) for r in bs)
                    self.used += nb
                    self.stats.peak_bytes = max(self.stats.peak_bytes, self.used)
                    results, bufs, hold = self._price(bs, payloads, now)
                    # the batch's stores stay allocated until its prices are home
                    deliveries.append((rt.record(), results, bufs, hold, nb))
                    tp = st.add("price", tp)
                self.stats.peak_bytes = max(self.stats.peak_bytes, self.used)
                # 3. this group's iterations and its convergence read
                sols = []
                for kind in SOLVERS:
                    if groups[g][kind]:
                        self.stats.max_active[kind] = max(self.stats.max_active.get(kind, 0), counts[kind] + len(
                            [r for r in adm if r["kind"] == kind]))
                        self._iterate(kind, groups[g][kind])
                        for s in groups[g][kind]:
                            s.it += self.C
                        sols += groups[g][kind]
                tp = st.add("iterate", tp)
                if sols:
                    arrs = []
                    for s in sols:
                        arrs += [s.bb, s.st.rho if s.res.kind == "cg" else s.st.rr]
                    work, vals = gbuf[g]
                    rd = rt.read_scalars_async(arrs, work, vals)
                    gbuf[g] = (rd.work, rd.vals)
                    pend[g] = (rd, sols, holds)
                    st.add("read", tp)
                self.stats.ticks += 1
                self._advance(0.0)
                g = (g + 1) % G
            rt.sync()
            complete(block=True)
        finally:
            self._inflight.clear()
            if t_ref is not None:
                rt.release_ticket(t_ref)
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

