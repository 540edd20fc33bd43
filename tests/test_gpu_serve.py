"""The serving loop on the device: continuous batching of CG, BiCGSTAB and
Black-Scholes requests.

Each request's result must be bit-identical alone and in the mix (the mix
admits requests while others are mid-solve, so they share batched launches),
and agree with the oracle.  Option prices: per option within 4 eps32 (S + K) of
the stored-dtype oracle.
Solves: the oracle, run with the same convergence test (every 4
iterations), stops within one test of the GPU (near convergence the updates
are dominated by rounding, which the two paths do in different orders, and
BiCGSTAB's residual is not monotone, so the two can cross the tolerance one
test apart); the solution's true residual ||b - A x|| (oracle SpMV) is within
1.5 tol ||b||; and it differs from the oracle's converged iterate by at most
2 tol kappa norm-wise -- two solutions whose residuals are both below
tol ||b|| can differ by that much, with kappa = cot^2(pi / (2 (m + 1))) the
condition number of the 3-D 7-point Laplacian."""
import numpy as np
import pytest

from oracle import programs
from paper_2406_18109_gb300 import arrays as A
from paper_2406_18109_gb300 import serve
from paper_2406_18109_gb300 import workloads as W
from synth import inputs
from tests.helpers import gpu_runtime

pytestmark = pytest.mark.gpu

# every solve spans at least two 256-element tiles (a one-point instance
# runs unbatched: its scalar and vector tasks share one launch domain)
LADDER = (7, 9, 12, 16)


def _requests():
    # 14 requests, 0.5 ms apart on average, against 1 ms ticks: several
    # arrive while earlier solves are running
    return inputs.serving_requests(14, seed=3, mean_gap_s=5e-4, ladder=LADDER, bs_log2=(9, 14))


def _serve(reqs, **kw):
    with gpu_runtime("persistent", tile=256) as rt:
        srv = serve.Server(rt, inputs.poisson3d_csr, tol=1e-8, iters_per_tick=4, clock=serve.TickClock(1e-3), **kw)
        out = srv.run(reqs, inputs.serving_payload)
        return {r.rid: r for r in out}, srv.stats, rt.stats()


def _same(a, b):
    if isinstance(a, tuple):
        return all(_same(x, y) for x, y in zip(a, b))
    return a.dtype == b.dtype and np.array_equal(a.view(np.uint8), b.view(np.uint8))


def test_mix_equals_alone_and_oracle():
    reqs = _requests()
    mix, st, rst = _serve(reqs)
    assert sorted(mix) == [r["rid"] for r in reqs]
    assert st.max_active.get("cg", 0) >= 2 and st.max_active.get("bicgstab", 0) >= 2
    assert rst["batches"] > 0 and rst["batch_fallbacks"] == 0, rst["batch_fallback_reason"]
    overlapped = [r for r in mix.values() if r.kind != "bs" and r.admitted > 0]
    assert overlapped, "no solve joined while others were running"
    prm = inputs.bs_params()
    for req in reqs:
        got = mix[req["rid"]]
        alone, _, _ = _serve([dict(req, arrival=0.0)])
        ref = alone[req["rid"]]
        assert got.iterations == ref.iterations, req
        assert _same(got.output, ref.output), req
        if req["kind"] == "bs":
            S, K, T = inputs.serving_payload(req)
            c, p = programs.black_scholes(S, K, T, prm["r"], prm["sigma"], np.float32)
            tol = 4 * np.finfo(np.float32).eps * (S.astype(np.float64) + K)   # stored-dtype oracle
            assert np.all(np.abs(got.output[0] - c) <= tol) and np.all(np.abs(got.output[1] - p) <= tol)
            continue
        k, tol, m = got.iterations, 1e-8, req["size"]
        assert got.converged and got.rel_residual <= tol and k % 4 == 0
        rp, col, val = inputs.poisson3d_csr(m)
        b = programs.spmv(rp, col, val, inputs.serving_payload(req))
        bn = np.linalg.norm(b)

        def oracle(iters):
            if req["kind"] == "cg":
                x, r, rho = programs.cg(rp, col, val, b, iters)
                return x, np.sqrt(rho) / bn
            x, it, rel = programs.bicgstab(rp, col, val, b, 0.0, iters)
            assert it == iters
            return x, rel
        ko = 4
        xo, rel_o = oracle(ko)
        while rel_o > tol:
            ko += 4
            xo, rel_o = oracle(ko)
        assert abs(k - ko) <= 4, (req, k, ko)
        assert np.linalg.norm(b - programs.spmv(rp, col, val, got.output)) <= 1.5 * tol * bn, req
        kappa = 1.0 / np.tan(np.pi / (2 * (m + 1))) ** 2
        assert np.linalg.norm(got.output - xo) / np.linalg.norm(xo) <= 2 * tol * kappa, req


def test_budget_limits_admission_and_evicts_operators():
    reqs = _requests()
    free, _, _ = _serve(reqs)
    # room for the largest request and its operator, little more: requests
    # queue for memory and idle operators are evicted
    big = max(serve.request_bytes(r["kind"], r["size"]) + (serve.operator_bytes(r["size"]) if r["kind"] != "bs" else 0)
              for r in reqs)
    tight, st, _ = _serve(reqs, budget_bytes=big + 4096)
    assert st.peak_bytes <= big + 4096 and st.evictions > 0
    for rid, r in free.items():
        assert tight[rid].iterations == r.iterations and _same(tight[rid].output, r.output)
        assert tight[rid].latency >= 0


def test_batch_repeat_equals_reissue():
    specs = [(7, 1), (9, 2), (12, 3)]
    xs = {}
    for repeat in (False, True):
        with gpu_runtime("persistent", tile=256) as rt:
            probs = []
            for m, seed in specs:
                rp, col, val = inputs.poisson3d_csr(m)
                Am = A.CSR(rt, rp, col, val)
                probs.append((Am, W.cg_start_inplace(Am @ rt.array(inputs.uniform(seed, -1, 1, m ** 3)))))
            rt.flush()
            W.batched_cg_iteration(rt, probs)
            if repeat:
                rt.batch_repeat(9)
                assert rt.stats()["batch_repeats"] == 9
            else:
                for _ in range(9):
                    W.batched_cg_iteration(rt, probs)
            xs[repeat] = [s.x.numpy() for _, s in probs]
            # a freed store ends the steady state: repeating is refused
            tmp = rt.array(np.ones(10))
            tmp2 = tmp * 2.0
            tmp2.numpy()
            del tmp, tmp2
            rt.flush()
            with pytest.raises(A.B.DfsError):
                rt.batch_repeat(1)
    for a, b in zip(xs[False], xs[True]):
        assert np.array_equal(a.view(np.uint64), b.view(np.uint64))


def test_read_scalars_matches_single_reads():
    with gpu_runtime("persistent", tile=256) as rt:
        a = rt.array(inputs.uniform(3, -1, 1, 5000))
        b = rt.array(inputs.uniform(4, -1, 1, 5000).astype(np.float32))
        ss = [A.dot(a, a), A.asum(a), A.dot(b, b), rt.scalar(2.5), rt.array(np.array(7, dtype=np.int32))]
        vals = rt.read_scalars(ss)
        for v, s in zip(vals, ss):
            assert v == float(s.numpy())


def test_serving_full_size_requests():
    """Eight requests drawn from the benchmark's serving distribution (3-D
    Poisson 64^3..256^3, options 2^16..2^24) in its launch configuration:
    every solve converged, its true residual ||b - A x|| (oracle SpMV) within
    1.5 tol ||b||; option prices on a sample of 4096 options per batch
    within 4 eps32 (S + K) of the stored-dtype oracle."""
    from paper_2406_18109_gb300 import configs
    cfg = configs.SERVING
    reqs = inputs.serving_requests(8, seed=cfg["seed"], mean_gap_s=cfg["mean_gap_ms"] * 1e-3)
    with gpu_runtime("persistent", tile=cfg["tile"], block=cfg["block"], unroll=cfg["unroll"]) as rt:
        srv = serve.Server(rt, inputs.poisson3d_csr, budget_bytes=int(cfg["budget_gb"] * 1e9), tol=cfg["tol"],
                           iters_per_tick=cfg["iters_per_tick"], max_active=cfg["max_active"])
        out = {r.rid: r for r in srv.run(reqs, inputs.serving_payload)}
    assert sorted(out) == [r["rid"] for r in reqs]
    prm = inputs.bs_params()
    rng = np.random.default_rng(5)
    for req in reqs:
        r = out[req["rid"]]
        if req["kind"] == "bs":
            S, K, T = inputs.serving_payload(req)
            idx = np.sort(rng.choice(len(S), 4096, replace=False))
            c, p = programs.black_scholes(S[idx], K[idx], T[idx], prm["r"], prm["sigma"], np.float32)
            tol = 4 * np.finfo(np.float32).eps * (S[idx].astype(np.float64) + K[idx])   # stored-dtype oracle
            assert np.all(np.abs(r.output[0][idx] - c) <= tol) and np.all(np.abs(r.output[1][idx] - p) <= tol)
            continue
        assert r.converged and r.iterations % cfg["iters_per_tick"] == 0, req
        rp, col, val = inputs.poisson3d_csr(req["size"])
        b = programs.spmv(rp, col, val, inputs.serving_payload(req))
        res = np.linalg.norm(b - programs.spmv(rp, col, val, r.output))
        assert res <= 1.5 * cfg["tol"] * np.linalg.norm(b), (req, res / np.linalg.norm(b))


def test_scalar_gather_and_repeat_refuse_bad_state():
    """dfs_read_scalars refuses a store that is not 0-d or holds no value;
    dfs_batch_repeat refuses a batch that was not steady (it created the
    stores it wrote) and works once the batch only updates stores in place."""
    with gpu_runtime("persistent", tile=256) as rt:
        v = rt.array(np.ones(300))
        with pytest.raises(A.B.DfsError) as e:
            rt.read_scalars([v])
        assert e.value.code == -1
        with pytest.raises(A.B.DfsError) as e:
            rt.read_scalars([rt.empty(())])
        assert e.value.code == -7
        xs = [rt.array(inputs.uniform(i, -1, 1, 700 + 300 * i)) for i in range(2)]
        rt.batch_begin()
        outs = []
        for x in xs:
            outs.append(x * 2.0)                 # creates its output: not steady
            rt.batch_next()
        rt.batch_end()
        with pytest.raises(A.B.DfsError) as e:
            rt.batch_repeat(1)
        assert e.value.code == -7
        rt.batch_begin()
        for x in xs:
            x *= 0.5                             # in place: steady
            rt.batch_next()
        rt.batch_end()
        rt.batch_repeat(3)
        for i, x in enumerate(xs):
            want = inputs.uniform(i, -1, 1, 700 + 300 * i) * 0.5 ** 4
            assert np.array_equal(x.numpy(), want)


def test_payloads_in_mapped_host_memory_give_the_same_results():
    """Request data in mapped page-locked buffers are read in place (x*
    streamed into a device copy; option inputs read directly) with the same
    results, bit for bit, as uploaded pageable data."""
    reqs = _requests()

    def pinned(req):
        p = inputs.serving_payload(req)
        out = []
        for a in (p if isinstance(p, tuple) else (p,)):
            h = A.Runtime.host_empty(a.shape, a.dtype)
            h[...] = a
            out.append(h)
        return tuple(out) if isinstance(p, tuple) else out[0]
    with gpu_runtime("persistent", tile=256) as rt:
        srv = serve.Server(rt, inputs.poisson3d_csr, tol=1e-8, iters_per_tick=4, clock=serve.TickClock(1e-3))
        got = {r.rid: r for r in srv.run(reqs, pinned)}
        assert rt.stats()["batch_fallbacks"] == 0
    ref, _, _ = _serve(reqs)
    for rid, r in ref.items():
        assert got[rid].iterations == r.iterations and _same(got[rid].output, r.output), rid


def test_replayed_iteration_windows_equal_issued_ones():
    """Iterations replayed from a recorded window per kind and size
    (dfs_template_replay) retire every solve after the same iterations with
    the same bits as iterations issued task by task."""
    reqs = _requests()
    rep, _, rst = _serve(reqs)
    plain, _, _ = _serve(reqs, templates=False)
    assert rst["batch_fallbacks"] == 0, rst["batch_fallback_reason"]
    for rid, r in rep.items():
        assert r.iterations == plain[rid].iterations, rid
        assert _same(r.output, plain[rid].output), rid


def test_one_group_and_two_pipelined_groups_agree():
    """The loop with two groups taking turns (the GPU iterates one group while
    the host reads the other's residuals) and with one group (the host waits
    for every read) retire every solve after the same iterations with the
    same bits: groups change when work runs, not what it computes."""
    reqs = _requests()
    two, _, _ = _serve(reqs)
    one, _, _ = _serve(reqs, overlap=False)
    assert sorted(two) == sorted(one) == [r["rid"] for r in reqs]
    for rid, r in two.items():
        assert r.iterations == one[rid].iterations, rid
        assert _same(r.output, one[rid].output), rid


def test_async_scalar_read_and_tickets():
    """dfs_read_scalars_async returns the values dfs_read_scalars returns,
    once its ticket has completed; tickets poll, wait, time and release, and
    a released ticket is unknown."""
    with gpu_runtime("persistent", tile=256) as rt:
        xs = [rt.array(inputs.uniform(i, -1, 1, 500 + 200 * i)) for i in range(5)]
        dots = [A.dot(x, x) for x in xs]
        want = rt.read_scalars(dots)
        t_a = rt.record()
        rd = rt.read_scalars_async(dots)
        for x in xs:
            x *= 2.0                             # work queued behind the read
        t_b = rt.record()
        assert rd.values() == want
        rt.wait(t_b)
        assert rt.poll(t_a) and rt.poll(t_b)
        assert rt.elapsed_ms(t_a, t_b) >= 0.0
        for t in (t_a, t_b):
            rt.release_ticket(t)
        with pytest.raises(A.B.DfsError) as e:
            rt.wait(t_a)
        assert e.value.code == -7
        # buffers reused by a second read of other values: (2x).(2x) = 4 x.x exactly
        dots2 = [A.dot(x, x) for x in xs]
        rd2 = rt.read_scalars_async(dots2[:3], rd.work, rd.vals)
        assert rd2.work is rd.work and rd2.values() == [4.0 * v for v in want[:3]]
        with pytest.raises(A.B.DfsError) as e:
            rt.read_scalars_async([xs[0]])       # not 0-d
        assert e.value.code == -1
