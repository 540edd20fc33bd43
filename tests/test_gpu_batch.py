"""Batched execution of isomorphic windows (many uneven problems, one launch).

Every instance of a batch must give exactly what it gives when run alone
with the same tiles (bit for bit: reductions keep per-point partials summed
in point order), and agree with the oracle."""
import numpy as np
import pytest

from oracle import programs
from paper_2406_18109_gb300 import arrays as A
from paper_2406_18109_gb300 import workloads as W
from synth import inputs
from tests.helpers import gpu_runtime

pytestmark = pytest.mark.gpu

SPECS = [("poisson", 33, 0, 1), ("spd", 5000, 7, 2), ("poisson", 71, 0, 3), ("spd", 1500, 8, 4),
         ("poisson", 45, 0, 5), ("poisson", 90, 0, 6), ("spd", 12000, 9, 7)]


def _problems(rt, specs, dtype=np.float64):
    out = []
    for spec in specs:
        rp, col, val, xs = inputs.batched_cg_matrix(spec)
        Am = A.CSR(rt, rp, col, val.astype(dtype))
        b = Am @ rt.array(xs.astype(dtype))
        out.append((Am, W.cg_start_inplace(b)))
    rt.flush()
    return out


def _run(specs, iters, batched, dtype=np.float64, graph=False):
    with gpu_runtime("persistent", tile=512) as rt:
        probs = _problems(rt, specs, dtype)
        if batched:
            W.batched_cg_iteration(rt, probs)
            if graph:
                rt.capture_begin()
                W.batched_cg_iteration(rt, probs)
                g = rt.capture_end()
                for _ in range(iters - 1):
                    rt.graph_launch(g)
            else:
                for _ in range(iters - 1):
                    W.batched_cg_iteration(rt, probs)
        else:
            for Am, s in probs:
                for _ in range(iters):
                    W.cg_iteration_inplace(Am, s)
                    rt.flush()
        xs = [s.x.numpy() for _, s in probs]
        st = rt.stats()
        if batched and graph:
            rt.graph_destroy(g)
        return xs, st


def test_batched_equals_alone_and_oracle():
    iters = 20
    xb, st = _run(SPECS, iters, batched=True)
    assert st["batches"] == iters and st["batched_instances"] == iters * len(SPECS)
    assert st["batch_fallbacks"] == 0
    xa, _ = _run(SPECS, iters, batched=False)
    for i, spec in enumerate(SPECS):
        assert np.array_equal(xb[i].view(np.uint64), xa[i].view(np.uint64)), spec
        rp, col, val, xs = inputs.batched_cg_matrix(spec)
        b = programs.spmv(rp, col, val, xs)
        xo, _, _ = programs.cg(rp, col, val, b, iters)
        assert np.linalg.norm(xb[i] - xo) / np.linalg.norm(xo) < 1e-12, spec


def test_batched_fp32():
    iters = 15
    xb, st = _run(SPECS[:4], iters, batched=True, dtype=np.float32)
    xa, _ = _run(SPECS[:4], iters, batched=False, dtype=np.float32)
    for i in range(4):
        assert xb[i].dtype == np.float32
        assert np.array_equal(xb[i].view(np.uint32), xa[i].view(np.uint32))
        rp, col, val, xs = inputs.batched_cg_matrix(SPECS[i])
        b = programs.spmv(rp, col, val.astype(np.float32), xs.astype(np.float32), np.float32)
        xo, _, _ = programs.cg(rp, col, val, b, iters, dt=np.float32)
        # FP32 reductions against the stored-dtype oracle: 1e-5 (measured on GB300: 1.4e-7)
        assert np.linalg.norm(xb[i] - xo) / np.linalg.norm(xo) < 1e-5


def test_batched_graph_replay():
    iters = 12
    xg, _ = _run(SPECS, iters, batched=True, graph=True)
    xb, _ = _run(SPECS, iters, batched=True)
    for i in range(len(SPECS)):
        assert np.array_equal(xg[i].view(np.uint64), xb[i].view(np.uint64))


def test_non_isomorphic_batch_falls_back_correctly():
    with gpu_runtime("persistent", tile=512) as rt:
        x = rt.array(inputs.uniform(1, 0.5, 2.0, 3000))
        y = rt.array(inputs.uniform(2, 0.5, 2.0, 5000))
        rt.batch_begin()
        a = x * 2.0 + 1.0
        rt.batch_next()
        b = A.sqrt(y)
        rt.batch_next()
        rt.batch_end()
        st = rt.stats()
        assert st["batch_fallbacks"] == 1 and st["batches"] == 0
        assert np.allclose(a.numpy(), x.numpy() * 2 + 1) and np.allclose(b.numpy(), np.sqrt(y.numpy()))


def test_batched_black_scholes_instances_equal_alone():
    sizes = [10_000, 70_001, 33_333]
    prm = inputs.bs_params()
    data = [inputs.bs_inputs(n, seed=20 + i) for i, n in enumerate(sizes)]
    with gpu_runtime("persistent", tile=4096) as rt:
        arrs = [[rt.array(v) for v in d] for d in data]
        outs = []
        rt.batch_begin()
        for S, K, T in arrs:
            outs.append(W.black_scholes(S, K, T, prm["r"], prm["sigma"]))
            rt.batch_next()
        rt.batch_end()
        assert rt.stats()["batches"] == 1
        got = [(c.numpy(), p.numpy()) for c, p in outs]
    for (S, K, T), (c, p) in zip(data, got):
        with gpu_runtime("persistent", tile=4096) as rt:
            c1, p1 = W.black_scholes(rt.array(S), rt.array(K), rt.array(T), prm["r"], prm["sigma"])
            assert np.array_equal(c.view(np.uint32), c1.numpy().view(np.uint32))
            assert np.array_equal(p.view(np.uint32), p1.numpy().view(np.uint32))


def test_cached_batch_kernel_serves_new_stores():
    """A second batch of the same structure over other stores reuses the
    memoised kernel with its own pointers."""
    prm = inputs.bs_params()
    with gpu_runtime("persistent", tile=256) as rt:
        for rnd in range(3):
            sizes = [1000 + 7 * rnd, 3001, 555 + rnd]
            data = [inputs.bs_inputs(n, seed=40 + 3 * rnd + i) for i, n in enumerate(sizes)]
            arrs = [[rt.array(v) for v in d] for d in data]
            rt.batch_begin()
            outs = []
            for S, K, T in arrs:
                outs.append(W.black_scholes(S, K, T, prm["r"], prm["sigma"]))
                rt.batch_next()
            rt.batch_end()
            st = rt.stats()
            assert st["batches"] == rnd + 1 and st["batch_fallbacks"] == 0
            for (S, K, T), (c, p) in zip(data, outs):
                co, po = programs.black_scholes(S, K, T, prm["r"], prm["sigma"], np.float32)
                tol = 4 * np.finfo(np.float32).eps * (S.astype(np.float64) + K)   # stored-dtype oracle
                assert np.all(np.abs(c.numpy() - co) <= tol) and np.all(np.abs(p.numpy() - po) <= tol)
            del arrs, outs


def test_autotuned_batch_matches_fresh_run_and_oracle():
    """Tuning changes the context's tile and launch shape between timed
    trials; afterwards (state reset) the solves equal a fresh context built
    with the chosen setting, bit for bit, and the oracle."""
    from paper_2406_18109_gb300 import autotune
    iters = 15

    def setup(rt):
        probs, bs = [], []
        for spec in SPECS:
            rp, col, val, xs = inputs.batched_cg_matrix(spec)
            Am = A.CSR(rt, rp, col, val)
            b = Am @ rt.array(xs)
            probs.append((Am, W.cg_start_inplace(b)))
            bs.append(b)
        rt.flush()
        return probs, bs

    with gpu_runtime("persistent", tile=512, time_launches=True) as rt:
        probs, bs = setup(rt)
        best, trials = autotune.tune(rt, lambda: W.batched_cg_iteration(rt, probs),
                                     space={"tile": [256, 512], "block": [128, 256], "unroll": [1, 2],
                                            "ctas_per_sm": [0, 2]}, warmup=1, reps=2)
        assert len(trials) == 5 and all(np.isfinite(ms) for _, ms in trials)
        assert autotune.current(rt) == best
        rt.batch_begin()
        for (_, s), b in zip(probs, bs):
            W.cg_reset_inplace(s, b)
            rt.batch_next()
        rt.batch_end()
        for _ in range(iters):
            W.batched_cg_iteration(rt, probs)
        tuned = [s.x.numpy() for _, s in probs]
    with gpu_runtime("persistent", tile=best["tile"], block=best["block"], unroll=best["unroll"],
                     ctas_per_sm=best["ctas_per_sm"]) as rt:
        probs, _ = setup(rt)
        for _ in range(iters):
            W.batched_cg_iteration(rt, probs)
        fresh = [s.x.numpy() for _, s in probs]
    for i, spec in enumerate(SPECS):
        assert np.array_equal(tuned[i].view(np.uint64), fresh[i].view(np.uint64)), spec
        rp, col, val, xs = inputs.batched_cg_matrix(spec)
        xo, _, _ = programs.cg(rp, col, val, programs.spmv(rp, col, val, xs), iters)
        assert np.linalg.norm(tuned[i] - xo) / np.linalg.norm(xo) < 1e-12, spec


def test_batched_full_size_sampled():
    """The full batch the benchmark times (256 uneven solves, 22.3 M unknowns,
    its tile policy and launch shape): after 10 batched iterations, the
    largest and smallest problem of each family and two random ones agree
    with the oracle one by one (1e-12 norm-wise)."""
    from paper_2406_18109_gb300 import configs
    cfg = configs.BATCHED_CG
    specs = inputs.batched_cg_problems(cfg["count"], cfg["seed"])
    iters = 10
    with gpu_runtime("persistent", tile_max=cfg["tile_max"], min_points=cfg["min_points"], block=cfg["block"],
                     unroll=cfg["unroll"]) as rt:
        mats = []
        for spec in specs:
            rp, col, val, xs = inputs.batched_cg_matrix(spec)
            mats.append((A.CSR(rt, rp, col, val), rt.array(xs)))
        probs = []
        rt.batch_begin()
        for Am, xs_d in mats:
            b = Am @ xs_d
            probs.append((Am, W.cg_start_inplace(b), b))
            rt.batch_next()
        rt.batch_end()
        for _ in range(iters):
            W.batched_cg_iteration(rt, [(Am, s) for Am, s, _ in probs])
        st = rt.stats()
        assert st["batch_fallbacks"] == 0 and st["batches"] == iters + 1
        sizes = [(spec[0], spec[1]) for spec in specs]
        pick = set()
        for fam in ("poisson", "spd"):
            idx = [i for i, s in enumerate(sizes) if s[0] == fam]
            pick.add(max(idx, key=lambda i: sizes[i][1]))
            pick.add(min(idx, key=lambda i: sizes[i][1]))
        rng = np.random.default_rng(11)
        pick.update(int(i) for i in rng.choice(len(specs), 2, replace=False))
        got = {i: probs[i][1].x.numpy() for i in sorted(pick)}
    for i, x in got.items():
        rp, col, val, xs = inputs.batched_cg_matrix(specs[i])
        xo, _, _ = programs.cg(rp, col, val, programs.spmv(rp, col, val, xs), iters)
        assert np.linalg.norm(x - xo) / np.linalg.norm(xo) < 1e-12, specs[i]


def test_batched_barrier_timeout_is_reported_and_next_batch_is_right():
    """A batched launch whose grid barrier runs out of time (CTA 0 withholds
    its arrival at barrier 2) ends instead of hanging and reports
    DFS_ERR_BARRIER_TIMEOUT at the next sync; the context stays usable, and
    batched launches on the same device afterwards deal every point."""
    from paper_2406_18109_gb300.binding import DfsError
    specs = SPECS[:3]
    with gpu_runtime("persistent", tile=512, timeout_s=0.05, debug_skip_arrival=2) as rt:
        probs = _problems(rt, specs)
        W.batched_cg_iteration(rt, probs)
        with pytest.raises(DfsError) as e:
            rt.sync()
        assert e.value.code == -6
        rt.sync()                                  # error consumed; context usable
    # a fresh context on the same device: the batched kernels deal every point
    xb, st = _run(specs, 6, batched=True)
    xa, _ = _run(specs, 6, batched=False)
    for i in range(len(specs)):
        assert np.array_equal(xb[i].view(np.uint64), xa[i].view(np.uint64))


def test_kernel_source_names_the_batch_on_cache_hits():
    """The source reported for the most recent launch is the batched kernel's
    also when that kernel comes from the batch cache after another kernel ran
    in between, and after steady repeats."""
    with gpu_runtime("persistent", tile=512) as rt:
        probs = _problems(rt, SPECS[:3])
        W.batched_cg_iteration(rt, probs)                 # generated here
        first = rt.kernel_source()
        assert "find_inst" in first
        (A.full(rt, (1000,), 1.0) * 3.0).numpy()          # a single-window launch in between
        assert "find_inst" not in rt.kernel_source()
        W.batched_cg_iteration(rt, probs)                 # a batch-cache hit
        assert rt.kernel_source() == first
        rt.batch_repeat(2)                                # steady repeats of the same kernel
        assert rt.kernel_source() == first
        assert rt.stats()["batch_fallbacks"] == 0
