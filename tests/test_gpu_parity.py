"""GPU parity: the generated sm_103a kernels against the CPU oracle.

Every comparison runs the same seeded inputs through the CUDA path (via the
C-ABI) and through ``oracle/``.  Tolerances: FP64 reductions/solvers 1e-12
norm-wise relative; FP32 Black-Scholes |diff| <= 1e-5 (S + K) per option
against the FP64 oracle and <= 4 eps32 (S + K) against the stored-dtype one;
element-wise FP32 work whose operations round the same way on both sides
(the Jacobi stencil: adds and a multiply) bit for bit.  Fused execution must
equal unfused execution bit for bit (every element operation rounds once).
"""
import numpy as np
import pytest

from oracle import programs
from oracle.interp import Imm, Machine, XTask
from oracle.ir import Arg, IDENTITY, Tiling
from paper_2406_18109_gb300 import arrays as A
from paper_2406_18109_gb300 import binding as B
from paper_2406_18109_gb300 import configs
from paper_2406_18109_gb300 import workloads as W
from synth import inputs
from tests.helpers import MODES, gpu_runtime

pytestmark = pytest.mark.gpu

BS = configs.BLACK_SCHOLES


def _bits(a):
    return np.ascontiguousarray(a).view(np.uint32 if a.dtype == np.float32 else np.uint64)


# ----------------------------------------------------------- Black-Scholes
def _bs_gpu(mode, S, K, T, **kw):
    with gpu_runtime(mode, **kw) as rt:
        call, put = W.black_scholes(rt.array(S), rt.array(K), rt.array(T), BS["r"], BS["sigma"])
        return call.numpy(), put.numpy(), rt.stats()


@pytest.mark.parametrize("mode", MODES)
def test_black_scholes_matches_oracle(mode):
    n = 100_003                                  # 25 tiles of 4096 and a ragged tail
    S, K, T = inputs.bs_inputs(n, seed=BS["seed"])
    c, p, st = _bs_gpu(mode, S, K, T, tile=4096)
    scale = S.astype(np.float64) + K.astype(np.float64)
    c64, p64 = programs.black_scholes(S, K, T, BS["r"], BS["sigma"], np.float64)
    assert np.all(np.abs(c - c64) <= 1e-5 * scale)
    assert np.all(np.abs(p - p64) <= 1e-5 * scale)
    _assert_stored_dtype_close(S, K, T, c, p)
    if mode == "persistent":
        assert st["launches"] == 1
    if mode == "unfused":
        assert st["launches"] == W.BLACK_SCHOLES_TASKS


def _assert_stored_dtype_close(S, K, T, c, p):
    """Against the stored-dtype oracle (the same 23 steps, each rounded to
    float32): the two sides differ only in the library's log, exp and erf
    (each within a couple of float32 ulp on both sides), so every price agrees
    to a few ulp of the terms it is made of: |diff| <= 4 eps32 (S + K).
    Measured on GB300 over 100,003 options: 2.1 eps32 (S + K) at most, 57 % of
    calls and 67 % of puts bit-identical.  A wrong constant in the chain (say
    1/sqrt 2 to four digits) moves prices by tens of eps32 S."""
    c32, p32 = programs.black_scholes(S, K, T, BS["r"], BS["sigma"], np.float32)
    tol = 4 * np.finfo(np.float32).eps * (S.astype(np.float64) + K.astype(np.float64))
    assert np.all(np.abs(c.astype(np.float64) - c32) <= tol)
    assert np.all(np.abs(p.astype(np.float64) - p32) <= tol)



def test_black_scholes_fused_equals_unfused_bitwise():
    n = 50_001
    S, K, T = inputs.bs_inputs(n, seed=3)
    res = {m: _bs_gpu(m, S, K, T, tile=2048)[:2] for m in MODES}
    for m in MODES[1:]:
        assert np.array_equal(_bits(res[m][0]), _bits(res["persistent"][0]))
        assert np.array_equal(_bits(res[m][1]), _bits(res["persistent"][1]))


def test_black_scholes_full_size_sampled():
    """2^26 options in the benchmark's launch configuration; sampled options
    are priced one by one by the oracle."""
    n = BS["n"]
    S, K, T = inputs.bs_inputs(n, seed=BS["seed"])
    c, p, _ = _bs_gpu("persistent", S, K, T, tile=BS["tile"], block=BS["block"], unroll=BS["unroll"])
    rng = np.random.default_rng(99)
    idx = np.concatenate([rng.integers(0, n, 4000), np.arange(8), np.arange(n - 8, n)])
    c_o, p_o = programs.black_scholes(S[idx], K[idx], T[idx], BS["r"], BS["sigma"], np.float64)
    scale = S[idx].astype(np.float64) + K[idx].astype(np.float64)
    assert np.all(np.abs(c[idx] - c_o) <= 1e-5 * scale)
    assert np.all(np.abs(p[idx] - p_o) <= 1e-5 * scale)
    _assert_stored_dtype_close(S[idx], K[idx], T[idx], c[idx], p[idx])
    # put-call parity holds at every one of the 2^26 options
    lhs = c.astype(np.float64) - p.astype(np.float64)
    rhs = S.astype(np.float64) - K.astype(np.float64) * np.exp(-BS["r"] * T.astype(np.float64))
    assert np.all(np.abs(lhs - rhs) <= 1e-5 * (S.astype(np.float64) + K.astype(np.float64)))


# ---------------------------------------------------------------------- CG
def _cg_gpu(mode, m, iters, tile, seed=0, **kw):
    rp, col, val, xs = inputs.cg_inputs(m=m, seed=seed)
    with gpu_runtime(mode, tile=tile, **kw) as rt:
        Am = A.CSR(rt, rp, col, val)
        b = Am @ rt.array(xs)                   # b = A x*, computed on the device
        st = W.cg_start(b)
        rt.flush()
        for _ in range(iters):
            W.cg_iteration(Am, st)
            rt.flush()
        return st.x.numpy(), st.r.numpy(), st.rho.item(), b.numpy(), rt.stats()


def _cg_oracle(m, iters, seed=0):
    rp, col, val, xs = inputs.cg_inputs(m=m, seed=seed)
    b = programs.spmv(rp, col, val, xs)
    x, r, rho = programs.cg(rp, col, val, b, iters)
    return x, r, rho, b


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("mode", MODES)
def test_cg_matches_oracle(mode):
    m, iters = 61, 50                           # n = 3721: 15 tiles of 256 and a ragged tail
    x, r, rho, b, st = _cg_gpu(mode, m, iters, tile=256)
    xo, ro, rhoo, bo = _cg_oracle(m, iters)
    assert _rel(b, bo) < 1e-14
    # measured on GB300: x 1.2e-15, r 2.6e-14, rho 4.8e-14 (relative)
    assert _rel(x, xo) < 1e-12
    assert _rel(r, ro) < 1e-12
    assert abs(rho - rhoo) <= 1e-12 * abs(rhoo)
    if mode == "persistent":
        # b = A x* and the CG start share one flush, then one launch per iteration
        assert st["launches"] == iters + 1 and st["barriers"] == 2 * iters


def test_cg_single_point_domain():
    # n = 400 < one 512-row tile: the launch domain has one point, so the
    # scalar divides share it and the paper's pass fuses them with vector tasks
    x, r, rho, b, st = _cg_gpu("persistent", 20, 25, tile=512)
    xo, ro, rhoo, bo = _cg_oracle(20, 25)
    assert _rel(x, xo) < 1e-12 and abs(rho - rhoo) <= 1e-12 * abs(rhoo)
    xu, *_ = _cg_gpu("unfused", 20, 25, tile=512)
    assert np.array_equal(_bits(x), _bits(xu))


def test_cg_fused_equals_unfused_bitwise():
    res = {m: _cg_gpu(m, 40, 20, tile=256) for m in MODES}
    for m in MODES[1:]:
        assert np.array_equal(_bits(res[m][0]), _bits(res["persistent"][0]))
        assert res[m][2] == res["persistent"][2]


def test_cg_full_size():
    cfg = configs.CG
    x, r, rho, b, st = _cg_gpu("persistent", cfg["m"], cfg["iters"], tile=cfg["tile"],
                               block=cfg["block"], unroll=cfg["unroll"])
    xo, ro, rhoo, bo = _cg_oracle(cfg["m"], cfg["iters"])
    assert _rel(x, xo) < 1e-12 and _rel(r, ro) < 1e-12
    assert abs(rho - rhoo) <= 1e-12 * abs(rhoo)
    assert st["kernels_compiled"] + st["kernel_disk_hits"] <= 4    # isomorphic iterations share one kernel
    assert st["plan_hits"] >= cfg["iters"] - 1


@pytest.mark.parametrize("mode", MODES)
def test_cg_fp32_matches_stored_dtype_oracle(mode):
    """CG with FP32 values: against the FP32 oracle (same operations in the
    stored dtype) to 1e-5 norm-wise; fused and unfused paths bit-identical
    is checked by the FP64 tests."""
    m, iters = 48, 25
    rp, col, val, xs = inputs.cg_inputs(m=m, seed=0)
    with gpu_runtime(mode, tile=256) as rt:
        Am = A.CSR(rt, rp, col, val.astype(np.float32))
        b = Am @ rt.array(xs.astype(np.float32))
        s = W.cg_start(b)
        for _ in range(iters):
            W.cg_iteration(Am, s)
            rt.flush()
        x = s.x.numpy()
    assert x.dtype == np.float32
    bo = programs.spmv(rp, col, val.astype(np.float32), xs.astype(np.float32), np.float32)
    xo, _, _ = programs.cg(rp, col, val, bo, iters, dt=np.float32)
    assert _rel(x.astype(np.float64), xo.astype(np.float64)) < 1e-5


def test_cg_full_size_as_benchmarked():
    """The benchmark's launch configuration: the whole 256^2 solve captured
    in a CUDA graph with five iterations per flush window, replayed."""
    cfg = configs.CG
    ipf = cfg["iters_per_flush"]
    rp, col, val, xs = inputs.cg_inputs(m=cfg["m"], seed=cfg["seed"])
    with gpu_runtime("persistent", tile=cfg["tile"], block=cfg["block"], unroll=cfg["unroll"],
                     window_size=cfg["window_size"]) as rt:
        Am = A.CSR(rt, rp, col, val)
        b = Am @ rt.array(xs)
        s = W.cg_start_inplace(b)
        for _ in range(ipf):
            W.cg_iteration_inplace(Am, s)
        rt.flush()
        rt.capture_begin()
        W.cg_reset_inplace(s, b)
        rt.flush()
        for it in range(cfg["iters"]):
            W.cg_iteration_inplace(Am, s)
            if (it + 1) % ipf == 0:
                rt.flush()
        g = rt.capture_end()
        for _ in range(2):
            rt.graph_launch(g)
        x = s.x.numpy()
        launches = rt.stats()["launches"]
        rt.graph_destroy(g)
    xo, _, _, _ = _cg_oracle(cfg["m"], cfg["iters"])
    assert _rel(x, xo) < 1e-12
    assert launches >= 2 * (1 + cfg["iters"] // ipf)


# ------------------------------------------------------------------ Jacobi
def _jacobi_gpu(mode, grid, sweeps, rows, per_flush=1, **kw):
    with gpu_runtime(mode, rows=rows, **kw) as rt:
        g = rt.array(grid)
        views = W.jacobi_views(g)
        for s in range(sweeps):
            W.jacobi_sweep(views)
            if (s + 1) % per_flush == 0:
                rt.flush()
        return g.numpy(), rt.stats()


@pytest.mark.parametrize("mode", MODES)
def test_jacobi_matches_oracle_bitwise(mode):
    grid = inputs.jacobi_grid(62, seed=2)        # 64x64: 4 bands of 16 rows, the last ragged
    out, st = _jacobi_gpu(mode, grid, 12, rows=16, per_flush=3)
    want = programs.jacobi(grid, 12, np.float32)
    assert np.array_equal(_bits(out), _bits(want))


def test_jacobi_full_size_sampled():
    """8192^2 grid, benchmark launch configuration, 3 sweeps: every sampled
    point is recomputed by the oracle on its (2k+3)^2 neighbourhood (values
    farther than k cells cannot reach it in k sweeps)."""
    cfg = configs.JACOBI
    k = 3
    grid = inputs.jacobi_grid(cfg["N"], seed=cfg["seed"])
    out, _ = _jacobi_gpu("persistent", grid, k, rows=cfg["rows"], block=cfg["block"], unroll=cfg["unroll"])
    assert out.min() >= grid.min() and out.max() <= 1.0
    n = grid.shape[0]
    rng = np.random.default_rng(5)
    pts = [(1, 1), (n - 2, n - 2), (1, n - 2), (n - 2, 1), (n // 2, n // 2)]
    pts += [tuple(x) for x in rng.integers(1, n - 1, (60, 2))]
    R = k + 1
    for (i, j) in pts:
        i0, i1 = max(0, i - R), min(n, i + R + 1)
        j0, j1 = max(0, j - R), min(n, j + R + 1)
        sub = programs.jacobi(grid[i0:i1, j0:j1], k, np.float32)
        assert _bits(out[i:i + 1, j:j + 1]) == _bits(sub[i - i0:i - i0 + 1, j - j0:j - j0 + 1]), (i, j)


# ------------------------------------------------------ random windows
OPS1 = ["NEG", "EXP", "SQRT", "ABS", "LOG", "NCDF", "ERF", "COPY"]
OPS2 = ["ADD", "SUB", "MUL", "DIV", "MAX", "MIN"]


def _random_stream(rng, nstores):
    stream = []
    for _ in range(rng.integers(3, 12)):
        out = int(rng.integers(0, nstores))
        if rng.random() < 0.4:
            stream.append((str(rng.choice(OPS1)), out, [int(rng.integers(0, nstores))]))
        else:
            b = int(rng.integers(0, nstores)) if rng.random() < 0.7 else float(rng.uniform(0.5, 2))
            stream.append((str(rng.choice(OPS2)), out, [int(rng.integers(0, nstores)), b]))
    return stream


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_random_elementwise_windows(dtype):
    rng = np.random.default_rng(2024)
    n, tile, ns = 3001, 512, 4
    dom = ((n + tile - 1) // tile,)
    for trial in range(6):
        stream = _random_stream(rng, ns)
        init = [inputs.uniform(100 + trial * 10 + s, 0.5, 2.0, n, dtype) for s in range(ns)]
        outs = {}
        for mode in MODES:
            with gpu_runtime(mode, tile=tile) as rt:
                arrs = [rt.array(x) for x in init]
                for op, o, ins in stream:
                    opnds = [arrs[i]._arg(B.DFS_PRIV_R) if isinstance(i, int) else i for i in ins]
                    rt.submit(op, dom, opnds + [arrs[o]._arg(B.DFS_PRIV_W)])
                outs[mode] = [a.numpy() for a in arrs]
        for mode in MODES[1:]:
            for s in range(ns):
                assert np.array_equal(_bits(outs[mode][s]), _bits(outs["persistent"][s])), (trial, mode, s)
        m = Machine("stored")
        P = Tiling((tile,), (0,), IDENTITY, ((0,), (n,)))
        for s in range(ns):
            m.add(s, init[s])
        for op, o, ins in stream:
            opnds = [Arg(i, P, "R") if isinstance(i, int) else Imm(i) for i in ins]
            m.run(XTask(op, dom, opnds + [Arg(o, P, "W")]))
        for s in range(ns):
            want = m.arrays[s]
            got = outs["persistent"][s]
            ok = np.isclose(got, want, rtol=2e-6 if dtype == np.float32 else 1e-14, atol=0, equal_nan=True)
            assert ok.all(), (trial, s)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_erf_of_a_value_and_its_negation(dtype):
    """ERF and NCDF of x and of NEG(x) in one window: the fused body evaluates
    erf(|.|) once per pair, and each result keeps the bits of its task run
    alone (unfused), ERF stays odd bit for bit, and the values match the
    stored-dtype oracle -- on zeros, infinities, NaN, subnormals and the
    largest finite values as well as ordinary ones."""
    fi = np.finfo(dtype)
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, fi.tiny, fi.tiny / 8, -fi.tiny / 8, fi.max, -fi.max,
                        1e-3, -0.5, 2.0, 3.9, -4.0, 6.0, 27.0], dtype)
    x = np.concatenate([special, inputs.uniform(7, -8.0, 8.0, 3000, dtype)])
    n, tile = x.size, 512
    dom = ((n + tile - 1) // tile,)
    stream = [("NEG", 1, [0]), ("ERF", 2, [0]), ("ERF", 3, [1]), ("NCDF", 4, [0]), ("NCDF", 5, [1])]
    outs = {}
    for mode in MODES:
        with gpu_runtime(mode, tile=tile) as rt:
            arrs = [rt.array(x)] + [rt.array(np.zeros(n, dtype)) for _ in range(5)]
            for op, o, ins in stream:
                rt.submit(op, dom, [arrs[i]._arg(B.DFS_PRIV_R) for i in ins] + [arrs[o]._arg(B.DFS_PRIV_W)])
            outs[mode] = [a.numpy() for a in arrs]
            if mode == "persistent":
                src = rt.kernel_source()
                mags = src.count("erf_mag(") + 2 * src.count("erf_mag2(")   # erf_mag2 serves two lanes
                assert mags * 2 == src.count("erf_sign(")                      # one erf per pair
    for mode in MODES[1:]:
        for s in range(6):
            assert np.array_equal(_bits(outs[mode][s]), _bits(outs["persistent"][s])), (mode, s)
    e, e_neg = outs["persistent"][2], outs["persistent"][3]
    nan = np.isnan(x)
    assert np.array_equal(_bits(e_neg[~nan]), _bits(-e[~nan]))
    assert np.isnan(e[nan]).all() and np.isnan(e_neg[nan]).all()
    m = Machine("stored")
    P = Tiling((tile,), (0,), IDENTITY, ((0,), (n,)))
    m.add(0, x)
    for s in range(1, 6):
        m.add(s, np.zeros(n, dtype))
    for op, o, ins in stream:
        m.run(XTask(op, dom, [Arg(i, P, "R") for i in ins] + [Arg(o, P, "W")]))
    for s in range(1, 6):
        # NCDF = 0.5 (1 + erf): for x << 0 the sum cancels, so its error is
        # absolute, a few units in the last place of 1
        rtol, atol = (2e-6 if dtype == np.float32 else 1e-14), (fi.tiny if s < 4 else 4 * fi.eps)
        ok = np.isclose(outs["persistent"][s], m.arrays[s], rtol=rtol, atol=atol, equal_nan=True)
        assert ok.all(), (s, x[~ok], outs["persistent"][s][~ok], m.arrays[s][~ok])


def test_packed_lanes_never_contract_a_product_into_a_sum():
    """FP32 bodies run some tasks two lanes per instruction; a packed product
    that reaches a sum would be contracted into one fused multiply-add by the
    compiler.  Sums of products and NCDFs (whose last step multiplies) that
    feed sums, directly or through NEG or COPY, stay scalar, MUL runs on single
    lanes, the rest is packed, and every store equals the unfused tasks bit
    for bit."""
    n, tile = 8195, 1024
    dom = ((n + tile - 1) // tile,)
    a, b, d = (inputs.uniform(40 + k, -2.0, 2.0, n, np.float32) for k in range(3))
    stream = [("MUL", 3, [0, 1]), ("ADD", 4, [3, 2]),          # a*b + d: scalar pair
              ("MUL", 5, [0, 2]), ("NEG", 6, [5]), ("SUB", 7, [2, 6]),   # d - (-(a*d)): scalar, through NEG
              ("MUL", 8, [1, 2]), ("MUL", 9, [8, 1.5]),      # product of a product: single lanes
              ("ADD", 10, [0, 2]), ("MUL", 11, [10, 0.25]),  # (a+d)*0.25: the sum packed
              ("NCDF", 12, [0]), ("ADD", 13, [12, 1.0])]     # N(a) + 1: scalar (NCDF ends with a multiply)
    nst = 14
    outs, srcs = {}, {}
    for mode in MODES:
        with gpu_runtime(mode, tile=tile) as rt:
            arrs = [rt.array(x) for x in (a, b, d)] + [rt.array(np.zeros(n, np.float32)) for _ in range(3, nst)]
            for op, o, ins in stream:
                opnds = [arrs[i]._arg(B.DFS_PRIV_R) if isinstance(i, int) else i for i in ins]
                rt.submit(op, dom, opnds + [arrs[o]._arg(B.DFS_PRIV_W)])
            outs[mode] = [x.numpy() for x in arrs]
            srcs[mode] = rt.kernel_source()
    for mode in MODES[1:]:
        for s in range(nst):
            assert np.array_equal(_bits(outs[mode][s]), _bits(outs["persistent"][s])), (mode, s)
    src = srcs["persistent"]
    assert "pk_add(" in src and "pk_mul(" not in src
    for blocked in ("v0_", "v1_", "v2_", "v4_", "v5_", "v6_", "v8_", "v9_", "v10_"):   # tasks kept scalar
        assert f"const float2 {blocked}" not in src, blocked
    assert "const float2 v7_" in src                               # a + d on lane pairs
    # and the values are the stored-dtype oracle's (each operation rounded once)
    m = Machine("stored")
    P = Tiling((tile,), (0,), IDENTITY, ((0,), (n,)))
    for s, x in enumerate((a, b, d)):
        m.add(s, x)
    for s in range(3, nst):
        m.add(s, np.zeros(n, np.float32))
    for op, o, ins in stream:
        m.run(XTask(op, dom, [Arg(i, P, "R") if isinstance(i, int) else Imm(i) for i in ins] + [Arg(o, P, "W")]))
    for s in (3, 4, 5, 6, 7, 8, 9, 10, 11):
        assert np.array_equal(_bits(outs["persistent"][s]), _bits(m.arrays[s])), s


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_erf_sharing_after_a_rewrite_in_the_window(dtype):
    """A value and its negation stop being negations once either store is
    rewritten inside the window: the fused body must then evaluate erf of the
    new value, not reuse the magnitude it computed for the old one.  Stores 0
    and 1 are rewritten between the NEG and the ERF/NCDF tasks that read them;
    fused results equal the unfused tasks bit for bit."""
    n, tile = 4099, 512
    dom = ((n + tile - 1) // tile,)
    x = inputs.uniform(31, -3.0, 3.0, n, dtype)
    z = inputs.uniform(32, -3.0, 3.0, n, dtype)
    stream = [("NEG", 1, [0]), ("ERF", 2, [0]), ("NCDF", 3, [1]),
              ("ADD", 0, [4, 0.25]),                        # store 0 rewritten after its negation
              ("ERF", 5, [0]), ("ERF", 6, [1]), ("NCDF", 7, [0]), ("NCDF", 8, [1]),
              ("NEG", 9, [0]), ("MUL", 1, [4, 1.5]),         # now store 1 (the old negation) rewritten
              ("ERF", 10, [9]), ("ERF", 11, [1]), ("NCDF", 12, [9]), ("NCDF", 13, [1])]
    nst = 14
    outs = {}
    for mode in MODES:
        with gpu_runtime(mode, tile=tile) as rt:
            arrs = [rt.array(x), rt.array(np.zeros(n, dtype)), rt.array(np.zeros(n, dtype)),
                    rt.array(np.zeros(n, dtype)), rt.array(z)] + [rt.array(np.zeros(n, dtype)) for _ in range(5, nst)]
            for op, o, ins in stream:
                opnds = [arrs[i]._arg(B.DFS_PRIV_R) if isinstance(i, int) else i for i in ins]
                rt.submit(op, dom, opnds + [arrs[o]._arg(B.DFS_PRIV_W)])
            outs[mode] = [a.numpy() for a in arrs]
    for mode in MODES[1:]:
        for s in range(nst):
            assert np.array_equal(_bits(outs[mode][s]), _bits(outs["persistent"][s])), (mode, s)
    got = outs["persistent"]
    # ERF is odd bit for bit; the rewritten values are no longer negations
    assert np.array_equal(_bits(got[10]), _bits(-got[5]))
    assert not np.array_equal(np.abs(got[5]), np.abs(got[6]))
    m = Machine("stored")
    P = Tiling((tile,), (0,), IDENTITY, ((0,), (n,)))
    init = {0: x, 4: z}
    for s in range(nst):
        m.add(s, init.get(s, np.zeros(n, dtype)))
    for op, o, ins in stream:
        m.run(XTask(op, dom, [Arg(i, P, "R") if isinstance(i, int) else Imm(i) for i in ins] + [Arg(o, P, "W")]))
    fi = np.finfo(dtype)
    for s in range(nst):
        ok = np.isclose(got[s], m.arrays[s], rtol=(2e-6 if dtype == np.float32 else 1e-14), atol=4 * fi.eps)
        assert ok.all(), s


# ---------------------------------------------------- reductions, SpMV
@pytest.mark.parametrize("n", [1, 5, 255, 256, 257, 10007])
def test_dot_and_sum(n):
    x = inputs.uniform(1, -1, 1, n)
    y = inputs.uniform(2, -1, 1, n)
    with gpu_runtime("persistent", tile=256) as rt:
        X, Y = rt.array(x), rt.array(y)
        d = A.dot(X, Y).item()
        s = A.asum(X).item()
        nr = A.norm(X).item()
    assert abs(d - x @ y) <= 1e-13 * np.abs(x * y).sum() + 1e-300
    assert abs(s - x.sum()) <= 1e-13 * np.abs(x).sum() + 1e-300
    assert abs(nr - np.linalg.norm(x)) <= 1e-14 * np.linalg.norm(x)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_spmv_random_spd(dtype):
    rp, col, val = inputs.random_spd_csr(2000, seed=4)
    x = inputs.uniform(6, -1, 1, 2000, dtype)
    with gpu_runtime("persistent", tile=256) as rt:
        Am = A.CSR(rt, rp, col, val.astype(dtype))
        y = (Am @ rt.array(x)).numpy()
    want = programs.spmv(rp, col, val, x.astype(np.float64))
    tol = 1e-13 if dtype == np.float64 else 1e-5
    assert np.max(np.abs(y - want)) <= tol * np.max(np.abs(want))


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_spmv_long_rows_share_lanes(dtype):
    """Rows of ~90 entries are summed by groups of 4 lanes (spmv_warp): 3000
    rows over 12 tiles of 256 with a ragged tail, against the oracle."""
    rp, col, val = inputs.random_spd_csr(3000, seed=7, kmin=30, kmax=60)
    assert len(col) // 3000 >= 64
    x = inputs.uniform(8, -1, 1, 3000, dtype)
    with gpu_runtime("persistent", tile=256) as rt:
        Am = A.CSR(rt, rp, col, val.astype(dtype))
        y = (Am @ rt.array(x)).numpy()
        assert "spmv_warp" in rt.kernel_source() and "act_, 4);" in rt.kernel_source()
    want = programs.spmv(rp, col, val, x.astype(np.float64))
    tol = 1e-13 if dtype == np.float64 else 1e-5
    assert np.max(np.abs(y - want)) <= tol * np.max(np.abs(want))


def test_cg_long_rows_fused_unfused_batched_agree():
    """CG on long-row matrices: fused, unfused and batched (mixed with Poisson
    problems, whose rows stay one per lane) are bit-identical, and match the
    oracle to 1e-12."""
    iters = 12
    mats = [inputs.random_spd_csr(2500, seed=9, kmin=30, kmax=60), inputs.poisson2d_csr(40),
            inputs.random_spd_csr(1200, seed=10, kmin=30, kmax=60)]
    xs = [inputs.uniform(20 + i, -1, 1, len(m[0]) - 1) for i, m in enumerate(mats)]

    def run(mode, batched):
        with gpu_runtime(mode, tile=256) as rt:
            probs = []
            for (rp, col, val), x in zip(mats, xs):
                Am = A.CSR(rt, rp, col, val)
                probs.append((Am, W.cg_start_inplace(Am @ rt.array(x))))
            rt.flush()
            for _ in range(iters):
                if batched:
                    W.batched_cg_iteration(rt, probs)
                else:
                    for Am, s in probs:
                        W.cg_iteration_inplace(Am, s)
                    rt.flush()
            assert rt.stats()["batch_fallbacks"] == 0
            return [s.x.numpy() for _, s in probs]
    fused, unfused, batched = run("persistent", False), run("unfused", False), run("persistent", True)
    for i, (rp, col, val) in enumerate(mats):
        assert np.array_equal(fused[i].view(np.uint64), unfused[i].view(np.uint64)), i
        assert np.array_equal(fused[i].view(np.uint64), batched[i].view(np.uint64)), i
        xo, _, _ = programs.cg(rp, col, val, programs.spmv(rp, col, val, xs[i]), iters)
        assert np.linalg.norm(fused[i] - xo) / np.linalg.norm(xo) < 1e-12, i


@pytest.mark.parametrize("mode", ["persistent", "unfused"])
def test_spmv_output_as_temporary(mode):
    """y = A x dies inside its window (Def. 4): read straight from registers
    by the fused consumers, never stored."""
    rp, col, val = inputs.random_spd_csr(3000, seed=5)
    x = inputs.uniform(7, -1, 1, 3000)
    with gpu_runtime(mode, tile=512) as rt:
        Am = A.CSR(rt, rp, col, val)
        y = Am @ rt.array(x)
        z = y * 2.0 + 1.0
        r = A.dot(y, y)
        del y
        zg, rg = z.numpy(), float(r.numpy())
    y = programs.spmv(rp, col, val, x)
    assert np.max(np.abs(zg - (y * 2.0 + 1.0))) <= 1e-13 * np.max(np.abs(y))
    assert abs(rg - y @ y) <= 1e-13 * (y @ y)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("rows", [3, 64])
def test_jacobi3d_matches_oracle_bitwise(mode, rows):
    """Slices with offsets in 3-D: a 7-point stencil over shifted views of a
    15^3 grid (blocks of 3 planes: 5 points with a ragged last one; or one
    block), fused rows of (plane, row) pairs and the flat sweep."""
    g = inputs.jacobi3d_grid(13, seed=3)
    with gpu_runtime(mode, rows=rows) as rt:
        grid = rt.array(g)
        views = W.jacobi3d_views(grid)
        for _ in range(4):
            W.jacobi3d_sweep(views)
            rt.flush()
        got = grid.numpy()
    want = programs.jacobi3d(g, 4, np.float32)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


def test_fig6_example_values_and_temporary():
    """Section 5.1's fragment with random x, y: v = (y + 2x)^2 within 1e-15
    relative per element (CUDA's pow and the host's may round differently by
    an ulp), the reduction over w[n/2:] within 1e-13, and z never allocated."""
    n = 10_000
    x, y = inputs.uniform(11, -1, 1, n), inputs.uniform(12, -1, 1, n)
    with gpu_runtime("persistent", tile=1024) as rt:
        X, Y = rt.array(x), rt.array(y)
        rt.flush()
        a0 = rt.stats()["allocations"]
        z = 2.0 * X
        w = Y + z
        v = w ** 2.0
        nrm = A.norm(w[n // 2:])
        del X, Y, z, w
        vg, ng = v.numpy(), float(nrm.numpy())
        allocs = rt.stats()["allocations"] - a0
    from oracle import ops
    wo = ops.binary("ADD", y, ops.binary("MUL", 2.0, x, np.float64), np.float64)
    vo = ops.binary("POW", wo, 2.0, np.float64)
    assert np.max(np.abs(vg - vo) / np.maximum(vo, 1e-300)) <= 1e-15
    want = np.sqrt(np.dot(wo[n // 2:], wo[n // 2:]))
    assert abs(ng - want) <= 1e-13 * want
    assert allocs == 3                           # w, v and the norm's 0-d result; z stays in registers


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_scalar_chains_between_reductions(dtype):
    """Reductions finished after a grid barrier feed chains of scalar tasks
    (divide, square root, multiply, maximum) whose results the next vector
    phase broadcasts: in the fused kernel warp 0 computes them and hands them
    to the CTA through shared memory.  All three execution modes agree bit
    for bit, and every value matches the FP64 definition within 1e-12 (FP64)
    or 1e-5 (FP32) relative to the magnitudes involved."""
    n = 10_007                                   # 10 tiles of 1024 and a ragged tail
    x, y, z = (inputs.uniform(s, 0.5, 2.0, n).astype(dtype) for s in (31, 32, 33))
    res = {}
    for mode in MODES:
        with gpu_runtime(mode, tile=1024) as rt:
            X, Y, Z = rt.array(x), rt.array(y), rt.array(z)
            s1 = A.dot(X, Y)
            s2 = s1 / A.dot(Z, Z)
            s3 = A.sqrt(s2) * s1
            Wv = X * s2 + Y
            s4 = A.dot(Wv, Wv)
            s5 = A.maximum(s4 / s3, s2)
            V = Wv - Z * s5
            res[mode] = [Wv.numpy(), V.numpy()] + [np.asarray(a.numpy()) for a in (s1, s2, s3, s4, s5)]
            if mode == "persistent":
                assert rt.stats()["launches"] == 1
    for mode in MODES[1:]:
        for k, (a, b) in enumerate(zip(res[mode], res["persistent"])):
            assert np.array_equal(_bits(np.atleast_1d(a)), _bits(np.atleast_1d(b))), (mode, k)
    tol = 1e-5 if dtype == np.float32 else 1e-12
    xd, yd, zd = (v.astype(np.float64) for v in (x, y, z))
    s1o = float(np.dot(xd, yd))
    s2o = s1o / float(np.dot(zd, zd))
    s3o = np.sqrt(s2o) * s1o
    Wo = xd * s2o + yd
    s4o = float(np.dot(Wo, Wo))
    s5o = max(s4o / s3o, s2o)
    Vo = Wo - zd * s5o
    Wg, Vg, *sg = res["persistent"]
    for got, want in zip(sg, (s1o, s2o, s3o, s4o, s5o)):
        assert abs(float(got) - want) <= tol * abs(want), (got, want)
    assert np.all(np.abs(Wg - Wo) <= tol * np.abs(Wo))
    assert np.all(np.abs(Vg - Vo) <= tol * (np.abs(Wo) + np.abs(zd * s5o)))


# ------------------------------------------------------- runtime behaviour
def test_temporaries_are_never_allocated():
    n = 1 << 16
    S, K, T = inputs.bs_inputs(n, seed=1)
    _, _, fused = _bs_gpu("persistent", S, K, T, tile=4096)
    _, _, unfused = _bs_gpu("unfused", S, K, T, tile=4096)
    assert fused["allocations"] == 5            # S, K, T, call, put
    assert unfused["allocations"] == 3 + W.BLACK_SCHOLES_TASKS


def test_barrier_timeout_is_reported_and_context_survives():
    rp, col, val, xs = inputs.cg_inputs(m=32, seed=0)
    with gpu_runtime("persistent", tile=256, timeout_s=0.05, debug_skip_arrival=1) as rt:
        Am = A.CSR(rt, rp, col, val)
        b = rt.array(xs)
        st = W.cg_start(b)
        rt.flush()
        W.cg_iteration(Am, st)
        with pytest.raises(B.DfsError) as e:
            rt.sync()
        assert e.value.code == -6
        rt.sync()                                # error consumed; context usable
        # the same time-out surfaces through a completion ticket
        W.cg_iteration(Am, st)
        t = rt.record()
        with pytest.raises(B.DfsError) as e:
            rt.wait(t)
        assert e.value.code == -6
        rt.release_ticket(t)
        rt.sync()
    # a fresh context on the same device computes correctly
    x, *_ = _cg_gpu("persistent", 32, 5, tile=256)
    xo, *_ = _cg_oracle(32, 5)
    assert _rel(x, xo) < 1e-12


def test_chunk_pipeline_equals_one_window():
    """Host arrays priced in chunks over three contexts (ragged last chunk)
    give exactly the single-window results."""
    from paper_2406_18109_gb300 import pipeline as PL
    import torch
    n = 300_001
    S, K, T = inputs.bs_inputs(n, seed=6)
    prm = inputs.bs_params()
    pin = lambda a: torch.from_numpy(a).pin_memory().numpy()
    hS, hK, hT = pin(S), pin(K), pin(T)
    hc, hp = pin(np.zeros(n, np.float32)), pin(np.zeros(n, np.float32))
    rts = PL.pipelined_runtimes(3, 0, tile=4096)
    try:
        pipe = PL.ChunkPipeline(rts, lambda a, b, c: W.black_scholes(a, b, c, prm["r"], prm["sigma"]), 65536,
                                [np.float32] * 3)
        for _ in range(2):
            pipe.run([hS, hK, hT], [hc, hp])
    finally:
        for r in rts:
            r.close()
    with gpu_runtime("persistent", tile=4096) as rt:
        c, p = W.black_scholes(rt.array(S), rt.array(K), rt.array(T), prm["r"], prm["sigma"])
        cw, pw = c.numpy(), p.numpy()
    assert np.array_equal(hc.view(np.uint32), cw.view(np.uint32))
    assert np.array_equal(hp.view(np.uint32), pw.view(np.uint32))


def test_wrap_host_zero_copy_equals_device_window():
    """Black-Scholes reading S, K, T from and writing call, put to mapped
    page-locked host memory gives exactly the device-resident results;
    pageable memory is refused before anything runs."""
    import torch
    n = 200_003
    S, K, T = inputs.bs_inputs(n, seed=8)
    prm = inputs.bs_params()
    pin = lambda a: torch.from_numpy(a).pin_memory().numpy()
    hS, hK, hT = pin(S), pin(K), pin(T)
    hc, hp = pin(np.zeros(n, np.float32)), pin(np.zeros(n, np.float32))
    with gpu_runtime("persistent", tile=4096) as rt:
        wc, wp = rt.wrap_host(hc), rt.wrap_host(hp)
        c, p = W.black_scholes(rt.wrap_host(hS), rt.wrap_host(hK), rt.wrap_host(hT), prm["r"], prm["sigma"])
        wc[...] = c
        wp[...] = p
        del c, p
        rt.flush()
        rt.sync()
        with pytest.raises(B.DfsError) as e:              # pageable memory is refused
            rt.wrap_host(np.zeros(1 << 20, np.float32))
        assert e.value.code == -1
        c2, p2 = W.black_scholes(rt.array(S), rt.array(K), rt.array(T), prm["r"], prm["sigma"])
        cw, pw = c2.numpy(), p2.numpy()
    assert np.array_equal(hc.view(np.uint32), cw.view(np.uint32))
    assert np.array_equal(hp.view(np.uint32), pw.view(np.uint32))
