"""C-ABI checks that need no GPU: the library loads, exports every declared
symbol, validates submissions, and its fusion pass produces the paper's plans.
Analysis-only contexts (device = -1) also compile every generated kernel with
NVRTC for sm_103a, which checks the code generator without a GPU."""
import re

import numpy as np
import pytest

from paper_2406_18109_gb300 import binding as B
from paper_2406_18109_gb300 import arrays as A
from paper_2406_18109_gb300 import workloads as W
from tests.helpers import HEADER, ensure_built


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dfs_[a-z_]+)\s*\(", text)))


def test_exports_every_declared_symbol():
    names = declared_functions()
    assert set(names) == set(B.EXPORTS)
    lib = B.lib()
    for n in names:
        assert hasattr(lib, n), n
    assert B.dfs_version() >= 100


def test_config_default_matches_header():
    cfg = B.dfs_config_default()
    assert cfg.fusion == 1 and cfg.launch_mode == B.DFS_LAUNCH_PERSISTENT
    assert cfg.block_threads == 256 and cfg.barrier_timeout_s == 2.0
    assert cfg.debug_skip_arrival == 0


def rt0(**kw):
    return A.Runtime(device=-1, **kw)


def expect_invalid(fn):
    with pytest.raises(B.DfsError) as e:
        fn()
    assert e.value.code in (-1, -7)


def test_submission_validation():
    rt = rt0(tile=4)
    a = rt.empty((8,), np.float32)
    b = rt.empty((8,), np.float64)
    s = rt.empty((), np.float32)
    T4 = rt.tiling((4,))
    none = rt.none
    # dtype mismatch
    expect_invalid(lambda: rt.submit("ADD", (2,), [(a.handle, T4, 1), (b.handle, T4, 1), (a.handle, T4, 2)]))
    # write through None with several points interferes
    expect_invalid(lambda: rt.submit("COPY", (2,), [1.0, (a.handle, none, 2)]))
    # 0-d output of a multi-point task
    expect_invalid(lambda: rt.submit("COPY", (2,), [(a.handle, T4, 1), (s.handle, none, 2)]))
    # reduction output must be RD(SUM) 0-d
    expect_invalid(lambda: rt.submit("DOT", (2,), [(a.handle, T4, 1), (a.handle, T4, 1), (s.handle, none, 2)]))
    # reading a store a task reduces to
    expect_invalid(lambda: rt.submit("DOT", (1,), [(s.handle, none, 1), (s.handle, none, 1), (s.handle, none, 4)]))
    # write one view while reading an aliasing one in the same task
    v1, v2 = a[0:4], a[2:6]
    T2 = rt.tiling((2,))
    expect_invalid(lambda: rt.submit("COPY", (2,), [(v1.handle, T2, 1), (v2.handle, T2, 2)]))
    # unknown op / wrong arity
    expect_invalid(lambda: B.dfs_submit(rt.ctx, 999, (1,), [1.0, (a.handle, T4, 2)]))
    expect_invalid(lambda: rt.submit("ADD", (2,), [(a.handle, T4, 1), (a.handle, T4, 2)]))
    # released stores cannot be used
    c = rt.empty((8,), np.float32)
    h = c.handle
    c.release()
    expect_invalid(lambda: rt.submit("COPY", (2,), [1.0, (h, T4, 2)]))
    assert rt.plan()["groups"] == []


def test_operands_must_touch_equal_sub_stores():
    """Element-wise and DOT operands need sub-stores of one shape at every
    point: equal extents, tiles, offsets from the view origin and projections.
    Views of different roots at different origins qualify; a different tile,
    extent or offset does not."""
    rt = rt0(tile=4)
    a = rt.empty((12,), np.float32)
    b = rt.empty((16,), np.float32)
    s = rt.empty((), np.float32)
    T4 = rt.tiling((4,))
    T2 = rt.tiling((2,))
    T4o = rt.tiling((4,), offset=(1,))
    av, bv = a[0:8], b[8:16]                     # 8 elements each, other origins
    rt.submit("ADD", (2,), [(av.handle, T4, 1), (bv.handle, T4, 1), (av.handle, T4, 2)])
    rt.submit("DOT", (2,), [(av.handle, T4, 1), (bv.handle, T4, 1), (s.handle, rt.none, 4)])
    n_ok = rt.stats()["tasks"]
    expect_invalid(lambda: rt.submit("ADD", (2,), [(av.handle, T4, 1), (bv.handle, T2, 1), (av.handle, T4, 2)]))
    expect_invalid(lambda: rt.submit("ADD", (3,), [(a.handle, T4, 1), (b[0:12].handle, T4o, 1), (a.handle, T4, 2)]))
    expect_invalid(lambda: rt.submit("ADD", (2,), [(av.handle, T4, 1), (b[0:12].handle, T4, 1), (av.handle, T4, 2)]))
    expect_invalid(lambda: rt.submit("DOT", (2,), [(av.handle, T4, 1), (bv.handle, T2, 1), (s.handle, rt.none, 4)]))
    assert rt.stats()["tasks"] == n_ok


def test_view_bounds_checked():
    rt = rt0()
    g = rt.empty((4, 4), np.float32)
    with pytest.raises(B.DfsError):
        B.dfs_store_view(rt.ctx, g.handle, [1, 1], [4, 4])


def test_fig1_plan_and_kernel_compiles():
    rt = rt0(rows=2)
    g = rt.empty((6, 6), np.float32)
    views = W.jacobi_views(g)
    W.jacobi_sweep(views)
    p = rt.plan()
    assert p["groups"] == [[0, 1, 2, 3, 4], [5]]
    assert len(p["temporaries"]) == 4
    assert p["barriers"] == 1
    with pytest.raises(B.DfsError) as e:
        rt.flush()
    assert e.value.code == -2      # compiled, not launched: no device here
    assert "grid_barrier" in rt.kernel_source()


def test_black_scholes_plan_fuses_everything():
    rt = rt0(tile=8)
    S, K, T = (rt.empty((30,), np.float32) for _ in range(3))
    call, put = W.black_scholes(S, K, T, 0.02, 0.3)
    p = rt.plan()
    assert p["groups"] == [list(range(W.BLACK_SCHOLES_TASKS))]
    assert len(p["temporaries"]) == W.BLACK_SCHOLES_TASKS - 2
    assert call.handle not in p["temporaries"] and put.handle not in p["temporaries"]
    with pytest.raises(B.DfsError):
        rt.flush()
    src = rt.kernel_source()
    # four N() tasks per element, replicated over vector lanes and loop
    # variants (a packed call, pk_ncdf_of_erf, serves two lanes); N(d) and
    # N(-d) share one erf evaluation
    packed = src.count("pk_ncdf_of_erf(")
    results = src.count("ncdf_of_erf(") - packed + 2 * packed
    assert packed > 0 and results % 4 == 0 and "ld4" in src and "st4" in src
    mags = src.count("erf_mag(") + 2 * src.count("erf_mag2(")      # erf_mag2 serves two lanes
    assert mags * 2 == results
    assert "log_f32x2(" in src                                         # LOG of S/K, two lanes at a time
    # only the two outputs are stored: the 21 temporaries live in registers
    assert src.count("st4(") == src.count("st4(r3") + src.count("st4(r4")


def test_batched_black_scholes_shares_erf_of_negations():
    """The batched generator emits the same erf sharing as the single-window
    one: per lane, N(-d1) and N(-d2) reuse erf(|.|) of N(d1) and N(d2)."""
    rt = rt0(tile=1024)
    arrs = [[rt.empty((n,), np.float32) for _ in range(3)] for n in (3000, 5000)]
    keep = []
    rt.batch_begin()
    for S, K, T in arrs:
        keep.append(W.black_scholes(S, K, T, 0.02, 0.3))
        rt.batch_next()
    with pytest.raises(B.DfsError) as e:
        rt.batch_end()
    assert e.value.code == -2
    assert rt.stats()["batch_fallbacks"] == 0
    src = rt.kernel_source()
    assert "find_inst" in src
    assert src.count("ncdf_of_erf(") > 0 and src.count("erf_mag(") * 2 == src.count("ncdf_of_erf(")


@pytest.mark.parametrize("stream, mags_per_sign", [
    # ERF of x and NCDF of -x take erf of different arguments: nothing shared
    ([("NEG", 1, 0), ("ERF", 2, 0), ("NCDF", 3, 1)], 1.0),
    # N(-x) first, then N(x): the pair shares one erf either way round
    ([("NEG", 1, 0), ("NCDF", 2, 1), ("NCDF", 3, 0)], 0.5),
    # erf(-x) and erf(x) share too
    ([("NEG", 1, 0), ("ERF", 2, 1), ("ERF", 3, 0)], 0.5),
    # -(-x) is x again, but only a direct negation is tracked: no sharing
    ([("NEG", 1, 0), ("NEG", 2, 1), ("NCDF", 3, 0), ("NCDF", 4, 2)], 1.0),
])
def test_erf_sharing_follows_negations_only(stream, mags_per_sign):
    """Where a fused body evaluates erf(|.|) once for two results: exactly for
    a value and its direct negation, and never across ERF and NCDF (whose erf
    arguments differ by the 1/sqrt 2 scaling)."""
    n, tile = 3001, 512
    rt = rt0(tile=tile)
    arrs = [rt.empty((n,), np.float32) for _ in range(5)]
    for op, o, i in stream:
        rt.submit(op, ((n + tile - 1) // tile,), [arrs[i]._arg(B.DFS_PRIV_R), arrs[o]._arg(B.DFS_PRIV_W)])
    with pytest.raises(B.DfsError) as e:
        rt.flush()
    assert e.value.code == -2
    src = rt.kernel_source()
    mags = src.count("erf_mag(") + 2 * src.count("erf_mag2(")      # erf_mag2 serves two lanes
    assert mags == mags_per_sign * src.count("erf_sign(")


def test_black_scholes_unfused_plan():
    rt = rt0(tile=8, fusion=False, launch="per_task")
    S, K, T = (rt.empty((30,), np.float32) for _ in range(3))
    W.black_scholes(S, K, T, 0.02, 0.3)
    p = rt.plan()
    assert len(p["groups"]) == W.BLACK_SCHOLES_TASKS and p["temporaries"] == []
    assert len(p["launches"]) == W.BLACK_SCHOLES_TASKS


def _cg_rt(**kw):
    rt = rt0(tile=8, **kw)
    Am = A.CSR.__new__(A.CSR)
    Am.rt, Am.nrows, Am.ncols, Am.nnz = rt, 16, 16, 40
    Am.rowptr = rt.empty((17,), np.int32)
    Am.col = rt.empty((40,), np.int32)
    Am.val = rt.empty((40,), np.float64)
    Am.dtype = np.dtype(np.float64)
    st = W.CGState(rt.empty((16,)), rt.empty((16,)), rt.empty((16,)), rt.empty(()))
    return rt, Am, st


def test_cg_plan():
    rt, Am, st = _cg_rt()
    W.cg_iteration(Am, st)
    p = rt.plan()
    # [SpMV, dot] | [alpha] | [x+=, r-=, dot] | [beta] | [p=]
    assert p["groups"] == [[0, 1], [2], [3, 4, 5, 6, 7], [8], [9, 10]]
    assert p["scalar_groups"] == [1, 3]
    assert p["launches"] == [[0, 1, 2, 3, 4]] and p["barriers"] == 2
    assert len(p["temporaries"]) == 3          # alpha*p, alpha*q, beta*p
    with pytest.raises(B.DfsError):
        rt.flush()


def test_cg_plan_two_iterations_memo_key():
    rt, Am, st = _cg_rt()
    W.cg_iteration(Am, st)
    k1 = rt.plan()["key"]
    with pytest.raises(B.DfsError):
        rt.flush()
    W.cg_iteration(Am, st)
    k2 = rt.plan()["key"]
    # isomorphic windows over different stores share one canonical key (Section 5.2)
    assert k1 == k2


def test_batched_kernel_compiles_and_checks_isomorphism():
    rt = rt0(tile=512)
    probs = []
    for m in (40, 33, 47):
        Am = A.CSR.__new__(A.CSR)
        Am.rt, Am.nrows, Am.ncols, Am.nnz = rt, m * m, m * m, 5 * m * m - 4 * m
        Am.rowptr = rt.empty((m * m + 1,), np.int32)
        Am.col = rt.empty((Am.nnz,), np.int32)
        Am.val = rt.empty((Am.nnz,), np.float64)
        Am.dtype = np.dtype(np.float64)
        probs.append((Am, W.CGInPlace(*(rt.empty((m * m,)) for _ in range(4)), rt.empty(()))))
    with pytest.raises(B.DfsError) as e:
        W.batched_cg_iteration(rt, probs)
    assert e.value.code == -2 and "batched kernel compiled" in str(e.value)
    src = rt.kernel_source()
    assert "find_inst" in src and src.count("grid_barrier") == 4
    assert rt.stats()["batch_fallbacks"] == 0
    # instances that are not isomorphic are flushed as an ordinary window
    rt.batch_begin()
    a = rt.empty((1000,))
    b = a * 2.0
    rt.batch_next()
    c = A.sqrt(a)
    rt.batch_next()
    with pytest.raises(B.DfsError):
        rt.batch_end()
    assert rt.stats()["batch_fallbacks"] == 1
    with pytest.raises(B.DfsError) as e:
        rt.batch_next()
    assert e.value.code == -7


def test_spmv_output_temporary_compiles():
    """An SpMV whose output dies in the window is eliminated (Def. 4); its row
    index still comes from the output's offset."""
    for batched in (False, True):
        rt = rt0(tile=512)
        keep = []
        if batched:
            rt.batch_begin()
        for n in (1433, 8587):
            Am = A.CSR.__new__(A.CSR)
            Am.rt, Am.nrows, Am.ncols, Am.nnz = rt, n, n, 16 * n
            Am.rowptr = rt.empty((n + 1,), np.int32)
            Am.col = rt.empty((16 * n,), np.int32)
            Am.val = rt.empty((16 * n,), np.float64)
            Am.dtype = np.dtype(np.float64)
            y = Am @ rt.empty((n,))
            keep.append((Am, y * 2.0, A.dot(y, y)))
            del y
            if batched:
                rt.batch_next()
        if not batched:
            p = rt.plan()
            assert len(p["temporaries"]) == 2
        with pytest.raises(B.DfsError) as e:
            rt.batch_end() if batched else rt.flush()
        assert e.value.code == -2
        assert rt.stats()["batch_fallbacks"] == 0
        assert "spmv_row" in rt.kernel_source()


def test_capture_api_needs_a_device_and_checks_state():
    rt = rt0()
    with pytest.raises(B.DfsError) as e:
        rt.capture_begin()
    assert e.value.code == -2
    with pytest.raises(B.DfsError) as e:
        rt.capture_end()
    assert e.value.code == -7
    with pytest.raises(B.DfsError) as e:
        rt.graph_launch(12345)
    assert e.value.code == -7
    # batch repetition and the scalar gather need a device; bad arguments first
    with pytest.raises(B.DfsError) as e:
        rt.batch_repeat(-1)
    assert e.value.code == -1
    with pytest.raises(B.DfsError) as e:
        rt.batch_repeat(1)
    assert e.value.code == -2
    s = rt.empty(())
    with pytest.raises(B.DfsError) as e:
        rt.read_scalars([s])
    assert e.value.code == -2


def test_tickets_and_async_scalar_read_check_their_arguments():
    """Completion tickets and the asynchronous gather: unknown tickets and
    null results are refused, and both need a device."""
    rt = rt0()
    lib, ctx = B.lib(), rt.ctx
    assert lib.dfs_record(ctx, None) == -1
    assert lib.dfs_wait(ctx, 99) == -7
    assert lib.dfs_poll(ctx, 99, None) == -1
    done = B.C.c_int32()
    assert lib.dfs_poll(ctx, 99, B.C.byref(done)) == -7
    ms = B.C.c_float()
    assert lib.dfs_ticket_elapsed_ms(ctx, 1, 2, B.C.byref(ms)) == -7
    assert lib.dfs_ticket_elapsed_ms(ctx, 1, 2, None) == -1
    assert lib.dfs_ticket_release(ctx, 99) == -7
    with pytest.raises(B.DfsError) as e:
        rt.record()
    assert e.value.code == -2
    s = rt.empty(())
    assert lib.dfs_read_scalars_async(ctx, 1, B._i64s([s.handle]), None, None) == -1
    assert lib.dfs_read_scalars_async(ctx, -1, None, None, None) == -1
    # host buffers that are not page-locked are refused before anything else
    work = (B.C.c_int64 * 2)()
    vals = (B.C.c_double * 1)()
    assert lib.dfs_read_scalars_async(ctx, 1, B._i64s([s.handle]), work, vals) == -1


def test_window_size_triggers_analysis():
    rt = rt0(tile=4, window_size=3)
    a = rt.empty((8,), np.float32)
    b = a + 1.0
    c = b * 2.0
    with pytest.raises(B.DfsError):
        d = c - 3.0                              # third task: window full, analysed
    st = rt.stats()
    assert st["flushes"] == 1 and st["tasks"] == 3


def test_window_grows_while_everything_fuses():
    """Section 7.2: the window size doubles whenever a full window fused into
    one task, up to the cap; a window that does not fuse completely keeps it."""
    rt = rt0(tile=4, window_size=2, window_growth=True, window_max=16)
    a = rt.empty((8,), np.float32)
    x = a
    sizes = []
    for _ in range(40):                      # an element-wise chain: every window fuses
        try:
            x = x * 1.5
        except B.DfsError as e:
            assert e.code == -2
        sizes.append(rt.stats()["window_size"])
    assert sizes[-1] == 16 and sorted(set(sizes)) == [2, 4, 8, 16]
    assert rt.stats()["window_growths"] == 3
    # reductions cut the window into several tasks: no growth
    rt = rt0(tile=4, window_size=4, window_growth=True)
    v = rt.empty((8,), np.float32)
    for _ in range(12):
        try:
            s = A.dot(v, v)
            v = v * s
        except B.DfsError:
            pass
    assert rt.stats()["window_size"] == 4 and rt.stats()["window_growths"] == 0
    # growth is off by default
    rt = rt0(tile=4, window_size=2)
    y = rt.empty((8,), np.float32)
    for _ in range(10):
        try:
            y = y + 1.0
        except B.DfsError:
            pass
    assert rt.stats()["window_size"] == 2


def test_3d_stencil_plan_and_kernel_compiles():
    """Slices with offsets in 3-D: the 7-point stencil fuses like Fig. 1's
    (six ADDs and the MULT in one task, COPY after the barrier)."""
    rt = rt0(rows=2)
    g = rt.empty((6, 7, 8), np.float32)
    W.jacobi3d_sweep(W.jacobi3d_views(g))
    p = rt.plan()
    assert p["groups"] == [[0, 1, 2, 3, 4, 5, 6], [7]]
    assert len(p["temporaries"]) == 6 and p["barriers"] == 1
    with pytest.raises(B.DfsError) as e:
        rt.flush()
    assert e.value.code == -2
    assert "% ext1" in rt.kernel_source()        # rows of a 3-D space are (plane, row) pairs


def test_fig6_temporary_example_plan():
    """Section 5.1's example: z = 2x; w = y + z; v = w**2; a reduction over the
    view w[n/2:]; del x, y, z, w.  MULT, ADD, POW fuse; the reduction over the
    view is a separate task; only z is temporary."""
    rt = rt0(tile=4)
    x = A.full(rt, (16,), 0.0)
    y = A.full(rt, (16,), 1.0)
    with pytest.raises(B.DfsError):
        rt.flush()
    z = 2.0 * x
    w = y + z
    v = w ** 2.0
    nrm = A.dot(w[8:], w[8:])
    zh, wh = z.handle, w.handle
    del x, y, z, w
    p = rt.plan()
    assert p["groups"][0] == [0, 1, 2] and [3] in p["groups"]
    assert p["temporaries"] == [zh] and wh not in p["temporaries"]


@pytest.mark.parametrize("per_row,lanes", [(5, 1), (16, 1), (31, 1), (32, 2), (100, 4), (700, 32)])
def test_spmv_lanes_follow_the_mean_row_length(per_row, lanes):
    """Rows of 32 or more entries are shared by a power-of-two group of lanes
    (16 or more entries per lane; one warp-cooperative row product,
    spmv_warp); shorter rows keep one row per lane (spmv_row)."""
    rt = rt0(tile=512)
    n = 3000
    Am = A.CSR.__new__(A.CSR)
    Am.rt, Am.nrows, Am.ncols, Am.nnz = rt, n, n, per_row * n
    Am.rowptr = rt.empty((n + 1,), np.int32)
    Am.col = rt.empty((per_row * n,), np.int32)
    Am.val = rt.empty((per_row * n,), np.float64)
    Am.dtype = np.dtype(np.float64)
    y = Am @ rt.empty((n,))
    _ = A.dot(y, y)
    with pytest.raises(B.DfsError):
        rt.flush()
    src = rt.kernel_source()
    if lanes == 1:
        assert "spmv_row" in src and "spmv_warp" not in src
    else:
        assert f"act_, {lanes});" in src


def _cg_inplace(rt, n=16, nnz=40):
    Am = A.CSR.__new__(A.CSR)
    Am.rt, Am.nrows, Am.ncols, Am.nnz = rt, n, n, nnz
    Am.rowptr = rt.empty((n + 1,), np.int32)
    Am.col = rt.empty((nnz,), np.int32)
    Am.val = rt.empty((nnz,), np.float64)
    Am.dtype = np.dtype(np.float64)
    st = W.CGInPlace(*(rt.empty((n,)) for _ in range(4)), rt.empty(()))
    return Am, st, [Am.rowptr, Am.col, Am.val, st.x, st.r, st.p, st.q, st.rho]


def test_template_replay_issues_the_recorded_window():
    """A recorded in-place CG iteration replayed over another solve's stores
    issues the same tasks as submitting that solve's iteration directly: the
    same canonical window key (Section 5.2), groups and temporaries."""
    rt = rt0(tile=8, window_size=4096)
    A1, s1, in1 = _cg_inplace(rt)
    A2, s2, in2 = _cg_inplace(rt)
    t0 = rt.stats()["tasks"]
    tpl = rt.record_template(W.cg_iteration_inplace, A1, s1)
    ntask = rt.stats()["tasks"] - t0
    assert ntask >= 10 and sorted(tpl.inputs) == sorted(a.handle for a in in1)
    with pytest.raises(B.DfsError):
        rt.flush()                               # no device: the window is analysed and dropped
    W.cg_iteration_inplace(A2, s2)
    direct = rt.plan()
    with pytest.raises(B.DfsError):
        rt.flush()
    t1 = rt.stats()["tasks"]
    tpl.replay(in1, in2)
    assert rt.stats()["tasks"] - t1 == ntask
    rep = rt.plan()
    for k in ("key", "groups", "scalar_groups", "barriers"):
        assert rep[k] == direct[k], k
    assert len(rep["temporaries"]) == len(direct["temporaries"]) >= 2   # alpha*p, alpha*q, ...
    with pytest.raises(B.DfsError):
        rt.flush()
    # every input must be mapped, to a store of the recorded shape
    with pytest.raises(B.DfsError) as e:
        tpl.replay(in1[:-1], in2[:-1])
    assert e.value.code == -1
    other = rt.empty((17,))
    with pytest.raises(B.DfsError) as e:
        tpl.replay(in1, in2[:3] + [other] + in2[4:])
    assert e.value.code == -1
    tpl.free()


def test_failed_replay_releases_the_stores_it_created():
    """A replay that fails part-way (here the window fills on its first task,
    and an analysis-only context cannot launch the flush) leaves no store of
    its own behind: the temporary it had created is released with it."""
    rt = rt0(tile=8, window_size=3)
    a, b = rt.empty((16,)), rt.empty((16,))

    def step(a, b):
        t = a * 2.0
        b += t
    tpl = rt.record_template(step, a, b)
    assert rt.stats()["tasks"] == 2
    with pytest.raises(B.DfsError):
        rt.flush()                                # analysed and dropped: the recorded t is freed
    base = rt.stats()["stores"]
    b += 1.0
    b += 1.0                                      # two tasks in the window, no new store
    with pytest.raises(B.DfsError) as e:
        tpl.replay([a, b], [a, b])                # its MUL is the window's third task
    assert e.value.code == -2
    assert rt.stats()["stores"] == base
    tpl.replay([a, b], [a, b])                    # a fresh window takes the whole replay
    assert rt.stats()["stores"] == base + 1       # t stays alive for the pending tasks
    with pytest.raises(B.DfsError):
        rt.flush()
    assert rt.stats()["stores"] == base


def test_template_recording_refuses_what_a_replay_cannot_repeat():
    rt = rt0(tile=8)
    x = rt.empty((16,))
    B.dfs_template_begin(rt.ctx)
    with pytest.raises(B.DfsError) as e:
        B.dfs_template_begin(rt.ctx)             # no nesting
    assert e.value.code == -7
    with pytest.raises(B.DfsError) as e:
        rt.batch_begin()
    assert e.value.code == -7
    with pytest.raises(B.DfsError) as e:
        B.dfs_store_write(rt.ctx, x.handle, np.zeros(16).ctypes.data, 128)
    assert e.value.code == -7
    with pytest.raises(B.DfsError) as e:
        B.dfs_template_end(rt.ctx)               # the refused call spoils the recording
    assert e.value.code == -7
    # a created store still alive at the end spoils it too
    B.dfs_template_begin(rt.ctx)
    keep = x * 2.0
    with pytest.raises(B.DfsError) as e:
        B.dfs_template_end(rt.ctx)
    assert e.value.code == -7
    del keep
    # releasing a store the recording did not create
    y = rt.empty((16,))
    B.dfs_template_begin(rt.ctx)
    del y
    with pytest.raises(B.DfsError) as e:
        B.dfs_template_end(rt.ctx)
    assert e.value.code == -7
    with pytest.raises(B.DfsError) as e:
        B.dfs_template_end(rt.ctx)               # not recording any more
    assert e.value.code == -7


# ------------------------------------------------- staged SpMV x windows
def _fake_csr(rt, m, tile, dtype=np.float64, windows=True):
    """A CSR of the 2-D Poisson pattern in an analysis-only context (stores
    without data), with a window store for `tile` when asked."""
    Am = A.CSR.__new__(A.CSR)
    Am.rt, Am.nrows, Am.ncols, Am.nnz = rt, m * m, m * m, 5 * m * m - 4 * m
    Am.rowptr = rt.empty((m * m + 1,), np.int32)
    Am.col = rt.empty((Am.nnz,), np.int32)
    Am.val = rt.empty((Am.nnz,), dtype)
    Am.dtype = np.dtype(dtype)
    Am._host = None
    npts = -(-m * m // tile)
    Am._win = {tile: rt.empty((6 * npts,), np.int32)} if windows else {}
    return Am


def test_staged_spmv_kernels_compile():
    rt = rt0(tile=512)
    Am = _fake_csr(rt, 40, 512)
    s = W.CGInPlace(*(rt.empty((1600,)) for _ in range(4)), rt.empty(()))
    W.cg_iteration_inplace(Am, s)
    with pytest.raises(B.DfsError) as e:
        rt.flush()
    assert e.value.code == -2
    src = rt.kernel_source()
    assert "xstage<double>" in src and "spmv_row_xs<double>" in src and "dfs_xs_raw" in src
    # batched: instances of different sizes, each with its own windows
    probs = []
    for m in (40, 33):
        Am = _fake_csr(rt, m, 512, np.float32)
        probs.append((Am, W.CGInPlace(*(rt.empty((m * m,), np.float32) for _ in range(4)),
                                      rt.empty((), np.float32))))
    with pytest.raises(B.DfsError) as e:
        W.batched_cg_iteration(rt, probs)
    assert e.value.code == -2 and "batched kernel compiled" in str(e.value)
    src = rt.kernel_source()
    assert "xstage<float>" in src and "spmv_row_xs<float>" in src and "find_inst" in src


def test_spmv_window_argument_is_validated():
    rt = rt0(tile=256)
    n = 1000
    rp, col = rt.empty((n + 1,), np.int32), rt.empty((5 * n,), np.int32)
    val, x, y = rt.empty((5 * n,)), rt.empty((n,)), rt.empty((n,))
    dom, part = rt.layout((n,))
    none = rt.none

    def submit(win, wpart, priv=B.DFS_PRIV_R):
        args = [(a.handle, none, B.DFS_PRIV_R) for a in (rp, col, val, x)]
        args += [(y.handle, part, B.DFS_PRIV_W), (win.handle, wpart, priv)]
        rt.submit("SPMV", dom, args)

    good = rt.empty((6 * dom[0],), np.int32)
    submit(good, rt.tiling((6,)))                     # accepted
    with pytest.raises(B.DfsError):
        submit(rt.empty((6 * dom[0],), np.int64), rt.tiling((6,)))      # not int32
    with pytest.raises(B.DfsError):
        submit(good, rt.tiling((4,)))                                   # records of 6
    with pytest.raises(B.DfsError):
        submit(rt.empty((6 * dom[0] - 6,), np.int32), rt.tiling((6,)))  # one record short
    with pytest.raises(B.DfsError):
        submit(good, rt.tiling((6,)), B.DFS_PRIV_RW)                    # read only


@pytest.mark.parametrize("kind", ["poisson2d", "poisson3d", "spd"])
@pytest.mark.parametrize("elem", [4, 8])
def test_spmv_windows_cover_the_rows(kind, elem):
    """dfs_spmv_windows against brute force: records are 16-byte aligned,
    inside the aligned part of x, within the budget, at most three disjoint
    intervals, and cover every column the point's rows read below that
    aligned end (or the point is not staged at all)."""
    from synth import inputs
    rp, col, _ = {"poisson2d": lambda: inputs.poisson2d_csr(45), "poisson3d": lambda: inputs.poisson3d_csr(13),
                  "spd": lambda: inputs.random_spd_csr(3000, seed=3)}[kind]()
    n = len(rp) - 1
    q = 16 // elem
    end_al = n // q * q
    for tile, budget in ((256, B.SPMV_STAGE_BYTES), (700, B.SPMV_STAGE_BYTES), (512, 4096)):
        rec = B.dfs_spmv_windows(rp, col, n, tile, elem, budget).reshape(-1, 6)
        assert len(rec) == -(-n // tile)
        staged = 0
        for p, r in enumerate(rec):
            lo, ln = r[0::2], r[1::2]
            if ln.sum() == 0:
                continue
            staged += 1
            assert ln.sum() * elem <= budget
            ivs = sorted((int(a), int(a) + int(b)) for a, b in zip(lo, ln) if b > 0)
            for a, b in ivs:
                assert a % q == 0 and (b - a) % q == 0 and 0 <= a < b <= end_al
            for (a0, b0), (a1, b1) in zip(ivs, ivs[1:]):
                assert b0 <= a1
            cols = np.unique(col[rp[p * tile]:rp[min((p + 1) * tile, n)]])
            inside = np.zeros(len(cols), bool)
            for a, b in ivs:
                inside |= (cols >= a) & (cols < b)
            assert inside[cols < end_al].all(), (p, tile)
        if kind != "spd" and budget == B.SPMV_STAGE_BYTES:
            assert staged == len(rec)                   # banded rows: every point fits
    with pytest.raises(B.DfsError):
        B.dfs_spmv_windows(rp, col, n, 0, elem)        # no tile
    with pytest.raises(B.DfsError):
        B.dfs_spmv_windows(rp, col, n, 256, 2)         # element size


def test_lane_pair_decisions():
    """Which FP32 tasks of a vector body run on lane pairs (generated code, no
    device): adds, NCDF, ERF and LOG pair up; multiplies stay on single lanes;
    a sum that a product (MUL, or NCDF through NEG) reaches stays scalar, and
    so does that NCDF."""
    rt = rt0(tile=1024)
    n = 8195
    a, b, d = (rt.empty((n,), np.float32) for _ in range(3))
    outs = [rt.empty((n,), np.float32) for _ in range(12)]
    dom, _ = rt.layout((n,))
    P = B.DFS_PRIV_R
    stream = [("MUL", [a, b], 0), ("ADD", [outs[0], d], 1),        # v0 product, v1 its sum: scalar
              ("ADD", [a, d], 2),                                  # v2 a sum of loads: pair
              ("NCDF", [a], 3), ("NEG", [outs[3]], 4), ("SUB", [d, outs[4]], 5),   # v3..v5: NCDF reaches a sum
              ("NCDF", [b], 6), ("MUL", [outs[6], b], 7),          # v6 NCDF into a product: pair; v7 MUL: single
              ("ERF", [a], 8), ("LOG", [b], 9), ("ADD", [outs[8], 1.0], 10)]        # v8, v9, v10: pair
    for op, ins, o in stream:
        args = [x._arg(P) if not isinstance(x, float) else x for x in ins]
        rt.submit(op, dom, args + [outs[o]._arg(B.DFS_PRIV_W)])
    with pytest.raises(B.DfsError):
        rt.flush()
    src = rt.kernel_source()
    paired = {k for k in range(11) if f"const float2 v{k}_" in src}
    assert paired == {2, 6, 8, 9, 10}, paired
    assert "pk_mul(" not in src and "log_f32x2(" in src and "erf_mag2(" in src
