"""Pins of the unfused interpreter (CPU only)."""
import numpy as np

from oracle import programs
from oracle.interp import Imm, Machine, XTask
from oracle.ir import Arg, IDENTITY, NonePart, Tiling
from synth import inputs


def _vec(n, tile):
    return Tiling((tile,), (0,), IDENTITY, ((0,), (n,)))


def test_interp_reductions_match_numpy():
    n, tile = 37, 8
    dom = ((n + tile - 1) // tile,)
    P = _vec(n, tile)
    s = NonePart(((), ()))
    m = Machine("fp64")
    x = inputs.uniform(1, -1, 1, n)
    y = inputs.uniform(2, -1, 1, n)
    m.add(0, x)
    m.add(1, y)
    m.alloc(2, (), np.float64)
    m.alloc(3, (), np.float64)
    m.run(XTask("DOT", dom, [Arg(0, P, "R"), Arg(1, P, "R"), Arg(2, s, "Rd")]))
    m.run(XTask("SUM", dom, [Arg(0, P, "R"), Arg(3, s, "Rd")]))
    assert abs(m.arrays[2][()] - x @ y) < 1e-14
    assert abs(m.arrays[3][()] - x.sum()) < 1e-14
    # a second reduction folds into the stored value
    m.run(XTask("SUM", dom, [Arg(0, P, "R"), Arg(3, s, "Rd")]))
    assert abs(m.arrays[3][()] - 2 * x.sum()) < 1e-14


def test_interp_spmv_matches_dense():
    rp, col, val = inputs.random_spd_csr(21, seed=3)
    x = inputs.uniform(4, -1, 1, 21)
    m = Machine("fp64")
    for i, a in enumerate((rp, col, val, x)):
        m.add(i, a)
    m.alloc(4, (21,), np.float64)
    whole = lambda k: NonePart(((0,), (k,)))
    m.run(XTask("SPMV", (3,), [Arg(0, whole(22), "R"), Arg(1, whole(len(col)), "R"),
                               Arg(2, whole(len(col)), "R"), Arg(3, whole(21), "R"),
                               Arg(4, _vec(21, 8), "W")]))
    np.testing.assert_allclose(m.arrays[4], programs.spmv(rp, col, val, x), atol=1e-14)


def test_interp_black_scholes_stream_equals_program():
    n, tile = 300, 64
    dom = ((n + tile - 1) // tile,)
    P = _vec(n, tile)
    S, K, T = inputs.bs_inputs(n, seed=5)
    prm = inputs.bs_params()
    r, sig = prm["r"], prm["sigma"]
    mu = r + 0.5 * sig * sig
    m = Machine("stored")
    ids = {}

    def st(name):
        if name not in ids:
            ids[name] = len(ids)
            m.alloc(ids[name], (n,), np.float32)
        return Arg(ids[name], P, "R")

    for name, arr in (("S", S), ("K", K), ("T", T)):
        ids[name] = len(ids)
        m.add(ids[name], arr)
    stream = [
        ("DIV", "t1", "S", "K"), ("LOG", "t2", "t1"), ("SQRT", "t3", "T"), ("MUL", "v", sig, "t3"),
        ("MUL", "t5", mu, "T"), ("ADD", "t6", "t2", "t5"), ("DIV", "d1", "t6", "v"),
        ("SUB", "d2", "d1", "v"), ("MUL", "t9", -r, "T"), ("EXP", "disc", "t9"),
        ("MUL", "kd", "K", "disc"), ("NCDF", "n1", "d1"), ("NCDF", "n2", "d2"),
        ("MUL", "c1", "S", "n1"), ("MUL", "c2", "kd", "n2"), ("SUB", "call", "c1", "c2"),
        ("NEG", "m1", "d1"), ("NCDF", "nm1", "m1"), ("NEG", "m2", "d2"), ("NCDF", "nm2", "m2"),
        ("MUL", "p1", "kd", "nm2"), ("MUL", "p2", "S", "nm1"), ("SUB", "put", "p1", "p2"),
    ]
    assert len(stream) == programs.BLACK_SCHOLES_TASKS
    for op, out, *ins in stream:
        operands = [Imm(i) if isinstance(i, float) else st(i) for i in ins]
        o = st(out)
        m.run(XTask(op, dom, operands + [Arg(o.store, P, "W")]))
    call, put = programs.black_scholes(S, K, T, r, sig, np.float32)
    np.testing.assert_array_equal(m.arrays[ids["call"]], call)
    np.testing.assert_array_equal(m.arrays[ids["put"]], put)
