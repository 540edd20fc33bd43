"""Pins of the oracle's IR definitions (CPU only): Sections 3-5 of the paper."""
import random

import numpy as np

from oracle import ir
from oracle.interp import Imm, Machine, XTask
from oracle.ir import Arg, IDENTITY, NonePart, Projection, Task, Tiling
from tests.ir_streams import fig1_stream, memo_streams, read_golden, temp_elim_stream

FULL44 = ((0, 0), (4, 4))


# ------------------------------------------------------------- Fig. 3 tilings
def test_tiling_2x2_of_4x4():
    P = Tiling((2, 2), (0, 0), IDENTITY, FULL44)
    assert P.sub_store((0, 0)) == ((0, 0), (2, 2))
    assert P.sub_store((0, 1)) == ((0, 2), (2, 4))
    assert P.sub_store((1, 1)) == ((2, 2), (4, 4))


def test_tiling_rows_1x4():
    P = Tiling((1, 4), (0, 0), IDENTITY, FULL44)
    for i in range(4):
        assert P.sub_store((i, 0)) == ((i, 0), (i + 1, 4))


def test_tiling_with_offset_starts_at_1_1():
    P = Tiling((2, 2), (1, 1), IDENTITY, ((1, 1), (4, 4)))
    assert P.sub_store((0, 0)) == ((1, 1), (3, 3))
    assert P.sub_store((1, 1)) == ((3, 3), (4, 4))   # clipped to the store


def test_aliased_blocking_by_projection():
    # a size-4 vector tiled over a 2x2 domain, the projection drops dimension 1
    P = Tiling((2,), (0,), Projection(1, (0,)), ((0,), (4,)))
    assert P.sub_store((0, 0)) == P.sub_store((0, 1)) == ((0,), (2,))
    assert P.sub_store((1, 0)) == P.sub_store((1, 1)) == ((2,), (4,))


# ------------------------------------------------------ Fig. 4 dependence maps
def _vec_tasks(read_parts, write_part=None, n=8, dom=(4,)):
    wp = write_part or Tiling((2,), (0,), IDENTITY, ((0,), (n,)))
    t1 = Task("W", dom, [Arg(0, wp, "W")])
    t2 = Task("R", dom, [Arg(0, p, "R") for p in read_parts] + [Arg(1, wp, "W")])
    return t1, t2


def test_pointwise_dependence_map():
    P = Tiling((2,), (0,), IDENTITY, ((0,), (8,)))
    t1, t2 = _vec_tasks([P])
    assert ir.dependence_map(t1, t2) == {(p,): {(p,)} for p in range(4)}
    assert ir.fusible_pair(t1, t2)


def test_stencil_dependence_map():
    right = Tiling((2,), (1,), IDENTITY, ((0,), (8,)))
    left = Tiling((2,), (-1,), IDENTITY, ((0,), (8,)))
    t1, t2 = _vec_tasks([left, right])
    D = ir.dependence_map(t1, t2)
    for p in range(4):
        assert D[(p,)] == {(q,) for q in (p - 1, p, p + 1) if 0 <= q < 4}
    assert not ir.fusible_pair(t1, t2)


def test_write_then_read_other_partition_depends_everywhere():
    t1, t2 = _vec_tasks([NonePart(((0,), (8,)))])
    D = ir.dependence_map(t1, t2)
    assert all(D[(p,)] == {(q,) for q in range(4)} for p in range(4))


def test_reductions_to_same_store_do_not_depend():
    P = Tiling((2,), (0,), IDENTITY, ((0,), (8,)))
    s = NonePart(((), ()))
    t1 = Task("DOT", (4,), [Arg(0, P, "R"), Arg(2, s, "Rd")])
    t2 = Task("DOT", (4,), [Arg(1, P, "R"), Arg(2, s, "Rd")])
    assert ir.fusible_pair(t1, t2)
    t3 = Task("USE", (4,), [Arg(2, s, "R"), Arg(1, P, "W")])
    assert not ir.fusible_pair(t1, t3)


# ----------------------------------------------------- Fig. 1 golden example
def test_fig1_stencil_fusion_and_temporaries():
    tasks, ids, boxes, app = fig1_stream()
    rows = read_golden("fig1_stencil_stream.txt")
    want_groups = [tuple(int(x) for x in g.split("-")) for g in
                   next(r for r in rows if r[0] == "groups")[1:]]
    want_temps = set(next(r for r in rows if r[0] == "temporaries")[1:])
    assert ir.partition_window(tasks) == want_groups
    # the COPY is excluded by the anti-dependence constraint (reads of aliasing
    # views of grid, then a write to the centre view)
    assert ir.true_dependence(tasks) and not ir.anti_dependence(tasks)
    assert ir.fusible_sequence(tasks[:5]) and not ir.fusible_sequence(tasks)
    f = want_groups[0][1]
    names = {v: k for k, v in ids.items()}
    temps = {names[s] for s in boxes if ir.is_temporary(tasks, f, s, boxes[s], s in app)}
    assert temps == want_temps


def test_fig1_next_iteration_is_cut_by_true_dependence():
    tasks, *_ = fig1_stream()
    two = tasks + tasks
    assert ir.partition_window(two) == [(0, 5), (5, 6), (6, 11), (11, 12)]
    assert not ir.true_dependence(two[5:7])


# ----------------------------------------------------- Fig. 6 golden example
def test_temp_elimination_example():
    tasks, ids, boxes, app = temp_elim_stream()
    rows = read_golden("temp_elim_example.txt")
    want_groups = [tuple(int(x) for x in g.split("-")) for g in
                   next(r for r in rows if r[0] == "groups")[1:]]
    want_temps = set(next(r for r in rows if r[0] == "temporaries")[1:])
    assert ir.partition_window(tasks) == want_groups
    f = want_groups[0][1]
    names = {v: k for k, v in ids.items()}
    temps = {names[s] for s in boxes
             if any(a.store == s for t in tasks[:f] for a in t.args)
             and ir.is_temporary(tasks, f, s, boxes[s], s in app)}
    assert temps == want_temps


def test_covers():
    P = Tiling((2,), (0,), IDENTITY, ((0,), (8,)))
    assert ir.covers(((0,), (8,)), P, (4,))
    assert not ir.covers(((0,), (8,)), P, (3,))
    half = Tiling((2,), (4,), IDENTITY, ((4,), (8,)))
    assert not ir.covers(((0,), (8,)), half, (2,))


def test_fused_arguments_promote_rw():
    P = Tiling((2,), (0,), IDENTITY, ((0,), (8,)))
    t1 = Task("A", (4,), [Arg(0, P, "R"), Arg(1, P, "W")])
    t2 = Task("B", (4,), [Arg(1, P, "R"), Arg(0, P, "W")])
    args = ir.fused_arguments([t1, t2])
    assert [(a.store, a.priv) for a in args] == [(0, "RW"), (1, "RW")]


# ----------------------------------------------------- Fig. 7 golden example
def test_memo_canonical_forms():
    streams, canon = memo_streams()
    A, B, C = (ir.canonical(streams[k]) for k in "ABC")
    assert A == B and A != C
    for key, form in canon.items():
        got = [(t[0], tuple((s, p) for s, _, p in t[2])) for t in ir.canonical(streams[key])]
        assert got == form


# ----------------------------------------- Theorem 1 on random tiny windows
def _random_window(rng, n=8):
    parts = [
        ((4,), Tiling((2,), (0,), IDENTITY, ((0,), (n,)))),
        ((2,), Tiling((4,), (0,), IDENTITY, ((0,), (n,)))),
        ((4,), Tiling((2,), (1,), IDENTITY, ((1,), (n,)))),
        ((4,), NonePart(((0,), (n,)))),
    ]
    win = []
    for _ in range(rng.randint(2, 6)):
        dom_choice = rng.choice([(4,), (2,)])
        cands = [p for d, p in parts if d == dom_choice or isinstance(p, NonePart)]
        while True:
            args = []
            for s in rng.sample(range(3), rng.randint(1, 3)):
                args.append(Arg(s, rng.choice(cands), rng.choice(["R", "W", "RW", "Rd"])))
            t = Task("T", dom_choice, args)
            if ir.non_interfering(t):
                break
        win.append(t)
    return win


def test_non_interfering():
    P = Tiling((2,), (0,), IDENTITY, ((0,), (8,)))
    whole = NonePart(((0,), (8,)))
    assert ir.non_interfering(Task("T", (4,), [Arg(0, P, "R"), Arg(0, P, "W")]))
    assert not ir.non_interfering(Task("T", (4,), [Arg(0, whole, "W")]))
    assert ir.non_interfering(Task("T", (1,), [Arg(0, whole, "W")]))
    assert not ir.non_interfering(Task("T", (4,), [Arg(0, whole, "R"), Arg(0, P, "W")]))
    assert ir.non_interfering(Task("T", (4,), [Arg(0, P, "R"), Arg(1, whole, "Rd")]))
    assert not ir.non_interfering(Task("T", (4,), [Arg(1, whole, "R"), Arg(1, whole, "Rd")]))


def test_greedy_prefixes_are_fusible_by_brute_force():
    rng = random.Random(1234)
    checked = 0
    for _ in range(400):
        win = _random_window(rng)
        for s, e in ir.partition_window(win):
            assert ir.satisfies_constraints(win[s:e])
            assert ir.fusible_sequence(win[s:e])
            checked += e - s > 1
    assert checked > 50


def test_fused_point_major_execution_equals_unfused():
    # Theorem 1 (2): executing a fusible group point by point (all tasks at point
    # p, then p+1, ...) gives the same stores as task-by-task execution.
    rng = random.Random(7)
    ops1 = ["NEG", "EXP", "SQRT", "ABS"]
    ops2 = ["ADD", "SUB", "MUL", "MAX"]
    n = 8
    tile = Tiling((2,), (0,), IDENTITY, ((0,), (n,)))
    for trial in range(60):
        tasks = []
        for _ in range(rng.randint(2, 6)):
            out = rng.randrange(4)
            if rng.random() < 0.5:
                ins = [Arg(rng.randrange(4), tile, "R")]
                name = rng.choice(ops1)
            else:
                ins = [Arg(rng.randrange(4), tile, "R"),
                       rng.choice([Arg(rng.randrange(4), tile, "R"), Imm(rng.uniform(-2, 2))])]
                name = rng.choice(ops2)
            tasks.append(XTask(name, (4,), ins + [Arg(out, tile, "W")]))
        ir_tasks = [Task(t.name, t.domain, [o for o in t.operands if isinstance(o, Arg)]) for t in tasks]
        assert ir.partition_window(ir_tasks) == [(0, len(tasks))]
        init = {s: np.random.default_rng(trial * 10 + s).uniform(0.5, 2.0, n) for s in range(4)}
        unf = Machine("fp64")
        fus = Machine("fp64")
        for s in range(4):
            unf.add(s, init[s])
            fus.add(s, init[s])
        unf.run_all(tasks)
        for p in range(4):
            for t in tasks:
                fus.run(XTask(t.name, (1,), [o if isinstance(o, Imm) else
                                              Arg(o.store, Tiling((2,), (2 * p,), IDENTITY, ((0,), (n,))), o.priv)
                                              for o in t.operands]))
        for s in range(4):
            np.testing.assert_array_equal(unf.arrays[s], fus.arrays[s])
