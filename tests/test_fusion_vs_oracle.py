"""The C++ fusion pass (through the C-ABI, analysis-only context) against the
oracle's brute-force restatement of Sections 4-5, on random legal windows.

Checked per window: the fused groups equal the oracle's greedy prefixes
(Fig. 5 constraints, Section 4.2.2); every group is fusible by brute-force
dependence maps (Def. 3, Theorem 1); the temporaries equal Def. 4 evaluated
by the oracle (exactly when a group has one iteration space, and as a subset
otherwise, since the runtime keeps a temporary in memory when its accesses
span loop nests that cannot share registers)."""
import random

import numpy as np
import pytest

from oracle import ir
from paper_2406_18109_gb300 import arrays as A
from paper_2406_18109_gb300 import binding as B
from tests.helpers import ensure_built

N = 8


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


class World:
    """Stores of one window, created through the C-ABI and mirrored as IR args."""

    def __init__(self, rt):
        self.rt = rt
        self.full = [rt.empty((N,), np.float64) for _ in range(3)]
        self.view_of = {}
        self.views = []
        for k, (lo, hi) in enumerate(((0, 4), (4, 8), (2, 6))):
            v = self.full[k % 2][lo:hi]
            self.views.append(v)
            self.view_of[v.handle] = (self.full[k % 2].handle, lo, hi)
        self.scal = [rt.empty((), np.float64) for _ in range(2)]
        self.full_h = [a.handle for a in self.full]
        self.scal_h = [a.handle for a in self.scal]
        self.T4 = rt.tiling((4,))
        self.T2 = rt.tiling((2,))

    def root(self, h):
        return self.view_of[h][0] if h in self.view_of else h

    def ir_part(self, h, part):
        if h in self.view_of:
            r, lo, hi = self.view_of[h]
            return ir.Tiling((2,), (lo,), ir.IDENTITY, ((lo,), (hi,)))
        if part == self.rt.none:
            return ir.NonePart(((), ())) if h in self.scal_h else ir.NonePart(((0,), (N,)))
        return ir.Tiling((4,), (0,), ir.IDENTITY, ((0,), (N,)))


PRIV = {1: "R", 2: "W", 3: "RW", 4: "Rd"}


def random_task(rng, w):
    kind = rng.random()
    if kind < 0.15:       # scalar task
        a, b = rng.sample(w.scal, 2) if rng.random() < 0.5 else (rng.choice(w.scal), None)
        out = rng.choice(w.scal)
        ins = [(a.handle, w.rt.none, 1), (b.handle, w.rt.none, 1) if b is not None else 1.5]
        return "ADD", (1,), ins + [(out.handle, w.rt.none, 2)]
    use_views = rng.random() < 0.35
    pool = w.views if use_views else w.full
    part = w.T2 if use_views else w.T4
    if kind < 0.3:        # reduction
        x, y = rng.choice(pool), rng.choice(pool)
        out = rng.choice(w.scal)
        return "DOT", (2,), [(x.handle, part, 1), (y.handle, part, 1), (out.handle, w.rt.none, 4)]
    x = rng.choice(pool)
    out = rng.choice(pool)
    ins = [(x.handle, part, 1)]
    if rng.random() < 0.6:
        if rng.random() < 0.3:
            ins.append((rng.choice(w.scal).handle, w.rt.none, 1))
        else:
            ins.append((rng.choice(pool).handle, part, 1))
        return rng.choice(["ADD", "MUL", "SUB"]), (2,), ins + [(out.handle, part, 2)]
    return rng.choice(["NEG", "EXP", "COPY"]), (2,), ins + [(out.handle, part, 2)]


def to_ir(w, op, dom, args):
    out = []
    for a in args:
        if not isinstance(a, tuple):
            continue
        h, part, pr = a
        out.append(ir.Arg(w.root(h), w.ir_part(h, part), PRIV[pr]))
    return ir.Task(op, dom, out)


def space_key(t):
    a = t.args[-1] if t.name != "DOT" else t.args[0]
    return (t.domain, a.part.shape if isinstance(a.part, ir.Tiling) else None,
            a.part.view[1][0] - a.part.view[0][0] if a.part.view[0] else 0)


@pytest.mark.parametrize("seed", range(6))
def test_random_windows_match_oracle(seed):
    rng = random.Random(seed)
    checked_groups = 0
    for trial in range(60):
        rt = A.Runtime(device=-1)
        w = World(rt)
        tasks = []
        for _ in range(rng.randint(2, 9)):
            op, dom, args = random_task(rng, w)
            try:
                rt.submit(op, dom, args)
            except B.DfsError:
                continue          # the C-ABI rejected an illegal task; the oracle never sees it
            t = to_ir(w, op, dom, args)
            assert ir.non_interfering(t), (op, args)
            tasks.append(t)
        # drop some application references before planning
        live = {h: True for h in w.full_h + w.scal_h}
        for arr in rng.sample(w.full + w.scal, rng.randint(0, 4)):
            live[arr.handle] = False
            arr.release()
        if any(not live[w.root(v.handle)] for v in w.views):
            pass
        for v in w.views:       # views keep their root alive while they live
            root = w.root(v.handle)
            if rng.random() < 0.5:
                v.release()
            else:
                live[root] = True
        plan = rt.plan()
        groups = [(g[0], g[-1] + 1) for g in plan["groups"]]
        assert groups == ir.partition_window(tasks), (trial, plan)
        for s, e in groups:
            assert ir.fusible_sequence(tasks[s:e])
        # temporaries: roots temporary in every group referencing them (Def. 4)
        roots = {a.store for t in tasks for a in t.args}
        shapes = {h: ((0,), (N,)) for h in w.full_h}
        shapes.update({h: ((), ()) for h in w.scal_h})
        want_exact, want_any = set(), set()
        for r in roots:
            refs, temp = 0, 0
            single_space = True
            for s, e in groups:
                if any(a.store == r for t in tasks[s:e] for a in t.args):
                    refs += 1
                    if ir.is_temporary(tasks, e, r, shapes[r], live.get(r, True), start=s):
                        temp += 1
                    if len({space_key(t) for t in tasks[s:e] if any(a.store == r for a in t.args)}) > 1 or \
                            len({space_key(t) for t in tasks[s:e]}) > 1:
                        single_space = False
            if refs and refs == temp:
                want_any.add(r)
                if single_space:
                    want_exact.add(r)
        got = set(plan["temporaries"])
        assert want_exact <= got <= want_any, (trial, got, want_exact, want_any)
        checked_groups += len(groups)
        rt.close()
    assert checked_groups > 50
