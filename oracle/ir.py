"""The paper's IR and its fusion definitions, written out plainly (oracle).

TEST INFRASTRUCTURE ONLY.  Everything here follows Sections 3-5 of the paper
literally and by brute force; nothing is optimised.

Data model (Section 3.1, Fig. 2a):
  * A store is a rectangular array identified by an id.  Array-library views
    (e.g. ``grid[1:-1, 1:-1]`` in Fig. 1a) are sub-stores of their parent: a
    view is described here by (root id, box) and every analysis works on the
    root store, as Def. 1 compares "sub-stores with the same parent".
  * ``NonePart`` replicates: every point maps to the whole (view) box.
  * ``Tiling(shape, offset, proj)``: the sub-store of point p is
    [proj(p)*shape, proj(p+1)*shape) + offset (Fig. 3e), clipped to the view
    box it was made on.  proj(p+1) is read as proj(p) + 1 per coordinate, which
    holds for the identity and for dimension-dropping projections (Fig. 3d).
Computation model (Section 3.2): IndexTask(launch domain, [(S, P, Pr)]) with
privileges R, W, RW (both R and W) and Rd (a single reduction operator).
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field
from typing import Optional

Box = tuple  # ((lo0, lo1, ...), (hi0, hi1, ...)) half-open


def box_empty(b: Box) -> bool:
    lo, hi = b
    return any(h <= l for l, h in zip(lo, hi))


def box_intersect(a: Box, b: Box) -> Box:
    lo = tuple(max(x, y) for x, y in zip(a[0], b[0]))
    hi = tuple(min(x, y) for x, y in zip(a[1], b[1]))
    return (lo, hi)


def boxes_overlap(a: Box, b: Box) -> bool:
    return not box_empty(box_intersect(a, b))


@dataclass(frozen=True)
class Projection:
    """Projection(id, Point -> Point) (Fig. 2a).  ``keep`` lists the launch-domain
    coordinates that survive; None means the identity."""
    pid: int = 0
    keep: Optional[tuple] = None

    def __call__(self, p):
        return tuple(p) if self.keep is None else tuple(p[i] for i in self.keep)


IDENTITY = Projection(0, None)


@dataclass(frozen=True)
class NonePart:
    """Replication: every point maps to the whole view box (Section 3.1)."""
    view: Box

    def sub_store(self, p) -> Box:
        return self.view


@dataclass(frozen=True)
class Tiling:
    """Affine tiling (Section 3.1; bounds per Fig. 3e).  ``offset`` is in root
    coordinates (the view's origin plus the tiling's own offset); ``view`` is
    the box of the store the tiling was made on."""
    shape: tuple
    offset: tuple
    proj: Projection
    view: Box

    def sub_store(self, p) -> Box:
        q = self.proj(p)
        lo = tuple(qi * s + o for qi, s, o in zip(q, self.shape, self.offset))
        hi = tuple((qi + 1) * s + o for qi, s, o in zip(q, self.shape, self.offset))
        return box_intersect((lo, hi), self.view)


@dataclass(frozen=True)
class Arg:
    store: int          # root store id
    part: object        # NonePart | Tiling
    priv: str           # 'R', 'W', 'RW', 'Rd'


@dataclass
class Task:
    name: str
    domain: tuple
    args: list = field(default_factory=list)


def R(a: Arg) -> bool:
    return a.priv in ("R", "RW")


def W(a: Arg) -> bool:
    return a.priv in ("W", "RW")


def Rd(a: Arg) -> bool:
    return a.priv == "Rd"


def points(domain):
    return itertools.product(*[range(d) for d in domain])


def non_interfering(t: Task) -> bool:
    """The input assumption of the fusion algorithm: an index task's point tasks
    do not race.  No two points write overlapping data or write what another
    point reads, a point never reads or writes data it (or another point)
    reduces to, and one point does not access aliasing but different sub-stores
    with a write among them.  (Overlapping reductions with one operator are
    allowed.)"""
    pts = list(points(t.domain))
    for ia, a in enumerate(t.args):
        for ib, b in enumerate(t.args):
            if a.store != b.store:
                continue
            for p in pts:
                sa = a.part.sub_store(p)
                for q in pts:
                    if p == q and ia == ib:
                        continue
                    if not boxes_overlap(sa, b.part.sub_store(q)):
                        continue
                    if Rd(a) and (R(b) or W(b)):
                        return False
                    if p != q and W(a) and (R(b) or W(b)):
                        return False
                    if p == q and W(a) and a.part != b.part:
                        return False
    return True


# ---------------------------------------------------------------- Section 4.1
def dep(t1: Task, p, t2: Task, p2) -> bool:
    """dep(T1^p, T2^p') of Def. 1: some sub-stores of the same parent overlap and
    the privileges form a true-, anti- or reduction-dependence."""
    for a in t1.args:
        sa = a.part.sub_store(p)
        for b in t2.args:
            if a.store != b.store:
                continue
            if not boxes_overlap(sa, b.part.sub_store(p2)):
                continue
            if W(a) and (R(b) or W(b) or Rd(b)):
                return True          # true-dep
            if R(a) and (W(b) or Rd(b)):
                return True          # anti-dep
            if Rd(a) and (R(b) or W(b)):
                return True          # reduction-dep
    return False


def dependence_map(t1: Task, t2: Task) -> dict:
    """D(T1, T2)[p] = {p' in domain(T2) : dep(T1^p, T2^p')} (Def. 2)."""
    return {p: {p2 for p2 in points(t2.domain) if dep(t1, p, t2, p2)}
            for p in points(t1.domain)}


def fusible_pair(t1: Task, t2: Task) -> bool:
    """Def. 3: for all p, D(T1, T2)[p] is a subset of {p}."""
    return all(s <= {p} for p, s in dependence_map(t1, t2).items())


def fusible_sequence(tasks) -> bool:
    """Every ordered pair of the sequence is fusible (the statement of Theorem 1)."""
    return all(fusible_pair(tasks[i], tasks[j])
               for i in range(len(tasks)) for j in range(i + 1, len(tasks)))


# ------------------------------------------------------------ Section 4.2.1
def launch_domain_equivalence(tasks) -> bool:
    return all(t.domain == tasks[0].domain for t in tasks)


def true_dependence(tasks) -> bool:
    for i, ti in enumerate(tasks):
        for a in ti.args:
            if not W(a):
                continue
            for tj in tasks[i + 1:]:
                for b in tj.args:
                    if b.store == a.store and (R(b) or W(b)) and b.part != a.part:
                        return False
    return True


def anti_dependence(tasks) -> bool:
    for i, ti in enumerate(tasks):
        for a in ti.args:
            if not R(a):
                continue
            for tj in tasks[i + 1:]:
                for b in tj.args:
                    if b.store == a.store and W(b) and b.part != a.part:
                        return False
    return True


def reduction(tasks) -> bool:
    for i, ti in enumerate(tasks):
        for a in ti.args:
            if not Rd(a):
                continue
            for j, tj in enumerate(tasks):
                if j == i:
                    continue
                for b in tj.args:
                    if b.store == a.store and (R(b) or W(b)):
                        return False
    return True


def satisfies_constraints(tasks) -> bool:
    """All four constraints of Fig. 5 hold for the sequence."""
    return (launch_domain_equivalence(tasks) and true_dependence(tasks)
            and anti_dependence(tasks) and reduction(tasks))


# ------------------------------------------------------------ Section 4.2.2
def longest_prefix(window) -> int:
    """Length of the longest prefix of the window meeting every constraint."""
    f = 1
    for k in range(2, len(window) + 1):
        if satisfies_constraints(window[:k]):
            f = k
        else:
            break
    return f


def partition_window(window):
    """Repeatedly cut the longest fusible prefix off the window; returns the
    list of groups as (start, end) index pairs."""
    groups, s = [], 0
    while s < len(window):
        f = longest_prefix(window[s:])
        groups.append((s, s + f))
        s += f
    return groups


def fused_arguments(tasks):
    """Argument list of the fused task (Section 4.2.2): the union of the
    arguments, a (store, partition) both read and written promoted to RW."""
    privs = {}
    order = []
    for t in tasks:
        for a in t.args:
            k = (a.store, a.part)
            if k not in privs:
                privs[k] = set()
                order.append(k)
            privs[k].add(a.priv)
    out = []
    for k in order:
        s = privs[k]
        r = bool(s & {"R", "RW"})
        w = bool(s & {"W", "RW"})
        if r and w:
            p = "RW"
        elif w:
            p = "W"
        elif r:
            p = "R"
        else:
            p = "Rd"
        out.append(Arg(k[0], k[1], p))
    return out


# --------------------------------------------------------------- Section 5.1
def covers(root_box: Box, part, domain) -> bool:
    """covers(S, P): the sub-stores of P over the launch domain contain every
    point of S (checked element by element)."""
    lo, hi = root_box
    covered = set()
    for p in points(domain):
        b = part.sub_store(p)
        if box_empty(b):
            continue
        covered.update(itertools.product(*[range(l, h) for l, h in zip(*b)]))
    return all(c in covered for c in itertools.product(*[range(l, h) for l, h in zip(lo, hi)]))


def is_temporary(window, f: int, store: int, root_box: Box, app_live: bool, start: int = 0) -> bool:
    """Def. 4 for the fusion of window[start:f] within the window.

    (1) every read of S in the fused prefix is preceded inside it by a write
        through the same partition that covers S;
    (2) no task after the prefix reads or reduces to S (the condition is read
        as "k > f and (R or Rd)");
    (3) the application holds no live reference to S.
    """
    if app_live:
        return False
    prefix = window[start:f]
    for j, tj in enumerate(prefix):
        for b in tj.args:
            if b.store != store or not R(b):
                continue
            ok = any(W(a) and a.store == store and a.part == b.part
                     and covers(root_box, a.part, ti.domain)
                     for ti in prefix[:j] for a in ti.args)
            if not ok:
                return False
    for tk in window[f:]:
        for b in tk.args:
            if b.store == store and (R(b) or Rd(b)):
                return False
    return True


# --------------------------------------------------------------- Section 5.2
def canonical(window):
    """Alpha-renamed form of a window: stores numbered by first occurrence,
    partitions and launch domains kept (the De Bruijn-like index form)."""
    ids = {}
    out = []
    for t in window:
        args = []
        for a in t.args:
            if a.store not in ids:
                ids[a.store] = len(ids)
            args.append((ids[a.store], a.part, a.priv))
        out.append((t.name, t.domain, tuple(args)))
    return tuple(out)
