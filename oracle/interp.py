"""Unfused task-stream interpreter (oracle; test infrastructure only).

Executes a stream of index tasks in program order, exactly as an unfused
runtime would (Section 3.2): every index task runs point by point over its
launch domain, each point task applying its body to the sub-stores its
partitions give it (Fig. 3e), and every store -- temporaries included -- is a
real array.  The result of any fusion must equal this (Theorem 1: the fused
task preserves all dependencies of the sequence it replaces).

Operand conventions of the task bodies:
  * element-wise ops (``oracle.ops``): inputs (store args read, or ``Imm``
    immediates) in order, then the written output;
  * ``DOT``: [x R, y R, out Rd] -- out gets sum over points of sum(x*y);
  * ``SUM``: [x R, out Rd];
  * ``SPMV``: [rowptr R, col R, val R, x R, y W] -- CSR product y = A x over
    the rows of y's sub-store (the Legate Sparse SpMV task of Section 7).
A reduction into a store that holds no value yet starts from the operator's
identity (zero); otherwise it folds into the stored value.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import ops
from .ir import Arg, points, box_empty


@dataclass(frozen=True)
class Imm:
    """An immediate scalar operand."""
    value: float


@dataclass
class XTask:
    name: str
    domain: tuple
    operands: list        # Arg | Imm


def _slice(b):
    lo, hi = b
    return tuple(slice(l, h) for l, h in zip(lo, hi))


class Machine:
    """Holds the stores (root arrays) and runs tasks on them.

    ``mode='stored'`` computes every task in its output store's dtype;
    ``mode='fp64'`` keeps every store in float64.
    """

    def __init__(self, mode: str = "stored"):
        self.mode = mode
        self.arrays = {}
        self.valid = set()

    def add(self, sid: int, array: np.ndarray, valid: bool = True):
        a = np.array(array, copy=True)
        if self.mode == "fp64" and a.dtype.kind == "f":
            a = a.astype(np.float64)
        self.arrays[sid] = a
        if valid:
            self.valid.add(sid)

    def alloc(self, sid: int, shape, dtype):
        dt = np.float64 if (self.mode == "fp64" and np.dtype(dtype).kind == "f") else dtype
        self.arrays[sid] = np.zeros(shape, dtype=dt)

    def _read(self, op, p):
        if isinstance(op, Imm):
            return op.value
        return self.arrays[op.store][_slice(op.part.sub_store(p))]

    def run(self, t: XTask):
        name = t.name
        if name in ops.UNARY or name in ops.BINARY:
            self._elementwise(t)
        elif name == "DOT" or name == "SUM":
            self._reduce(t)
        elif name == "SPMV":
            self._spmv(t)
        else:
            raise ValueError(f"unknown task {name}")

    def run_all(self, tasks):
        for t in tasks:
            self.run(t)

    def _elementwise(self, t: XTask):
        out = t.operands[-1]
        ins = t.operands[:-1]
        dt = self.arrays[out.store].dtype
        for p in points(t.domain):
            ob = out.part.sub_store(p)
            if box_empty(ob) and len(ob[0]) > 0:
                continue
            vals = [self._read(o, p) for o in ins]
            if t.name in ops.UNARY:
                r = ops.unary(t.name, vals[0], dt)
            else:
                r = ops.binary(t.name, vals[0], vals[1], dt)
            self.arrays[out.store][_slice(ob)] = r
        self.valid.add(out.store)

    def _reduce(self, t: XTask):
        out = t.operands[-1]
        ins = t.operands[:-1]
        dt = self.arrays[out.store].dtype
        partials = []
        for p in points(t.domain):
            b = ins[0].part.sub_store(p)
            if box_empty(b) and len(b[0]) > 0:
                partials.append(dt.type(0))
                continue
            x = np.asarray(self._read(ins[0], p), dtype=dt)
            if t.name == "DOT":
                y = np.asarray(self._read(ins[1], p), dtype=dt)
                partials.append(np.sum(x * y, dtype=dt))
            else:
                partials.append(np.sum(x, dtype=dt))
        acc = self.arrays[out.store][()] if out.store in self.valid else dt.type(0)
        acc = np.asarray(acc, dtype=dt)
        for s in partials:
            acc = np.asarray(acc + s, dtype=dt)
        self.arrays[out.store][()] = acc
        self.valid.add(out.store)

    def _spmv(self, t: XTask):
        rp_a, col_a, val_a, x_a, y_a = t.operands
        rowptr = self.arrays[rp_a.store]
        col = self.arrays[col_a.store]
        val = self.arrays[val_a.store]
        x = self.arrays[x_a.store]
        y = self.arrays[y_a.store]
        dt = y.dtype
        for p in points(t.domain):
            lo, hi = y_a.part.sub_store(p)
            for r in range(lo[0], hi[0]):
                a, b = int(rowptr[r]), int(rowptr[r + 1])
                y[r] = np.sum(val[a:b].astype(dt) * x[col[a:b]].astype(dt), dtype=dt)
        self.valid.add(y_a.store)
