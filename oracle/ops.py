"""Element operations of the task bodies (oracle; test infrastructure only).

Each index task of the array libraries applies one operation to every element
of its sub-stores (Section 2, Fig. 1e: ADD, MULT, COPY; Section 6, Fig. 8a:
an element-wise addition body).  These are the plain definitions, evaluated
with numpy in a chosen dtype: float64 for the FP64 oracle, or the stored dtype
(float32) where every operation rounds to float32 after each step, exactly as
an unfused task that writes its result to a float32 store would.

Operation set (names are the task names used throughout the tests):
  unary   COPY NEG ABS EXP LOG SQRT ERF NCDF
  binary  ADD SUB MUL DIV POW MAX MIN
  NCDF(x) = 0.5 * (1 + erf(x * (1/sqrt 2))), the standard normal CDF written
  with erf, evaluated step by step in the working dtype.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special

UNARY = ("COPY", "NEG", "ABS", "EXP", "LOG", "SQRT", "ERF", "NCDF")
BINARY = ("ADD", "SUB", "MUL", "DIV", "POW", "MAX", "MIN")
REDUCTIONS = ("DOT", "SUM")


def as_dtype(x, dt):
    """Round a value or array to the working dtype."""
    return np.asarray(x, dtype=dt)


def unary(op: str, x, dt):
    """out = op(x), every step rounded to dt."""
    x = as_dtype(x, dt)
    if op == "COPY":
        return x.copy()
    if op == "NEG":
        return -x
    if op == "ABS":
        return np.abs(x)
    if op == "EXP":
        return np.exp(x)
    if op == "LOG":
        return np.log(x)
    if op == "SQRT":
        return np.sqrt(x)
    if op == "ERF":
        return as_dtype(special.erf(x), dt)
    if op == "NCDF":
        t = x * as_dtype(math.sqrt(0.5), dt)
        e = as_dtype(special.erf(t), dt)
        u = as_dtype(1.0, dt) + e
        return as_dtype(0.5, dt) * u
    raise ValueError(f"unknown unary op {op}")


def binary(op: str, x, y, dt):
    """out = x op y, rounded to dt."""
    x = as_dtype(x, dt)
    y = as_dtype(y, dt)
    if op == "ADD":
        return x + y
    if op == "SUB":
        return x - y
    if op == "MUL":
        return x * y
    if op == "DIV":
        return x / y
    if op == "POW":
        return np.power(x, y)
    if op == "MAX":
        return np.maximum(x, y)
    if op == "MIN":
        return np.minimum(x, y)
    raise ValueError(f"unknown binary op {op}")


def arity(op: str) -> int:
    if op in UNARY:
        return 1
    if op in BINARY:
        return 2
    raise ValueError(op)
