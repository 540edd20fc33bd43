"""The workloads as plain unfused programs (oracle; test infrastructure only).

Each function is the program an array-library user writes, run eagerly in
program order: one whole-array operation per task, every intermediate kept as
its own array.  ``dt`` is the working dtype: float64 for the FP64 oracle, or
the stored dtype (float32) for the stored-dtype oracle, in which case every
step rounds to float32.

  * ``black_scholes`` -- European call and put prices.  The paper evaluates a
    Black-Scholes pricing micro-benchmark (Section 7.1) but prints no formula;
    the formula is the textbook one:
        d1 = (ln(S/K) + (r + sigma^2/2) T) / (sigma sqrt T),  d2 = d1 - sigma sqrt T
        call = S N(d1) - K e^{-rT} N(d2),   put = K e^{-rT} N(-d2) - S N(-d1)
    with N the standard normal CDF written through erf.  It is issued as the
    23-task stream below (one line per task).
  * ``cg`` -- conjugate gradients (Hestenes-Stiefel form, x0 = 0), the sparse
    Krylov solver of Section 7.1, one line per task of a naturally written
    NumPy/SciPy program: q = A p; pq = p.q; alpha = rho/pq; x += alpha p;
    r -= alpha q; rho' = r.r; beta = rho'/rho; p = r + beta p.
  * ``jacobi`` -- the 5-point stencil of Section 2, Fig. 1a: five aliased views
    of one grid summed left to right, scaled by 0.2, copied back into the
    centre view; the boundary is never written.
  * ``bicgstab`` -- BiCGSTAB (van der Vorst form; the paper names the solver in
    Section 7.1 without printing it):
        rho = rhat.r; beta = (rho/rho_prev)(alpha/omega); p = r + beta (p - omega v)
        v = A p; alpha = rho / (rhat.v); s = r - alpha v; t = A s
        omega = (t.s)/(t.t); x += alpha p + omega s; r = s - omega t.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import sparse

from . import ops


def _c(v, dt):
    return np.asarray(v, dtype=dt)


def black_scholes(S, K, T, r: float, sigma: float, dt=np.float64):
    """Call and put prices by the 23-task unfused stream (task number: line)."""
    S = _c(S, dt)
    K = _c(K, dt)
    T = _c(T, dt)
    mu = r + 0.5 * sigma * sigma            # host-side constant (an immediate)
    t1 = ops.binary("DIV", S, K, dt)         # 1  S / K
    t2 = ops.unary("LOG", t1, dt)            # 2  ln(S/K)
    t3 = ops.unary("SQRT", T, dt)            # 3  sqrt T
    v = ops.binary("MUL", sigma, t3, dt)     # 4  sigma sqrt T
    t5 = ops.binary("MUL", mu, T, dt)        # 5  (r + sigma^2/2) T
    t6 = ops.binary("ADD", t2, t5, dt)       # 6
    d1 = ops.binary("DIV", t6, v, dt)        # 7
    d2 = ops.binary("SUB", d1, v, dt)        # 8
    t9 = ops.binary("MUL", -r, T, dt)        # 9  -rT
    disc = ops.unary("EXP", t9, dt)          # 10 e^{-rT}
    kd = ops.binary("MUL", K, disc, dt)      # 11 K e^{-rT}
    n1 = ops.unary("NCDF", d1, dt)           # 12 N(d1)
    n2 = ops.unary("NCDF", d2, dt)           # 13 N(d2)
    c1 = ops.binary("MUL", S, n1, dt)        # 14
    c2 = ops.binary("MUL", kd, n2, dt)       # 15
    call = ops.binary("SUB", c1, c2, dt)     # 16
    m1 = ops.unary("NEG", d1, dt)            # 17
    nm1 = ops.unary("NCDF", m1, dt)          # 18 N(-d1)
    m2 = ops.unary("NEG", d2, dt)            # 19
    nm2 = ops.unary("NCDF", m2, dt)          # 20 N(-d2)
    p1 = ops.binary("MUL", kd, nm2, dt)      # 21
    p2 = ops.binary("MUL", S, nm1, dt)       # 22
    put = ops.binary("SUB", p1, p2, dt)      # 23
    return call, put


BLACK_SCHOLES_TASKS = 23


def csr_matrix(rowptr, col, val, n_cols=None, dt=np.float64):
    n = len(rowptr) - 1
    return sparse.csr_matrix((np.asarray(val, dtype=dt), np.asarray(col), np.asarray(rowptr)),
                             shape=(n, n if n_cols is None else n_cols))


def spmv(rowptr, col, val, x, dt=np.float64):
    """y = A x for a CSR matrix (the library's sparse product serves as the step)."""
    return _c(csr_matrix(rowptr, col, val, len(x), dt) @ _c(x, dt), dt)


def dot(x, y, dt=np.float64):
    return _c(np.dot(_c(x, dt), _c(y, dt)), dt)


def cg(rowptr, col, val, b, iters: int, dt=np.float64, x0=None, history=None):
    """CG for `iters` iterations from x0 (default zero); returns x, r, rho.

    ``history``, when a list, receives x after every iteration.
    """
    b = _c(b, dt)
    x = np.zeros_like(b) if x0 is None else _c(x0, dt).copy()
    r = b - spmv(rowptr, col, val, x, dt) if x0 is not None else b.copy()
    p = r.copy()
    rho = dot(r, r, dt)
    for _ in range(iters):
        q = spmv(rowptr, col, val, p, dt)          # SPMV
        pq = dot(p, q, dt)                          # DOT
        alpha = _c(rho / pq, dt)                    # scalar DIV
        t1 = ops.binary("MUL", alpha, p, dt)        # MUL
        x = ops.binary("ADD", x, t1, dt)            # ADD  (x += alpha p)
        t2 = ops.binary("MUL", alpha, q, dt)        # MUL
        r = ops.binary("SUB", r, t2, dt)            # SUB  (r -= alpha q)
        rho_new = dot(r, r, dt)                     # DOT
        beta = _c(rho_new / rho, dt)                # scalar DIV
        rho = rho_new
        t3 = ops.binary("MUL", beta, p, dt)         # MUL
        p = ops.binary("ADD", r, t3, dt)            # ADD  (p = r + beta p)
        if history is not None:
            history.append(x.copy())
    return x, r, rho


CG_TASKS_PER_ITERATION = 11


def jacobi(grid, sweeps: int, dt=np.float32):
    """Fig. 1a on an (N+2)x(N+2) grid: returns the grid after `sweeps` sweeps."""
    g = _c(grid, dt).copy()
    center = g[1:-1, 1:-1]
    north = g[0:-2, 1:-1]
    east = g[1:-1, 2:]
    west = g[1:-1, 0:-2]
    south = g[2:, 1:-1]
    for _ in range(sweeps):
        t1 = ops.binary("ADD", center, north, dt)
        t2 = ops.binary("ADD", t1, east, dt)
        t3 = ops.binary("ADD", t2, west, dt)
        avg = ops.binary("ADD", t3, south, dt)
        work = ops.binary("MUL", 0.2, avg, dt)
        center[:] = ops.unary("COPY", work, dt)
    return g


JACOBI_TASKS_PER_SWEEP = 6


def jacobi3d(grid, sweeps: int, dt=np.float32):
    """The Fig. 1a pattern carried to a 3-D (N+2)^3 grid (a 7-point average
    over shifted interior slices; not a program of the paper): per sweep
    work = (1/7) * ((((((c + zm) + zp) + ym) + yp) + xm) + xp), summed left to
    right, then COPY(work, center).  The boundary is never written."""
    g = _c(grid, dt).copy()
    c = g[1:-1, 1:-1, 1:-1]
    nb = (g[0:-2, 1:-1, 1:-1], g[2:, 1:-1, 1:-1], g[1:-1, 0:-2, 1:-1], g[1:-1, 2:, 1:-1],
          g[1:-1, 1:-1, 0:-2], g[1:-1, 1:-1, 2:])
    for _ in range(sweeps):
        acc = c
        for v in nb:
            acc = ops.binary("ADD", acc, v, dt)
        work = ops.binary("MUL", 1.0 / 7.0, acc, dt)
        c[:] = ops.unary("COPY", work, dt)
    return g


def bicgstab(rowptr, col, val, b, tol: float, max_iters: int, dt=np.float64):
    """BiCGSTAB from x0 = 0 until ||r|| <= tol ||b||; returns (x, iterations, ||r||/||b||)."""
    b = _c(b, dt)
    x = np.zeros_like(b)
    r = b.copy()
    rhat = r.copy()
    p = np.zeros_like(b)
    v = np.zeros_like(b)
    rho_prev = _c(1.0, dt)
    alpha = _c(1.0, dt)
    omega = _c(1.0, dt)
    bnorm = math.sqrt(float(dot(b, b, dt)))
    it = 0
    rel = math.sqrt(float(dot(r, r, dt))) / bnorm
    while it < max_iters and rel > tol:
        rho = dot(rhat, r, dt)
        beta = _c((rho / rho_prev) * (alpha / omega), dt)
        p = r + beta * (p - omega * v)
        v = spmv(rowptr, col, val, p, dt)
        alpha = _c(rho / dot(rhat, v, dt), dt)
        s = r - alpha * v
        t = spmv(rowptr, col, val, s, dt)
        omega = _c(dot(t, s, dt) / dot(t, t, dt), dt)
        x = x + alpha * p + omega * s
        r = s - omega * t
        rho_prev = rho
        it += 1
        rel = math.sqrt(float(dot(r, r, dt))) / bnorm
    return x, it, rel
