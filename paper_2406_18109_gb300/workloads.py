"""The evaluated programs written naturally against the array front end.

Each line is one array operation, hence one index task, as an application of
the array libraries would issue them (Section 7.1): the runtime decides what
fuses.  The task counts are those of the unfused streams.

  * Black-Scholes call/put pricing: 23 tasks per batch.
  * Conjugate gradients: 11 tasks per iteration (SpMV, two dots, two scalar
    divides, three scaled updates written as multiply + add/sub).
  * The Fig. 1a stencil (Jacobi relaxation over five aliased views): 6 tasks
    per sweep.
  * BiCGSTAB: 4 dots, 2 SpMVs, scalar arithmetic and vector updates per
    iteration (plus r.r for the convergence test).

The *_inplace variants keep a solve's whole state in stores created once and
updated in place, so one iteration is a steady window: it can be captured in
a CUDA graph, batched with other solves of other sizes, and re-run with
dfs_batch_repeat.
"""
from __future__ import annotations

from dataclasses import dataclass

from . import arrays as A
from .arrays import Array, CSR, Runtime

BLACK_SCHOLES_TASKS = 23
CG_TASKS_PER_ITERATION = 11
JACOBI_TASKS_PER_SWEEP = 6


def black_scholes(S: Array, K: Array, T: Array, r: float, sigma: float, out=None):
    """European call and put under Black-Scholes, N(x) = 0.5 (1 + erf(x/sqrt 2)).
    out: optional (call, put) stores the last two tasks write into."""
    mu = r + 0.5 * sigma * sigma
    t1 = S / K
    t2 = A.log(t1)
    t3 = A.sqrt(T)
    v = sigma * t3
    t5 = mu * T
    t6 = t2 + t5
    d1 = t6 / v
    d2 = d1 - v
    t9 = (-r) * T
    disc = A.exp(t9)
    kd = K * disc
    n1 = A.ncdf(d1)
    n2 = A.ncdf(d2)
    c1 = S * n1
    c2 = kd * n2
    call = A.subtract(c1, c2, out=out[0] if out else None)
    m1 = -d1
    nm1 = A.ncdf(m1)
    m2 = -d2
    nm2 = A.ncdf(m2)
    p1 = kd * nm2
    p2 = S * nm1
    put = A.subtract(p1, p2, out=out[1] if out else None)
    return call, put


@dataclass
class CGState:
    x: Array
    r: Array
    p: Array
    rho: Array


def cg_start(b: Array) -> CGState:
    """x0 = 0, r0 = b, p0 = r0, rho0 = r0.r0."""
    x = A.full(b.rt, b.shape, 0.0, b.dtype)
    r = A.copy(b)
    p = A.copy(b)
    rho = A.dot(r, r)
    return CGState(x, r, p, rho)


def cg_iteration(Amat: CSR, s: CGState) -> None:
    """One CG iteration as a naturally written NumPy/SciPy program."""
    q = Amat @ s.p
    alpha = s.rho / A.dot(s.p, q)
    s.x += alpha * s.p
    s.r -= alpha * q
    rho_new = A.dot(s.r, s.r)
    beta = rho_new / s.rho
    s.rho = rho_new
    s.p = s.r + beta * s.p


@dataclass
class CGInPlace:
    """CG state held in fixed stores, updated in place (q, x, r, p, rho), so
    that one iteration is a steady-state window sequence that can be captured
    once and replayed (no store is created that outlives the iteration)."""
    x: Array
    r: Array
    p: Array
    q: Array
    rho: Array


def cg_start_inplace(b: Array) -> CGInPlace:
    """cg_start plus q = 0, so that every state store holds a value and the
    first iteration is already a steady window."""
    st = cg_start(b)
    q = A.full(b.rt, b.shape, 0.0, b.dtype)
    return CGInPlace(st.x, st.r, st.p, q, st.rho)


def cg_reset_inplace(s: CGInPlace, b: Array) -> None:
    """x = 0, r = b, p = b, rho = r.r, written into the existing state stores."""
    s.x[...] = 0.0
    s.r[...] = b
    s.p[...] = b
    s.rho[...] = A.dot(s.r, s.r)


def cg_iteration_inplace(Amat: CSR, s: CGInPlace) -> None:
    """One CG iteration writing only into the state stores (12 tasks)."""
    Amat.spmv(s.p, s.q)
    alpha = s.rho / A.dot(s.p, s.q)
    s.x += alpha * s.p
    s.r -= alpha * s.q
    rho_new = A.dot(s.r, s.r)
    beta = rho_new / s.rho
    s.rho[...] = rho_new
    s.p *= beta
    s.p += s.r


def batched_cg_iteration(rt: Runtime, problems) -> None:
    """One CG iteration of every (matrix, in-place state) pair in one batched
    launch: each solve's 12 tasks form one instance of the batch."""
    rt.batch_begin()
    for Amat, s in problems:
        cg_iteration_inplace(Amat, s)
        rt.batch_next()
    rt.batch_end()


def jacobi_views(grid: Array):
    """center, north, east, west, south views of an (N+2)x(N+2) grid (Fig. 1a)."""
    return (grid[1:-1, 1:-1], grid[0:-2, 1:-1], grid[1:-1, 2:], grid[1:-1, 0:-2], grid[2:, 1:-1])


def jacobi_sweep(views) -> None:
    center, north, east, west, south = views
    avg = center + north + east + west + south
    work = 0.2 * avg
    center[:] = work


def jacobi3d_views(grid: Array):
    """center and its six face neighbours of an (N+2)^3 grid, as shifted
    interior views (the Fig. 1a pattern in 3-D)."""
    i, lo, hi = slice(1, -1), slice(0, -2), slice(2, None)
    return (grid[i, i, i], grid[lo, i, i], grid[hi, i, i], grid[i, lo, i], grid[i, hi, i],
            grid[i, i, lo], grid[i, i, hi])


def jacobi3d_sweep(views) -> None:
    """work = (1/7)(c + z- + z+ + y- + y+ + x- + x+), then center[:] = work (8 tasks)."""
    center = views[0]
    acc = center
    for v in views[1:]:
        acc = acc + v
    work = (1.0 / 7.0) * acc
    center[:] = work


@dataclass
class BiCGState:
    x: Array
    r: Array
    rhat: Array
    p: Array
    v: Array
    rho: Array
    alpha: Array
    omega: Array


def bicgstab_start(b: Array) -> BiCGState:
    rt = b.rt
    x = A.full(rt, b.shape, 0.0, b.dtype)
    r = A.copy(b)
    rhat = A.copy(b)
    p = A.full(rt, b.shape, 0.0, b.dtype)
    v = A.full(rt, b.shape, 0.0, b.dtype)
    one = rt.scalar(1.0, b.dtype)
    return BiCGState(x, r, rhat, p, v, one, A.copy(one), A.copy(one))


def bicgstab_iteration(Amat: CSR, s: BiCGState) -> Array:
    """One BiCGSTAB iteration (van der Vorst); returns r.r of the new residual."""
    rho = A.dot(s.rhat, s.r)
    beta = (rho / s.rho) * (s.alpha / s.omega)
    s.p = s.r + beta * (s.p - s.omega * s.v)
    s.v = Amat @ s.p
    s.alpha = rho / A.dot(s.rhat, s.v)
    sv = s.r - s.alpha * s.v
    t = Amat @ sv
    s.omega = A.dot(t, sv) / A.dot(t, t)
    s.x += s.alpha * s.p + s.omega * sv
    s.r = sv - s.omega * t
    s.rho = rho
    return A.dot(s.r, s.r)


@dataclass
class BiCGInPlace:
    """BiCGSTAB state in fixed stores (vectors x, r, rhat, p, v, s, t; scalars
    rho, alpha, omega and rr = r.r after the last iteration)."""
    x: Array
    r: Array
    rhat: Array
    p: Array
    v: Array
    s: Array
    t: Array
    rho: Array
    alpha: Array
    omega: Array
    rr: Array


def bicgstab_start_inplace(b: Array) -> BiCGInPlace:
    """x0 = 0, r0 = rhat = b, p0 = v0 = 0, rho = alpha = omega = 1, rr = b.b."""
    rt = b.rt
    st = BiCGInPlace(A.full(rt, b.shape, 0.0, b.dtype), A.copy(b), A.copy(b), A.full(rt, b.shape, 0.0, b.dtype),
                     A.full(rt, b.shape, 0.0, b.dtype), A.full(rt, b.shape, 0.0, b.dtype),
                     A.full(rt, b.shape, 0.0, b.dtype), A.full(rt, (), 1.0, b.dtype), A.full(rt, (), 1.0, b.dtype),
                     A.full(rt, (), 1.0, b.dtype), None)
    st.rr = A.dot(st.r, st.r)
    return st


def bicgstab_iteration_inplace(Amat: CSR, st: BiCGInPlace) -> None:
    """One BiCGSTAB iteration (van der Vorst) written into the state stores, in
    the oracle's operation order; leaves r.r in st.rr."""
    rho = A.dot(st.rhat, st.r)
    beta = (rho / st.rho) * (st.alpha / st.omega)
    st.p[...] = st.r + beta * (st.p - st.omega * st.v)
    Amat.spmv(st.p, st.v)
    st.alpha[...] = rho / A.dot(st.rhat, st.v)
    st.s[...] = st.r - st.alpha * st.v
    Amat.spmv(st.s, st.t)
    st.omega[...] = A.dot(st.t, st.s) / A.dot(st.t, st.t)
    st.x += st.alpha * st.p
    st.x += st.omega * st.s
    st.r[...] = st.s - st.omega * st.t
    st.rr[...] = A.dot(st.r, st.r)
    st.rho[...] = rho
