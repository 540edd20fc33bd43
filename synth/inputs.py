"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module draws random numbers and builds matrix *structure*; it holds none
of the method's arithmetic (no task, no fusion, no solver step).  Both the CPU
oracle and the CUDA path take their inputs from here, so neither has to import
the other.

Workloads (shapes and value distributions of the paper's evaluation, Section 7):
  * Black-Scholes option batches: spot U[5,30], strike U[1,100], expiry
    U[0.25,10] years, drawn in that order from numpy's PCG64 with the seed given.
  * CG on the 2-D 5-point Poisson matrix (Dirichlet, natural row-major order,
    diagonal 4, off-diagonals -1, columns ascending, int32 CSR indices) with a
    manufactured solution x* ~ U[-1,1].
  * Jacobi relaxation on an (N+2)x(N+2) grid whose interior is U[0,1] and whose
    boundary is 1.0 (the aliased-view stencil of Section 2, Fig. 1).
  * BiCGSTAB on the 3-D 7-point Poisson matrix (diagonal 6, off-diagonals -1).
  * Random diagonally dominant SPD CSR matrices for batched solves.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "bs_inputs", "bs_params", "poisson2d_csr", "poisson3d_csr", "cg_inputs",
    "jacobi_grid", "random_spd_csr", "uniform",
]


def uniform(seed: int, lo: float, hi: float, n: int, dtype=np.float64) -> np.ndarray:
    """n draws of U[lo, hi) from numpy's default PCG64 generator."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, n).astype(dtype)


def bs_params() -> dict:
    """Market parameters of the Black-Scholes workload: r = 0.02, sigma = 0.3."""
    return {"r": 0.02, "sigma": 0.3}


def bs_inputs(n: int, seed: int = 1, dtype=np.float32):
    """Spot, strike and expiry arrays of an n-option batch (drawn S, K, T in order)."""
    rng = np.random.default_rng(seed)
    S = rng.uniform(5.0, 30.0, n).astype(dtype)
    K = rng.uniform(1.0, 100.0, n).astype(dtype)
    T = rng.uniform(0.25, 10.0, n).astype(dtype)
    return S, K, T


def poisson2d_csr(m: int):
    """CSR arrays (rowptr, col, val) of the m*m-unknown 2-D 5-point Laplacian.

    Row i = r*m + c couples to (r-1,c), (r,c-1), (r,c), (r,c+1), (r+1,c) when those
    lie inside the grid; columns within a row ascend.  nnz = 5 m^2 - 4 m.
    """
    n = m * m
    idx = np.arange(n, dtype=np.int64)
    r, c = idx // m, idx % m
    cols = []
    vals = []
    # neighbour offsets in ascending column order
    for dr, dc, v in ((-1, 0, -1.0), (0, -1, -1.0), (0, 0, 4.0), (0, 1, -1.0), (1, 0, -1.0)):
        ok = (r + dr >= 0) & (r + dr < m) & (c + dc >= 0) & (c + dc < m)
        cols.append(np.where(ok, idx + dr * m + dc, -1))
        vals.append(np.where(ok, v, 0.0))
    C = np.stack(cols, axis=1)
    V = np.stack(vals, axis=1)
    mask = C >= 0
    counts = mask.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return rowptr.astype(np.int32), C[mask].astype(np.int32), V[mask].astype(np.float64)


def poisson3d_csr(m: int):
    """CSR arrays of the m^3-unknown 3-D 7-point Laplacian (diag 6, off -1)."""
    n = m * m * m
    idx = np.arange(n, dtype=np.int64)
    z, y, x = idx // (m * m), (idx // m) % m, idx % m
    cols, vals = [], []
    for dz, dy, dx, v in ((-1, 0, 0, -1.0), (0, -1, 0, -1.0), (0, 0, -1, -1.0), (0, 0, 0, 6.0),
                          (0, 0, 1, -1.0), (0, 1, 0, -1.0), (1, 0, 0, -1.0)):
        ok = ((z + dz >= 0) & (z + dz < m) & (y + dy >= 0) & (y + dy < m)
              & (x + dx >= 0) & (x + dx < m))
        cols.append(np.where(ok, idx + dz * m * m + dy * m + dx, -1))
        vals.append(np.where(ok, v, 0.0))
    C = np.stack(cols, axis=1)
    V = np.stack(vals, axis=1)
    mask = C >= 0
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(mask.sum(axis=1), out=rowptr[1:])
    return rowptr.astype(np.int32), C[mask].astype(np.int32), V[mask].astype(np.float64)


def batched_cg_problems(count: int = 256, seed: int = 4, mmin: int = 32, mmax: int = 1024,
                        spd_min: int = 1024, spd_max: int = 65536):
    """Specifications of a batch of uneven CG problems.

    Each problem is, with probability 1/2, the 2-D 5-point Poisson matrix of an
    m x m grid with m log-uniform in [mmin, mmax], else a random diagonally
    dominant SPD matrix of n rows, n log-uniform in [spd_min, spd_max].
    Returns (kind, size, matrix seed, solution seed) tuples; the matrices are
    built by batched_cg_matrix.
    """
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        if rng.random() < 0.5:
            m = int(round(np.exp(rng.uniform(np.log(mmin), np.log(mmax)))))
            out.append(("poisson", m, 0, 1000 + i))
        else:
            nn = int(round(np.exp(rng.uniform(np.log(spd_min), np.log(spd_max)))))
            out.append(("spd", nn, 10_000 + i, 1000 + i))
    return out


def batched_cg_matrix(spec):
    """(rowptr, col, val, x*) of one problem of batched_cg_problems."""
    kind, size, mseed, xseed = spec
    if kind == "poisson":
        rp, col, val = poisson2d_csr(size)
    else:
        rp, col, val = random_spd_csr(size, mseed)
    return rp, col, val, uniform(xseed, -1.0, 1.0, len(rp) - 1)


def cg_inputs(m: int = 256, seed: int = 0):
    """Poisson matrix of an m x m grid and the manufactured solution x* ~ U[-1,1]."""
    rowptr, col, val = poisson2d_csr(m)
    xstar = uniform(seed, -1.0, 1.0, m * m)
    return rowptr, col, val, xstar


def jacobi_grid(N: int, seed: int = 2, dtype=np.float32) -> np.ndarray:
    """(N+2)x(N+2) grid: interior U[0,1] (row-major draw order), boundary 1.0."""
    rng = np.random.default_rng(seed)
    g = np.ones((N + 2, N + 2), dtype=dtype)
    g[1:-1, 1:-1] = rng.uniform(0.0, 1.0, (N, N)).astype(dtype)
    return g


def random_spd_csr(n: int, seed: int, kmin: int = 2, kmax: int = 13):
    """Random symmetric, strictly diagonally dominant CSR matrix (hence SPD).

    Each row draws k in [kmin, kmax] off-diagonal column positions (uniform
    over the other n-1 columns, repeats merged) with values U[-1, 0); the
    pattern is symmetrised as B + B^T and the diagonal set to the row's
    absolute off-diagonal sum plus one.  Rows hold about 5-27 entries.
    Returned with ascending columns.
    """
    rng = np.random.default_rng(seed)
    k = np.minimum(rng.integers(kmin, kmax + 1, n), max(0, n - 1))
    R = np.repeat(np.arange(n, dtype=np.int64), k)
    off = rng.integers(0, max(1, n - 1), R.size)
    Cc = (R + 1 + off) % n
    Vv = rng.uniform(-1.0, 0.0, R.size)
    # symmetrise: entries (i,j) and (j,i) summed
    R2 = np.concatenate([R, Cc])
    C2 = np.concatenate([Cc, R])
    V2 = np.concatenate([Vv, Vv])
    key = R2 * n + C2
    order = np.argsort(key, kind="stable")
    key, V2 = key[order], V2[order]
    ukey, start = np.unique(key, return_index=True)
    Vs = np.add.reduceat(V2, start) if len(V2) else V2
    Ru, Cu = ukey // n, ukey % n
    offsum = np.zeros(n)
    np.add.at(offsum, Ru, np.abs(Vs))
    Rall = np.concatenate([Ru, np.arange(n)])
    Call = np.concatenate([Cu, np.arange(n)])
    Vall = np.concatenate([Vs, offsum + 1.0])
    key = Rall * n + Call
    order = np.argsort(key, kind="stable")
    Rall, Call, Vall = Rall[order], Call[order], Vall[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, Rall + 1, 1)
    rowptr = np.cumsum(rowptr)
    return rowptr.astype(np.int32), Call.astype(np.int32), Vall.astype(np.float64)


# 3-D grid sides of the served Poisson operators: log-spaced from 64 to 256
# (64 * 2^(k/4), k = 0..8), so that drawing a side uniformly from the ladder is
# a log-uniform draw of m in [64, 256]
SERVE_LADDER = tuple(int(round(64 * 2 ** (k / 4))) for k in range(9))


def serving_requests(count: int, seed: int = 3, mean_gap_s: float = 2e-3, ladder=SERVE_LADDER,
                     bs_log2=(16, 24)):
    """A Poisson-arrival request stream (exponential gaps of mean mean_gap_s).

    Each request is, with probability 1/3 each, a CG solve or a BiCGSTAB solve
    on the 3-D 7-point Poisson matrix of an m^3 grid (m drawn uniformly from
    `ladder`), or a Black-Scholes batch of n = 2^u options, u uniform in
    bs_log2.  Returns dicts {rid, arrival, kind, size, seed} in arrival order;
    the request's data come from serving_payload.
    """
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(mean_gap_s, count)
    kinds = rng.integers(0, 3, count)
    rungs = rng.integers(0, len(ladder), count)
    u = rng.uniform(bs_log2[0], bs_log2[1], count)
    t = np.cumsum(gaps) - gaps[0]
    out = []
    for i in range(count):
        kind = ("cg", "bicgstab", "bs")[int(kinds[i])]
        size = int(ladder[int(rungs[i])]) if kind != "bs" else int(round(2.0 ** u[i]))
        out.append({"rid": i, "arrival": float(t[i]), "kind": kind, "size": size, "seed": 100_000 + seed * 10_000 + i})
    return out


def serving_payload(req: dict):
    """Host data of one request: x* ~ U[-1,1] over the m^3 unknowns of a
    solve (its right-hand side is b = A x*), or (S, K, T) of an option batch."""
    if req["kind"] == "bs":
        return bs_inputs(req["size"], seed=req["seed"])
    return uniform(req["seed"], -1.0, 1.0, req["size"] ** 3)


def jacobi3d_grid(N: int, seed: int = 2, dtype=np.float32) -> np.ndarray:
    """(N+2)^3 grid: interior U[0,1] from `seed`, boundary 1.0."""
    g = np.ones((N + 2, N + 2, N + 2), dtype=np.float64)
    g[1:-1, 1:-1, 1:-1] = np.random.default_rng(seed).uniform(0.0, 1.0, (N, N, N))
    return g.astype(dtype)
