"""Pins of the oracle's workload programs (CPU only).

Every check here is fixed by something other than the oracle: textbook values,
closed forms, invariants of the mathematics, or brute force on tiny inputs.
"""
import math
import os

import numpy as np
import pytest

from oracle import ops, programs
from synth import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ---------------------------------------------------------------- Black-Scholes
def test_ncdf_table_values():
    for row in _golden("black_scholes_textbook.txt"):
        if row[0] != "ncdf":
            continue
        x, want = float(row[1]), float(row[2])
        got = float(ops.unary("NCDF", x, np.float64))
        assert abs(got - want) < 1e-9, (x, got, want)


def test_black_scholes_textbook_example():
    rows = [r for r in _golden("black_scholes_textbook.txt") if r[0] == "option"]
    assert rows
    for _, S, K, r, sig, T, c, p, dec in rows:
        call, put = programs.black_scholes(np.array([float(S)]), np.array([float(K)]),
                                           np.array([float(T)]), float(r), float(sig), np.float64)
        assert round(float(call[0]), int(dec)) == float(c)
        assert round(float(put[0]), int(dec)) == float(p)
        call32, put32 = programs.black_scholes(np.array([float(S)]), np.array([float(K)]),
                                               np.array([float(T)]), float(r), float(sig), np.float32)
        assert call32.dtype == np.float32
        assert round(float(call32[0]), int(dec)) == float(c)
        assert round(float(put32[0]), int(dec)) == float(p)


@pytest.mark.parametrize("dt,tol", [(np.float64, 1e-12), (np.float32, 1e-5)])
def test_black_scholes_put_call_parity(dt, tol):
    S, K, T = inputs.bs_inputs(4096, seed=11, dtype=np.float64)
    prm = inputs.bs_params()
    call, put = programs.black_scholes(S, K, T, prm["r"], prm["sigma"], dt)
    S64, K64, T64 = (np.asarray(a, dtype=dt).astype(np.float64) for a in (S, K, T))
    lhs = call.astype(np.float64) - put.astype(np.float64)
    rhs = S64 - K64 * np.exp(-prm["r"] * T64)
    assert np.all(np.abs(lhs - rhs) <= tol * (S64 + K64))


def test_black_scholes_zero_volatility_limit():
    # As sigma -> 0 the call tends to max(S - K e^{-rT}, 0) and the put to max(K e^{-rT} - S, 0).
    S = np.array([10.0, 10.0, 50.0, 20.0])
    K = np.array([5.0, 20.0, 49.0, 21.0])
    T = np.array([1.0, 2.0, 0.5, 3.0])
    r = 0.05
    call, put = programs.black_scholes(S, K, T, r, 1e-6, np.float64)
    fwd = S - K * np.exp(-r * T)
    assert np.allclose(call, np.maximum(fwd, 0.0), atol=1e-9)
    assert np.allclose(put, np.maximum(-fwd, 0.0), atol=1e-9)


def test_black_scholes_monotone_in_spot_and_strike():
    S = np.linspace(5, 30, 200)
    K = np.full_like(S, 17.0)
    T = np.full_like(S, 1.5)
    call, put = programs.black_scholes(S, K, T, 0.02, 0.3, np.float64)
    assert np.all(np.diff(call) > 0) and np.all(np.diff(put) < 0)
    call_k, put_k = programs.black_scholes(np.full_like(S, 17.0), S, T, 0.02, 0.3, np.float64)
    assert np.all(np.diff(call_k) < 0) and np.all(np.diff(put_k) > 0)
    # price bounds: max(S - K e^{-rT}, 0) <= call <= S
    assert np.all(call <= S) and np.all(call >= np.maximum(S - 17.0 * np.exp(-0.03), 0) - 1e-12)


def test_black_scholes_stored_dtype_close_to_fp64():
    S, K, T = inputs.bs_inputs(1 << 14, seed=1)
    prm = inputs.bs_params()
    c32, p32 = programs.black_scholes(S, K, T, prm["r"], prm["sigma"], np.float32)
    c64, p64 = programs.black_scholes(S, K, T, prm["r"], prm["sigma"], np.float64)
    scale = S.astype(np.float64) + K.astype(np.float64)
    assert np.all(np.abs(c32 - c64) <= 1e-5 * scale)
    assert np.all(np.abs(p32 - p64) <= 1e-5 * scale)


# ------------------------------------------------------------------------- SpMV
def test_spmv_matches_dense_product():
    for seed in range(3):
        rp, col, val = inputs.random_spd_csr(30, seed=seed)
        dense = np.zeros((30, 30))
        for i in range(30):
            for k in range(rp[i], rp[i + 1]):
                dense[i, col[k]] += val[k]
        x = inputs.uniform(seed + 7, -1, 1, 30)
        assert np.allclose(programs.spmv(rp, col, val, x), dense @ x, rtol=0, atol=1e-13)
        # the generator's matrix is symmetric positive definite
        assert np.allclose(dense, dense.T)
        assert np.all(np.linalg.eigvalsh(dense) > 0)


def test_poisson_structure():
    m = 7
    rp, col, val = inputs.poisson2d_csr(m)
    assert len(col) == 5 * m * m - 4 * m
    dense = np.zeros((m * m, m * m))
    for i in range(m * m):
        for k in range(rp[i], rp[i + 1]):
            dense[i, col[k]] = val[k]
        assert np.all(np.diff(col[rp[i]:rp[i + 1]]) > 0)
    # Kronecker-sum form of the 5-point Laplacian
    T1 = 2 * np.eye(m) - np.eye(m, k=1) - np.eye(m, k=-1)
    assert np.array_equal(dense, np.kron(np.eye(m), T1) + np.kron(T1, np.eye(m)))
    rp3, col3, val3 = inputs.poisson3d_csr(4)
    assert len(col3) == 7 * 64 - 6 * 16


# --------------------------------------------------------------------------- CG
def _dense_to_csr(A):
    rp, col, val = [0], [], []
    for i in range(A.shape[0]):
        nz = np.nonzero(A[i])[0]
        col.extend(nz.tolist())
        val.extend(A[i, nz].tolist())
        rp.append(len(col))
    return np.array(rp, np.int32), np.array(col, np.int32), np.array(val)


def test_cg_exact_termination_in_n_steps():
    rng = np.random.default_rng(5)
    for n in (2, 5, 8):
        M = rng.standard_normal((n, n))
        A = M @ M.T + n * np.eye(n)
        b = rng.standard_normal(n)
        rp, col, val = _dense_to_csr(A)
        x, r, _ = programs.cg(rp, col, val, b, n)
        assert np.linalg.norm(b - A @ x) / np.linalg.norm(b) < 1e-10
        assert np.allclose(x, np.linalg.solve(A, b), rtol=1e-9, atol=1e-12)


def test_cg_k_distinct_eigenvalues_k_steps():
    # CG on a matrix with k distinct eigenvalues terminates in k steps.
    d = np.array([1.0, 1.0, 3.0, 3.0, 3.0, 7.0, 7.0, 1.0])
    A = np.diag(d)
    b = np.arange(1.0, 9.0)
    rp, col, val = _dense_to_csr(A)
    x2, _, _ = programs.cg(rp, col, val, b, 2)
    x3, _, _ = programs.cg(rp, col, val, b, 3)
    assert np.linalg.norm(b - A @ x2) / np.linalg.norm(b) > 1e-3
    assert np.linalg.norm(b - A @ x3) / np.linalg.norm(b) < 1e-13


def test_cg_first_step_is_steepest_descent():
    rp, col, val, xs = inputs.cg_inputs(m=12, seed=3)
    b = programs.spmv(rp, col, val, xs)
    x1, _, _ = programs.cg(rp, col, val, b, 1)
    Ab = programs.spmv(rp, col, val, b)
    assert np.allclose(x1, (b @ b) / (b @ Ab) * b, rtol=1e-14, atol=0)


def test_cg_recovers_manufactured_solution():
    rp, col, val, xs = inputs.cg_inputs(m=16, seed=0)
    b = programs.spmv(rp, col, val, xs)
    x, _, _ = programs.cg(rp, col, val, b, 200)
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-10


def test_cg_a_norm_error_decreases():
    rp, col, val, xs = inputs.cg_inputs(m=32, seed=0)
    b = programs.spmv(rp, col, val, xs)
    hist = []
    programs.cg(rp, col, val, b, 50, history=hist)
    errs = []
    for x in hist:
        e = x - xs
        errs.append(e @ programs.spmv(rp, col, val, e))
    assert np.all(np.diff(errs) < 0)


def test_cg_stored_dtype_runs_in_float32():
    rp, col, val, xs = inputs.cg_inputs(m=16, seed=0)
    b = programs.spmv(rp, col, val, xs)
    x32, _, _ = programs.cg(rp, col, val, b, 30, dt=np.float32)
    x64, _, _ = programs.cg(rp, col, val, b, 30, dt=np.float64)
    assert x32.dtype == np.float32
    assert np.linalg.norm(x32 - x64) / np.linalg.norm(x64) < 1e-4


# ----------------------------------------------------------------------- Jacobi
def test_jacobi_two_by_two_interior_closed_form():
    # Boundary 1, interior 0: by symmetry every interior cell has the same value v_k,
    # two boundary neighbours and two interior neighbours, so v_{k+1} = 0.2 (3 v_k + 2).
    g = np.ones((4, 4))
    g[1:-1, 1:-1] = 0.0
    v = 0.0
    for k in range(1, 6):
        v = 0.2 * (3 * v + 2)
        out = programs.jacobi(g, k, np.float64)
        assert np.allclose(out[1:-1, 1:-1], v, rtol=0, atol=1e-15)
        assert np.all(out[0] == 1) and np.all(out[-1] == 1)
    assert abs(programs.jacobi(g, 1, np.float64)[1, 1] - 0.4) < 1e-15
    assert abs(programs.jacobi(g, 2, np.float64)[1, 1] - 0.64) < 1e-15


def test_jacobi_single_sweep_spreads_a_delta():
    # One sweep of a unit delta gives 0.2 on the cell and its four neighbours:
    # each view offset is exercised (a wrong offset moves the pattern).
    g = np.zeros((7, 9))
    g[3, 5] = 1.0
    out = programs.jacobi(g, 1, np.float64)
    want = np.zeros((7, 9))
    for (i, j) in ((3, 5), (2, 5), (4, 5), (3, 4), (3, 6)):
        want[i, j] = 0.2
    assert np.allclose(out, want, atol=1e-16)
    # asymmetric check: a delta on the boundary only affects its interior neighbour
    g = np.zeros((5, 6))
    g[0, 2] = 1.0
    out = programs.jacobi(g, 1, np.float64)
    want = np.zeros((5, 6))
    want[0, 2] = 1.0
    want[1, 2] = 0.2
    assert np.allclose(out, want, atol=1e-16)


def test_jacobi_fixed_points_and_max_principle():
    # affine grids are fixed points of the 5-point average that includes the centre
    i, j = np.meshgrid(np.arange(10.0), np.arange(12.0), indexing="ij")
    g = 0.5 * i - 0.25 * j + 3.0
    assert np.allclose(programs.jacobi(g, 3, np.float64), g, atol=1e-13)
    g = inputs.jacobi_grid(30, seed=2, dtype=np.float32)
    out = programs.jacobi(g, 20, np.float32)
    assert out.dtype == np.float32
    assert out.min() >= g.min() and out.max() <= 1.0
    assert np.array_equal(out[0], g[0]) and np.array_equal(out[:, -1], g[:, -1])


def test_jacobi_is_jacobi_not_gauss_seidel():
    # every sweep reads the old grid only: compare with an explicit double-buffered sweep
    g = inputs.jacobi_grid(6, seed=4, dtype=np.float64)
    new = g.copy()
    for a in range(1, 7):
        for b in range(1, 7):
            new[a, b] = 0.2 * ((((g[a, b] + g[a - 1, b]) + g[a, b + 1]) + g[a, b - 1]) + g[a + 1, b])
    assert np.array_equal(programs.jacobi(g, 1, np.float64), new)


def test_jacobi3d_matches_explicit_loops_and_delta():
    # an explicit double-buffered triple loop in the stated summation order
    g = np.random.default_rng(5).uniform(0, 1, (5, 6, 7)).astype(np.float32)
    new = g.copy()
    sev = np.float32(1.0 / 7.0)
    for a in range(1, 4):
        for b in range(1, 5):
            for c in range(1, 6):
                acc = g[a, b, c]
                for v in (g[a - 1, b, c], g[a + 1, b, c], g[a, b - 1, c], g[a, b + 1, c], g[a, b, c - 1],
                          g[a, b, c + 1]):
                    acc = np.float32(acc + v)
                new[a, b, c] = np.float32(sev * acc)
    assert np.array_equal(programs.jacobi3d(g, 1, np.float32), new)
    # a unit delta spreads 1/7 onto itself and its six face neighbours only
    d = np.zeros((5, 5, 5))
    d[2, 2, 2] = 1.0
    out = programs.jacobi3d(d, 1, np.float64)
    want = np.zeros((5, 5, 5))
    for (a, b, c) in ((2, 2, 2), (1, 2, 2), (3, 2, 2), (2, 1, 2), (2, 3, 2), (2, 2, 1), (2, 2, 3)):
        want[a, b, c] = 1.0 / 7.0
    assert np.allclose(out, want, atol=1e-16)


def test_jacobi3d_affine_fixed_point_and_max_principle():
    i, j, k = np.meshgrid(np.arange(6.0), np.arange(7.0), np.arange(8.0), indexing="ij")
    g = 0.5 * i - 0.25 * j + 0.125 * k + 2.0
    assert np.allclose(programs.jacobi3d(g, 3, np.float64), g, atol=1e-13)
    g = np.ones((8, 8, 8), np.float32)
    g[1:-1, 1:-1, 1:-1] = np.random.default_rng(6).uniform(0, 1, (6, 6, 6))
    out = programs.jacobi3d(g, 10, np.float32)
    assert out[1:-1, 1:-1, 1:-1].min() >= g[1:-1, 1:-1, 1:-1].min() and out.max() <= 1.0


# --------------------------------------------------------------------- BiCGSTAB
def test_bicgstab_manufactured_solution():
    rp, col, val = inputs.poisson3d_csr(8)
    xs = inputs.uniform(9, -1, 1, 512)
    b = programs.spmv(rp, col, val, xs)
    x, it, rel = programs.bicgstab(rp, col, val, b, 1e-10, 500)
    assert rel <= 1e-10 and it < 500
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-8


def test_bicgstab_nonsymmetric_dense():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((12, 12)) + 12 * np.eye(12)
    rp, col, val = _dense_to_csr(A)
    b = rng.standard_normal(12)
    x, it, rel = programs.bicgstab(rp, col, val, b, 1e-12, 100)
    assert np.allclose(x, np.linalg.solve(A, b), atol=1e-10)
