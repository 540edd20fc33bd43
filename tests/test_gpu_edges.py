"""Edge cases of the CUDA path against the oracle: empty inputs, inputs
smaller than one vector of lanes, CSR rows without entries (and a matrix
without any), the smallest Jacobi grids, and degenerate option parameters
(at the money, expiry at zero, very long expiry, deep in and out of the
money).  Tolerances as in test_gpu_parity.py; fused execution equals the
unfused tasks bit for bit."""
import numpy as np
import pytest

from oracle import programs
from paper_2406_18109_gb300 import arrays as A
from paper_2406_18109_gb300 import configs
from paper_2406_18109_gb300 import workloads as W
from synth import inputs
from tests.helpers import MODES, gpu_runtime

pytestmark = pytest.mark.gpu

BS = configs.BLACK_SCHOLES


def _bits(a):
    return np.ascontiguousarray(a).view(np.uint32 if a.dtype == np.float32 else np.uint64)


def _bs(mode, S, K, T):
    with gpu_runtime(mode, tile=4096) as rt:
        c, p = W.black_scholes(rt.array(S), rt.array(K), rt.array(T), BS["r"], BS["sigma"])
        return c.numpy(), p.numpy()


def _bs_close(S, K, T, c, p):
    """Stored-dtype oracle, 4 eps32 (S + K) per option; NaN exactly where the
    oracle has NaN."""
    c32, p32 = programs.black_scholes(S, K, T, BS["r"], BS["sigma"], np.float32)
    tol = 4 * np.finfo(np.float32).eps * (S.astype(np.float64) + K.astype(np.float64))
    for got, want in ((c, c32), (p, p32)):
        nan = np.isnan(want)
        assert np.array_equal(np.isnan(got), nan)
        assert np.all(np.abs(got[~nan].astype(np.float64) - want[~nan]) <= tol[~nan])


def test_empty_inputs():
    z32 = np.zeros(0, np.float32)
    for mode in MODES:
        c, p = _bs(mode, z32, z32, z32)
        assert c.shape == (0,) and p.shape == (0,)
    with gpu_runtime("persistent", tile=256) as rt:
        x = rt.array(np.zeros(0))
        assert A.dot(x, x).item() == 0.0
        assert A.asum(x).item() == 0.0
        y = (x * 2.0 + 1.0).numpy()
        assert y.shape == (0,)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 7])
def test_black_scholes_below_one_vector(n):
    S, K, T = inputs.bs_inputs(n, seed=11 + n)
    outs = {m: _bs(m, S, K, T) for m in MODES}
    for m in MODES[1:]:
        assert np.array_equal(_bits(outs[m][0]), _bits(outs["persistent"][0]))
        assert np.array_equal(_bits(outs[m][1]), _bits(outs["persistent"][1]))
    _bs_close(S, K, T, *outs["persistent"])


def test_black_scholes_degenerate_options():
    # at the money; expiry near zero and at zero (d1, d2 = +-inf: the payoff);
    # a 1000-year expiry; deep in and out of the money; repeated to fill
    # several vectors and a ragged tail
    S0 = np.array([20, 20, 30, 5, 30, 5, 20, 20, 1e-3, 1e4, 20, 7], np.float32)
    K0 = np.array([20, 20, 1, 100, 1, 100, 20, 10, 50, 1, 30, 7], np.float32)
    T0 = np.array([1, 1e-6, 0.25, 0.25, 1e3, 1e3, 0, 0, 1, 1, 0, 1e-30], np.float32)
    S, K, T = (np.tile(a, 9)[:101] for a in (S0, K0, T0))
    outs = {m: _bs(m, S, K, T) for m in MODES}
    for m in MODES[1:]:
        assert np.array_equal(_bits(outs[m][0]), _bits(outs["persistent"][0]))
        assert np.array_equal(_bits(outs[m][1]), _bits(outs["persistent"][1]))
    c, p = outs["persistent"]
    _bs_close(S, K, T, c, p)
    # expiry zero away from the money: the payoff, exactly
    z = (T == 0) & (S != K)
    assert np.array_equal(c[z], np.maximum(S[z] - K[z], 0).astype(np.float32))
    assert np.array_equal(p[z], np.maximum(K[z] - S[z], 0).astype(np.float32))


def _csr_with_empty_rows(n, seed):
    rng = np.random.default_rng(seed)
    lens = np.minimum(rng.integers(0, 6, n), n)
    lens[rng.random(n) < 0.3] = 0
    lens[0] = lens[-1] = 0
    rp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    col = np.concatenate([np.sort(rng.choice(n, k, replace=False)) for k in lens]).astype(np.int32)
    val = rng.uniform(-1, 1, rp[-1])
    return rp, col, val


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_spmv_rows_without_entries(dtype):
    for n, seed in ((1, 1), (3, 2), (517, 3), (4099, 4)):
        rp, col, val = _csr_with_empty_rows(n, seed)
        x = inputs.uniform(seed + 10, -1.0, 1.0, n, dtype)
        with gpu_runtime("persistent", tile=256) as rt:
            y = (A.CSR(rt, rp, col, val.astype(dtype)) @ rt.array(x)).numpy()
        want = programs.spmv(rp, col, val.astype(dtype), x, np.float64)
        bound = programs.csr_matrix(rp, col, np.abs(val), n) @ np.abs(x.astype(np.float64))
        eps = np.finfo(dtype).eps
        assert np.all(np.abs(y - want) <= 8 * eps * bound)
        assert np.all(y[np.diff(rp) == 0] == 0)
    # no entries at all
    n = 1000
    rp = np.zeros(n + 1, np.int32)
    with gpu_runtime("persistent", tile=256) as rt:
        y = (A.CSR(rt, rp, np.zeros(0, np.int32), np.zeros(0, dtype)) @ rt.array(np.ones(n, dtype))).numpy()
    assert y.shape == (n,) and np.all(y == 0)


@pytest.mark.parametrize("N", [1, 2, 3, 5, 9])
def test_jacobi_smallest_grids(N):
    grid = inputs.jacobi_grid(N, seed=20 + N)
    want = programs.jacobi(grid, 4, np.float32)
    for mode in MODES:
        with gpu_runtime(mode, rows=16) as rt:
            g = rt.array(grid)
            views = W.jacobi_views(g)
            for _ in range(4):
                W.jacobi_sweep(views)
                rt.flush()
            out = g.numpy()
        assert np.array_equal(_bits(out), _bits(want)), mode
