"""Captured windows replayed as CUDA graphs (memoised windows + graphs).

An in-place CG iteration is captured once and replayed; the result must match
the oracle's CG (and, bit for bit, the same iterations issued normally)."""
import numpy as np
import pytest

from oracle import programs
from paper_2406_18109_gb300 import arrays as A
from paper_2406_18109_gb300 import binding as B
from paper_2406_18109_gb300 import workloads as W
from synth import inputs
from tests.helpers import MODES, gpu_runtime

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _cg_inplace(mode, m, iters, graph: bool):
    rp, col, val, xs = inputs.cg_inputs(m=m, seed=0)
    with gpu_runtime(mode, tile=256) as rt:
        Am = A.CSR(rt, rp, col, val)
        b = Am @ rt.array(xs)
        s = W.cg_start_inplace(b)
        W.cg_iteration_inplace(Am, s)          # first iteration issued normally (compiles, sizes scratch)
        rt.flush()
        if graph:
            rt.capture_begin()
            W.cg_iteration_inplace(Am, s)
            g = rt.capture_end()
            for _ in range(iters - 1):
                rt.graph_launch(g)
        else:
            for _ in range(iters - 1):
                W.cg_iteration_inplace(Am, s)
                rt.flush()
        x, rho = s.x.numpy(), s.rho.item()
        if graph:
            rt.graph_destroy(g)
        return x, rho


@pytest.mark.parametrize("mode", MODES)
def test_replayed_cg_iteration_matches_oracle(mode):
    m, iters = 61, 30
    x, rho = _cg_inplace(mode, m, iters, graph=True)
    rp, col, val, xs = inputs.cg_inputs(m=m, seed=0)
    bo = programs.spmv(rp, col, val, xs)
    xo, _, rhoo = programs.cg(rp, col, val, bo, iters)
    assert _rel(x, xo) < 1e-12
    assert abs(rho - rhoo) <= 1e-12 * abs(rhoo)
    xi, rhoi = _cg_inplace(mode, m, iters, graph=False)
    assert np.array_equal(x.view(np.uint64), xi.view(np.uint64)) and rho == rhoi


def test_whole_solve_captured_and_replayed_twice():
    rp, col, val, xs = inputs.cg_inputs(m=40, seed=0)
    with gpu_runtime("persistent", tile=256) as rt:
        Am = A.CSR(rt, rp, col, val)
        b = Am @ rt.array(xs)
        s = W.cg_start_inplace(b)
        W.cg_iteration_inplace(Am, s)
        rt.flush()
        rt.capture_begin()
        W.cg_reset_inplace(s, b)
        for _ in range(12):
            W.cg_iteration_inplace(Am, s)
        g = rt.capture_end()
        rt.graph_launch(g)
        x1 = s.x.numpy()
        rt.graph_launch(g)                       # the reset makes each replay a full solve
        x2 = s.x.numpy()
        rt.graph_destroy(g)
    bo = programs.spmv(rp, col, val, xs)
    xo, _, _ = programs.cg(rp, col, val, bo, 12)
    assert _rel(x1, xo) < 1e-12 and np.array_equal(x1, x2)


def test_capture_rejects_a_store_that_escapes():
    with gpu_runtime("persistent", tile=256) as rt:
        a = rt.array(np.ones(1000))
        rt.capture_begin()
        b = a * 2.0                              # created inside the capture and kept
        with pytest.raises(B.DfsError) as e:
            rt.capture_end()
        assert e.value.code == -7
        del b
        c = a * 3.0                              # the context still works afterwards
        assert np.allclose(c.numpy(), 3.0)
