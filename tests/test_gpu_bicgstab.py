"""BiCGSTAB (Section 7.1) through the fused runtime against the oracle.

The iteration is the naturally written program of workloads.bicgstab_iteration
(two SpMVs, five dot products, scalar updates, vector updates per iteration).
FP64 results must agree with the FP64 oracle to 1e-12 norm-wise after a fixed
number of iterations (measured on GB300: 1.1e-14), and fused must equal
unfused bit for bit.  The residual norm is the norm of a difference that
cancels, so it is compared to 1e-12 of ||b|| and to 1e-10 of itself
(measured: 4.7e-12 of itself)."""
import numpy as np
import pytest

from oracle import programs
from paper_2406_18109_gb300 import arrays as A
from paper_2406_18109_gb300 import workloads as W
from synth import inputs
from tests.helpers import MODES, gpu_runtime

pytestmark = pytest.mark.gpu


def _gpu(mode, m, iters):
    rp, col, val = inputs.poisson3d_csr(m)
    xs = inputs.uniform(9, -1, 1, m ** 3)
    with gpu_runtime(mode, tile=512) as rt:
        Am = A.CSR(rt, rp, col, val)
        b = Am @ rt.array(xs)
        s = W.bicgstab_start(b)
        rt.flush()
        for _ in range(iters):
            rr = W.bicgstab_iteration(Am, s)
            rt.flush()
        return s.x.numpy(), rr.item(), rt.stats()


@pytest.mark.parametrize("mode", MODES)
def test_bicgstab_matches_oracle(mode):
    m, iters = 13, 15                         # 2197 unknowns: 5 tiles of 512 with a ragged tail
    x, rr, st = _gpu(mode, m, iters)
    rp, col, val = inputs.poisson3d_csr(m)
    xs = inputs.uniform(9, -1, 1, m ** 3)
    b = programs.spmv(rp, col, val, xs)
    xo, it, rel = programs.bicgstab(rp, col, val, b, 0.0, iters)
    assert it == iters
    assert np.linalg.norm(x - xo) / np.linalg.norm(xo) < 1e-12
    assert abs(np.sqrt(rr) / np.linalg.norm(b) - rel) <= min(1e-12, 1e-10 * rel)
    if mode == "persistent":
        # set-up takes at most two launches, then one launch per iteration
        assert st["launches"] <= iters + 2


def test_bicgstab_fused_equals_unfused_bitwise():
    res = {m: _gpu(m, 10, 8) for m in MODES}
    for m in MODES[1:]:
        assert np.array_equal(res[m][0].view(np.uint64), res["persistent"][0].view(np.uint64))


def test_bicgstab_converges_to_manufactured_solution():
    m = 10
    rp, col, val = inputs.poisson3d_csr(m)
    xs = inputs.uniform(9, -1, 1, m ** 3)
    with gpu_runtime("persistent", tile=512) as rt:
        Am = A.CSR(rt, rp, col, val)
        b = Am @ rt.array(xs)
        bn = np.sqrt(A.dot(b, b).item())
        s = W.bicgstab_start(b)
        for it in range(200):
            rr = W.bicgstab_iteration(Am, s)
            if (it + 1) % 10 == 0 and np.sqrt(rr.item()) <= 1e-10 * bn:
                break
        x = s.x.numpy()
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-8


def test_inplace_iteration_matches_oracle():
    """The in-place form (state stores updated in place, used by batching and
    serving) before convergence: 1e-12 norm-wise, as the naturally written one."""
    m, iters = 13, 15
    rp, col, val = inputs.poisson3d_csr(m)
    xs = inputs.uniform(9, -1, 1, m ** 3)
    with gpu_runtime("persistent", tile=512) as rt:
        Am = A.CSR(rt, rp, col, val)
        s = W.bicgstab_start_inplace(Am @ rt.array(xs))
        for _ in range(iters):
            W.bicgstab_iteration_inplace(Am, s)
            rt.flush()
        x, rr = s.x.numpy(), float(s.rr.numpy())
    b = programs.spmv(rp, col, val, xs)
    xo, it, rel = programs.bicgstab(rp, col, val, b, 0.0, iters)
    assert np.linalg.norm(x - xo) / np.linalg.norm(xo) < 1e-12
    assert abs(np.sqrt(rr) / np.linalg.norm(b) - rel) <= min(1e-12, 1e-10 * rel)
