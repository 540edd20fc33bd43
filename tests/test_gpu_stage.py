"""SpMV with x windows staged in shared memory (the optional window argument
of DFS_OP_SPMV): the rows read the same x values in the same order, so every
result must equal the unstaged run bit for bit, and the oracle as before.
Covered: the persistent CG window (2-D Poisson, one window per point; 3-D
Poisson, three; random SPD, the whole vector or, when too large, nothing),
BiCGSTAB (two SpMVs per iteration), batched CG in FP64 and FP32 over uneven
problems, and window records that are out of bounds or misaligned, which the
kernel must ignore."""
import numpy as np
import pytest

from oracle import programs
from paper_2406_18109_gb300 import arrays as A
from paper_2406_18109_gb300 import workloads as W
from synth import inputs
from tests.helpers import gpu_runtime

pytestmark = pytest.mark.gpu


def _bits(a):
    return np.ascontiguousarray(a).view(np.uint32 if a.dtype == np.float32 else np.uint64)


def _cg(stage, rp, col, val, xs, iters, tile, corrupt=None):
    with gpu_runtime("persistent", tile=tile, stage_x=stage) as rt:
        Am = A.CSR(rt, rp, col, val)
        if corrupt is not None:
            w = Am._win[rt.tile_1d(Am.nrows)]
            w.write(corrupt(w.numpy()))
        s = W.cg_start_inplace(Am @ rt.array(xs))
        rt.flush()
        for _ in range(iters):
            W.cg_iteration_inplace(Am, s)
            rt.flush()
        src = rt.kernel_source()
        return s.x.numpy(), float(s.rho.numpy()), src


MATS = {
    "poisson2d": lambda: (*inputs.poisson2d_csr(61), inputs.uniform(3, -1, 1, 61 * 61)),
    "poisson3d": lambda: (*inputs.poisson3d_csr(17), inputs.uniform(4, -1, 1, 17 ** 3)),
    "spd_small": lambda: (*inputs.random_spd_csr(2000, seed=4), inputs.uniform(5, -1, 1, 2000)),
    "spd_large": lambda: (*inputs.random_spd_csr(12000, seed=5), inputs.uniform(6, -1, 1, 12000)),
}


@pytest.mark.parametrize("name", sorted(MATS))
def test_staged_cg_equals_unstaged_and_oracle(name):
    rp, col, val, xs = MATS[name]()
    iters = 25
    xs_, rho_s, src = _cg(True, rp, col, val, xs, iters, 256)
    xu, rho_u, _ = _cg(False, rp, col, val, xs, iters, 256)
    assert "xstage<double>" in src
    assert np.array_equal(_bits(xs_), _bits(xu)) and rho_s == rho_u
    xo, _, _ = programs.cg(rp, col, val, programs.spmv(rp, col, val, xs), iters)
    assert np.linalg.norm(xs_ - xo) / np.linalg.norm(xo) < 1e-12


def test_windows_cover_what_the_tests_need():
    # the cases above stage what they claim: every point of the banded and
    # small matrices, no point of the large random one
    from paper_2406_18109_gb300 import binding as B
    for name, want in (("poisson2d", "all"), ("poisson3d", "all"), ("spd_small", "all"), ("spd_large", "none")):
        rp, col, _, _ = MATS[name]()
        rec = B.dfs_spmv_windows(rp, col, len(rp) - 1, 256, 8).reshape(-1, 6)
        staged = (rec[:, 1::2].sum(axis=1) > 0)
        assert staged.all() if want == "all" else not staged.any(), name


def test_corrupt_window_records_are_ignored():
    rp, col, val, xs = MATS["poisson2d"]()
    iters = 10
    xu, rho_u, _ = _cg(False, rp, col, val, xs, iters, 256)
    n = len(rp) - 1

    def bad(rec):
        r = rec.reshape(-1, 6).copy()
        r[0::4, 0] = n - 2                 # past the end of x
        r[0::4, 1] = 64
        r[1::4, 0] = 1                     # not 16-byte aligned
        r[2::4, 1] = 3                     # a size that is not a multiple of 16 bytes
        r[3::4, 1] = 1 << 30               # more than the shared memory holds
        return r.reshape(-1)
    xb, rho_b, src = _cg(True, rp, col, val, xs, iters, 256, corrupt=bad)
    assert "xstage<double>" in src
    assert np.array_equal(_bits(xb), _bits(xu)) and rho_b == rho_u


def test_staged_bicgstab_equals_unstaged():
    m, iters = 13, 12
    rp, col, val = inputs.poisson3d_csr(m)
    xs = inputs.uniform(9, -1, 1, m ** 3)
    out = {}
    for stage in (True, False):
        with gpu_runtime("persistent", tile=512, stage_x=stage) as rt:
            Am = A.CSR(rt, rp, col, val)
            s = W.bicgstab_start_inplace(Am @ rt.array(xs))
            for _ in range(iters):
                W.bicgstab_iteration_inplace(Am, s)
                rt.flush()
            out[stage] = s.x.numpy()
    assert np.array_equal(_bits(out[True]), _bits(out[False]))
    b = programs.spmv(rp, col, val, xs)
    xo, _, _ = programs.bicgstab(rp, col, val, b, 0.0, iters)
    assert np.linalg.norm(out[True] - xo) / np.linalg.norm(xo) < 1e-12


SPECS = [("poisson", 33, 0, 1), ("spd", 5000, 7, 2), ("poisson", 71, 0, 3), ("spd", 1500, 8, 4),
         ("poisson", 45, 0, 5), ("poisson", 90, 0, 6)]


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_staged_batched_cg_equals_unstaged(dtype):
    iters = 12
    res = {}
    for stage in (True, False):
        with gpu_runtime("persistent", tile=512, stage_x=stage) as rt:
            probs = []
            for spec in SPECS:
                rp, col, val, xs = inputs.batched_cg_matrix(spec)
                Am = A.CSR(rt, rp, col, val.astype(dtype))
                probs.append((Am, W.cg_start_inplace(Am @ rt.array(xs.astype(dtype)))))
            rt.flush()
            for _ in range(iters):
                W.batched_cg_iteration(rt, probs)
            st = rt.stats()
            assert st["batch_fallbacks"] == 0
            if stage:
                assert "xstage<" in rt.kernel_source()
            res[stage] = [s.x.numpy() for _, s in probs]
    for i, spec in enumerate(SPECS):
        assert np.array_equal(_bits(res[True][i]), _bits(res[False][i])), spec
        rp, col, val, xs = inputs.batched_cg_matrix(spec)
        if dtype == np.float64:
            xo, _, _ = programs.cg(rp, col, val, programs.spmv(rp, col, val, xs), iters)
            assert np.linalg.norm(res[True][i] - xo) / np.linalg.norm(xo) < 1e-12, spec
