"""Row-block CG and Jacobi with the runtime's kernels as each rank's local
windows, on one GPU.

One rank runs through dist.rowblock_cg / rowblock_jacobi with nothing to
exchange.  Several ranks are emulated in one process, one runtime context per
rank: the test runs every rank's window of a phase in turn and then performs
the exchanges itself (the halo all-to-all as copies between the ranks'
wrapped buffers, the all-reduce as a sum in rank order), so no kernel ever
waits for another rank.  The concatenated CG solution must match the
single-process oracle CG to 1e-12, and the Jacobi grid bit for bit.
"""
import numpy as np
import pytest

from oracle import programs
from paper_2406_18109_gb300 import dist as D
from synth import inputs
from tests.helpers import gpu_runtime

pytestmark = pytest.mark.gpu


def _cg_problem(name):
    if name == "poisson":
        return inputs.cg_inputs(m=45, seed=0)
    rp, col, val = inputs.random_spd_csr(4000, seed=6)
    return rp, col, val, inputs.uniform(8, -1, 1, 4000)


def _emulated_cg(steps, iters):
    """rowblock_cg's sequence over all ranks at once, with the exchanges done
    here between the ranks' buffers."""
    def allreduce(attr):
        tot = sum(getattr(s, attr).item() for s in steps)   # rank order
        for s in steps:
            getattr(s, attr).fill_(tot)

    def halo():
        offs = {}
        for r, s in enumerate(steps):
            offs[r] = (np.concatenate([[0], np.cumsum(s.block.send_counts)]),
                       np.concatenate([[0], np.cumsum(s.block.recv_counts)]))
        for r, s in enumerate(steps):
            for q, t in enumerate(steps):
                if r != q and s.block.send_counts[q]:
                    so, ro = offs[r][0], offs[q][1]
                    t.halo[ro[r]:ro[r + 1]].copy_(s.send[so[q]:so[q + 1]])
    for s in steps:
        s.start()
    allreduce("rr")
    for s in steps:
        s.set_rho()
    for _ in range(iters):
        for s in steps:
            s.pack_halo()
        for s in steps:
            s.rt.sync()
        halo()
        for s in steps:
            s.spmv_dot()
        allreduce("pq")
        for s in steps:
            s.update_xr()
        allreduce("rr")
        for s in steps:
            s.update_p()


@pytest.mark.parametrize("name", ["poisson", "spd"])
@pytest.mark.parametrize("P", [1, 2, 3])
def test_rowblock_cg_matches_oracle(name, P):
    torch = pytest.importorskip("torch")
    iters = 30
    rp, col, val, xs = _cg_problem(name)
    b = programs.spmv(rp, col, val, xs)
    xo, _, _ = programs.cg(rp, col, val, b, iters)
    rts, steps = [], []
    st = torch.cuda.Stream()
    try:
        torch.cuda.set_stream(st)              # torch copies and every context share one stream
        for r in range(P):
            rt = gpu_runtime("persistent", tile=256, stream=st.cuda_stream).__enter__()
            rts.append(rt)
            blk = D.RowBlock(rp, col, val, P, r)
            steps.append(D.RuntimeCG(rt, blk, b[blk.lo:blk.hi], torch))
        if P == 1:
            D.rowblock_cg(steps[0], D.SelfComm(), iters)
        else:
            _emulated_cg(steps, iters)
        x = np.concatenate([s.solution() for s in steps])
    finally:
        for rt in rts:
            rt.close()
        torch.cuda.set_stream(torch.cuda.default_stream())
    assert np.linalg.norm(x - xo) / np.linalg.norm(xo) < 1e-12


@pytest.mark.parametrize("P", [1, 2, 3])
def test_rowblock_jacobi_matches_oracle_bitwise(P):
    torch = pytest.importorskip("torch")
    N, sweeps = 70, 7
    g = inputs.jacobi_grid(N, seed=2, dtype=np.float32)
    want = programs.jacobi(g, sweeps, np.float32)[1:-1]
    rts, steps = [], []
    st = torch.cuda.Stream()
    try:
        torch.cuda.set_stream(st)
        for r in range(P):
            rt = gpu_runtime("persistent", rows=8, stream=st.cuda_stream).__enter__()
            rts.append(rt)
            lo, hi = D.jacobi_block_rows(N, P, r)
            steps.append(D.RuntimeJacobi(rt, g[lo:hi], torch))
        if P == 1:
            D.rowblock_jacobi(steps[0], D.SelfComm(), sweeps)
        else:
            for _ in range(sweeps):
                for s in steps:
                    s.before_exchange()
                    s.rt.sync()
                for r in range(P - 1):
                    # ghost rows: the next block's first row below, this block's last row above
                    steps[r].row(-1).copy_(steps[r + 1].row(1))
                    steps[r + 1].row(0).copy_(steps[r].row(-2))
                for s in steps:
                    s.sweep()
        got = np.concatenate([s.owned_rows() for s in steps])
    finally:
        for rt in rts:
            rt.close()
        torch.cuda.set_stream(torch.cuda.default_stream())
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
