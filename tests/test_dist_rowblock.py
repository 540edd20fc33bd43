"""Row-block partition of the iterative solvers over ranks (CPU only).

Section 3.2 runs an index task's point tasks one per processor; across GPUs a
solver's vectors are tiled by row blocks.  Checked here without a GPU:
  * the plan of the C-ABI (dfs_rowblock_plan) against brute force: owned
    rows, local columns, halo slots, and that what rank r sends to rank q is
    exactly what q's halo slots expect from r;
  * the orchestration (halo all-to-all, SUM all-reduces of the dot products,
    ghost-row swaps) on 2 and 3 gloo ranks, each rank running its local
    windows with the CPU oracle: the concatenated CG solution equals the
    single-process oracle CG to 1e-12, and the Jacobi grid bit for bit.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from oracle import ops, programs  # noqa: E402
from paper_2406_18109_gb300 import binding as B  # noqa: E402
from paper_2406_18109_gb300 import dist as D  # noqa: E402
from synth import inputs  # noqa: E402
from tests.helpers import ensure_built  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


MATRICES = {
    "poisson": lambda: inputs.poisson2d_csr(9),
    "spd": lambda: inputs.random_spd_csr(70, seed=3),
}


@pytest.mark.parametrize("name", sorted(MATRICES))
@pytest.mark.parametrize("P", [1, 2, 3, 4])
def test_plan_against_brute_force(name, P):
    rp, col, val = MATRICES[name]()
    n = len(rp) - 1
    plans = [D.RowBlock(rp, col, val, P, r) for r in range(P)]
    # the blocks cover the rows once, in order, balanced to within one row
    assert plans[0].lo == 0 and plans[-1].hi == n
    for a, b in zip(plans, plans[1:]):
        assert a.hi == b.lo
    sizes = [p.n_own for p in plans]
    assert max(sizes) - min(sizes) <= 1
    x = inputs.uniform(5, -1, 1, n)
    y = programs.spmv(rp, col, val, x)
    for r, p in enumerate(plans):
        # halo: the distinct outside columns the owned rows read, ascending
        cols = set(col[rp[p.lo]:rp[p.hi]].tolist())
        want = sorted(c for c in cols if not p.lo <= c < p.hi)
        assert p.halo_cols.tolist() == want
        # the local matrix on [owned x, halo x] gives the owned rows of A x bit for bit
        x_ext = np.concatenate([x[p.lo:p.hi], x[p.halo_cols]])
        assert np.array_equal(programs.spmv(p.rowptr, p.col, p.val, x_ext), y[p.lo:p.hi])
        for q in range(P):
            # recv: halo slots owned by q; send: q's halo slots owned by r, in order
            owned_q = (plans[q].lo <= p.halo_cols) & (p.halo_cols < plans[q].hi)
            assert p.recv_counts[q] == owned_q.sum()
            so = np.concatenate([[0], np.cumsum(p.send_counts)])
            sent = p.lo + p.send_idx[so[q]:so[q + 1]]
            ro = np.concatenate([[0], np.cumsum(plans[q].recv_counts)])
            assert sent.tolist() == plans[q].halo_cols[ro[r]:ro[r + 1]].tolist()
        assert p.send_counts[r] == 0 and p.recv_counts[r] == 0


def test_poisson_halo_is_one_grid_row_per_neighbour():
    m = 12
    rp, col, val = inputs.poisson2d_csr(m)
    p = D.RowBlock(rp, col, val, 3, 1)           # middle block of 48 rows = 4 grid rows
    assert p.n_own == 48 and p.n_halo == 2 * m
    assert p.recv_counts.tolist() == [m, 0, m] and p.send_counts.tolist() == [m, 0, m]


def test_plan_rejects_malformed_input():
    rp, col, val = inputs.poisson2d_csr(4)
    with pytest.raises(B.DfsError):
        B.dfs_rowblock_plan(rp, col, 2, 2)                      # rank out of range
    with pytest.raises(B.DfsError):
        B.dfs_rowblock_plan(rp, col, 0, 0)                      # no ranks
    bad = col.copy()
    bad[3] = len(rp) + 5
    with pytest.raises(B.DfsError):
        B.dfs_rowblock_plan(rp, bad, 2, 0)                      # column out of range
    rp2 = rp.copy()
    rp2[2], rp2[3] = rp2[3], rp2[2]
    with pytest.raises(B.DfsError):
        B.dfs_rowblock_plan(rp2, col, 2, 0)                     # decreasing row pointers
    assert B.dfs_rowblock_bounds(10, 4, 3) == (7, 10)
    assert B.dfs_rowblock_bounds(2, 3, 0) == (0, 0)             # more ranks than rows: empty blocks
    with pytest.raises(B.DfsError):
        B.dfs_rowblock_bounds(10, 4, 4)


# ---------------------------------------------------- oracle local windows
class OracleCG:
    """The local windows of dist.rowblock_cg run by the CPU oracle; the
    exchange buffers are CPU torch tensors sharing memory with numpy."""

    def __init__(self, block, b_own):
        self.block = block
        f64 = torch.float64
        self.p_ext_t = torch.zeros(block.n_own + block.n_halo, dtype=f64)
        self.p_ext = self.p_ext_t.numpy()
        self.halo = self.p_ext_t[block.n_own:]
        self.send = torch.zeros(block.n_send, dtype=f64)
        self.pq = torch.zeros((), dtype=f64)
        self.rr = torch.zeros((), dtype=f64)
        self.b = b_own

    def start(self):
        self.x = np.zeros(self.block.n_own)
        self.r = self.b.copy()
        self.p_ext[:self.block.n_own] = self.b
        self.rr.fill_(float(programs.dot(self.r, self.r)))

    def set_rho(self):
        self.rho = float(self.rr)

    def pack_halo(self):
        self.send.numpy()[:] = self.p_ext[self.block.send_idx]

    def spmv_dot(self):
        b = self.block
        self.q = programs.spmv(b.rowptr, b.col, b.val, self.p_ext)
        self.pq.fill_(float(programs.dot(self.p_ext[:b.n_own], self.q)))

    def update_xr(self):
        p = self.p_ext[:self.block.n_own]
        alpha = self.rho / float(self.pq)
        self.x = ops.binary("ADD", self.x, ops.binary("MUL", alpha, p, np.float64), np.float64)
        self.r = ops.binary("SUB", self.r, ops.binary("MUL", alpha, self.q, np.float64), np.float64)
        self.rr.fill_(float(programs.dot(self.r, self.r)))

    def update_p(self):
        n = self.block.n_own
        beta = float(self.rr) / self.rho
        self.rho = float(self.rr)
        self.p_ext[:n] = ops.binary("ADD", self.r, ops.binary("MUL", beta, self.p_ext[:n], np.float64), np.float64)


class OracleJacobi:
    def __init__(self, rows):
        self.t = torch.from_numpy(np.ascontiguousarray(rows))

    def before_exchange(self):
        pass

    def row(self, i):
        return self.t[i]

    def sweep(self):
        g = programs.jacobi(self.t.numpy(), 1, np.float32)
        self.t[1:-1] = torch.from_numpy(g[1:-1])


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        comm = D.Comm()
        out = {}
        for name, iters in (("poisson", 30), ("spd", 25)):
            rp, col, val, xs = (inputs.cg_inputs(m=23, seed=0) if name == "poisson"
                                else (*inputs.random_spd_csr(300, seed=6), inputs.uniform(8, -1, 1, 300)))
            b = programs.spmv(rp, col, val, xs)
            blk = D.RowBlock(rp, col, val, world, rank)
            st = OracleCG(blk, b[blk.lo:blk.hi].copy())
            D.rowblock_cg(st, comm, iters)
            out[name] = (blk.lo, st.x)
        N = 37
        g = inputs.jacobi_grid(N, seed=2, dtype=np.float32)
        lo, hi = D.jacobi_block_rows(N, world, rank)
        sj = OracleJacobi(g[lo:hi])
        D.rowblock_jacobi(sj, comm, 9)
        out["jacobi"] = (lo, sj.t[1:-1].numpy().copy())
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_rowblock_solvers_on_gloo_ranks(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29000 + (os.getpid() % 400) + 7 * world
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for name, iters in (("poisson", 30), ("spd", 25)):
        rp, col, val, xs = (inputs.cg_inputs(m=23, seed=0) if name == "poisson"
                            else (*inputs.random_spd_csr(300, seed=6), inputs.uniform(8, -1, 1, 300)))
        b = programs.spmv(rp, col, val, xs)
        xo, _, _ = programs.cg(rp, col, val, b, iters)
        x = np.concatenate([res[r][name][1] for r in range(world)])
        assert [res[r][name][0] for r in range(world)] == sorted(res[r][name][0] for r in range(world))
        assert np.linalg.norm(x - xo) / np.linalg.norm(xo) < 1e-12, name
    g = inputs.jacobi_grid(37, seed=2, dtype=np.float32)
    want = programs.jacobi(g, 9, np.float32)[1:-1]
    got = np.concatenate([res[r]["jacobi"][1] for r in range(world)])
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
