"""Multi-rank execution (one process per GPU).

Independent work units (Black-Scholes batches) are sharded by giving every
rank its own batch: there is no collective on the data path.  The only
cross-rank communication is control: the slowest rank's time and the total
number of units, combined after the timed region.

Iterative solvers shard by row blocks (Section 3.2: the point tasks of an
index task run one per processor; the paper's evaluation scales this way
over GPUs).  Rank r owns a block of rows of the matrix and of every vector.
Per CG iteration the ranks exchange two things only:
  * the HALO of p: the entries of p that their SpMV rows read from other
    blocks, one all-to-all with the counts of the row-block plan
    (dfs_rowblock_plan), received into p's halo slots;
  * the partial sums of the two dot products, one SUM all-reduce of one
    value each.
A Jacobi sweep exchanges one ghost row with each neighbouring block.
Everything else is the rank's own fused windows.  The orchestration below is
written once against a small set of steps: ``RuntimeCG`` / ``RuntimeJacobi``
run them as the runtime's kernels on this rank's GPU; a test can supply other
steps (the CPU oracle) to check the partition and the exchanges.
"""
from __future__ import annotations

import numpy as np


def rank_seed(base_seed: int, rank: int) -> int:
    """Seed of rank r's batch: the configured seed on rank 0, distinct elsewhere."""
    return base_seed if rank == 0 else base_seed + 1000 * rank


def combine(ms_local: float, units_local: float, device=None):
    """(value, ms_max, units_total): whole-job throughput in units/s over all
    ranks, timed by the slowest rank.  Works with gloo (CPU) or NCCL."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return units_local / (ms_local / 1e3), ms_local, units_local
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    u = torch.tensor([units_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    ms = float(t.item())
    units = float(u.item())
    return units / (ms / 1e3), ms, units


# ------------------------------------------------------------ collectives
class Comm:
    """The exchanges of the row-block solvers over torch.distributed (NCCL
    between GPUs, gloo between CPU processes).  Tensors are contiguous."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist, self.group = dist, group
        self.rank = dist.get_rank(group)
        self.size = dist.get_world_size(group)

    def allreduce_sum(self, t) -> None:
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM, group=self.group)

    def exchange(self, send, send_counts, recv, recv_counts) -> None:
        """All-to-all: send[segment q] goes to rank q, recv[segment q] comes
        from rank q; segments are consecutive, with the given counts."""
        if sum(send_counts) == 0 and sum(recv_counts) == 0 and self.size == 1:
            return
        self.dist.all_to_all_single(recv, send, [int(c) for c in recv_counts], [int(c) for c in send_counts],
                                    group=self.group)

    def neighbours(self, to_prev, from_prev, to_next, from_next) -> None:
        """Swaps rows with ranks r - 1 and r + 1 (None where there is none)."""
        ops = []
        if to_prev is not None:
            ops += [self.dist.P2POp(self.dist.isend, to_prev, self.rank - 1, self.group),
                    self.dist.P2POp(self.dist.irecv, from_prev, self.rank - 1, self.group)]
        if to_next is not None:
            ops += [self.dist.P2POp(self.dist.isend, to_next, self.rank + 1, self.group),
                    self.dist.P2POp(self.dist.irecv, from_next, self.rank + 1, self.group)]
        if ops:
            for w in self.dist.batch_isend_irecv(ops):
                w.wait()


class SelfComm:
    """One rank: nothing to exchange."""
    rank, size = 0, 1

    def allreduce_sum(self, t) -> None:
        pass

    def exchange(self, send, send_counts, recv, recv_counts) -> None:
        assert sum(send_counts) == 0 and sum(recv_counts) == 0

    def neighbours(self, to_prev, from_prev, to_next, from_next) -> None:
        assert to_prev is None and to_next is None


# --------------------------------------------------------- row-block plan
class RowBlock:
    """Rank `rank`'s block of a square CSR matrix (dfs_rowblock_plan): owned
    rows [lo, hi), the local matrix with owned columns first and halo slots
    after, and the exchange counts."""

    def __init__(self, rowptr, col, val, nranks: int, rank: int):
        from . import binding as B
        p = B.dfs_rowblock_plan(rowptr, col, nranks, rank)
        self.lo, self.hi = p["row_lo"], p["row_hi"]
        self.n_own = self.hi - self.lo
        self.n_halo = len(p["halo_cols"])
        self.rowptr, self.col = p["local_rowptr"], p["local_col"]
        self.val = np.ascontiguousarray(np.asarray(val)[rowptr[self.lo]:rowptr[self.hi]])
        self.halo_cols, self.send_idx = p["halo_cols"], p["send_idx"]
        self.recv_counts, self.send_counts = p["recv_counts"], p["send_counts"]
        self.n_send = len(self.send_idx)


def rowblock_cg(steps, comm, iters: int) -> None:
    """CG (Hestenes-Stiefel, the stream of a naturally written solver) over a
    row-block partition: per iteration the halo exchange of p, then
    [q = A p, p.q] and a SUM all-reduce, [alpha; x +=, r -=, r.r] and a SUM
    all-reduce, [beta; p = r + beta p].  `steps` runs the local windows and
    owns the buffers the exchanges read and write."""
    steps.start()
    comm.allreduce_sum(steps.rr)
    steps.set_rho()
    for _ in range(iters):
        steps.pack_halo()
        comm.exchange(steps.send, steps.block.send_counts, steps.halo, steps.block.recv_counts)
        steps.spmv_dot()
        comm.allreduce_sum(steps.pq)
        steps.update_xr()
        comm.allreduce_sum(steps.rr)
        steps.update_p()


def rowblock_jacobi(steps, comm, sweeps: int) -> None:
    """The Fig. 1 sweep over row blocks of the interior: before each sweep
    every block sends its first owned row to the previous block and its last
    to the next one, which keep them as ghost rows; the sweep then reads
    nothing else from other blocks."""
    for _ in range(sweeps):
        steps.before_exchange()
        first = comm.rank == 0
        last = comm.rank == comm.size - 1
        comm.neighbours(None if first else steps.row(1), None if first else steps.row(0),
                        None if last else steps.row(-2), None if last else steps.row(-1))
        steps.sweep()


def _check_stream(rt, torch) -> None:
    """The exchanges run on torch's current stream; the context must launch
    on that same (non-default) stream for the two to stay ordered."""
    cur = torch.cuda.current_stream().cuda_stream
    if not rt.stream or rt.stream != cur:
        raise ValueError("the runtime context must be created on torch's current stream (a non-default "
                         "torch.cuda.Stream), which the exchanges also use")


def jacobi_block_rows(N: int, nranks: int, rank: int):
    """Global rows [lo, hi) of the (N+2)-row grid that rank `rank` holds:
    its owned interior rows plus one ghost (or boundary) row on each side."""
    from . import binding as B
    lo, hi = B.dfs_rowblock_bounds(N, nranks, rank)
    if hi <= lo:
        raise ValueError("every rank needs at least one interior row")
    return lo, hi + 2


# ------------------------------------------------- steps on the runtime
class RuntimeCG:
    """The local windows of rowblock_cg as the runtime's fused kernels on this
    rank's GPU.  Exchange buffers are torch tensors wrapped as stores, so
    NCCL reads and writes the memory the kernels use; every step flushes
    its window before the host issues the next collective, and the runtime's
    stream is the current torch stream, so the two stay ordered."""

    def __init__(self, rt, block: RowBlock, b_own: np.ndarray, torch):
        from . import arrays as A
        _check_stream(rt, torch)
        self.A, self.rt, self.block, self.torch = A, rt, block, torch
        dev = torch.device("cuda", torch.cuda.current_device())
        f64 = torch.float64
        n_own, n_halo = block.n_own, block.n_halo
        self.Aloc = A.CSR(rt, block.rowptr, block.col, block.val, ncols=n_own + n_halo)
        self.p_ext_t = torch.zeros(n_own + n_halo, dtype=f64, device=dev)
        self.p_ext = rt.wrap(self.p_ext_t)
        self.p = self.p_ext[0:n_own]
        self.halo = self.p_ext_t[n_own:]
        self.send = torch.zeros(max(1, block.n_send), dtype=f64, device=dev)[:block.n_send]
        if block.n_send:
            # packing the halo is a gather: a selection matrix with one unit
            # entry per sent value, applied by the SpMV kernel
            self.G = A.CSR(rt, np.arange(block.n_send + 1, dtype=np.int32), block.send_idx,
                           np.ones(block.n_send), ncols=n_own)
            self.send_arr = rt.wrap(self.send)
        self.pq = torch.zeros((), dtype=f64, device=dev)
        self.rr = torch.zeros((), dtype=f64, device=dev)
        self.pq_a, self.rr_a = rt.wrap(self.pq), rt.wrap(self.rr)
        self.b = rt.array(np.ascontiguousarray(b_own, dtype=np.float64))
        self.x = A.full(rt, (n_own,), 0.0)
        self.r = A.full(rt, (n_own,), 0.0)
        self.q = A.full(rt, (n_own,), 0.0)
        self.rho = A.full(rt, (), 0.0)

    def start(self):
        self.x[...] = 0.0
        self.r[...] = self.b
        self.p[...] = self.b
        self.rr_a[...] = self.A.dot(self.r, self.r)
        self.rt.flush()

    def set_rho(self):
        self.rho[...] = self.rr_a

    def pack_halo(self):
        if self.block.n_send:
            self.G.spmv(self.p, self.send_arr)
        self.rt.flush()

    def spmv_dot(self):
        self.Aloc.spmv(self.p_ext, self.q)
        self.pq_a[...] = self.A.dot(self.p, self.q)
        self.rt.flush()

    def update_xr(self):
        alpha = self.rho / self.pq_a
        self.x += alpha * self.p
        self.r -= alpha * self.q
        self.rr_a[...] = self.A.dot(self.r, self.r)
        self.rt.flush()

    def update_p(self):
        beta = self.rr_a / self.rho
        self.rho[...] = self.rr_a
        self.p *= beta
        self.p += self.r

    def solution(self) -> np.ndarray:
        return self.x.numpy()


class RuntimeJacobi:
    """The local sweep of rowblock_jacobi as the runtime's fused window
    (Fig. 1) on a wrapped torch grid holding this rank's rows plus the ghost
    rows; rows are exchanged in place."""

    def __init__(self, rt, grid_rows: np.ndarray, torch):
        from . import arrays as A
        from . import workloads as W
        _check_stream(rt, torch)
        self.rt, self.W = rt, W
        dev = torch.device("cuda", torch.cuda.current_device())
        self.t = torch.from_numpy(np.ascontiguousarray(grid_rows)).to(dev)
        self.g = rt.wrap(self.t)
        self.views = W.jacobi_views(self.g)
        self.A = A

    def before_exchange(self):
        self.rt.flush()

    def row(self, i: int):
        return self.t[i]

    def sweep(self):
        self.W.jacobi_sweep(self.views)
        self.rt.flush()

    def owned_rows(self) -> np.ndarray:
        self.rt.sync()
        return self.t[1:-1].cpu().numpy()
