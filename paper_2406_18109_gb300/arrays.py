"""A NumPy-style array front end that issues index tasks to the runtime.

This plays the role of the task-based array libraries of the paper (Section 1
and Section 3: cuPyNumeric and Legate Sparse translate array operations into
a stream of index tasks over partitioned stores).  Each operator below submits
exactly one task through the C-ABI; all computation happens in the generated
kernels.  Arrays drop their store reference when Python frees them, which
feeds the split reference count used by temporary elimination (Section 5.1).

Partitioning: an array of shape (n,) is tiled into blocks of ``tile`` elements
over the launch domain (ceil(n/tile),); a 2-D array (or view) of shape (m, w)
into bands of ``rows`` rows, launch domain (ceil(m/rows), 1).  Arrays of equal
shape therefore share launch domain and tiling, which is what lets the fusion
pass fuse their tasks.  0-d arrays are read through the None partition.
"""
from __future__ import annotations

import math
import weakref

import numpy as np

from . import binding as B

_DT = {np.dtype(np.float32): B.DFS_F32, np.dtype(np.float64): B.DFS_F64,
       np.dtype(np.int32): B.DFS_I32, np.dtype(np.int64): B.DFS_I64}


def _dfs_dtype(dt) -> int:
    return _DT[np.dtype(dt)]


class Runtime:
    """One fusion context (C-ABI ``dfs_ctx``) plus the library's partitioning policy."""

    def __init__(self, device: int = 0, fusion: bool = True, launch: str = "persistent",
                 window_size: int = 256, block: int = 256, unroll: int = 2, ctas_per_sm: int = 0,
                 stream: int | None = None, cache_dir: str | None = None, timeout_s: float = 2.0,
                 tile: int | None = None, rows: int | None = None, sms: int = 152,
                 debug_skip_arrival: int = 0):
        cfg = B.dfs_config_default()
        cfg.device = device
        cfg.fusion = 1 if fusion else 0
        cfg.launch_mode = B.DFS_LAUNCH_PERSISTENT if launch == "persistent" else B.DFS_LAUNCH_PER_TASK
        cfg.window_size = window_size
        cfg.block_threads = block
        cfg.unroll = unroll
        cfg.ctas_per_sm = ctas_per_sm
        cfg.barrier_timeout_s = timeout_s
        cfg.stream = stream
        cfg.debug_skip_arrival = debug_skip_arrival
        self._cache_dir = cache_dir.encode() if cache_dir else None
        cfg.cache_dir = self._cache_dir
        self.ctx = B.dfs_init(cfg)
        self.device = device
        self.none = B.dfs_partition_none(self.ctx)
        self._tilings = {}
        self.tile = tile
        self.rows = rows
        self.sms = sms
        self._alive = True

    # ------------------------------------------------------------ lifetime
    def close(self):
        if self._alive:
            self._alive = False
            B.dfs_shutdown(self.ctx)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---------------------------------------------------------- partitions
    def tiling(self, tile, offset=None) -> int:
        key = (tuple(tile), tuple(offset) if offset else None)
        h = self._tilings.get(key)
        if h is None:
            h = B.dfs_partition_tiling(self.ctx, tile, offset)
            self._tilings[key] = h
        return h

    def tile_1d(self, n: int) -> int:
        if self.tile:
            return self.tile
        # a few points per SM, tiles a multiple of 256 elements, at most 16384
        t = math.ceil(n / (self.sms * 4))
        t = max(256, min(16384, ((t + 255) // 256) * 256))
        return t

    def rows_2d(self, m: int, w: int) -> int:
        if self.rows:
            return self.rows
        return max(1, min(m, (1 << 17) // max(1, w)))

    def layout(self, shape):
        """(launch domain, partition handle) the library uses for this shape."""
        if len(shape) == 0:
            return (1,), self.none
        if len(shape) == 1:
            t = self.tile_1d(shape[0])
            return (max(1, math.ceil(shape[0] / t)),), self.tiling((t,))
        if len(shape) == 2:
            r = self.rows_2d(shape[0], shape[1])
            return (max(1, math.ceil(shape[0] / r)), 1), self.tiling((r, shape[1]))
        raise ValueError("arrays of rank > 2 are not supported by the front end")

    # -------------------------------------------------------------- arrays
    def empty(self, shape, dtype=np.float64) -> "Array":
        shape = tuple(int(s) for s in shape)
        h = B.dfs_store_create(self.ctx, _dfs_dtype(dtype), shape)
        return Array(self, h, shape, np.dtype(dtype))

    def array(self, host: np.ndarray) -> "Array":
        host = np.ascontiguousarray(host)
        a = self.empty(host.shape, host.dtype)
        a.write(host)
        return a

    def scalar(self, value: float, dtype=np.float64) -> "Array":
        return self.array(np.array(value, dtype=dtype))

    def wrap(self, tensor) -> "Array":
        """Wraps a contiguous CUDA tensor (torch) without copying."""
        import torch  # plumbing only: device memory owned by PyTorch
        assert tensor.is_cuda and tensor.is_contiguous()
        dt = {torch.float32: np.float32, torch.float64: np.float64,
              torch.int32: np.int32, torch.int64: np.int64}[tensor.dtype]
        h = B.dfs_store_wrap(self.ctx, _dfs_dtype(dt), tuple(tensor.shape), tensor.data_ptr())
        return Array(self, h, tuple(tensor.shape), np.dtype(dt), keep=tensor)

    def submit(self, op, domain, args):
        B.dfs_submit(self.ctx, op, domain, args)

    def flush(self):
        B.dfs_flush(self.ctx)

    def sync(self):
        B.dfs_sync(self.ctx)

    def plan(self) -> dict:
        return B.dfs_plan_json(self.ctx)

    def stats(self) -> dict:
        return B.dfs_stats_json(self.ctx)

    def kernel_source(self) -> str:
        return B.dfs_last_kernel_source(self.ctx)


def _release(rt_ref, handle):
    rt = rt_ref()
    if rt is not None and rt._alive:
        try:
            B.dfs_store_release(rt.ctx, handle)
        except B.DfsError:
            pass


class Array:
    """A store (or view) handle; operators submit one index task each."""

    __array_priority__ = 100

    def __init__(self, rt: Runtime, handle: int, shape, dtype, keep=None):
        self.rt = rt
        self.handle = handle
        self.shape = tuple(shape)
        self.dtype = np.dtype(dtype)
        self._keep = keep
        self._fin = weakref.finalize(self, _release, weakref.ref(rt), handle)

    @property
    def ndim(self):
        return len(self.shape)

    @property
    def size(self):
        return int(np.prod(self.shape)) if self.shape else 1

    def release(self):
        self._fin()

    # ------------------------------------------------------------ host I/O
    def write(self, host: np.ndarray):
        host = np.ascontiguousarray(host, dtype=self.dtype)
        B.dfs_store_write(self.rt.ctx, self.handle, host.ctypes.data, host.nbytes)

    def numpy(self) -> np.ndarray:
        out = np.empty(self.shape, dtype=self.dtype)
        B.dfs_store_read(self.rt.ctx, self.handle, out.ctypes.data, out.nbytes)
        return out

    def read_into(self, out: np.ndarray):
        B.dfs_store_read(self.rt.ctx, self.handle, out.ctypes.data, out.nbytes)

    def item(self) -> float:
        return float(self.numpy())

    def device_ptr(self) -> int:
        return B.dfs_store_device_ptr(self.rt.ctx, self.handle)

    # --------------------------------------------------------------- views
    def __getitem__(self, idx) -> "Array":
        if not isinstance(idx, tuple):
            idx = (idx,)
        if len(idx) > self.ndim:
            raise IndexError("too many indices")
        idx = idx + (slice(None),) * (self.ndim - len(idx))
        off, shp = [], []
        for s, n in zip(idx, self.shape):
            if not isinstance(s, slice) or s.step not in (None, 1):
                raise IndexError("views are unit-stride slices")
            lo, hi, _ = s.indices(n)
            off.append(lo)
            shp.append(max(0, hi - lo))
        h = B.dfs_store_view(self.rt.ctx, self.handle, off, shp)
        return Array(self.rt, h, shp, self.dtype)

    def __setitem__(self, idx, value):
        view = self[idx]
        view._unary("COPY", value, out=view)

    # ------------------------------------------------------------ tasking
    def _arg(self, priv):
        _, part = self.rt.layout(self.shape)
        return (self.handle, part, priv)

    def _operand(self, v):
        if isinstance(v, Array):
            return v._arg(B.DFS_PRIV_R)
        return float(v)

    def _domain_of(self, *xs):
        best = None
        for x in xs:
            if isinstance(x, Array) and x.ndim > 0:
                best = x
                break
        return self.rt.layout(best.shape if best is not None else ())[0], best

    def _binary(self, op, a, b, out=None):
        dom, big = self._domain_of(a, b)
        shape = big.shape if big is not None else ()
        if out is None:
            out = self.rt.empty(shape, self.dtype)
        self.rt.submit(op, dom, [self._operand(a), self._operand(b), out._arg(B.DFS_PRIV_W)])
        return out

    def _unary(self, op, a, out=None):
        dom, big = self._domain_of(a if isinstance(a, Array) else self)
        target = out if out is not None else self.rt.empty(self.shape, self.dtype)
        dom = self.rt.layout(target.shape)[0]
        self.rt.submit(op, dom, [self._operand(a), target._arg(B.DFS_PRIV_W)])
        return target

    def __add__(self, o): return self._binary("ADD", self, o)
    def __radd__(self, o): return self._binary("ADD", o, self)
    def __sub__(self, o): return self._binary("SUB", self, o)
    def __rsub__(self, o): return self._binary("SUB", o, self)
    def __mul__(self, o): return self._binary("MUL", self, o)
    def __rmul__(self, o): return self._binary("MUL", o, self)
    def __truediv__(self, o): return self._binary("DIV", self, o)
    def __rtruediv__(self, o): return self._binary("DIV", o, self)
    def __pow__(self, o): return self._binary("POW", self, o)
    def __neg__(self): return self._unary("NEG", self)

    def __iadd__(self, o): return self._binary("ADD", self, o, out=self)
    def __isub__(self, o): return self._binary("SUB", self, o, out=self)
    def __imul__(self, o): return self._binary("MUL", self, o, out=self)
    def __itruediv__(self, o): return self._binary("DIV", self, o, out=self)


# ------------------------------------------------------------- functions
def _map(op, x: Array) -> Array:
    return x._unary(op, x)


def exp(x): return _map("EXP", x)
def log(x): return _map("LOG", x)
def sqrt(x): return _map("SQRT", x)
def erf(x): return _map("ERF", x)
def absolute(x): return _map("ABS", x)
def ncdf(x): return _map("NCDF", x)
def copy(x): return _map("COPY", x)
def maximum(a, b): return (a if isinstance(a, Array) else b)._binary("MAX", a, b)
def minimum(a, b): return (a if isinstance(a, Array) else b)._binary("MIN", a, b)


def full(rt: Runtime, shape, value: float, dtype=np.float64) -> Array:
    out = rt.empty(shape, dtype)
    dom = rt.layout(out.shape)[0]
    rt.submit("COPY", dom, [float(value), out._arg(B.DFS_PRIV_W)])
    return out


def dot(x: Array, y: Array) -> Array:
    out = x.rt.empty((), x.dtype)
    dom = x.rt.layout(x.shape)[0]
    x.rt.submit("DOT", dom, [x._arg(B.DFS_PRIV_R), y._arg(B.DFS_PRIV_R),
                             (out.handle, x.rt.none, B.DFS_PRIV_RD, B.DFS_REDOP_SUM)])
    return out


def asum(x: Array) -> Array:
    out = x.rt.empty((), x.dtype)
    dom = x.rt.layout(x.shape)[0]
    x.rt.submit("SUM", dom, [x._arg(B.DFS_PRIV_R), (out.handle, x.rt.none, B.DFS_PRIV_RD, B.DFS_REDOP_SUM)])
    return out


def norm(x: Array) -> Array:
    return sqrt(dot(x, x))


class CSR:
    """CSR matrix (int32 row pointers and columns), the Legate Sparse layout."""

    def __init__(self, rt: Runtime, rowptr: np.ndarray, col: np.ndarray, val: np.ndarray, ncols: int | None = None):
        self.rt = rt
        self.nrows = len(rowptr) - 1
        self.ncols = self.nrows if ncols is None else ncols
        self.nnz = len(col)
        self.rowptr = rt.array(np.asarray(rowptr, dtype=np.int32))
        self.col = rt.array(np.asarray(col, dtype=np.int32))
        self.val = rt.array(np.asarray(val))
        self.dtype = self.val.dtype

    def __matmul__(self, x: Array) -> Array:
        y = self.rt.empty((self.nrows,), self.dtype)
        self.spmv(x, y)
        return y

    def spmv(self, x: Array, y: Array):
        dom, part = self.rt.layout(y.shape)
        n = self.rt.none
        self.rt.submit("SPMV", dom, [(self.rowptr.handle, n, B.DFS_PRIV_R), (self.col.handle, n, B.DFS_PRIV_R),
                                     (self.val.handle, n, B.DFS_PRIV_R), (x.handle, n, B.DFS_PRIV_R),
                                     (y.handle, part, B.DFS_PRIV_W)])
        return y
