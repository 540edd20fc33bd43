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

The issue path is kept short (cached layouts, one packed argument buffer per
runtime) because the host issues one task per array operation.
"""
from __future__ import annotations

import ctypes as C
import math
import struct
import weakref

import numpy as np

from . import binding as B

_DT = {np.dtype(np.float32): B.DFS_F32, np.dtype(np.float64): B.DFS_F64,
       np.dtype(np.int32): B.DFS_I32, np.dtype(np.int64): B.DFS_I64}
_ARG = struct.Struct("=qqiid")      # dfs_arg: store, partition, privilege, redop, imm (32 bytes)
assert _ARG.size == C.sizeof(B.dfs_arg)
_R, _W, _RD, _IMM = B.DFS_PRIV_R, B.DFS_PRIV_W, B.DFS_PRIV_RD, B.DFS_PRIV_IMM
_SUM = B.DFS_REDOP_SUM
_OP = B.OPS


def _dfs_dtype(dt) -> int:
    return _DT[np.dtype(dt)]


class Runtime:
    """One fusion context (C-ABI ``dfs_ctx``) plus the library's partitioning policy."""

    def __init__(self, device: int = 0, fusion: bool = True, launch: str = "persistent",
                 window_size: int = 256, block: int = 256, unroll: int = 2, ctas_per_sm: int = 0,
                 stream: int | None = None, cache_dir: str | None = None, timeout_s: float = 2.0,
                 tile: int | None = None, rows: int | None = None, sms: int = 152,
                 debug_skip_arrival: int = 0, time_launches: bool = False, tile_max: int = 16384,
                 min_points: int | None = None, window_growth: bool = False, window_max: int = 0,
                 stage_x: bool = False):
        cfg = B.dfs_config_default()
        cfg.device = device
        cfg.fusion = 1 if fusion else 0
        cfg.launch_mode = B.DFS_LAUNCH_PERSISTENT if launch == "persistent" else B.DFS_LAUNCH_PER_TASK
        cfg.window_size = window_size
        cfg.block_threads = block
        cfg.unroll = unroll
        cfg.ctas_per_sm = ctas_per_sm
        self.block, self.unroll, self.ctas_per_sm = block, unroll, ctas_per_sm
        cfg.barrier_timeout_s = timeout_s
        cfg.stream = stream
        cfg.debug_skip_arrival = debug_skip_arrival
        cfg.time_launches = 1 if time_launches else 0
        cfg.window_growth = 1 if window_growth else 0
        cfg.window_max = window_max
        self._cache_dir = cache_dir.encode() if cache_dir else None
        cfg.cache_dir = self._cache_dir
        self.ctx = B.dfs_init(cfg)
        self.device = device
        self.stream = stream or None          # the caller's cudaStream_t handle, or None: the context's own
        self.none = B.dfs_partition_none(self.ctx)
        self._tilings = {}
        self._layouts = {}
        self._shapes = {}
        self.tile = tile
        self.rows = rows
        self.sms = sms
        self.tile_max = tile_max
        self.min_points = min_points
        self._alive = True
        # SpMV x windows staged in shared memory (the optional window argument
        # of DFS_OP_SPMV); matrices register here to follow tiling changes
        self.stage_x = stage_x
        self._csrs = weakref.WeakSet()
        L = B.lib()
        self._lib_submit = L.dfs_submit
        self._lib_create = L.dfs_store_create
        self._lib_release = L.dfs_store_release
        self._argbuf = (B.dfs_arg * 8)()
        self._argptr = C.cast(self._argbuf, C.POINTER(B.dfs_arg))
        self._out = C.c_int64()
        self._outref = C.byref(self._out)

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
        """Elements per point of a length-n vector: the fixed `tile`, else the
        smallest multiple of 256 giving at most `min_points` points (default
        4 per SM), within [256, tile_max]."""
        if self.tile:
            return self.tile
        t = math.ceil(n / (self.min_points or self.sms * 4))
        return max(256, min(self.tile_max, ((t + 255) // 256) * 256))

    def rows_2d(self, m: int, w: int) -> int:
        if self.rows:
            return self.rows
        return max(1, min(m, (1 << 17) // max(1, w)))

    def layout(self, shape):
        """(launch domain, partition handle) the library uses for this shape."""
        lay = self._layouts.get(shape)
        if lay is None:
            lay = self._make_layout(shape)
        return lay[0], lay[1]

    def _make_layout(self, shape):
        if len(shape) == 0:
            dom, part = (1,), self.none
        elif len(shape) == 1:
            t = self.tile_1d(shape[0])
            dom, part = (max(1, math.ceil(shape[0] / t)),), self.tiling((t,))
        elif len(shape) == 2:
            r = self.rows_2d(shape[0], shape[1])
            dom, part = (max(1, math.ceil(shape[0] / r)), 1), self.tiling((r, shape[1]))
        elif len(shape) == 3:
            # blocks of whole planes, as many as rows_2d allows for a plane's elements
            r = self.rows_2d(shape[0], shape[1] * shape[2])
            dom, part = (max(1, math.ceil(shape[0] / r)), 1, 1), self.tiling((r, shape[1], shape[2]))
        else:
            raise ValueError("arrays of rank > 3 are not supported by the front end")
        lay = (dom, part, (C.c_int64 * len(dom))(*dom), len(dom))
        self._layouts[shape] = lay
        return lay

    # ------------------------------------------------------------- tasking
    def _pack(self, i, x):
        if x.__class__ is Array:
            lay = self._layouts.get(x.shape) or self._make_layout(x.shape)
            _ARG.pack_into(self._argbuf, i * 32, x.handle, lay[1], _R, 0, 0.0)
        else:
            _ARG.pack_into(self._argbuf, i * 32, 0, 0, _IMM, 0, float(x))

    def _issue(self, opcode, lay, n):
        rc = self._lib_submit(self.ctx, opcode, lay[3], lay[2], n, self._argptr)
        if rc:
            B._check(self.ctx, rc)

    def _new(self, shape, dtype) -> "Array":
        sc = self._shapes.get(shape)
        if sc is None:
            sc = self._shapes[shape] = (C.c_int64 * max(1, len(shape)))(*shape)
        rc = self._lib_create(self.ctx, _DT[dtype], len(shape), sc, self._outref)
        if rc:
            B._check(self.ctx, rc)
        return Array(self, self._out.value, shape, dtype)

    def empty(self, shape, dtype=np.float64) -> "Array":
        return self._new(tuple(int(s) for s in shape), np.dtype(dtype))

    def array(self, host: np.ndarray) -> "Array":
        host = np.asarray(host)
        if not host.flags.c_contiguous:       # (ascontiguousarray would make 0-d arrays 1-d)
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
        a = Array(self, h, tuple(tensor.shape), np.dtype(dt))
        a._keep = tensor
        return a

    @staticmethod
    def host_empty(shape, dtype=np.float64) -> np.ndarray:
        """A numpy array in mapped page-locked host memory (dfs_host_alloc),
        freed with the array; wrap it with wrap_host for kernels to read or
        write it in place."""
        import weakref
        dt = np.dtype(dtype)
        shape = tuple(int(d) for d in shape) if isinstance(shape, (tuple, list)) else (int(shape),)
        nbytes = max(1, int(np.prod(shape)) * dt.itemsize)
        ptr = B.dfs_host_alloc(nbytes)
        buf = (C.c_char * nbytes).from_address(ptr)
        arr = np.frombuffer(buf, dtype=dt, count=int(np.prod(shape))).reshape(shape)
        weakref.finalize(buf, B.dfs_host_free, ptr)
        return arr

    def wrap_host(self, host: np.ndarray) -> "Array":
        """Wraps a contiguous numpy array that lives in mapped page-locked
        host memory (e.g. a pinned torch tensor's .numpy()): kernels read and
        write it directly, without copies (dfs_store_wrap_host)."""
        assert host.flags["C_CONTIGUOUS"]
        h = B.dfs_store_wrap_host(self.ctx, _dfs_dtype(host.dtype), tuple(host.shape), host.ctypes.data)
        a = Array(self, h, tuple(host.shape), host.dtype)
        a._keep = host
        return a

    def submit(self, op, domain, args):
        B.dfs_submit(self.ctx, op, domain, args)

    def flush(self):
        B.dfs_flush(self.ctx)

    def sync(self):
        B.dfs_sync(self.ctx)

    def sync_quiet(self):
        """Synchronise and drop any deferred device error (after a failed trial)."""
        try:
            B.dfs_sync(self.ctx)
        except B.DfsError:
            pass

    def plan(self) -> dict:
        return B.dfs_plan_json(self.ctx)

    def stats(self) -> dict:
        return B.dfs_stats_json(self.ctx)

    def kernel_source(self) -> str:
        return B.dfs_last_kernel_source(self.ctx)

    # ------------------------------------------------------------ batching
    def batch_begin(self):
        """Start a batch of isomorphic instances (see dfs_batch_begin)."""
        B.dfs_batch_begin(self.ctx)

    def batch_next(self):
        """End the current instance of the batch."""
        B.dfs_batch_next(self.ctx)

    def batch_end(self):
        """Run the batch: one launch over every instance."""
        B.dfs_batch_end(self.ctx)

    def batch_repeat(self, n: int):
        """Run the last (steady, in-place) batch n more times (dfs_batch_repeat)."""
        B.dfs_batch_repeat(self.ctx, n)

    def set_launch(self, block: int, unroll: int, ctas_per_sm: int = 0):
        """New launch parameters for the following windows (dfs_set_launch_config)."""
        B.dfs_set_launch_config(self.ctx, block, unroll, ctas_per_sm)
        self.block, self.unroll, self.ctas_per_sm = block, unroll, ctas_per_sm

    def set_tiling(self, tile: int | None = None, rows: int | None = None, tile_max: int | None = None,
                   min_points: int | None = None):
        """New tiling policy for arrays' partitions from now on: a fixed tile
        (1-D, elements) and row block (2-D), or (tile None) the size-dependent
        policy of tile_1d.  Tasks already submitted keep theirs; a store may be
        partitioned differently by later tasks."""
        self.flush()
        self.tile, self.rows = tile, rows
        if tile_max is not None:
            self.tile_max = tile_max
        if min_points is not None:
            self.min_points = min_points
        self._layouts.clear()
        for m in list(self._csrs):
            m.prepare_windows()

    def read_scalars(self, arrays) -> list:
        """Values of many 0-d arrays with one gather and one copy (dfs_read_scalars)."""
        return B.dfs_read_scalars(self.ctx, [a.handle for a in arrays])

    def read_scalars_async(self, arrays, work=None, vals=None) -> "ScalarRead":
        """Enqueues one gather of many 0-d arrays into page-locked host memory
        and returns at once (dfs_read_scalars_async, then a ticket); the
        result's values() waits for it.  work / vals: reusable page-locked
        buffers (host_empty) of at least 2 n int64 and n float64."""
        return ScalarRead(self, arrays, work, vals)

    # ----------------------------------------------------------- templates
    def record_template(self, step, *args):
        """Runs step(*args) while recording its store creations, views, tasks
        and releases (dfs_template_begin/end) and returns the Template.  The
        step must release everything it creates (its temporaries go out of
        scope when it returns)."""
        B.dfs_template_begin(self.ctx)
        try:
            step(*args)
        except BaseException:
            try:
                B.dfs_template_end(self.ctx)
            except B.DfsError:
                pass
            raise
        return Template(self, B.dfs_template_end(self.ctx))

    # ------------------------------------------------------------- tickets
    def record(self) -> int:
        """A ticket for the work issued so far (dfs_record)."""
        return B.dfs_record(self.ctx)

    def wait(self, ticket: int) -> None:
        B.dfs_wait(self.ctx, ticket)

    def poll(self, ticket: int) -> bool:
        return B.dfs_poll(self.ctx, ticket)

    def elapsed_ms(self, t_from: int, t_to: int) -> float:
        return B.dfs_ticket_elapsed_ms(self.ctx, t_from, t_to)

    def release_ticket(self, ticket: int) -> None:
        B.dfs_ticket_release(self.ctx, ticket)

    # ------------------------------------------------------- graph capture
    def capture_begin(self):
        B.dfs_capture_begin(self.ctx)

    def capture_end(self) -> int:
        return B.dfs_capture_end(self.ctx)

    def graph_launch(self, graph: int):
        B.dfs_graph_launch(self.ctx, graph)

    def graph_destroy(self, graph: int):
        B.dfs_graph_destroy(self.ctx, graph)




class Template:
    """A recorded instance window (Runtime.record_template): replay() issues
    it again with its input stores replaced, in one call."""

    def __init__(self, rt: "Runtime", tid: int):
        self.rt, self.id = rt, tid
        self.inputs = B.dfs_template_inputs(rt.ctx, tid)

    def replay(self, src, dst) -> None:
        """src, dst: arrays (or store handles) pairwise; every input of the
        template must appear in src."""
        h = [a.handle if isinstance(a, Array) else int(a) for a in src]
        g = [a.handle if isinstance(a, Array) else int(a) for a in dst]
        B.dfs_template_replay(self.rt.ctx, self.id, h, g)

    def free(self) -> None:
        if self.id is not None:
            B.dfs_template_free(self.rt.ctx, self.id)
            self.id = None


class ScalarRead:
    """An asynchronous gather of 0-d arrays (Runtime.read_scalars_async): the
    values land in page-locked host memory when the stream reaches the copy.
    The arrays' stores and the buffers stay referenced until values() returns."""

    def __init__(self, rt: "Runtime", arrays, work=None, vals=None):
        n = len(arrays)
        if work is None or len(work) < 2 * n:
            work = Runtime.host_empty((max(1, 2 * n),), np.int64)
        if vals is None or len(vals) < n:
            vals = Runtime.host_empty((max(1, n),), np.float64)
        self.rt, self.n, self.arrays, self.work, self.vals = rt, n, list(arrays), work, vals
        B.dfs_read_scalars_async(rt.ctx, [a.handle for a in self.arrays], work.ctypes.data, vals.ctypes.data)
        self.ticket = B.dfs_record(rt.ctx)

    def done(self) -> bool:
        return self.ticket is None or B.dfs_poll(self.rt.ctx, self.ticket)

    def values(self) -> list:
        """Waits for the gather; the n values as floats."""
        if self.ticket is not None:
            B.dfs_wait(self.rt.ctx, self.ticket)
            B.dfs_ticket_release(self.rt.ctx, self.ticket)
            self.ticket = None
            self.arrays = []
        return [float(v) for v in self.vals[:self.n]]


class Array:
    """A store (or view) handle; operators submit one index task each."""

    __slots__ = ("rt", "handle", "shape", "dtype", "_keep", "__weakref__")
    __array_priority__ = 100

    def __init__(self, rt: Runtime, handle: int, shape, dtype):
        self.rt = rt
        self.handle = handle
        self.shape = shape
        self.dtype = dtype
        self._keep = None

    def __del__(self):
        rt = self.rt
        if self.handle and rt._alive:
            rt._lib_release(rt.ctx, self.handle)
            self.handle = 0

    def release(self):
        rt = self.rt
        if self.handle and rt._alive:
            B.dfs_store_release(rt.ctx, self.handle)
        self.handle = 0

    @property
    def ndim(self):
        return len(self.shape)

    @property
    def size(self):
        return int(np.prod(self.shape)) if self.shape else 1

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
        if idx is Ellipsis:
            idx = ()
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
        return Array(self.rt, h, tuple(shp), self.dtype)

    def __setitem__(self, idx, value):
        view = self[idx]
        _unary(_OP["COPY"], value, view, view)

    # ------------------------------------------------------------ tasking
    def _arg(self, priv):
        _, part = self.rt.layout(self.shape)
        return (self.handle, part, priv)

    def __add__(self, o): return _binary(32, self, o, self)
    def __radd__(self, o): return _binary(32, o, self, self)
    def __sub__(self, o): return _binary(33, self, o, self)
    def __rsub__(self, o): return _binary(33, o, self, self)
    def __mul__(self, o): return _binary(34, self, o, self)
    def __rmul__(self, o): return _binary(34, o, self, self)
    def __truediv__(self, o): return _binary(35, self, o, self)
    def __rtruediv__(self, o): return _binary(35, o, self, self)
    def __pow__(self, o): return _binary(36, self, o, self)
    def __neg__(self): return _unary(2, self, self)

    def __iadd__(self, o): return _binary(32, self, o, self, out=self)
    def __isub__(self, o): return _binary(33, self, o, self, out=self)
    def __imul__(self, o): return _binary(34, self, o, self, out=self)
    def __itruediv__(self, o): return _binary(35, self, o, self, out=self)


def _binary(opcode, a, b, like: Array, out: Array | None = None) -> Array:
    rt = like.rt
    big = a if (a.__class__ is Array and a.shape) else (b if (b.__class__ is Array and b.shape) else like)
    shape = big.shape
    if out is None:
        out = rt._new(shape, like.dtype)
    lay = rt._layouts.get(shape) or rt._make_layout(shape)
    rt._pack(0, a)
    rt._pack(1, b)
    olay = rt._layouts.get(out.shape) or rt._make_layout(out.shape)
    _ARG.pack_into(rt._argbuf, 64, out.handle, olay[1], _W, 0, 0.0)
    rt._issue(opcode, lay, 3)
    return out


def _unary(opcode, a, like: Array, out: Array | None = None) -> Array:
    rt = like.rt
    if out is None:
        out = rt._new(like.shape, like.dtype)
    lay = rt._layouts.get(out.shape) or rt._make_layout(out.shape)
    rt._pack(0, a)
    _ARG.pack_into(rt._argbuf, 32, out.handle, lay[1], _W, 0, 0.0)
    rt._issue(opcode, lay, 2)
    return out


# ------------------------------------------------------------- functions
def exp(x): return _unary(4, x, x)
def log(x): return _unary(5, x, x)
def sqrt(x): return _unary(6, x, x)
def erf(x): return _unary(7, x, x)
def absolute(x): return _unary(3, x, x)
def ncdf(x): return _unary(8, x, x)
def copy(x): return _unary(1, x, x)
def subtract(a, b, out: Array | None = None):
    """a - b, into `out` when given (as numpy.subtract(a, b, out=...))."""
    return _binary(33, a, b, a if isinstance(a, Array) else b, out=out)


def maximum(a, b): return _binary(37, a, b, a if isinstance(a, Array) else b)
def minimum(a, b): return _binary(38, a, b, a if isinstance(a, Array) else b)


def full(rt: Runtime, shape, value: float, dtype=np.float64) -> Array:
    out = rt.empty(shape, dtype)
    return _unary(1, float(value), out, out)


def _reduce(opcode, x: Array, y: Array | None) -> Array:
    rt = x.rt
    out = rt._new((), x.dtype)
    lay = rt._layouts.get(x.shape) or rt._make_layout(x.shape)
    rt._pack(0, x)
    n = 1
    if y is not None:
        rt._pack(1, y)
        n = 2
    _ARG.pack_into(rt._argbuf, 32 * n, out.handle, rt.none, _RD, _SUM, 0.0)
    rt._issue(opcode, lay, n + 1)
    return out


def dot(x: Array, y: Array) -> Array:
    return _reduce(64, x, y)


def asum(x: Array) -> Array:
    return _reduce(65, x, None)


def norm(x: Array) -> Array:
    return sqrt(dot(x, x))


class CSR:
    """CSR matrix (int32 row pointers and columns), the Legate Sparse layout."""

    _win = None    # tile -> window store (staged SpMV), when the runtime stages x
    _host = None   # host copies of (rowptr, col), kept only while staging

    def __init__(self, rt: Runtime, rowptr: np.ndarray, col: np.ndarray, val: np.ndarray, ncols: int | None = None):
        self.rt = rt
        self.nrows = len(rowptr) - 1
        self.ncols = self.nrows if ncols is None else ncols
        self.nnz = len(col)
        self.rowptr = rt.array(np.asarray(rowptr, dtype=np.int32))
        self.col = rt.array(np.asarray(col, dtype=np.int32))
        self.val = rt.array(np.asarray(val))
        self.dtype = self.val.dtype
        # x windows per tile of rows (staged SpMV); the structure is kept on
        # the host to compute them for the tile in use, outside batches,
        # captures and recordings (an upload is not allowed inside them)
        if rt.stage_x:
            self._win = {}
            self._host = (np.asarray(rowptr, dtype=np.int32), np.asarray(col, dtype=np.int32))
            rt._csrs.add(self)
            self.prepare_windows()

    def prepare_windows(self):
        """Computes and uploads the x windows for the runtime's current tile
        of this matrix's rows (no-op when staging is off or they exist)."""
        if self._host is None:
            return
        t = self.rt.tile_1d(self.nrows)
        if t not in self._win:
            rec = B.dfs_spmv_windows(self._host[0], self._host[1], self.ncols, t, self.dtype.itemsize)
            self._win[t] = self.rt.array(rec)

    def __matmul__(self, x: Array) -> Array:
        y = self.rt._new((self.nrows,), self.dtype)
        self.spmv(x, y)
        return y

    def spmv(self, x: Array, y: Array):
        rt = self.rt
        lay = rt._layouts.get(y.shape) or rt._make_layout(y.shape)
        n = rt.none
        _ARG.pack_into(rt._argbuf, 0, self.rowptr.handle, n, _R, 0, 0.0)
        _ARG.pack_into(rt._argbuf, 32, self.col.handle, n, _R, 0, 0.0)
        _ARG.pack_into(rt._argbuf, 64, self.val.handle, n, _R, 0, 0.0)
        _ARG.pack_into(rt._argbuf, 96, x.handle, n, _R, 0, 0.0)
        _ARG.pack_into(rt._argbuf, 128, y.handle, lay[1], _W, 0, 0.0)
        win = self._win.get(rt.tile_1d(self.nrows)) if self._win and y.shape[0] == self.nrows else None
        if win is not None:
            _ARG.pack_into(rt._argbuf, 160, win.handle, rt.tiling((6,)), _R, 0, 0.0)
            rt._issue(96, lay, 6)
        else:
            rt._issue(96, lay, 5)
        return y
