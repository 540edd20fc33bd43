"""ctypes binding of the C-ABI in ``include/diffuse.h`` (argument marshalling only).

Every function keeps the C name and raises :class:`DfsError` on a negative
status.  The shared library is the in-tree ``_lib/libdiffuse.so`` built by
``paper_2406_18109_gb300._build.build()``; importing this module does not
build it, and calling into a missing library raises at once -- there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import json
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libdiffuse.so")

# enums of diffuse.h
DFS_OK = 0
STATUS = {0: "DFS_OK", -1: "DFS_ERR_INVALID", -2: "DFS_ERR_NO_DEVICE", -3: "DFS_ERR_CUDA",
          -4: "DFS_ERR_COMPILE", -5: "DFS_ERR_OOM", -6: "DFS_ERR_BARRIER_TIMEOUT",
          -7: "DFS_ERR_STATE", -8: "DFS_ERR_BUFFER", -9: "DFS_ERR_TOO_LARGE"}
DFS_F32, DFS_F64, DFS_I32, DFS_I64 = 0, 1, 2, 3
DFS_PRIV_R, DFS_PRIV_W, DFS_PRIV_RW, DFS_PRIV_RD, DFS_PRIV_IMM = 1, 2, 3, 4, 8
DFS_REDOP_NONE, DFS_REDOP_SUM = 0, 1
DFS_LAUNCH_PER_TASK, DFS_LAUNCH_PERSISTENT = 0, 1
OPS = {"COPY": 1, "NEG": 2, "ABS": 3, "EXP": 4, "LOG": 5, "SQRT": 6, "ERF": 7, "NCDF": 8,
       "ADD": 32, "SUB": 33, "MUL": 34, "DIV": 35, "POW": 36, "MAX": 37, "MIN": 38,
       "DOT": 64, "SUM": 65, "SPMV": 96}
MAX_DIM = 3

# every symbol include/diffuse.h declares
EXPORTS = ("dfs_config_default", "dfs_init", "dfs_shutdown", "dfs_store_create", "dfs_store_wrap",
           "dfs_store_view", "dfs_store_release", "dfs_store_write", "dfs_store_read",
           "dfs_store_device_ptr", "dfs_partition_none", "dfs_partition_tiling", "dfs_submit",
           "dfs_flush", "dfs_sync", "dfs_last_error", "dfs_plan_json", "dfs_stats_json",
           "dfs_last_kernel_source", "dfs_version", "dfs_dot_noalloc", "dfs_capture_begin",
           "dfs_capture_end", "dfs_graph_launch", "dfs_graph_destroy", "dfs_batch_begin",
           "dfs_batch_next", "dfs_batch_end", "dfs_batch_repeat", "dfs_read_scalars",
           "dfs_set_launch_config", "dfs_store_wrap_host", "dfs_host_alloc", "dfs_host_free",
           "dfs_read_scalars_async", "dfs_record", "dfs_wait", "dfs_poll", "dfs_ticket_elapsed_ms",
           "dfs_ticket_release", "dfs_template_begin", "dfs_template_end", "dfs_template_inputs",
           "dfs_template_replay", "dfs_template_free", "dfs_rowblock_bounds", "dfs_rowblock_sizes",
           "dfs_rowblock_plan", "dfs_spmv_windows")
SPMV_STAGE_BYTES = 53248          # DFS_SPMV_STAGE_BYTES


class dfs_config(C.Structure):
    _fields_ = [("device", C.c_int32), ("fusion", C.c_int32), ("launch_mode", C.c_int32),
                ("window_size", C.c_int32), ("stream", C.c_void_p), ("block_threads", C.c_int32),
                ("ctas_per_sm", C.c_int32), ("unroll", C.c_int32), ("barrier_timeout_s", C.c_double),
                ("cache_dir", C.c_char_p), ("debug_skip_arrival", C.c_int32), ("time_launches", C.c_int32),
                ("window_growth", C.c_int32), ("window_max", C.c_int32)]


class dfs_arg(C.Structure):
    _fields_ = [("store", C.c_int64), ("partition", C.c_int64), ("privilege", C.c_int32),
                ("redop", C.c_int32), ("imm", C.c_double)]


class dfs_rowblock_sizes_t(C.Structure):
    _fields_ = [("row_lo", C.c_int64), ("row_hi", C.c_int64), ("nnz", C.c_int64), ("n_halo", C.c_int64),
                ("n_send", C.c_int64)]


class DfsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        self.code = code
        super().__init__(f"{STATUS.get(code, code)}: {msg}")


_lib = None


def lib():
    """The loaded shared library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run paper_2406_18109_gb300._build.build() first")
        L = C.CDLL(LIB_PATH)
        P, I64, I32 = C.c_void_p, C.c_int64, C.c_int32
        pI64 = C.POINTER(C.c_int64)
        sig = {
            "dfs_config_default": (None, [C.POINTER(dfs_config)]),
            "dfs_init": (C.c_int, [C.POINTER(P), C.POINTER(dfs_config)]),
            "dfs_shutdown": (C.c_int, [P]),
            "dfs_store_create": (C.c_int, [P, I32, I32, pI64, pI64]),
            "dfs_store_wrap": (C.c_int, [P, I32, I32, pI64, P, pI64]),
            "dfs_store_view": (C.c_int, [P, I64, pI64, pI64, pI64]),
            "dfs_store_release": (C.c_int, [P, I64]),
            "dfs_store_write": (C.c_int, [P, I64, P, C.c_size_t]),
            "dfs_store_read": (C.c_int, [P, I64, P, C.c_size_t]),
            "dfs_store_device_ptr": (C.c_int, [P, I64, C.POINTER(P)]),
            "dfs_partition_none": (C.c_int, [P, pI64]),
            "dfs_partition_tiling": (C.c_int, [P, I32, pI64, pI64, C.POINTER(C.c_int32), pI64]),
            "dfs_submit": (C.c_int, [P, I32, I32, pI64, I32, C.POINTER(dfs_arg)]),
            "dfs_flush": (C.c_int, [P]),
            "dfs_sync": (C.c_int, [P]),
            "dfs_last_error": (C.c_char_p, [P]),
            "dfs_plan_json": (C.c_int, [P, C.c_char_p, C.c_size_t, C.POINTER(C.c_size_t)]),
            "dfs_stats_json": (C.c_int, [P, C.c_char_p, C.c_size_t, C.POINTER(C.c_size_t)]),
            "dfs_last_kernel_source": (C.c_int, [P, C.c_char_p, C.c_size_t, C.POINTER(C.c_size_t)]),
            "dfs_version": (C.c_int, []),
            "dfs_dot_noalloc": (C.c_int, [P, P, I64, P, P]),
            "dfs_capture_begin": (C.c_int, [P]),
            "dfs_capture_end": (C.c_int, [P, pI64]),
            "dfs_graph_launch": (C.c_int, [P, I64]),
            "dfs_graph_destroy": (C.c_int, [P, I64]),
            "dfs_batch_begin": (C.c_int, [P]),
            "dfs_batch_next": (C.c_int, [P]),
            "dfs_batch_end": (C.c_int, [P]),
            "dfs_batch_repeat": (C.c_int, [P, I32]),
            "dfs_read_scalars": (C.c_int, [P, I32, pI64, C.POINTER(C.c_double)]),
            "dfs_set_launch_config": (C.c_int, [P, I32, I32, I32]),
            "dfs_store_wrap_host": (C.c_int, [P, I32, I32, pI64, P, pI64]),
            "dfs_host_alloc": (C.c_int, [C.c_size_t, C.POINTER(P)]),
            "dfs_host_free": (C.c_int, [P]),
            "dfs_read_scalars_async": (C.c_int, [P, I32, pI64, P, P]),
            "dfs_record": (C.c_int, [P, C.POINTER(C.c_uint64)]),
            "dfs_wait": (C.c_int, [P, C.c_uint64]),
            "dfs_poll": (C.c_int, [P, C.c_uint64, C.POINTER(C.c_int32)]),
            "dfs_ticket_elapsed_ms": (C.c_int, [P, C.c_uint64, C.c_uint64, C.POINTER(C.c_float)]),
            "dfs_ticket_release": (C.c_int, [P, C.c_uint64]),
            "dfs_template_begin": (C.c_int, [P]),
            "dfs_template_end": (C.c_int, [P, C.POINTER(C.c_uint64)]),
            "dfs_template_inputs": (C.c_int, [P, C.c_uint64, I32, pI64, C.POINTER(C.c_int32)]),
            "dfs_template_replay": (C.c_int, [P, C.c_uint64, I32, pI64, pI64]),
            "dfs_template_free": (C.c_int, [P, C.c_uint64]),
            "dfs_rowblock_bounds": (C.c_int, [I64, I32, I32, pI64, pI64]),
            "dfs_rowblock_sizes": (C.c_int, [P, P, I64, I32, I32, C.POINTER(dfs_rowblock_sizes_t)]),
            "dfs_rowblock_plan": (C.c_int, [P, P, I64, I32, I32, P, P, P, P, P, P]),
            "dfs_spmv_windows": (C.c_int, [P, P, I64, I64, I64, I32, I64, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(ctx, rc: int):
    if rc != DFS_OK:
        msg = lib().dfs_last_error(ctx).decode() if ctx else ""
        raise DfsError(rc, msg)


def _i64s(vals):
    vals = list(vals)
    return (C.c_int64 * max(1, len(vals)))(*vals)


# ------------------------------------------------------------------ C names
def dfs_config_default() -> dfs_config:
    cfg = dfs_config()
    lib().dfs_config_default(C.byref(cfg))
    return cfg


def dfs_init(cfg: dfs_config | None = None):
    ctx = C.c_void_p()
    rc = lib().dfs_init(C.byref(ctx), C.byref(cfg) if cfg is not None else None)
    if rc != DFS_OK:
        raise DfsError(rc, "dfs_init failed")
    return ctx


def dfs_shutdown(ctx) -> None:
    _check(None, lib().dfs_shutdown(ctx))


def dfs_store_create(ctx, dtype: int, shape) -> int:
    out = C.c_int64()
    _check(ctx, lib().dfs_store_create(ctx, dtype, len(shape), _i64s(shape), C.byref(out)))
    return out.value


def dfs_store_wrap(ctx, dtype: int, shape, dev_ptr: int) -> int:
    out = C.c_int64()
    _check(ctx, lib().dfs_store_wrap(ctx, dtype, len(shape), _i64s(shape), C.c_void_p(dev_ptr), C.byref(out)))
    return out.value


def dfs_store_view(ctx, parent: int, offset, shape) -> int:
    out = C.c_int64()
    _check(ctx, lib().dfs_store_view(ctx, parent, _i64s(offset), _i64s(shape), C.byref(out)))
    return out.value


def dfs_store_release(ctx, store: int) -> None:
    _check(ctx, lib().dfs_store_release(ctx, store))


def dfs_store_write(ctx, store: int, host_ptr: int, nbytes: int) -> None:
    _check(ctx, lib().dfs_store_write(ctx, store, C.c_void_p(host_ptr), nbytes))


def dfs_store_read(ctx, store: int, host_ptr: int, nbytes: int) -> None:
    _check(ctx, lib().dfs_store_read(ctx, store, C.c_void_p(host_ptr), nbytes))


def dfs_store_device_ptr(ctx, store: int) -> int:
    out = C.c_void_p()
    _check(ctx, lib().dfs_store_device_ptr(ctx, store, C.byref(out)))
    return out.value or 0


def dfs_partition_none(ctx) -> int:
    out = C.c_int64()
    _check(ctx, lib().dfs_partition_none(ctx, C.byref(out)))
    return out.value


def dfs_partition_tiling(ctx, tile, offset=None, proj=None) -> int:
    out = C.c_int64()
    nd = len(tile)
    off = _i64s(offset if offset is not None else [0] * nd)
    pj = (C.c_int32 * nd)(*proj) if proj is not None else None
    _check(ctx, lib().dfs_partition_tiling(ctx, nd, _i64s(tile), off, pj, C.byref(out)))
    return out.value


def make_args(args) -> C.Array:
    """args: list of (store, partition, privilege[, redop]) tuples or floats (immediates)."""
    arr = (dfs_arg * len(args))()
    for i, a in enumerate(args):
        if isinstance(a, (int, float)) and not isinstance(a, bool) and not isinstance(a, tuple):
            arr[i].privilege = DFS_PRIV_IMM
            arr[i].imm = float(a)
        else:
            arr[i].store = a[0]
            arr[i].partition = a[1]
            arr[i].privilege = a[2]
            arr[i].redop = a[3] if len(a) > 3 else (DFS_REDOP_SUM if a[2] == DFS_PRIV_RD else DFS_REDOP_NONE)
    return arr


def dfs_submit(ctx, op, domain, args) -> None:
    opc = OPS[op] if isinstance(op, str) else int(op)
    arr = make_args(args)
    _check(ctx, lib().dfs_submit(ctx, opc, len(domain), _i64s(domain), len(args), arr))


def dfs_flush(ctx) -> None:
    _check(ctx, lib().dfs_flush(ctx))


def dfs_sync(ctx) -> None:
    _check(ctx, lib().dfs_sync(ctx))


def dfs_last_error(ctx) -> str:
    return lib().dfs_last_error(ctx).decode()


def _json_call(fn, ctx) -> str:
    need = C.c_size_t(0)
    fn(ctx, None, 0, C.byref(need))
    buf = C.create_string_buffer(need.value + 1)
    _check(ctx, fn(ctx, buf, need.value + 1, C.byref(need)))
    return buf.value.decode()


def dfs_plan_json(ctx) -> dict:
    return json.loads(_json_call(lib().dfs_plan_json, ctx))


def dfs_stats_json(ctx) -> dict:
    return json.loads(_json_call(lib().dfs_stats_json, ctx))


def dfs_last_kernel_source(ctx) -> str:
    return _json_call(lib().dfs_last_kernel_source, ctx)


def dfs_capture_begin(ctx) -> None:
    _check(ctx, lib().dfs_capture_begin(ctx))


def dfs_capture_end(ctx) -> int:
    out = C.c_int64()
    _check(ctx, lib().dfs_capture_end(ctx, C.byref(out)))
    return out.value


def dfs_graph_launch(ctx, graph: int) -> None:
    _check(ctx, lib().dfs_graph_launch(ctx, graph))


def dfs_graph_destroy(ctx, graph: int) -> None:
    _check(ctx, lib().dfs_graph_destroy(ctx, graph))


def dfs_batch_begin(ctx) -> None:
    _check(ctx, lib().dfs_batch_begin(ctx))


def dfs_batch_next(ctx) -> None:
    _check(ctx, lib().dfs_batch_next(ctx))


def dfs_batch_end(ctx) -> None:
    _check(ctx, lib().dfs_batch_end(ctx))


def dfs_batch_repeat(ctx, n: int) -> None:
    _check(ctx, lib().dfs_batch_repeat(ctx, n))


def dfs_read_scalars(ctx, stores, out=None):
    """Values of the 0-d stores `stores` as a list of floats (or written into
    `out`, a C double array of at least len(stores) elements)."""
    n = len(stores)
    hs = _i64s(stores)
    buf = out if out is not None else (C.c_double * max(1, n))()
    _check(ctx, lib().dfs_read_scalars(ctx, n, hs, buf))
    return buf[:n]


def dfs_read_scalars_async(ctx, stores, host_work: int, host_vals: int) -> None:
    """Enqueues the gather of the 0-d `stores` into page-locked host memory
    (addresses host_work: 2 int64 per store, host_vals: 1 double per store)."""
    _check(ctx, lib().dfs_read_scalars_async(ctx, len(stores), _i64s(stores), host_work, host_vals))


def dfs_record(ctx) -> int:
    t = C.c_uint64()
    _check(ctx, lib().dfs_record(ctx, C.byref(t)))
    return t.value


def dfs_wait(ctx, ticket: int) -> None:
    _check(ctx, lib().dfs_wait(ctx, ticket))


def dfs_poll(ctx, ticket: int) -> bool:
    done = C.c_int32()
    _check(ctx, lib().dfs_poll(ctx, ticket, C.byref(done)))
    return bool(done.value)


def dfs_ticket_elapsed_ms(ctx, t_from: int, t_to: int) -> float:
    ms = C.c_float()
    _check(ctx, lib().dfs_ticket_elapsed_ms(ctx, t_from, t_to, C.byref(ms)))
    return float(ms.value)


def dfs_ticket_release(ctx, ticket: int) -> None:
    _check(ctx, lib().dfs_ticket_release(ctx, ticket))


def dfs_template_begin(ctx) -> None:
    _check(ctx, lib().dfs_template_begin(ctx))


def dfs_template_end(ctx) -> int:
    t = C.c_uint64()
    _check(ctx, lib().dfs_template_end(ctx, C.byref(t)))
    return t.value


def dfs_template_inputs(ctx, tid: int) -> list:
    n = C.c_int32()
    _check(ctx, lib().dfs_template_inputs(ctx, tid, 0, None, C.byref(n)))
    out = (C.c_int64 * max(1, n.value))()
    _check(ctx, lib().dfs_template_inputs(ctx, tid, n.value, out, C.byref(n)))
    return list(out[:n.value])


def dfs_template_replay(ctx, tid: int, src, dst) -> None:
    _check(ctx, lib().dfs_template_replay(ctx, tid, len(src), _i64s(src), _i64s(dst)))


def dfs_template_free(ctx, tid: int) -> None:
    _check(ctx, lib().dfs_template_free(ctx, tid))


def dfs_set_launch_config(ctx, block_threads: int, unroll: int, ctas_per_sm: int) -> None:
    _check(ctx, lib().dfs_set_launch_config(ctx, block_threads, unroll, ctas_per_sm))


def dfs_store_wrap_host(ctx, dtype: int, shape, host_ptr: int) -> int:
    out = C.c_int64()
    _check(ctx, lib().dfs_store_wrap_host(ctx, dtype, len(shape), _i64s(shape), C.c_void_p(host_ptr), C.byref(out)))
    return out.value


def dfs_host_alloc(nbytes: int) -> int:
    out = C.c_void_p()
    _check(None, lib().dfs_host_alloc(nbytes, C.byref(out)))
    return out.value or 0


def dfs_host_free(ptr: int) -> None:
    _check(None, lib().dfs_host_free(C.c_void_p(ptr)))


def dfs_version() -> int:
    return lib().dfs_version()


NOALLOC_TILE = 4096
NOALLOC_MAX_N = 16384 * NOALLOC_TILE


def dfs_dot_noalloc(x_ptr: int, y_ptr: int, n: int, out_ptr: int, stream: int = 0) -> None:
    """Dot product of two device vectors into a device double, allocating nothing."""
    rc = lib().dfs_dot_noalloc(C.c_void_p(x_ptr), C.c_void_p(y_ptr), n, C.c_void_p(out_ptr),
                               C.c_void_p(stream) if stream else None)
    if rc != DFS_OK:
        raise DfsError(rc, "dfs_dot_noalloc failed")


def dfs_rowblock_bounds(n: int, nranks: int, rank: int):
    """(lo, hi): the global rows rank `rank` of `nranks` owns out of n."""
    lo, hi = C.c_int64(), C.c_int64()
    _check(None, lib().dfs_rowblock_bounds(n, nranks, rank, C.byref(lo), C.byref(hi)))
    return lo.value, hi.value


def dfs_rowblock_plan(rowptr, col, nranks: int, rank: int) -> dict:
    """Rank `rank`'s row-block plan of a square int32 CSR matrix: a dict of
    row_lo, row_hi, local_rowptr, local_col, halo_cols, recv_counts, send_idx,
    send_counts (numpy arrays; see dfs_rowblock_plan in diffuse.h)."""
    import numpy as np
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    n = len(rowptr) - 1
    sz = dfs_rowblock_sizes_t()
    L = lib()
    _check(None, L.dfs_rowblock_sizes(rowptr.ctypes.data, col.ctypes.data, n, nranks, rank, C.byref(sz)))
    n_own = sz.row_hi - sz.row_lo
    out = {"row_lo": sz.row_lo, "row_hi": sz.row_hi,
           "local_rowptr": np.empty(n_own + 1, np.int32), "local_col": np.empty(sz.nnz, np.int32),
           "halo_cols": np.empty(sz.n_halo, np.int64), "recv_counts": np.empty(nranks, np.int64),
           "send_idx": np.empty(sz.n_send, np.int32), "send_counts": np.empty(nranks, np.int64)}
    _check(None, L.dfs_rowblock_plan(rowptr.ctypes.data, col.ctypes.data, n, nranks, rank,
                                     out["local_rowptr"].ctypes.data, out["local_col"].ctypes.data,
                                     out["halo_cols"].ctypes.data, out["recv_counts"].ctypes.data,
                                     out["send_idx"].ctypes.data, out["send_counts"].ctypes.data))
    return out


def dfs_spmv_windows(rowptr, col, ncols: int, tile: int, elem_bytes: int, budget_bytes: int = SPMV_STAGE_BYTES):
    """The x windows of every SpMV point (tiles of `tile` rows) of a CSR
    matrix: an int32 array of 6 entries per point (see dfs_spmv_windows in
    diffuse.h)."""
    import numpy as np
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    nrows = len(rowptr) - 1
    out = np.zeros(6 * max(1, -(-nrows // tile) if tile > 0 else 1), np.int32)   # the C call checks tile
    _check(None, lib().dfs_spmv_windows(rowptr.ctypes.data, col.ctypes.data, nrows, ncols, tile, elem_bytes,
                                        budget_bytes, out.ctypes.data))
    return out
