"""Shared helpers of the test-suite."""
import os
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "diffuse.h")

_built = False


def ensure_built():
    """Builds the shared library once per session (no-op when up to date)."""
    global _built
    if not _built:
        from paper_2406_18109_gb300 import _build
        _build.build()
        _built = True


def kernel_cache_dir() -> str:
    d = os.path.join(tempfile.gettempdir(), "dfs_test_cubins")
    os.makedirs(d, exist_ok=True)
    return d


def gpu_runtime(mode: str = "persistent", **kw):
    """A device context: mode is persistent (fused, one kernel per flush),
    per_task (fused, one kernel per fused task) or unfused."""
    from paper_2406_18109_gb300 import arrays as A
    ensure_built()
    if mode == "unfused":
        return A.Runtime(device=0, fusion=False, launch="per_task", cache_dir=kernel_cache_dir(), **kw)
    return A.Runtime(device=0, fusion=True, launch=mode, cache_dir=kernel_cache_dir(), **kw)


MODES = ("persistent", "per_task", "unfused")
