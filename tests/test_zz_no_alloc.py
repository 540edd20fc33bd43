"""dfs_dot_noalloc -- the dot product for callers that cannot allocate device
memory (stream capture in progress, fixed-budget serving loops, plug-ins of a
framework that owns all allocations) -- checked through the C-ABI against the
runtime's own DOT task on the same device data, on two calls in a row (the
second smaller, so stale scratch from the first call would show up).

Collected last on purpose: a failure here leaves every other test already run.
"""
import pytest

from paper_2406_18109_gb300 import arrays as A
from paper_2406_18109_gb300 import binding as B
from synth import inputs
from tests.helpers import ensure_built, gpu_runtime

pytestmark = pytest.mark.gpu


def _runtime_dot(x_t, y_t) -> float:
    with gpu_runtime("persistent", tile=256) as rt:
        return A.dot(rt.wrap(x_t), rt.wrap(y_t)).item()


def test_noalloc_dot_matches_runtime_dot_twice():
    torch = pytest.importorskip("torch")
    ensure_built()
    dev = torch.device("cuda:0")
    out = torch.zeros(1, dtype=torch.float64, device=dev)   # caller-owned output
    stream = torch.cuda.current_stream().cuda_stream
    for call, n in enumerate((1_000_003, 77_777)):
        x = torch.from_numpy(inputs.uniform(10 + call, -1, 1, n)).to(dev)
        y = torch.from_numpy(inputs.uniform(20 + call, -1, 1, n)).to(dev)
        B.dfs_dot_noalloc(x.data_ptr(), y.data_ptr(), n, out.data_ptr(), stream)
        torch.cuda.synchronize()
        got = float(out.item())
        want = _runtime_dot(x, y)
        scale = float(torch.sum(torch.abs(x * y)).item())
        assert abs(got - want) <= 1e-13 * scale, (call, got, want)
    # a size beyond the fixed scratch is refused before anything is launched
    with pytest.raises(B.DfsError) as e:
        B.dfs_dot_noalloc(x.data_ptr(), y.data_ptr(), B.NOALLOC_MAX_N + 1, out.data_ptr(), stream)
    assert e.value.code == -9
