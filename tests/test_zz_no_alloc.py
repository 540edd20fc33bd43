"""dfs_dot_noalloc -- the dot product for callers that cannot allocate device
memory: serving loops that reserve all their memory at start-up (a later
cudaMalloc could block, synchronise the device or fail under the budget) and
plug-ins whose host framework owns every allocation.

Checked through the C-ABI on two calls in a row (the second smaller, so stale
partials left in the shared scratch by the first call would show up):
  * against the runtime's own DOT task on the same device data;
  * against an exactly summed reference (math.fsum of the products), which
    shares nothing with the device code;
  * the same inputs twice give the same bits (fixed summation order);
  * n == 0 writes 0.0; a size beyond the fixed scratch is refused.

Collected last on purpose: a failure here leaves every other test already run.
"""
import math

import numpy as np
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
        xh = inputs.uniform(10 + call, -1, 1, n)
        yh = inputs.uniform(20 + call, -1, 1, n)
        x = torch.from_numpy(xh).to(dev)
        y = torch.from_numpy(yh).to(dev)
        B.dfs_dot_noalloc(x.data_ptr(), y.data_ptr(), n, out.data_ptr(), stream)
        torch.cuda.synchronize()
        got = float(out.item())
        # the sum of n products can cancel, so the error is measured against
        # sum |x_i y_i| (the condition of the sum), not |x . y|
        scale = math.fsum(np.abs(xh * yh))
        exact = math.fsum(xh * yh)
        assert abs(got - exact) <= 1e-13 * scale, (call, got, exact)
        want = _runtime_dot(x, y)
        assert abs(got - want) <= 1e-13 * scale, (call, got, want)
        # a repeat on the same inputs gives the same bits
        B.dfs_dot_noalloc(x.data_ptr(), y.data_ptr(), n, out.data_ptr(), stream)
        torch.cuda.synchronize()
        assert np.float64(out.item()).view(np.uint64) == np.float64(got).view(np.uint64)
    # n == 0 writes 0.0 into the output (set to NaN first)
    out.fill_(float("nan"))
    B.dfs_dot_noalloc(x.data_ptr(), y.data_ptr(), 0, out.data_ptr(), stream)
    torch.cuda.synchronize()
    assert float(out.item()) == 0.0
    # a size beyond the fixed scratch is refused before anything is launched
    with pytest.raises(B.DfsError) as e:
        B.dfs_dot_noalloc(x.data_ptr(), y.data_ptr(), B.NOALLOC_MAX_N + 1, out.data_ptr(), stream)
    assert e.value.code == -9
