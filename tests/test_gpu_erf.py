"""The FP32 erf of the element operations ERF and NCDF (this library's own
approximation in dfs_device.cuh): within 2 ulp of erf evaluated in FP64, the
bound CUDA documents for its erff; odd bit for bit; and the two-lane packed
evaluation gives exactly the bits of the scalar one."""
import numpy as np
import pytest
from scipy import special

from paper_2406_18109_gb300 import binding as B
from tests.helpers import gpu_runtime

pytestmark = pytest.mark.gpu


def _erf_gpu(x, view_offset=0):
    """ERF of x on the GPU; with view_offset the input is a view starting that
    many elements into its store (unaligned, so the body runs one lane per
    thread instead of packed lane pairs)."""
    n = x.size
    with gpu_runtime("persistent", tile=8192) as rt:
        if view_offset:
            base = rt.array(np.concatenate([np.zeros(view_offset, np.float32), x]))
            X = base[view_offset:view_offset + n]
        else:
            X = rt.array(x)
        out = rt.array(np.zeros(n, np.float32))
        dom, part = rt.layout((n,))
        rt.submit("ERF", dom, [X._arg(B.DFS_PRIV_R), out._arg(B.DFS_PRIV_W)])
        got = out.numpy()                      # flushes, launches and reads back
        return got, rt.kernel_source()


def _ulp(v):
    v = np.abs(v).astype(np.float32)
    return (np.nextafter(v, np.float32(np.inf)) - v).astype(np.float64)


def test_erf_within_two_ulp():
    hi = np.float32(4.2).view(np.uint32)
    grid = np.arange(0, hi, 64, dtype=np.uint32).view(np.float32)           # every 64th float in [0, 4.2]
    dense = np.concatenate([np.arange(np.float32(0.95).view(np.uint32), np.float32(1.05).view(np.uint32),
                                      dtype=np.uint32).view(np.float32),
                            np.arange(np.float32(3.9).view(np.uint32), np.float32(3.94).view(np.uint32),
                                      dtype=np.uint32).view(np.float32)])
    rnd = np.random.default_rng(7).uniform(0, 5, 1 << 20).astype(np.float32)
    x = np.concatenate([grid, dense, rnd, np.array([0.0, 1e-45, 1e-38, 1e-20, 0.5, 1.0, 3.92, 10.0, 1e30,
                                                    np.inf], np.float32)])
    got, src = _erf_gpu(x)
    assert "erf_mag2(" in src                         # the lane-pair path ran
    want = special.erf(x.astype(np.float64))
    err = np.abs(got.astype(np.float64) - want) / _ulp(want)
    worst = int(np.argmax(err))
    assert err.max() <= 2.0, (float(x[worst]), float(got[worst]), float(want[worst]), float(err.max()))
    assert np.mean(err <= 0.5) > 0.7                  # correctly rounded for most arguments
    # special values and the odd extension, bit for bit
    sp = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1e-40, -1e-40, 2.0, -2.0, 0.3, -0.3], np.float32)
    g, _ = _erf_gpu(sp)
    assert g[0] == 0 and np.signbit(g[1]) and g[1] == 0 and g[2] == 1 and g[3] == -1 and np.isnan(g[4])
    assert np.array_equal(g[5::2].view(np.uint32) ^ np.uint32(0x80000000), g[6::2].view(np.uint32))


def test_lane_pairs_equal_one_lane_bitwise():
    x = np.concatenate([np.random.default_rng(8).uniform(-5, 5, 1 << 18).astype(np.float32),
                        np.array([0.0, -0.0, 1.0, -1.0, 3.92, np.inf, np.nan], np.float32)])
    packed, src_p = _erf_gpu(x)
    single, src_s = _erf_gpu(x, view_offset=1)
    assert "erf_mag2(" in src_p and "erf_mag2(" not in src_s
    assert np.array_equal(packed.view(np.uint32), single.view(np.uint32))
