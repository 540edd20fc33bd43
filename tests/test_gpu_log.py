"""The FP32 log of the element operation LOG (this library's own
approximation in dfs_device.cuh): within 1 ulp of log evaluated in FP64, the
bound CUDA documents for its logf, over normal and subnormal arguments; the
IEEE results at 0, below 0, inf and NaN; and the two-lane packed evaluation
gives exactly the bits of the scalar one."""
import numpy as np
import pytest

from paper_2406_18109_gb300 import binding as B
from tests.helpers import gpu_runtime

pytestmark = pytest.mark.gpu


def _log_gpu(x, view_offset=0):
    """LOG of x on the GPU; with view_offset the input is a view starting that
    many elements into its store (unaligned, so the body runs one lane per
    thread instead of packed lane pairs)."""
    n = x.size
    with gpu_runtime("persistent", tile=8192) as rt:
        if view_offset:
            base = rt.array(np.concatenate([np.ones(view_offset, np.float32), x]))
            X = base[view_offset:view_offset + n]
        else:
            X = rt.array(x)
        out = rt.array(np.zeros(n, np.float32))
        dom, part = rt.layout((n,))
        rt.submit("LOG", dom, [X._arg(B.DFS_PRIV_R), out._arg(B.DFS_PRIV_W)])
        got = out.numpy()                      # flushes, launches and reads back
        return got, rt.kernel_source()


def _ulp(v):
    v = np.abs(v).astype(np.float32)
    return (np.nextafter(v, np.float32(np.inf)) - v).astype(np.float64)


def _bits(lo, hi, step=1):
    return np.arange(np.float32(lo).view(np.uint32), np.float32(hi).view(np.uint32), step,
                     dtype=np.uint32).view(np.float32)


def test_log_within_one_ulp():
    x = np.concatenate([
        _bits(0.5, 2.0),                                            # every float around 1
        np.arange(0x00800000, 0x7f800000, 251, dtype=np.uint32).view(np.float32),  # all binades
        np.arange(1, 0x00800000, 61, dtype=np.uint32).view(np.float32),            # subnormals
        np.array([1e-45, 1.1754942e-38, 1.17549435e-38, 3.4028235e38, 1.0, 2.0, 0.70710677, 0.7071068,
                  1.4142135, 1.4142137], np.float32)])
    got, src = _log_gpu(x)
    assert "log_f32x2(" in src                        # the lane-pair path ran
    want = np.log(x.astype(np.float64))
    err = np.abs(got.astype(np.float64) - want) / _ulp(want)
    worst = int(np.argmax(err))
    assert err.max() <= 1.0, (float(x[worst]), float(got[worst]), float(want[worst]), float(err.max()))
    assert np.mean(err <= 0.5) > 0.85                 # correctly rounded for most arguments
    assert got[x == 1.0][0] == 0.0 and not np.signbit(got[x == 1.0][0])


def test_log_special_values():
    sp = np.array([0.0, -0.0, -1.0, -1e-40, -np.inf, np.inf, np.nan, 1e-40, 5.0, 1.0], np.float32)
    for off in (0, 1):                                # lane pairs, and one lane per thread
        g, _ = _log_gpu(sp, view_offset=off)
        assert g[0] == -np.inf and g[1] == -np.inf
        assert np.isnan(g[2]) and np.isnan(g[3]) and np.isnan(g[4])
        assert g[5] == np.inf and np.isnan(g[6])
        want7 = np.log(np.float64(sp[7]))
        assert abs(float(g[7]) - want7) <= _ulp(want7)
        assert g[9] == 0.0


def test_lane_pairs_equal_one_lane_bitwise():
    rng = np.random.default_rng(9)
    x = np.concatenate([np.exp(rng.uniform(-80, 80, 1 << 18)).astype(np.float32),
                        rng.uniform(0.5, 2.0, 1 << 16).astype(np.float32),
                        np.array([0.0, -1.0, 1e-40, np.inf, np.nan, 1.0], np.float32)])
    packed, src_p = _log_gpu(x)
    single, src_s = _log_gpu(x, view_offset=1)
    assert "log_f32x2(" in src_p and "log_f32x2(" not in src_s
    assert np.array_equal(packed.view(np.uint32), single.view(np.uint32))
