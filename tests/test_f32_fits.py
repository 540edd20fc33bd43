"""The FP32 erf and log of the device templates (dfs_device.cuh) against the
scripts that fit them: the header's coefficients are exactly what the
committed fits print, and the float32 evaluation of those steps, emulated
here with one rounding per fused multiply-add, stays within the stated bounds
(erf 2 ulp, log 1 ulp).  The GPU tests check the same bounds on the device."""
import importlib.util
import pathlib
import re

import numpy as np
import pytest

pytest.importorskip("mpmath")

CSRC = pathlib.Path(__file__).resolve().parents[1] / "paper_2406_18109_gb300" / "csrc"
HEADER = (CSRC / "dfs_device.cuh").read_text()


def _load(name):
    spec = importlib.util.spec_from_file_location(name, CSRC / f"{name}.py")
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _header_literal(name):
    m = re.search(rf"#define {name} (\S+)", HEADER)
    assert m, name
    return m.group(1)


def test_log_coefficients_are_the_fit():
    fit = _load("log_f32_fit")
    c = fit.fit_q()
    assert len(c) == 9
    for k, v in enumerate(c):
        assert fit.literal(v) == _header_literal(f"DFS_LOG_C{k}"), k
    assert fit.literal(fit.LN2_HI) == _header_literal("DFS_LN2_HI")
    assert fit.literal(fit.LN2_LO) == _header_literal("DFS_LN2_LO")
    assert int(_header_literal("DFS_SQRT_HALF_BITS"), 16) == fit.SQRT_HALF_BITS
    # ln2 split: the high part has few enough bits that k * ln2_hi is exact
    # for every exponent a float can have, and hi + lo is ln 2 to 2^-44
    hi = float(fit.LN2_HI)
    assert hi * 2 ** 15 == int(hi * 2 ** 15) and abs(hi + float(fit.LN2_LO) - np.log(2.0)) < 2.0 ** -44


def test_log_emulated_within_one_ulp():
    fit = _load("log_f32_fit")
    c = np.array([float.fromhex(_header_literal(f"DFS_LOG_C{k}")[:-1]) for k in range(9)], np.float32)
    lo, hi = np.float32(0.5).view(np.uint32), np.float32(2.0).view(np.uint32)
    x = np.arange(lo, hi, 7, dtype=np.uint32).view(np.float32)          # every 7th float around 1
    rnd = np.exp(np.random.default_rng(5).uniform(np.log(1.2e-38), np.log(3.4e38), 200_000)).astype(np.float32)
    x = np.concatenate([x, rnd])
    truth = np.log(x.astype(np.float64))
    err = np.abs(fit.emulate(x, c).astype(np.float64) - truth) / fit.ulp32(truth)
    assert err.max() <= 1.0, float(err.max())


def test_erf_coefficients_are_the_fit():
    fit = _load("erf_f32_fit")
    ca, cb = fit.fit_small(), fit.fit_large()
    for k, v in enumerate(ca):
        assert fit.literal(v) == _header_literal(f"DFS_ERF_A{k}"), k
    for k, v in enumerate(cb):
        assert fit.literal(v) == _header_literal(f"DFS_ERF_B{k}"), k


def test_erf_emulated_within_two_ulp():
    fit = _load("erf_f32_fit")
    ca = np.array([float.fromhex(_header_literal(f"DFS_ERF_A{k}")[:-1]) for k in range(7)], np.float32)
    cb = np.array([float.fromhex(_header_literal(f"DFS_ERF_B{k}")[:-1]) for k in range(7)], np.float32)
    for d in (0.0, 2.0, -2.0):                 # the hardware exp2 off by up to 2 ulp either way
        assert fit.emulated_error(ca, cb, d) <= 2.0
