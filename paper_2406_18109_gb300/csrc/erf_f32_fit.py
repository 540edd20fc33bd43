"""Fits the coefficients of the FP32 erf in dfs_device.cuh (erf_mag, erf_mag2)
and reports the error of its float32 evaluation.  Run on the build host (it
needs mpmath); it prints the DFS_ERF_A* and DFS_ERF_B* literals.

The approximation, written from the mathematics:
  x < 1:         erf(x) = x + x q(x^2)   q: degree 6 in t = x^2, fitted to
                                          erf(x)/x - 1, relative weights
  1 <= x < 3.92: erf(x) = 1 - 2^p(x)     p: degree 6 in x, fitted to
                                          log2 erfc(x), weighted by erfc(x)
                                          (the absolute error that reaches erf)
  x >= 3.92:     1                        (erfc(x) < 2^-25)
Fits are weighted least squares on Chebyshev nodes against 40-digit values.
The evaluation is emulated in float32 (each fused multiply-add rounded once)
with the hardware exp2 off by 0 or +-2 ulp, and compared with erf in FP64 over
a dense grid of [0, 4.2].
"""
import numpy as np
import mpmath as mp
from scipy import special

mp.mp.dps = 40
F32 = np.float32


def cheb(a, b, n):
    k = np.arange(n)
    return 0.5 * (a + b) + 0.5 * (b - a) * np.cos((2 * k + 1) * np.pi / (2 * n))


def fit_small(split=1.0, deg=6):
    t = cheb(0.0, split * split, 800)
    x = np.sqrt(t)
    ratio = np.array([float(mp.erf(mp.mpf(v)) / mp.mpf(v)) for v in x])
    V = np.vander(t, deg + 1, increasing=True)
    c, *_ = np.linalg.lstsq(V / ratio[:, None], (ratio - 1) / ratio, rcond=None)
    return c.astype(F32)


def fit_large(split=1.0, top=3.92, deg=6):
    x = cheb(split, top, 1200)
    q = np.array([float(mp.log(mp.erfc(mp.mpf(v)), 2)) for v in x])
    w = np.array([float(mp.erfc(mp.mpf(v))) for v in x])
    V = np.vander(x, deg + 1, increasing=True)
    c, *_ = np.linalg.lstsq(V * w[:, None], q * w, rcond=None)
    return c.astype(F32)


def fma32(a, b, c):
    return (np.asarray(a, np.float64) * np.asarray(b, np.float64) + np.asarray(c, np.float64)).astype(F32)


def horner(c, z):
    p = np.full(z.shape, c[-1], F32)
    for k in range(len(c) - 2, -1, -1):
        p = fma32(p, z, np.full(z.shape, c[k], F32))
    return p


def ulp32(v):
    v = np.abs(v).astype(F32)
    return (np.nextafter(v, F32(np.inf)) - v).astype(np.float64)


def emulated_error(ca, cb, exp2_ulp=0.0):
    xs = np.unique(np.concatenate([np.linspace(0, 4.2, 4_000_001).astype(F32),
                                   np.linspace(0.95, 1.3, 400_001).astype(F32)]))
    t = (xs.astype(np.float64) ** 2).astype(F32)
    ra = fma32(xs, horner(ca, t), xs)
    e = np.exp2(horner(cb, xs).astype(np.float64)).astype(F32)
    e = (e.astype(np.float64) * (1 + exp2_ulp * 2.0 ** -23)).astype(F32)
    rb = (1.0 - e.astype(np.float64)).astype(F32)
    r = np.where(xs < F32(1.0), ra, np.where(xs < F32(3.92), rb, F32(1))).astype(F32)
    truth = special.erf(xs.astype(np.float64))
    return float((np.abs(r.astype(np.float64) - truth) / ulp32(truth)).max())


def literal(c):
    return float(c).hex().replace("0000000p", "p") + "f"


if __name__ == "__main__":
    ca, cb = fit_small(), fit_large()
    for k, c in enumerate(ca):
        print(f"#define DFS_ERF_A{k} {literal(c)}")
    for k, c in enumerate(cb):
        print(f"#define DFS_ERF_B{k} {literal(c)}")
    for d in (0.0, 2.0, -2.0):
        print(f"exp2 off by {d:+.0f} ulp: worst error {emulated_error(ca, cb, d):.2f} ulp")
