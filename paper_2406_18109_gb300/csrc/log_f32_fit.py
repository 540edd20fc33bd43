"""Fits the coefficients of the FP32 log in dfs_device.cuh (log_f32,
log_f32x2) and reports the error of its float32 evaluation.  Run on the build
host (it needs mpmath); it prints the DFS_LOG_C* literals.

The approximation, written from the mathematics:
  a = 2^k m, m in [sqrt(1/2), sqrt(2)) taken from the bits of a
  f = m - 1 (exact), log(m) = f + f^2 Q(f)
      Q: degree 8 in f, fitted to (log1p(f) - f) / f^2, weighted by |f|
         (an error dQ moves log(m) by f^2 dQ, about |f| dQ relative to log(m))
  log(a) = k ln2_hi + (k ln2_lo + log(m)), ln2_hi with 15 significant bits so
  that k ln2_hi is exact for every k a float can have
The fit is weighted least squares on Chebyshev nodes against 40-digit values.
The evaluation is emulated in float32 (each fused multiply-add rounded once)
over every float in [1/16, 16) and 4 M random normal floats, and compared
with log in FP64.
"""
import numpy as np
import mpmath as mp

mp.mp.dps = 40
F32 = np.float32
SQRT_HALF_BITS = 0x3f3504f3
LN2_HI = F32(0.693145751953125)
LN2_LO = F32(np.log(2.0) - 0.693145751953125)


def cheb(a, b, n):
    k = np.arange(n)
    return 0.5 * (a + b) + 0.5 * (b - a) * np.cos((2 * k + 1) * np.pi / (2 * n))


def fit_q(deg=8, nodes=2000):
    m0 = float(np.uint32(SQRT_HALF_BITS).view(F32))
    f = cheb(m0 - 1, 2 * m0 - 1, nodes)
    q = np.array([float((mp.log1p(mp.mpf(v)) - mp.mpf(v)) / mp.mpf(v) ** 2) for v in f])
    w = np.abs(f)
    V = np.vander(f, deg + 1, increasing=True)
    c, *_ = np.linalg.lstsq(V * w[:, None], q * w, rcond=None)
    return c.astype(F32)


def fma32(a, b, c):
    return (np.asarray(a, np.float64) * np.asarray(b, np.float64) + np.asarray(c, np.float64)).astype(F32)


def ulp32(v):
    v = np.abs(v).astype(F32)
    return (np.nextafter(v, F32(np.inf)) - v).astype(np.float64)


def emulate(x, c):
    """The steps of log_f32 for positive normal float32 x."""
    d = x.view(np.int32).astype(np.int64) - SQRT_HALF_BITS
    kf = (d >> 23).astype(F32)
    m = ((d & 0x7fffff) + SQRT_HALF_BITS).astype(np.uint32).view(F32)
    f = (m.astype(np.float64) - 1.0).astype(F32)
    ff = (f.astype(np.float64) ** 2).astype(F32)
    q = np.full(x.shape, c[-1], F32)
    for j in range(len(c) - 2, -1, -1):
        q = fma32(q, f, c[j])
    return fma32(kf, LN2_HI, fma32(kf, LN2_LO, fma32(ff, q, f)))


def worst_error(c):
    worst, at = 0.0, None
    for e in range(-4, 4):
        bits = np.arange(F32(2.0 ** e).view(np.uint32), F32(2.0 ** (e + 1)).view(np.uint32), dtype=np.uint32)
        for part in np.array_split(bits, 4):
            x = part.view(F32)
            truth = np.log(x.astype(np.float64))
            err = np.abs(emulate(x, c).astype(np.float64) - truth) / ulp32(truth)
            i = int(np.argmax(err))
            if err[i] > worst:
                worst, at = float(err[i]), float(x[i])
    rnd = np.exp(np.random.default_rng(1).uniform(np.log(1.2e-38), np.log(3.4e38), 4_000_000)).astype(F32)
    truth = np.log(rnd.astype(np.float64))
    wide = float((np.abs(emulate(rnd, c).astype(np.float64) - truth) / ulp32(truth)).max())
    return worst, at, wide


def literal(c):
    return float(c).hex().replace("0000000p", "p") + "f"


if __name__ == "__main__":
    c = fit_q()
    for k, v in enumerate(c):
        print(f"#define DFS_LOG_C{k} {literal(v)}")
    print(f"#define DFS_LN2_HI {literal(LN2_HI)}")
    print(f"#define DFS_LN2_LO {literal(LN2_LO)}")
    worst, at, wide = worst_error(c)
    print(f"every float in [1/16, 16): worst error {worst:.2f} ulp (at {at!r}); random normal floats: {wide:.2f} ulp")
