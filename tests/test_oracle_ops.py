"""Pins of the oracle's element operations and of the Black-Scholes pricing
(CPU only).

The task bodies are the array libraries' operators (Section 2, Fig. 1e;
Section 6, Fig. 8a).  Each operation is pinned here by values a reader can
check by hand -- chosen so that a swapped operand order (POW, SUB, DIV), a
swapped pair of operations (MAX/MIN), a dropped sign (ABS, NEG) or a missing
rounding to the stored dtype fails -- and ERF by a printed table.

Black-Scholes (the Section 7.1 benchmark; the paper prints no formula) is
pinned by the closed form evaluated in 50-digit arithmetic, written out in
this file, on options that span moneyness and expiry: put-call parity holds
for any d1, d2, so it cannot catch a mistake in them, while these values do.
"""
import math
import os

import numpy as np
import pytest

from oracle import ops, programs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
F32 = np.float32
F64 = np.float64


def _val(x):
    return np.asarray(x).item()


# ------------------------------------------------------- hand-known values
# (op, operands, exact result) -- every result is exact in float32 and float64
EXACT = [
    ("COPY", (3.5,), 3.5),
    ("NEG", (2.25,), -2.25),
    ("NEG", (-7.0,), 7.0),
    ("ABS", (-3.5,), 3.5),
    ("ABS", (2.0,), 2.0),
    ("EXP", (0.0,), 1.0),
    ("LOG", (1.0,), 0.0),
    ("SQRT", (16.0,), 4.0),
    ("SQRT", (0.25,), 0.5),
    ("ERF", (0.0,), 0.0),
    ("NCDF", (0.0,), 0.5),
    ("ADD", (2.0, 3.0), 5.0),
    ("SUB", (5.0, 3.0), 2.0),
    ("SUB", (3.0, 5.0), -2.0),
    ("MUL", (4.0, 2.5), 10.0),
    ("DIV", (6.0, 3.0), 2.0),
    ("DIV", (3.0, 6.0), 0.5),
    ("POW", (2.0, 3.0), 8.0),           # x ** y, not y ** x (3 ** 2 = 9)
    ("POW", (3.0, 2.0), 9.0),
    ("POW", (4.0, 0.5), 2.0),
    ("POW", (2.0, -2.0), 0.25),
    ("POW", (-2.0, 3.0), -8.0),
    ("MAX", (-1.0, 2.0), 2.0),
    ("MAX", (2.0, -1.0), 2.0),
    ("MAX", (-3.0, -7.0), -3.0),
    ("MIN", (-1.0, 2.0), -1.0),
    ("MIN", (2.0, -1.0), -1.0),
    ("MIN", (-3.0, -7.0), -7.0),
]


@pytest.mark.parametrize("dt", [F64, F32])
@pytest.mark.parametrize("op,args,want", EXACT)
def test_exact_values(op, args, want, dt):
    got = ops.unary(op, args[0], dt) if len(args) == 1 else ops.binary(op, args[0], args[1], dt)
    assert np.asarray(got).dtype == dt
    assert _val(got) == want, (op, args, _val(got), want)


def test_abs_and_neg_signs_of_zero():
    # ABS clears the sign bit; NEG flips it (IEEE 754 abs / negate)
    assert math.copysign(1.0, _val(ops.unary("ABS", -0.0, F64))) == 1.0
    assert math.copysign(1.0, _val(ops.unary("NEG", 0.0, F64))) == -1.0
    assert math.copysign(1.0, _val(ops.unary("NEG", -0.0, F32))) == 1.0


def test_elementwise_on_arrays_and_scalar_broadcast():
    x = np.array([1.0, 2.0, 3.0, -4.0])
    # an immediate on either side of a non-commutative operation
    assert ops.binary("POW", x[:3], 2.0, F64).tolist() == [1.0, 4.0, 9.0]
    assert ops.binary("POW", 2.0, x[:3], F64).tolist() == [2.0, 4.0, 8.0]
    assert ops.binary("SUB", 10.0, x, F64).tolist() == [9.0, 8.0, 7.0, 14.0]
    assert ops.binary("DIV", x, 2.0, F64).tolist() == [0.5, 1.0, 1.5, -2.0]
    assert ops.binary("MAX", x, 2.0, F64).tolist() == [2.0, 2.0, 3.0, 2.0]
    assert ops.binary("MIN", x, 2.0, F64).tolist() == [1.0, 2.0, 2.0, -4.0]
    assert ops.unary("ABS", x, F64).tolist() == [1.0, 2.0, 3.0, 4.0]


def test_transcendental_values():
    # e, ln 8 = 3 ln 2, sqrt 2 and 2^(1/2): correctly rounded binary64 values
    assert abs(_val(ops.unary("EXP", 1.0, F64)) - 2.718281828459045) <= 4.5e-16
    assert abs(_val(ops.unary("LOG", 8.0, F64)) - 2.0794415416798357) <= 4.5e-16
    assert abs(_val(ops.unary("SQRT", 2.0, F64)) - 1.4142135623730951) <= 2.3e-16
    assert _val(ops.binary("POW", 2.0, 0.5, F64)) == _val(ops.unary("SQRT", 2.0, F64))
    assert _val(ops.unary("LOG", ops.unary("EXP", 3.0, F64), F64)) == 3.0


def test_stored_dtype_rounds_every_step():
    # float32 has 24 significant bits: 1 + 2^-24 rounds (ties to even) to 1,
    # while float64 keeps it
    tiny = 2.0 ** -24
    assert _val(ops.binary("ADD", 1.0, tiny, F32)) == 1.0
    assert _val(ops.binary("ADD", 1.0, tiny, F64)) == 1.0 + tiny
    # (1 + 2^-12)^2 = 1 + 2^-11 + 2^-24: the last term is half an ulp of
    # float32 at 1 and the tie goes to the even neighbour 1 + 2^-11
    a = 1.0 + 2.0 ** -12
    assert _val(ops.binary("MUL", a, a, F32)) == 1.0 + 2.0 ** -11
    assert _val(ops.binary("MUL", a, a, F64)) == 1.0 + 2.0 ** -11 + 2.0 ** -24
    # 1/3 in float32 is 11184811 * 2^-25
    assert _val(ops.binary("DIV", 1.0, 3.0, F32)) == 11184811 * 2.0 ** -25


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def test_erf_table():
    rows = _golden("erf_table.txt")
    assert len(rows) >= 5
    for _, x, want in rows:
        x, want = float(x), float(want)
        assert abs(_val(ops.unary("ERF", x, F64)) - want) <= 1e-15, x
        # odd function
        assert _val(ops.unary("ERF", -x, F64)) == -_val(ops.unary("ERF", x, F64))
        assert abs(_val(ops.unary("ERF", x, F32)) - want) <= 2.0 ** -23
    assert _val(ops.unary("ERF", np.inf, F64)) == 1.0
    assert _val(ops.unary("ERF", -np.inf, F64)) == -1.0


def test_ncdf_is_written_through_erf():
    # N(x) = (1 + erf(x / sqrt 2)) / 2: N(sqrt 2) = (1 + erf 1) / 2 from the table
    erf1 = float([r for r in _golden("erf_table.txt") if float(r[1]) == 1.0][0][2])
    assert abs(_val(ops.unary("NCDF", math.sqrt(2.0), F64)) - 0.5 * (1 + erf1)) <= 2e-15
    assert abs(_val(ops.unary("NCDF", -math.sqrt(2.0), F64)) - 0.5 * (1 - erf1)) <= 2e-15


# ----------------------------------------------- Black-Scholes closed form
# (S, K, T, r, sigma): deep out of and in the money, at the money, short and
# long expiries across the benchmark's ranges (S in [5, 30], K in [1, 100],
# T in [0.25, 10]) and a few other rates and volatilities
OPTIONS = [
    (5.0, 100.0, 0.25, 0.02, 0.3),
    (30.0, 1.0, 10.0, 0.02, 0.3),
    (17.0, 17.0, 1.0, 0.02, 0.3),
    (20.0, 25.0, 0.25, 0.02, 0.3),
    (25.0, 20.0, 0.5, 0.02, 0.3),
    (12.0, 50.0, 10.0, 0.02, 0.3),
    (28.0, 60.0, 5.0, 0.03, 0.5),
    (8.0, 7.5, 7.5, 0.01, 0.15),
    (10.0, 12.0, 2.0, 0.05, 0.2),
    (42.0, 40.0, 0.5, 0.10, 0.2),
    (100.0, 95.0, 3.0, 0.04, 0.25),
    (6.0, 5.0, 0.3, 0.0, 0.4),
]


def _bs_closed_form(S, K, T, r, sigma):
    """European call and put from the Black-Scholes-Merton formulas in
    50-digit arithmetic: d1 = (ln(S/K) + (r + sigma^2/2) T) / (sigma sqrt T),
    d2 = d1 - sigma sqrt T, N(x) = (1 + erf(x / sqrt 2)) / 2,
    call = S N(d1) - K e^{-rT} N(d2), put = K e^{-rT} N(-d2) - S N(-d1)."""
    mp = pytest.importorskip("mpmath")
    with mp.workdps(50):
        S, K, T, r, sigma = (mp.mpf(v) for v in (S, K, T, r, sigma))
        vol = sigma * mp.sqrt(T)
        d1 = (mp.log(S / K) + (r + sigma ** 2 / 2) * T) / vol
        d2 = d1 - vol
        N = lambda x: (1 + mp.erf(x / mp.sqrt(2))) / 2
        kd = K * mp.exp(-r * T)
        return float(S * N(d1) - kd * N(d2)), float(kd * N(-d2) - S * N(-d1))


@pytest.mark.parametrize("S,K,T,r,sigma", OPTIONS)
def test_black_scholes_fp64_against_50_digit_closed_form(S, K, T, r, sigma):
    want_c, want_p = _bs_closed_form(S, K, T, r, sigma)
    c, p = programs.black_scholes(np.array([S]), np.array([K]), np.array([T]), r, sigma, F64)
    tol = 1e-12 * (S + K)
    assert abs(c[0] - want_c) <= tol, (c[0], want_c)
    assert abs(p[0] - want_p) <= tol, (p[0], want_p)


@pytest.mark.parametrize("S,K,T,r,sigma", OPTIONS)
def test_black_scholes_stored_dtype_against_closed_form(S, K, T, r, sigma):
    # the float32 chain of 23 rounded steps stays within 1e-5 (S + K)
    want_c, want_p = _bs_closed_form(S, K, T, r, sigma)
    c, p = programs.black_scholes(np.array([S]), np.array([K]), np.array([T]), r, sigma, F32)
    assert c.dtype == F32
    assert abs(float(c[0]) - want_c) <= 1e-5 * (S + K)
    assert abs(float(p[0]) - want_p) <= 1e-5 * (S + K)


def test_closed_form_matches_the_printed_worked_example():
    # the 50-digit closed form of this file reproduces the textbook's printed
    # prices (tests/golden/black_scholes_textbook.txt), so it is itself pinned
    for row in _golden("black_scholes_textbook.txt"):
        if row[0] != "option":
            continue
        _, S, K, r, sig, T, c, p, dec = row
        want_c, want_p = _bs_closed_form(float(S), float(K), float(T), float(r), float(sig))
        assert round(want_c, int(dec)) == float(c) and round(want_p, int(dec)) == float(p)
