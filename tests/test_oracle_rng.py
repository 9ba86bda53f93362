"""Pins for the oracle's Gaussian test matrices (Sec. 2.2, Algorithm 4 step 3).

The generator itself is pinned by the published Philox4x32-10 known-answer
vectors; the field split by exact integer arithmetic on Python ints; the
bfloat16 rounding by exhaustive comparison with the exact rational rounding
rule; the quantile table by the normal CDF written with math.erfc (a routine
independent of the ndtri the oracle uses).
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import rng

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            rows.append([int(t, 16) for t in line.split()])
    return rows


def test_philox_known_answers():
    rows = _kat_rows()
    assert len(rows) == 3
    for r in rows:
        out = rng.philox4x32_10(*r[:6])
        assert [int(x) for x in out] == r[6:]


def test_philox_vectorised_matches_scalar():
    c = np.arange(50, dtype=np.uint64) * 977
    out = rng.philox4x32_10(c, c + 1, c + 2, c + 3, 123, 456)
    for i in (0, 7, 49):
        one = rng.philox4x32_10(int(c[i]), int(c[i]) + 1, int(c[i]) + 2, int(c[i]) + 3, 123, 456)
        assert [int(o[i]) for o in out] == [int(x) for x in one]


def test_twelve_bit_fields_exact():
    g = np.random.default_rng(5)
    words = g.integers(0, 2**32, size=(4, 64), dtype=np.uint64)
    fields = rng.twelve_bit_fields(*words)
    for col in range(64):
        big = sum(int(words[w, col]) << (32 * w) for w in range(4))
        expect = [(big >> (12 * f)) & 0xFFF for f in range(10)]
        assert fields[col].tolist() == expect


def _bf16_exact(x):
    """Nearest-even rounding to 8 significant bits with exact rationals."""
    fx = Fraction(x)
    if fx == 0:
        return 0.0
    sign = -1 if fx < 0 else 1
    fx = abs(fx)
    e = math.floor(math.log2(fx))
    while Fraction(2) ** e > fx:
        e -= 1
    while Fraction(2) ** (e + 1) <= fx:
        e += 1
    ulp = Fraction(2) ** (e - 7)
    q, r = divmod(fx, ulp)
    if r * 2 > ulp or (r * 2 == ulp and q % 2 == 1):
        q += 1
    return sign * float(q * ulp)


def test_bf16_rounding_against_exact_rule():
    g = np.random.default_rng(7)
    xs = np.concatenate([g.normal(size=2000) * 3,
                         # exact ties: 8 significant bits plus one half ulp
                         np.array([1.0 + 2**-8, 1.0 + 3 * 2**-8, -(2.0 + 2**-7), 3.0 + 2**-7])])
    vals, pats = rng.bf16_round_f64(xs)
    for x, v in zip(xs, vals):
        assert v == _bf16_exact(float(x))
    # bit pattern is the top half of the float32 encoding of the rounded value
    assert np.all((vals.astype(np.float32).view(np.uint32) & 0xFFFF) == 0)
    assert np.all(pats == (vals.astype(np.float32).view(np.uint32) >> 16))


def _phi(x):
    return 0.5 * math.erfc(-x / math.sqrt(2.0))


def test_gaussian_table_is_rounded_quantile():
    t = rng.gaussian_table()
    assert t.shape == (4096,)
    for u in range(4096):
        p = (u + 0.5) / 4096
        q = t[u]
        # the true quantile lies within half a bf16 ulp of q
        e = math.floor(math.log2(abs(q))) if q != 0 else -126
        half_ulp = 2.0 ** (e - 8)
        lo, hi = q - half_ulp * 1.0000001, q + half_ulp * 1.0000001
        assert _phi(lo) <= p <= _phi(hi), u
    # symmetry of the mid-point quantiles
    assert np.array_equal(t, -t[::-1])
    assert np.all(np.diff(t) >= 0)
    # textbook values: Phi^-1(0.975) = 1.95996...; the table entry nearest
    # p = 0.975 is within the bf16 rounding of it
    u = int(round(0.975 * 4096 - 0.5))
    assert abs(t[u] - 1.959964) < 0.01


def test_table_moments():
    t = rng.gaussian_table()
    assert abs(t.mean()) < 1e-12
    assert 0.99 < (t * t).mean() < 1.01


def test_psi_omega_layout_and_subsets():
    P = oracle.psi(23, 37, seed=11)
    assert P.shape == (23, 37)
    rows = np.array([0, 5, 36, 17])
    assert np.array_equal(oracle.psi(23, 37, seed=11, rows=rows), P[:, rows])
    O = oracle.omega(19, 23, seed=11)
    assert O.shape == (19, 23)
    cols = np.array([3, 18])
    assert np.array_equal(oracle.omega(19, 23, seed=11, cols=cols), O[cols])
    # the two streams and different seeds give different matrices
    assert not np.array_equal(P[:, :19], O.T)
    assert not np.array_equal(P, oracle.psi(23, 37, seed=12))
    # widening l only appends rows (counter layout is independent of l)
    assert np.array_equal(oracle.psi(30, 37, seed=11)[:23], P)


def test_psi_entry_from_counter():
    # entry Psi[s, i] is field s%10 of the block at counter (i, 0, s//10, 1)
    P = oracle.psi(30, 40, seed=0x1234_5678_9ABC)
    table = rng.gaussian_table()
    seed = 0x1234_5678_9ABC
    for s, i in [(0, 0), (9, 3), (10, 3), (29, 39), (17, 21)]:
        out = rng.philox4x32_10(i, 0, s // 10, 1, seed & 0xFFFFFFFF, seed >> 32)
        big = sum(int(o) << (32 * w) for w, o in enumerate(out))
        assert P[s, i] == table[(big >> (12 * (s % 10))) & 0xFFF]


def test_gaussian_statistics():
    P = oracle.psi(60, 20000, seed=3)
    x = P.ravel()
    assert abs(x.mean()) < 0.01
    assert abs(x.var() - (rng.gaussian_table() ** 2).mean()) < 0.01
    # Kolmogorov-Smirnov distance to N(0,1), allowing for the 12-bit grid
    xs = np.sort(x)
    emp = np.arange(1, len(xs) + 1) / len(xs)
    cdf = np.array([_phi(v) for v in xs[::97]])
    assert np.max(np.abs(emp[::97] - cdf)) < 0.01
    # neighbouring entries are uncorrelated
    assert abs(np.corrcoef(P[0], P[1])[0, 1]) < 0.05
