"""Pins of the FP8-E4M3 precision form's oracle (oracle/fp8.py) against the
format's own definition: every E4M3 value decoded from its 8-bit code (sign,
4 exponent bits with bias 7, 3 mantissa bits, subnormals at exponent 0, no
infinities, S.1111.111 NaN), brute-force nearest-value rounding with ties to
the even code, saturation at 448, and the per-column exponent rule checked
by its defining inequalities."""
import numpy as np
import pytest

from oracle import fp8


def e4m3_table():
    """(value, code) of every finite E4M3 code, decoded from the bits."""
    out = []
    for code in range(256):
        s, e, m = code >> 7, (code >> 3) & 0xF, code & 7
        if e == 15 and m == 7:
            continue                                  # NaN
        v = (m / 8.0) * 2.0 ** -6 if e == 0 else (1.0 + m / 8.0) * 2.0 ** (e - 7)
        out.append((-v if s else v, code))
    return out


def nearest_even(x, table):
    """Brute force: the table value nearest to x; on a tie the one whose code
    has an even mantissa field; beyond the largest value, the largest."""
    vals = np.array([v for v, _ in table])
    codes = np.array([c for _, c in table])
    d = np.abs(vals - x)
    best = np.flatnonzero(d == d.min())
    if len(best) > 1:
        even = [i for i in best if (codes[i] & 1) == 0]
        best = even
    return vals[best[0]]


def test_table_extremes():
    vals = sorted({v for v, _ in e4m3_table()})
    assert vals[-1] == 448.0 and vals[0] == -448.0
    assert min(v for v in vals if v > 0) == 2.0 ** -9
    assert len([v for v in vals if v > 0]) == 126


def test_every_value_is_a_fixed_point():
    vals = np.array([v for v, _ in e4m3_table()])
    assert np.array_equal(fp8.e4m3_round(vals), vals)


def test_midpoints_round_to_even_code():
    table = e4m3_table()
    pos = sorted({v for v, _ in table if v >= 0})
    mids = [(a + b) / 2 for a, b in zip(pos[:-1], pos[1:])]
    for x in mids + [-x for x in mids]:
        assert fp8.e4m3_round(np.array([x]))[0] == nearest_even(x, table), x


def test_random_values_and_saturation():
    rng = np.random.default_rng(5)
    x = np.exp(rng.uniform(np.log(2.0 ** -13), np.log(600.0), 3000)) * rng.choice([-1, 1], 3000)
    x = np.concatenate([x, [0.0, -0.0, 448.0, 460.0, 480.0, 1e6, -1e6, 2.0 ** -10, 3 * 2.0 ** -11]])
    table = e4m3_table()
    got = fp8.e4m3_round(x)
    want = np.array([nearest_even(v, table) for v in x])
    assert np.array_equal(got, want)


def test_column_exponents_defining_inequalities():
    rng = np.random.default_rng(6)
    A = rng.standard_normal((300, 40)) * np.exp(rng.uniform(-30, 30, 40))[None, :]
    A[:, 3] = 0.0
    A[:, 4] = 448.0
    A[:, 5] = 448.0000001
    e = fp8.column_exponents(A)
    mx = np.max(np.abs(A), axis=0)
    for c in range(A.shape[1]):
        if mx[c] == 0.0:
            assert e[c] == 0
            continue
        assert np.ldexp(mx[c], e[c]) <= 448.0 < np.ldexp(mx[c], e[c] + 1)
    assert e[4] == 0 and e[5] == -1


@pytest.mark.parametrize("seed", [1, 2])
def test_quantized_columns_error_bound(seed):
    """Every entry in E4M3's normal range is within 2^-4 relative of A
    (half a unit of 3 mantissa bits); the column maximum maps into
    (224, 448]; quantised entries stay as they are under the same scales."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((500, 30)) * np.exp(rng.uniform(-8, 8, 30))[None, :]
    Aq, e = fp8.quantize_columns(A)
    xs = np.ldexp(A, e[None, :])
    normal = np.abs(xs) >= 2.0 ** -6
    rel = np.abs(Aq - A)[normal] / np.abs(A)[normal]
    assert rel.max() <= 2.0 ** -4
    top = np.max(np.abs(xs), axis=0)
    assert np.all((top > 224.0) & (top <= 448.0))
    again = np.ldexp(fp8.e4m3_round(np.ldexp(Aq, e[None, :])), -e[None, :])
    assert np.array_equal(again, Aq)
