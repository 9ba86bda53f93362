"""FP8-E4M3 precision form of the sketch products (oracle; test
infrastructure only, used by tests/ alone).

The build's reading of the precision form "sketch GEMMs in FP8-E4M3 with
per-column scales": every column c of A is scaled by the power of two 2^e_c
that brings its largest magnitude as close to the largest E4M3 value (448)
as possible without passing it, each entry is rounded to the nearest E4M3
value (ties to even), and the sketches are the products of the dequantised
matrix A_q(:, c) = e4m3(A(:, c) 2^e_c) 2^-e_c with Psi and Omega in exact
arithmetic.  Psi and Omega keep their bfloat16 quantile values.

E4M3 (the OCP 8-bit format with 4 exponent bits, bias 7, 3 mantissa bits, no
infinities): normal values 1.f x 2^E for E = -6..8 up to 448 = 1.75 x 2^8,
subnormal values m/8 x 2^-6 for m = 1..7.
"""
import numpy as np

E4M3_MAX = 448.0
E4M3_MIN_NORMAL = 2.0 ** -6
E4M3_SUBNORMAL_QUANTUM = 2.0 ** -9
EXP_CLAMP = 100   # the scales' exponents are kept in [-100, 100]


def e4m3_round(x):
    """x (float64 array) rounded to the nearest E4M3 value, ties to even,
    saturating at +-448 (finite inputs)."""
    x = np.asarray(x, dtype=np.float64)
    ax = np.abs(x)
    out = np.empty_like(x)
    sub = ax < E4M3_MIN_NORMAL
    # subnormal range: a fixed grid of 2^-9 (np.rint rounds half to even)
    out[sub] = np.rint(x[sub] / E4M3_SUBNORMAL_QUANTUM) * E4M3_SUBNORMAL_QUANTUM
    # normal range: 4 significant bits (1 implicit + 3 stored)
    m, p = np.frexp(x[~sub])                 # x = m 2^p, 0.5 <= |m| < 1
    out[~sub] = np.ldexp(np.rint(m * 16.0) / 16.0, p)
    return np.clip(out, -E4M3_MAX, E4M3_MAX)


def column_exponents(A):
    """e_c: the largest integer with max_r |A(r, c)| 2^e_c <= 448 (0 for a
    zero column), clamped to [-100, 100]."""
    A = np.asarray(A, dtype=np.float64)
    mx = np.max(np.abs(A), axis=0) if A.shape[0] else np.zeros(A.shape[1])
    e = np.zeros(A.shape[1], dtype=np.int64)
    for c, v in enumerate(mx):
        if v == 0.0:
            continue
        f, p = np.frexp(v)                   # v = f 2^p, 0.5 <= f < 1
        ec = 9 - int(p) if f <= 0.875 else 8 - int(p)
        while np.ldexp(v, ec) > E4M3_MAX:
            ec -= 1
        while np.ldexp(v, ec + 1) <= E4M3_MAX:
            ec += 1
        e[c] = min(EXP_CLAMP, max(-EXP_CLAMP, ec))
    return e


def quantize_columns(A):
    """A_q = e4m3(A 2^e) 2^-e column by column, and the exponents e."""
    A = np.asarray(A, dtype=np.float64)
    e = column_exponents(A)
    Aq = np.ldexp(e4m3_round(np.ldexp(A, e[None, :])), -e[None, :])
    return Aq, e
