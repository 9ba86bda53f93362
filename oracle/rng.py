"""Counter-based Gaussian test matrices for the oracle (FP64, numpy).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library; both sides implement the same published generator
definition independently, so that the oracle draws the same Psi and Omega.

Paper passage: Sec. 2.2 (eq. ``eq:sampmatrix``) and Algorithm 4 draw the
sketching matrices with i.i.d. Gaussian entries and width l = k + p.  The paper
names no generator; the reading adopted here is:

* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
  as 1, 2, 3", SC'11): a 10-round counter-based bijection on four 32-bit words
  keyed by two 32-bit words.
* key = (seed mod 2^32, seed >> 32).
* Psi (l x m), entry Psi[s, i]:   counter = (i mod 2^32, i >> 32, s // 10, 1)
  Omega (n x l), entry Omega[j, s]: counter = (j mod 2^32, j >> 32, s // 10, 2)
* The 128-bit block x0 | x1<<32 | x2<<64 | x3<<96 is cut into ten 12-bit
  fields; field f (bits 12f .. 12f+11) gives the entry with s mod 10 == f.
* A 12-bit field u maps to q[u] = bf16_rn(Phi^-1((u + 0.5) / 4096)), the
  mid-point quantile of the standard normal rounded to nearest-even bfloat16
  directly from FP64.  The result is a discretised Gaussian with tails clipped
  near +-3.6 sigma; every value is exactly representable in bfloat16.

Here Phi^-1 is ``scipy.special.ndtri`` (a library routine used as a step).
"""
from __future__ import annotations

import numpy as np
from scipy.special import ndtri

_MASK32 = np.uint64(0xFFFFFFFF)
# Philox4x32 round multipliers and Weyl key increments (Salmon et al., SC'11).
_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)

STREAM_PSI = 1
STREAM_OMEGA = 2
TABLE_BITS = 12
TABLE_SIZE = 1 << TABLE_BITS
FIELDS_PER_BLOCK = 10


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32 with 10 rounds on arrays of 32-bit words held in uint64.

    Each round: the products M0*c0 and M1*c2 are split into (hi, lo) words and
    the new counter is (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); the key is
    bumped by the Weyl constants between rounds.
    """
    c0, c1, c2, c3 = (np.asarray(x, dtype=np.uint64) & _MASK32 for x in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & _MASK32
    k1 = np.asarray(k1, dtype=np.uint64) & _MASK32
    for rnd in range(10):
        if rnd:
            k0 = (k0 + _W0) & _MASK32
            k1 = (k1 + _W1) & _MASK32
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def twelve_bit_fields(x0, x1, x2, x3):
    """Split each 128-bit block into its ten 12-bit fields -> array [..., 10]."""
    lo = x0 | (x1 << np.uint64(32))
    hi = x2 | (x3 << np.uint64(32))
    m12 = np.uint64(0xFFF)
    out = []
    for f in range(FIELDS_PER_BLOCK):
        b = 12 * f
        if b + 12 <= 64:
            v = (lo >> np.uint64(b)) & m12
        elif b < 64:  # straddles the two 64-bit halves
            nlo = 64 - b
            v = (lo >> np.uint64(b)) | ((hi & np.uint64((1 << (12 - nlo)) - 1)) << np.uint64(nlo))
        else:
            v = (hi >> np.uint64(b - 64)) & m12
        out.append(v)
    return np.stack(out, axis=-1).astype(np.int64)


def bf16_round_f64(x):
    """Round FP64 values to the nearest bfloat16 (ties to even), in one step.

    Returns the rounded values as FP64 and their bfloat16 bit patterns.
    A bfloat16 keeps 8 significant bits, so the 45 low mantissa bits of the
    double are rounded away.  Only finite, normal inputs are expected.
    """
    x = np.asarray(x, dtype=np.float64)
    bits = x.view(np.uint64)
    drop = np.uint64(45)
    lsb = (bits >> drop) & np.uint64(1)
    half = np.uint64((1 << 44) - 1)
    r = (bits + half + lsb) & ~np.uint64((1 << 45) - 1)
    val = r.view(np.float64)
    pattern = (val.astype(np.float32).view(np.uint32) >> np.uint32(16)).astype(np.uint16)
    return val, pattern


def gaussian_table():
    """The 4096 mid-point normal quantiles rounded to bfloat16 (FP64 values)."""
    u = np.arange(TABLE_SIZE, dtype=np.float64)
    q = ndtri((u + 0.5) / TABLE_SIZE)
    val, _ = bf16_round_f64(q)
    return val


def gaussian_table_bits():
    """The same table as bfloat16 bit patterns (uint16)."""
    u = np.arange(TABLE_SIZE, dtype=np.float64)
    _, pat = bf16_round_f64(ndtri((u + 0.5) / TABLE_SIZE))
    return pat


def _gauss(index, width, stream, seed):
    """Matrix G[index_pos, s] for s in [0, width) drawn with the counter layout."""
    index = np.asarray(index, dtype=np.uint64)
    seed = int(seed) & ((1 << 64) - 1)
    k0, k1 = seed & 0xFFFFFFFF, seed >> 32
    nblk = (width + FIELDS_PER_BLOCK - 1) // FIELDS_PER_BLOCK
    table = gaussian_table()
    cols = []
    for sb in range(nblk):
        x = philox4x32_10(index & _MASK32, index >> np.uint64(32),
                          np.full_like(index, sb), np.full_like(index, stream), k0, k1)
        cols.append(table[twelve_bit_fields(*x)])
    g = np.concatenate(cols, axis=-1)[..., :width]
    return np.ascontiguousarray(g, dtype=np.float64)


def psi(l, m, seed, rows=None):
    """Psi (l x m), or only the columns ``rows`` of it (Algorithm 4, transposed)."""
    idx = np.arange(m, dtype=np.uint64) if rows is None else np.asarray(rows, dtype=np.uint64)
    return _gauss(idx, l, STREAM_PSI, seed).T.copy()


def omega(n, l, seed, cols=None):
    """Omega (n x l), or only the rows ``cols`` of it (Algorithm 4 step 3)."""
    idx = np.arange(n, dtype=np.uint64) if cols is None else np.asarray(cols, dtype=np.uint64)
    return _gauss(idx, l, STREAM_OMEGA, seed)
