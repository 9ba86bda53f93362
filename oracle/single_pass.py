"""Single-pass ID (Algorithm 6, Sec. 2.6), FP64, step by step.

TEST INFRASTRUCTURE ONLY (see the package header).

The paper's single-pass ID keeps only the coarse data: the row skeleton of the
coarse matrix is interpolated back to the fine grid instead of being read from
the data a second time (eq. ``eqn:single_ID``).  In this package's column
orientation (A = grid points x snapshots) that reads

    A ~ A_hat = M A_c(:, J_c) P_c,

with (J_c, P_c) the ID of A_c = A(rows_c, :) (Algorithm 5 / ``subsampled_id``)
and M (m x m_c) the coarse-to-fine interpolation operator of Algorithm 6 step
4.  The paper leaves the interpolant open; it discusses piecewise-linear
interpolation (H^2 error) and t coarse points per fine point.  The reading
taken here is trilinear interpolation on the mesh (t = 8):

* per direction, a fine index i lies between the coarse points a = floor(i/s)
  and a + 1 (coarse points are every s-th index from 0, as in ``coarse_rows``);
  the weight of the upper point is the fraction of the physical distance,
  w = (x_i - x_{a s}) / (x_{(a+1) s} - x_{a s});
* a fine index on a coarse point takes that point alone (w = 0);
* past the last coarse point a periodic direction wraps to coarse point 0 at
  x_0 + period; a non-periodic one extrapolates linearly from the last two
  coarse points (w > 1);
* the three directions combine as a tensor product (8 corners), each velocity
  component interpolates its own coarse field.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .interp_decomp import column_id, coarse_rows, spectral_norm


def axis_weights(x, stride, period):
    """(lo, hi, w) per fine index of one direction: the value at fine index i
    is (1 - w) f[lo] + w f[hi], lo/hi being coarse indices."""
    x = np.asarray(x, dtype=np.float64)
    n = len(x)
    c = (n + stride - 1) // stride
    lo = np.zeros(n, dtype=np.int64)
    hi = np.zeros(n, dtype=np.int64)
    w = np.zeros(n)
    for i in range(n):
        a = i // stride
        if i % stride == 0:
            lo[i] = hi[i] = a
        elif a + 1 < c:
            lo[i], hi[i] = a, a + 1
            w[i] = (x[i] - x[a * stride]) / (x[(a + 1) * stride] - x[a * stride])
        elif period > 0:
            lo[i], hi[i] = a, 0
            w[i] = (x[i] - x[a * stride]) / (x[0] + period - x[a * stride])
        elif c >= 2:
            lo[i], hi[i] = c - 2, c - 1
            w[i] = (x[i] - x[(c - 2) * stride]) / (x[(c - 1) * stride] - x[(c - 2) * stride])
        else:
            lo[i] = hi[i] = 0
    return lo, hi, w


def coarse_to_fine(grid, ncomp, stride, coords, periods, rows=None):
    """The interpolation operator M (m x m_c, sparse, 8 entries per row), or
    only its rows ``rows``.

    grid = (nx, ny, nz); coords = (x, y, z) coordinate arrays; periods =
    (px, py, pz), 0 for a non-periodic direction.  Fine row
    r = ((c ny + j) nz + kz) nx + i; coarse row ((c cy + jy) cz + kc) cx + ic,
    the order of ``coarse_rows``.  Entry (r, corner) = fx * fy * fz, the
    product of the one-dimensional weights of ``axis_weights``.
    """
    nx, ny, nz = grid
    sx, sy, sz = stride
    cx, cy, cz = (nx + sx - 1) // sx, (ny + sy - 1) // sy, (nz + sz - 1) // sz
    m, mc = ncomp * nx * ny * nz, ncomp * cx * cy * cz
    r = np.arange(m, dtype=np.int64) if rows is None else np.asarray(rows, dtype=np.int64)
    i = r % nx
    kz = (r // nx) % nz
    j = (r // (nx * nz)) % ny
    c = r // (nx * ny * nz)
    X = axis_weights(coords[0], sx, periods[0])
    Y = axis_weights(coords[1], sy, periods[1])
    Z = axis_weights(coords[2], sz, periods[2])
    cols, vals = [], []
    for by, fy in ((Y[0][j], 1.0 - Y[2][j]), (Y[1][j], Y[2][j])):
        for bz, fz in ((Z[0][kz], 1.0 - Z[2][kz]), (Z[1][kz], Z[2][kz])):
            for bx, fx in ((X[0][i], 1.0 - X[2][i]), (X[1][i], X[2][i])):
                cols.append(((c * cy + by) * cz + bz) * cx + bx)
                vals.append(fx * fy * fz)
    out_rows = np.tile(np.arange(len(r), dtype=np.int64), 8)
    return sp.csr_matrix((np.concatenate(vals), (out_rows, np.concatenate(cols))),
                         shape=(len(r), mc))


def single_pass_id(A, k, grid, ncomp, stride, coords, periods):
    """Algorithm 6 transposed.  Returns (J_c, P_c, k_out, margin, A_c, M, S)
    with S = M A_c(:, J_c) (m x k_out), the interpolated skeleton."""
    rows = coarse_rows(grid, ncomp, stride)
    Ac = np.asarray(A, dtype=np.float64)[rows, :]
    Jc, Pc, kout, margin = column_id(Ac, k)
    M = coarse_to_fine(grid, ncomp, stride, coords, periods)
    S = M @ Ac[:, Jc[:kout]]
    return Jc, Pc, kout, margin, Ac, M, S


def single_pass_error(A, S, Pc):
    """Errors of A_hat = S P_c (S = M A_c(:, J_c)): relative Frobenius and
    maximum entry-wise ratio over A_ij != 0 (the metrics of Sec. 3)."""
    A64 = np.asarray(A, dtype=np.float64)
    Rm = A64 - np.asarray(S, dtype=np.float64) @ np.asarray(Pc, dtype=np.float64)
    rel_fro = np.sqrt(np.sum(Rm * Rm)) / np.sqrt(np.sum(A64 * A64))
    nz = A64 != 0.0
    rel_max = float(np.max(np.abs(Rm[nz]) / np.abs(A64[nz]))) if np.any(nz) else 0.0
    return float(rel_fro), rel_max


def theorem22_bound(A, Ac, M, k):
    """Right side of Theorem 2.2 (column orientation):
    ||E_I||_2 + ||M||_2 sqrt(1 + k (n - k)) sigma_{k+1}(A_c), E_I = A - M A_c.
    Dense SVDs: small matrices only."""
    A64 = np.asarray(A, dtype=np.float64)
    Md = M.toarray() if sp.issparse(M) else np.asarray(M, dtype=np.float64)
    n = A64.shape[1]
    EI = A64 - Md @ Ac
    s = np.linalg.svd(Ac, compute_uv=False)
    sk1 = s[k] if k < len(s) else 0.0
    return spectral_norm(EI) + spectral_norm(Md) * np.sqrt(1.0 + k * (n - k)) * sk1
