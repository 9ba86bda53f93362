"""Pins of the single-pass ID oracle (Algorithm 6, Sec. 2.6) against what the
mathematics fixes: the interpolation operator M reproduces what trilinear
interpolation must reproduce, matches an independent trilinear fit, converges
like H^2 on smooth data, and the single-pass error obeys Theorem 2.2."""

import numpy as np
import pytest

import oracle.single_pass as osp
from oracle import coarse_rows, subsampled_id, recon_error
from synthetic.channel import LX, LZ, wall_normal_points, channel_field

GRID, NC, STRIDE = (12, 9, 8), 2, (4, 4, 3)   # ragged: 9 % 4 and 8 % 3 leave a tail


def mesh(grid):
    nx, ny, nz = grid
    x = np.arange(nx) * (LX / nx)
    z = np.arange(nz) * (LZ / nz)
    return (x, wall_normal_points(ny), z), (LX, 0.0, LZ)


def fine_points(grid, ncomp):
    nx, ny, nz = grid
    coords, _ = mesh(grid)
    c, j, kz, i = np.meshgrid(np.arange(ncomp), np.arange(ny), np.arange(nz), np.arange(nx),
                              indexing="ij")
    return (c.ravel(), coords[0][i.ravel()], coords[1][j.ravel()], coords[2][kz.ravel()],
            i.ravel(), kz.ravel())


def test_rows_sum_to_one_and_coarse_points_are_injected():
    coords, per = mesh(GRID)
    M = osp.coarse_to_fine(GRID, NC, STRIDE, coords, per)
    assert np.allclose(M @ np.ones(M.shape[1]), 1.0, atol=1e-14, rtol=0)
    rows = coarse_rows(GRID, NC, STRIDE)
    Mc = M[rows].toarray()
    assert np.array_equal(Mc, np.eye(len(rows)))


def test_trilinear_fields_are_reproduced():
    """A product of linear functions of the coordinates is reproduced exactly
    wherever no periodic wrap is involved, including the linear extrapolation
    past the last coarse y-plane."""
    coords, per = mesh(GRID)
    M = osp.coarse_to_fine(GRID, NC, STRIDE, coords, per)
    c, x, y, z, i, kz = fine_points(GRID, NC)
    f = (1.0 + 0.3 * x) * (2.0 - y) * (3.0 + 0.7 * z) * (1.0 + c)
    rows = coarse_rows(GRID, NC, STRIDE)
    g = M @ f[rows]
    nx, ny, nz = GRID
    last_x = ((nx - 1) // STRIDE[0]) * STRIDE[0]
    last_z = ((nz - 1) // STRIDE[2]) * STRIDE[2]
    inside = (i <= last_x) & (kz <= last_z)
    assert inside.sum() > 0 and (~inside).sum() > 0
    assert np.max(np.abs(g[inside] - f[inside])) <= 1e-12 * np.max(np.abs(f))
    # y alone (constant in x, z): exact everywhere, wrap cells included
    fy = 1.5 - 0.25 * y
    assert np.max(np.abs(M @ fy[rows] - fy)) <= 1e-13


def test_rows_match_an_independent_trilinear_fit():
    """Each fine point's value equals the trilinear polynomial through its
    eight corner values, found by solving the 8 x 8 system (no weights)."""
    coords, per = mesh(GRID)
    M = osp.coarse_to_fine(GRID, NC, STRIDE, coords, per).tocsr()
    rng = np.random.default_rng(3)
    fc = rng.standard_normal(M.shape[1])
    g = M @ fc
    nx, ny, nz = GRID
    sx, sy, sz = STRIDE
    cx, cy, cz = -(-nx // sx), -(-ny // sy), -(-nz // sz)
    x, y, z = coords

    def corners(idx, n, s, c, xs, period):
        a = idx // s
        if a + 1 < c:
            return [a, a + 1], [xs[a * s], xs[(a + 1) * s]]
        if period > 0:
            return [a, 0], [xs[a * s], xs[0] + period]
        return [c - 2, c - 1], [xs[(c - 2) * s], xs[(c - 1) * s]]

    for r in rng.choice(M.shape[0], size=40, replace=False):
        comp, rem = divmod(r, nx * ny * nz)
        j, rem = divmod(rem, nz * nx)
        kk, i = divmod(rem, nx)
        ix, px = corners(i, nx, sx, cx, x, per[0])
        iy, py = corners(j, ny, sy, cy, y, per[1])
        iz, pz = corners(kk, nz, sz, cz, z, per[2])
        rows_sys, rhs = [], []
        for a in range(2):
            for b in range(2):
                for d in range(2):
                    X, Y, Z = px[a], py[b], pz[d]
                    rows_sys.append([1, X, Y, Z, X * Y, X * Z, Y * Z, X * Y * Z])
                    rhs.append(fc[((comp * cy + iy[b]) * cz + iz[d]) * cx + ix[a]])
        coef = np.linalg.solve(np.array(rows_sys), np.array(rhs))
        X, Y, Z = x[i], y[j], z[kk]
        val = coef @ np.array([1, X, Y, Z, X * Y, X * Z, Y * Z, X * Y * Z])
        assert abs(val - g[r]) <= 1e-9 * max(1.0, abs(val))


def test_interpolation_error_converges_like_h_squared():
    """On a smooth field the interpolation error drops about 4x when the
    coarse spacing halves (the H^2 behaviour the paper cites)."""
    grid = (64, 33, 32)
    coords, per = mesh(grid)
    c, x, y, z, _, _ = fine_points(grid, 1)
    f = np.sin(2 * np.pi * x / LX) * np.cos(2 * np.pi * z / LZ) * np.cos(1.3 * y)
    errs = []
    for s in (2, 4, 8):
        st = (s, s, s)
        M = osp.coarse_to_fine(grid, 1, st, coords, per)
        rows = coarse_rows(grid, 1, st)
        errs.append(np.linalg.norm(M @ f[rows] - f))
    r1, r2 = errs[1] / errs[0], errs[2] / errs[1]
    assert 3.0 < r1 < 5.0 and 3.0 < r2 < 5.0, (errs, r1, r2)


def test_stride_one_reduces_to_subsampled_id():
    grid, nc = (8, 6, 8), 2
    A = channel_field(grid, nc, 40, seed=1).double().numpy()
    coords, per = mesh(grid)
    Jc, Pc, kout, _, Ac, M, S = osp.single_pass_id(A, 6, grid, nc, (1, 1, 1), coords, per)
    Js, Ps, ks, _, _ = subsampled_id(A, 6, grid, nc, (1, 1, 1))
    assert np.array_equal(Jc, Js) and kout == ks
    assert np.array_equal(S, A[:, Jc[:kout]])
    assert np.allclose(osp.single_pass_error(A, S, Pc), recon_error(A, Jc[:kout], Pc), rtol=1e-12)


@pytest.mark.parametrize("k", [3, 8])
def test_theorem_2_2_bound(k):
    grid, nc, st = (16, 9, 12), 2, (4, 4, 3)
    A = channel_field(grid, nc, 30, seed=2).double().numpy()
    coords, per = mesh(grid)
    Jc, Pc, kout, _, Ac, M, S = osp.single_pass_id(A, k, grid, nc, st, coords, per)
    Ahat = S @ Pc
    lhs = np.linalg.norm(A - Ahat, 2)
    assert lhs <= osp.theorem22_bound(A, Ac, M, k) * (1 + 1e-12)
    # and the single-pass error is at least the interpolation error's share:
    # A_hat lies in range(M), so ||A - A_hat|| >= ||(I - proj_M) A||
    Q, _ = np.linalg.qr(M.toarray())
    assert lhs >= np.linalg.norm(A - Q @ (Q.T @ A), 2) * (1 - 1e-12)


def test_planted_mistake_swapped_weights_is_caught(monkeypatch):
    orig = osp.axis_weights

    def swapped(x, stride, period):
        lo, hi, w = orig(x, stride, period)
        return lo, hi, np.where(w != 0, 1.0 - w, w)

    monkeypatch.setattr(osp, "axis_weights", swapped)
    with pytest.raises(AssertionError):
        test_trilinear_fields_are_reproduced()


def test_theorem22_bound_hand_computed_value():
    """Right side of Theorem 2.2 on a 3 x 3 example worked by hand (two-sided
    pin).  A_c = [[3, 0, 0], [0, 1, 0]] (singular values 3, 1; k = 1 gives
    sigma_2 = 1); M = [[1, 0], [0, 1], [1/2, 1/2]] has M^T M = [[5/4, 1/4],
    [1/4, 5/4]] with eigenvalues 3/2 and 1, so ||M||_2 = sqrt(3/2); A = M A_c
    + E with E zero except E[2, 2] = 2, so ||E_I||_2 = 2; n = 3 snapshots, so
    sqrt(1 + k (n - k)) = sqrt(3).  Bound: 2 + sqrt(3/2) sqrt(3) = 2 +
    sqrt(9/2)."""
    Ac = np.array([[3.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    M = np.array([[1.0, 0.0], [0.0, 1.0], [0.5, 0.5]])
    E = np.zeros((3, 3))
    E[2, 2] = 2.0
    A = M @ Ac + E
    b = osp.theorem22_bound(A, Ac, M, 1)
    assert abs(b - (2.0 + np.sqrt(4.5))) <= 1e-12
    assert abs(b - 4.121320343559643) <= 1e-12
    # k = 2 = rank(A_c): sigma_3 = 0 and the bound is the interpolation error
    assert abs(osp.theorem22_bound(A, Ac, M, 2) - 2.0) <= 1e-12
