"""GPU parity of the single-pass ID (Algorithm 6, Sec. 2.6):
A ~ M A_c(:, J_c) P_c, against the oracle's interpolation operator.

Bars: the lifted skeleton S = M A_c(:, J_c) within 1e-6 relative Frobenius
for FP32 data (FP32 interpolation: weights and 8-term sums rounded to FP32)
and 1e-13 for FP64; the errors as for the plain ID error pass
(|e - e_oracle| <= 1e-4 e_oracle for FP32 data, 1e-10 e_oracle for FP64).
"""
import numpy as np
import pytest
import torch

import oracle.single_pass as osp
from oracle import coarse_rows
from synthetic.channel import LX, LZ, channel_field, wall_normal_points

pytestmark = pytest.mark.gpu

DEV = "cuda"


def _sk(**kw):
    from paper_1905_13257_gb300 import IdSketch
    return IdSketch(**kw)


def mesh(grid):
    nx, ny, nz = grid
    return (np.arange(nx) * (LX / nx), wall_normal_points(ny), np.arange(nz) * (LZ / nz)), \
        (LX, 0.0, LZ)


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("dtype,stol,etol", [(torch.float32, 1e-6, 1e-4),
                                              (torch.float64, 1e-13, 1e-10)])
@pytest.mark.parametrize("grid,nc,stride,n,k", [
    ((20, 13, 12), 3, (4, 4, 3), 150, 12),   # ragged tails in y and z; m >= 128: tensor cores (FP32)
    ((9, 7, 5), 2, (2, 3, 2), 40, 6),        # small m: SIMT error pass
    ((16, 12, 16), 3, (4, 4, 4), 300, 40),   # several 256-column tiles
])
def test_single_pass_lift_and_error(dtype, stol, etol, grid, nc, stride, n, k):
    A = channel_field(grid, nc, n, seed=8, dtype=dtype, device=DEV)
    m = A.shape[0]
    sk = _sk(m=m, n_max=n, k=k, l=k + 8, seed=2, dtype=dtype, grid=grid, ncomp=nc,
             coarse_stride=stride, want_coarse=True)
    for j0 in range(0, n, 32):
        sk.stream_columns(A[:, j0:j0 + 32])
    Jc, Pc, kc = sk.coarse_factor()
    coords, per = mesh(grid)
    sk.set_mesh(*coords, per)
    S = sk.single_pass_lift(Jc[:kc], kc)
    fro, mx = sk.single_pass_error(A, Jc[:kc], Pc[:kc])
    An = A.cpu().double().numpy()
    rows = coarse_rows(grid, nc, stride)
    M = osp.coarse_to_fine(grid, nc, stride, coords, per)
    Jn = Jc[:kc].cpu().numpy()
    So = M @ An[rows][:, Jn]
    assert rel(S.cpu().numpy(), So) <= stol
    fo, mo = osp.single_pass_error(An, So, Pc[:kc].cpu().numpy())
    assert abs(fro - fo) <= etol * fo
    assert abs(mx - mo) <= etol * mo
    # two calls in a row give the same numbers (the skeleton buffer is rebuilt)
    assert sk.single_pass_error(A, Jc[:kc], Pc[:kc]) == (fro, mx)
    sk.close()


def test_stride_one_matches_the_plain_error_pass():
    """With coarse stride 1, M = I and A_c = A: the single-pass error equals
    the plain ID error of the same skeleton."""
    grid, nc, n = (16, 8, 16), 3, 96
    A = channel_field(grid, nc, n, seed=9, dtype=torch.float32, device=DEV)
    sk = _sk(m=A.shape[0], n_max=n, k=10, l=20, seed=1, dtype=torch.float32, grid=grid,
             ncomp=nc, coarse_stride=(1, 1, 1), want_coarse=True)
    sk.stream_columns(A)
    Jc, Pc, kc = sk.coarse_factor()
    sk.set_mesh(*mesh(grid)[0], mesh(grid)[1])
    assert torch.equal(sk.single_pass_lift(Jc[:kc], kc), A[:, Jc[:kc].long()])
    a = sk.single_pass_error(A, Jc[:kc], Pc[:kc])
    b = sk.reconstruct_error(A, Jc[:kc], Pc[:kc])
    assert abs(a[0] - b[0]) <= 1e-6 * b[0] and abs(a[1] - b[1]) <= 1e-5 * b[1]
    sk.close()


def test_single_pass_state_and_argument_errors():
    from paper_1905_13257_gb300 import IdError
    grid = (8, 6, 8)
    coords, per = mesh(grid)
    A = channel_field(grid, 3, 20, seed=1, dtype=torch.float32, device=DEV)
    sk = _sk(m=A.shape[0], n_max=20, k=4, l=8, seed=0, dtype=torch.float32)
    with pytest.raises(IdError) as e:   # no coarse grid
        sk.set_mesh(*coords, per)
    assert e.value.status == 2
    sk.close()
    sk = _sk(m=A.shape[0], n_max=20, k=4, l=8, seed=0, dtype=torch.float32, grid=grid, ncomp=3,
             coarse_stride=(2, 2, 2), want_coarse=True)
    sk.stream_columns(A)
    Jc, Pc, kc = sk.coarse_factor()
    with pytest.raises(IdError) as e:   # no mesh yet
        sk.single_pass_lift(Jc[:kc], kc)
    assert e.value.status == 2
    bad = (coords[0][::-1].copy(), coords[1], coords[2])
    with pytest.raises(IdError) as e:   # decreasing coordinates
        sk.set_mesh(*bad, per)
    assert e.value.status == 1
    sk.set_mesh(*coords, per)
    with pytest.raises(IdError) as e:   # J_c outside the streamed columns
        sk.single_pass_lift(torch.tensor([0, 20], dtype=torch.int32), 2)
    assert e.value.status == 1
    sk.close()
