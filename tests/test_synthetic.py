"""The seeded channel-field generator: structure the tests rely on."""
import numpy as np
import torch

from synthetic import channel_field, factors, wall_normal_points


def test_clean_field_is_rank_le_128_and_unit_rms():
    A = channel_field((16, 8, 16), 3, 300, seed=1, noise=0.0, dtype=torch.float64).numpy()
    assert A.shape == (3 * 16 * 8 * 16, 300)
    assert abs(np.sqrt(np.mean(A * A)) - 1.0) < 1e-9
    s = np.linalg.svd(A, compute_uv=False)
    assert s[128] < 1e-10 * s[0]
    assert s[60] > 1e-3 * s[0]          # rich spectrum: k = 50 is not at the noise floor


def test_layout_and_walls():
    grid = (8, 6, 4)
    S, T = factors(grid, 3, 10, seed=0)
    A = (S @ T).numpy()
    nx, ny, nz = grid
    # wall rows (j = 0 and ny-1) vanish for every component
    for c in range(3):
        for j in (0, ny - 1):
            r0 = ((c * ny + j) * nz) * nx
            assert np.allclose(A[r0:r0 + nz * nx], 0.0, atol=1e-12)
    y = wall_normal_points(ny)
    assert y[0] == -1.0 and y[-1] == 1.0 and np.all(np.diff(y) > 0)
    # stretched: finer spacing at the wall than in the centre
    assert (y[1] - y[0]) < (y[3] - y[2])


def test_gap_input_has_gap():
    A = channel_field((8, 8, 8), 3, 80, seed=2, gap_k=10, dtype=torch.float64).numpy()
    s = np.linalg.svd(A, compute_uv=False)
    assert s[10] / s[9] < 5e-3


def test_seeded_and_column_major():
    A1 = channel_field((4, 4, 4), 3, 7, seed=5)
    A2 = channel_field((4, 4, 4), 3, 7, seed=5)
    assert torch.equal(A1, A2)
    assert A1.stride() == (1, 192)
