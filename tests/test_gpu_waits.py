"""Device-side bounded waits give up and report a status instead of hanging.

Every wait in the library's kernels (mbarrier phases of the tensor-core
kernels, the grid barrier of the cooperative coarse QR) is bounded; on
timeout the kernel raises a status word that the host returns as
ID_ERR_TIMEOUT.  id_check_wait runs those wait routines with a ~1 ms limit on
a phase or barrier that nothing completes (no fault, no hang) and on one
that completes; the context must stay usable afterwards.
"""
import numpy as np
import pytest
import torch

import oracle
from synthetic import gaussian_matrix, low_rank_matrix

pytestmark = pytest.mark.gpu

ID_OK, ID_ERR_TIMEOUT = 0, 6


@pytest.mark.parametrize("mode,expected", [(0, ID_ERR_TIMEOUT), (1, ID_OK),
                                           (2, ID_ERR_TIMEOUT), (3, ID_OK)])
def test_bounded_wait_gives_up(mode, expected):
    from paper_1905_13257_gb300 import check_wait
    assert check_wait(mode) == expected


def test_context_usable_after_timeouts():
    from paper_1905_13257_gb300 import IdSketch, check_wait
    for mode in (0, 2, 0):
        assert check_wait(mode) == ID_ERR_TIMEOUT
    m, n, k = 4096, 96, 8
    A = gaussian_matrix(m, n, seed=3, dtype=torch.float32, device="cuda")
    A = A + low_rank_matrix(m, n, 6, seed=4, dtype=torch.float32, device="cuda") * 10
    g = np.random.default_rng(1)
    J = torch.tensor(g.choice(n, size=k, replace=False), dtype=torch.int32)
    P = torch.tensor(g.normal(size=(k, n)) * 0.3)
    sk = IdSketch(m=m, n_max=n, k=k, l=16, seed=0, dtype=torch.float32)
    fro, mx = sk.reconstruct_error(A, J, P)
    fo, mo = oracle.recon_error(A.cpu().double().numpy(), J.numpy(), P.numpy())
    assert abs(fro - fo) <= 1e-4 * fo
    sk.close()


def test_check_wait_rejects_bad_mode():
    from paper_1905_13257_gb300 import IdError, check_wait
    with pytest.raises(IdError):
        check_wait(7)
