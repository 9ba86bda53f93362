"""GPU parity of the FP8-E4M3 precision form (ID_SKETCH_FP8E4M3): the
sketches of the library against the oracle's sketches of the dequantised
matrix (oracle/fp8.py: per-column power-of-two scales, E4M3 rounding with
ties to even) on the same Psi and Omega, both tensor-core feeds, with and
without Y, ragged m and n, columns whose magnitudes span 12 decades.

Bars: W and Y within 1e-5 relative Frobenius of the oracle's products of the
dequantised matrix (exact tensor-core products, FP32 accumulation); A_c
exactly the data's own coarse rows; against the FP64 sketches of the
unquantised data, within 2^-4 relative Frobenius (every entry of the
dequantised matrix in E4M3's normal range is within 2^-4 of the data).
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import fp8 as ofp8
from synthetic import channel_field

pytestmark = pytest.mark.gpu

DEV = "cuda"


def rel(a, b):
    return np.linalg.norm(np.asarray(a, dtype=np.float64) - b) / np.linalg.norm(b)


def wide_columns(A):
    """Column c scaled by 10^(-6 + 12 c / (n - 1)): per-column scales matter."""
    n = A.shape[1]
    f = torch.logspace(-6, 6, n, dtype=torch.float64, device=A.device).to(A.dtype)
    return A * f[None, :]


@pytest.mark.parametrize("tma", ["1", "0"])
def test_fp8_sketches_match_oracle(monkeypatch, tma):
    monkeypatch.setenv("IDSKETCH_SKETCH_TMA", tma)
    from paper_1905_13257_gb300 import IdSketch
    grid, nc, n, l, seed = (20, 13, 12), 3, 300, 60, 6
    A = wide_columns(channel_field(grid, nc, n, seed=4, dtype=torch.float32, device=DEV))
    A = A.T.contiguous().T
    m = A.shape[0]
    sk = IdSketch(m, n, 10, l, seed=seed, prec="fp8", grid=grid, ncomp=nc,
                  coarse_stride=(2, 3, 2), want_Y=True, want_coarse=True, window_cols=256)
    for j0 in range(0, n, 32):
        sk.stream_columns(A[:, j0:j0 + 32])
    W, Y, Ac = sk.sketches()
    An = A.double().cpu().numpy()
    Aq, _ = ofp8.quantize_columns(An)
    Psi, Om = oracle.psi(l, m, seed), oracle.omega(n, l, seed)
    Wo, Yo = oracle.sketch(Aq, Psi, Om)
    assert rel(W.cpu().numpy(), Wo) <= 1e-5
    assert rel(Y.cpu().double().numpy(), Yo) <= 1e-5
    rows = oracle.coarse_rows(grid, nc, (2, 3, 2))
    assert np.array_equal(Ac.cpu().numpy(), A.cpu().numpy()[rows])
    Wx, Yx = oracle.sketch(An, Psi, Om)
    assert rel(W.cpu().numpy(), Wx) <= 2.0 ** -4
    assert rel(Y.cpu().double().numpy(), Yx) <= 2.0 ** -4
    J, P, kout = sk.factor()
    assert kout == 10
    Pn = P.cpu().numpy()
    assert np.array_equal(Pn[:, J.cpu().numpy()], np.eye(10))
    sk.close()


@pytest.mark.parametrize("tma", ["1", "0"])
def test_fp8_wide_sketch_without_y(monkeypatch, tma):
    """l = 90 without Y: one pass with 96-wide accumulators (TMA feed) or two
    passes of Psi rows (register feed), the scales applied once per window."""
    monkeypatch.setenv("IDSKETCH_SKETCH_TMA", tma)
    from paper_1905_13257_gb300 import IdSketch
    grid, nc, n, k, l, seed = (16, 12, 16), 3, 240, 80, 90, 9
    A = wide_columns(channel_field(grid, nc, n, seed=7, gap_k=k, dtype=torch.float32,
                                   device=DEV))
    A = A.T.contiguous().T
    m = A.shape[0]
    sk = IdSketch(m, n, k, l, seed=seed, prec="fp8", want_Y=False, window_cols=n)
    for j0 in range(0, n, 32):
        sk.stream_columns(A[:, j0:j0 + 32])
    W = sk.sketches()[0]
    An = A.double().cpu().numpy()
    Aq, _ = ofp8.quantize_columns(An)
    Wo, _ = oracle.sketch(Aq, oracle.psi(l, m, seed), oracle.omega(n, l, seed))
    assert rel(W.cpu().numpy(), Wo) <= 1e-5
    sk.close()
