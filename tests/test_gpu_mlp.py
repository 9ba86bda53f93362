"""GPU parity of the learned proposal's network kernels (id_mlp_*) against
the FP64 oracle (oracle/learned.py): the feature gather, the forward scores,
every gradient, and a training run whose trajectory follows the oracle's.

Bars (FP32 kernels, FP64 oracle on the same FP32 inputs): features exact;
scores within 1e-5 of max |s|; gradients within 1e-4 of each gradient's
largest entry; after 50 SGD steps the parameters within 1e-3 of their scale.
"""
import numpy as np
import pytest
import torch

import oracle.learned as L
from synthetic import channel_field

pytestmark = pytest.mark.gpu

DEV = "cuda"


def _params(F, H, seed):
    p = L.init_params(F, H, seed=seed)
    rng = np.random.default_rng(seed + 1)
    p["b1"] = rng.standard_normal(H) * 0.2
    p["b2"] = 0.05
    # the oracle runs on the FP32-rounded values the kernels see
    return {k: np.asarray(v, dtype=np.float32).astype(np.float64) for k, v in p.items()}


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_features_match_the_oracle(dtype):
    from paper_1905_13257_gb300 import mlp_features
    grid = (16, 12, 16)
    A = channel_field(grid, 3, 40, seed=5, dtype=dtype, device=DEV)
    rows = L.feature_rows(grid)
    X = mlp_features(A, rows, scale=1.0).cpu().numpy()
    Xo = L.column_features(A.cpu().numpy(), grid).astype(np.float32)
    assert np.array_equal(X, Xo)
    bad = np.array([rows[0], A.shape[0], -1])            # rows outside [0, m): NaN
    Xb = mlp_features(A, bad).cpu().numpy()
    assert np.all(np.isfinite(Xb[:, 0])) and np.all(np.isnan(Xb[:, 1:]))


@pytest.mark.parametrize("n,F,H", [(70, 100, 40), (33, 257, 64), (512, 96, 256)])
def test_forward_matches_the_oracle(n, F, H):
    from paper_1905_13257_gb300 import Mlp
    rng = np.random.default_rng(n + F)
    X = rng.standard_normal((n, F)).astype(np.float32)
    p = _params(F, H, seed=3)
    net = Mlp(p)
    s = net.forward(torch.from_numpy(X).to(DEV)).cpu().numpy()
    so, (Zo, Go) = L.forward(X.astype(np.float64), p)
    assert np.max(np.abs(s - so)) <= 1e-5 * max(1.0, np.abs(so).max())
    assert np.max(np.abs(net.G.cpu().numpy() - Go)) <= 1e-5 * max(1.0, np.abs(Go).max())


@pytest.mark.parametrize("pos_weight", [1.0, 3.0])
def test_backward_matches_the_oracle(pos_weight):
    from paper_1905_13257_gb300 import Mlp
    n, F, H = 70, 100, 40
    rng = np.random.default_rng(9)
    X = rng.standard_normal((n, F)).astype(np.float32)
    y = (rng.random(n) < 0.3).astype(np.float32)
    p = _params(F, H, seed=4)
    net = Mlp(p)
    Xd = torch.from_numpy(X).to(DEV)
    net.forward(Xd)
    g = net.backward(Xd, torch.from_numpy(y).to(DEV), pos_weight)
    go = L.backward(X.astype(np.float64), y.astype(np.float64), p, pos_weight)
    for key in ("W1", "b1", "w2", "b2"):
        a = g[key].cpu().numpy().reshape(-1)
        b = np.atleast_1d(np.asarray(go[key], dtype=np.float64)).reshape(-1)
        assert np.max(np.abs(a - b)) <= 1e-4 * max(1e-12, np.abs(b).max()), key


def test_gpu_training_follows_the_oracle():
    from paper_1905_13257_gb300 import Mlp
    rng = np.random.default_rng(0)
    n, F, H = 200, 16, 12
    X = rng.standard_normal((n, F)).astype(np.float32)
    y = (X[:, 0] + 0.5 * X[:, 1] > 0.8).astype(np.float32)
    p = _params(F, H, seed=1)
    net = Mlp(p)
    Xd, yd = torch.from_numpy(X).to(DEV), torch.from_numpy(y).to(DEV)
    q = dict(p)
    X64, y64 = X.astype(np.float64), y.astype(np.float64)
    first = L.bce_loss(L.forward(X64, q)[0], y64)
    for _ in range(50):
        net.forward(Xd)
        net.step(net.backward(Xd, yd), lr=0.5)
        q = L.sgd_step(q, L.backward(X64, y64, q), lr=0.5)
    for key in ("W1", "b1", "w2", "b2"):
        a = getattr(net, key).cpu().numpy().reshape(-1)
        b = np.atleast_1d(q[key]).reshape(-1)
        assert np.max(np.abs(a - b)) <= 1e-3 * max(1.0, np.abs(b).max()), key
    last = L.bce_loss(net.forward(Xd).cpu().numpy().astype(np.float64), y64)
    assert last < 0.7 * first
