"""GPU parity of the learned proposal's network kernels (id_mlp_*) against
the FP64 oracle (oracle/learned.py): the feature gather, the forward scores,
every gradient, and a training run whose trajectory follows the oracle's.

The two dense products run on the tensor cores with bfloat16 operands and
FP32 accumulation; the oracle takes the same bfloat16-rounded operands
(product_round=bf16_operands) with exact accumulation.  Bars: features
exact; scores within 1e-5 of max |s|; gradients within 1e-4 of each
gradient's largest entry; after 50 SGD steps the parameters within 1e-3 of
their scale.
"""
import numpy as np
import pytest
import torch

import oracle
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
    so, (Zo, Go) = L.forward(X.astype(np.float64), p, product_round=L.bf16_operands)
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
    go = L.backward(X.astype(np.float64), y.astype(np.float64), p, pos_weight,
                    product_round=L.bf16_operands)
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
    r = L.bf16_operands
    first = L.bce_loss(L.forward(X64, q, product_round=r)[0], y64)
    for _ in range(50):
        net.forward(Xd)
        net.step(net.backward(Xd, yd), lr=0.5)
        q = L.sgd_step(q, L.backward(X64, y64, q, product_round=r), lr=0.5)
    for key in ("W1", "b1", "w2", "b2"):
        a = getattr(net, key).cpu().numpy().reshape(-1)
        b = np.atleast_1d(q[key]).reshape(-1)
        assert np.max(np.abs(a - b)) <= 1e-3 * max(1.0, np.abs(b).max()), key
    last = L.bce_loss(net.forward(Xd).cpu().numpy().astype(np.float64), y64)
    assert last < 0.7 * first


# ------------------------------------------- QR restricted to the candidates

def test_factor_restricted_matches_the_oracle():
    """id_factor_restricted against oracle.learned.restricted_id on the same
    W: J identical (the candidate draw gives the restricted pivots a margin),
    P within 1e-9;
    with every column a candidate it is the plain randomized ID."""
    from paper_1905_13257_gb300 import IdError, IdSketch
    grid, n, k, l = (16, 12, 16), 200, 12, 22
    A = channel_field(grid, 3, n, seed=7, gap_k=k, dtype=torch.float32, device=DEV)
    sk = IdSketch(m=A.shape[0], n_max=n, k=k, l=l, seed=9, dtype=torch.float32, want_Y=False)
    sk.stream_columns(A)
    W = sk.sketches()[0].cpu().numpy()
    J0, P0, k0 = sk.factor(device="cpu")
    assert k0 == k
    # candidate sets: the first draw (from seed 2) whose restricted pivots have
    # an oracle margin >= 1e-4, so that J is unique and always compared
    for cseed in range(2, 34):
        rng = np.random.default_rng(cseed)
        others = rng.choice(np.setdiff1d(np.arange(n), J0.numpy()), 12, replace=False)
        cand = np.sort(np.concatenate([J0.numpy(), others]))
        if oracle.column_id(W[:, cand], k)[3] >= 1e-4:
            break
    assert oracle.column_id(W[:, cand], k)[3] >= 1e-4
    J, P, kk = sk.factor_restricted(cand, device="cpu")
    Jo, Po, ko = L.restricted_id(W, cand, k)
    assert kk == ko == k
    assert J.tolist() == Jo.tolist()
    assert np.max(np.abs(P.numpy() - Po)) <= 1e-9 * max(1.0, np.abs(Po).max())
    assert np.array_equal(P.numpy()[:, J.numpy()], np.eye(k))
    # every column a candidate: the plain ID (P = R11^-1 R12)
    J2, P2, k2 = sk.factor_restricted(np.arange(n), device="cuda")
    assert k2 == k and J2.cpu().tolist() == J0.tolist()
    assert np.max(np.abs(P2.cpu().numpy() - P0.numpy())) <= 1e-9 * max(1.0, P0.abs().max().item())
    for bad in ([3, 3, 5], [0, n], [-1, 4]):
        with pytest.raises(IdError) as e:
            sk.factor_restricted(np.array(bad))
        assert e.value.status == 1
    sk.close()


# ------------------------------------------------------------ the proposal

@pytest.mark.parametrize("n,count", [(512, 100), (37, 37), (4096, 1), (300, 17)])
def test_propose_matches_the_oracle(n, count):
    """id_mlp_propose against oracle.learned.propose: the count highest
    scores, ties to the lower index, in increasing column order (with many
    exact ties and a NaN, which ranks last)."""
    from paper_1905_13257_gb300 import _binding as B
    lib = B.load()
    rng = np.random.default_rng(n + count)
    s = np.round(rng.standard_normal(n) * 4) / 4          # many ties
    s = s.astype(np.float32)
    if n > 3:
        s[3] = np.nan
    sd = torch.from_numpy(s).to(DEV)
    cand = torch.empty(count, dtype=torch.int32, device=DEV)
    st = lib.id_mlp_propose(B.C.c_void_p(sd.data_ptr()), n, count, B.C.c_void_p(cand.data_ptr()),
                            B.C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    so = np.where(np.isnan(s), -np.inf, s.astype(np.float64))
    assert cand.cpu().tolist() == L.propose(so, count).tolist()
    assert lib.id_mlp_check(B.C.c_void_p(torch.cuda.current_stream().cuda_stream)) == 0


@pytest.mark.parametrize("n,strata,per", [(512, 50, 2), (100, 7, 2), (9, 3, 3), (4096, 64, 1)])
def test_propose_stratified_matches_the_oracle(n, strata, per):
    from paper_1905_13257_gb300 import _binding as B
    lib = B.load()
    rng = np.random.default_rng(n + strata)
    s = (np.round(rng.standard_normal(n) * 4) / 4).astype(np.float32)
    sd = torch.from_numpy(s).to(DEV)
    cand = torch.full((strata * per,), -7, dtype=torch.int32, device=DEV)
    cnt = torch.zeros(1, dtype=torch.int32, device=DEV)
    sh = B.C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.id_mlp_propose_stratified(B.C.c_void_p(sd.data_ptr()), n, strata, per,
                                         B.C.c_void_p(cand.data_ptr()),
                                         B.C.c_void_p(cnt.data_ptr()), sh) == 0
    want = L.propose_stratified(s.astype(np.float64), strata, per)
    assert int(cnt.item()) == len(want)
    assert cand[: len(want)].cpu().tolist() == want.tolist()
