"""Pins of the learned-proposal oracle (oracle/learned.py) against what the
mathematics fixes: the GELU's closed form and odd-part identity, analytic
gradients against central finite differences of the loss (and a planted
wrong derivative that the check catches), the cross entropy's definition,
the feature rows by brute force, the restricted ID reducing to the plain ID
when every column is a candidate and recovering exactly rank-k data, and a
training run that fits a separable toy problem."""
import math

import numpy as np
import pytest

import oracle
import oracle.learned as L
from synthetic import low_rank_matrix


def test_gelu_closed_form_and_identities():
    for z in (-3.0, -1.0, -0.25, 0.0, 0.5, 2.0):
        phi_cdf = 0.5 * (1.0 + math.erf(z / math.sqrt(2.0)))
        assert L.gelu(z) == pytest.approx(z * phi_cdf, rel=1e-14, abs=1e-300)
        # z Phi(z) - (-z) Phi(-z) = z (Phi(z) + Phi(-z)) = z
        assert L.gelu(z) - L.gelu(-z) == pytest.approx(z, abs=1e-14)
        h = 1e-6
        fd = (float(L.gelu(z + h)) - float(L.gelu(z - h))) / (2 * h)
        assert float(L.gelu_grad(z)) == pytest.approx(fd, rel=1e-8, abs=1e-9)
    assert float(L.gelu_grad(0.0)) == 0.5


def test_forward_one_unit_closed_form():
    p = {"W1": np.array([[0.7]]), "b1": np.array([-0.2]), "w2": np.array([1.5]), "b2": 0.3}
    x = np.array([[1.2]])
    z = 1.2 * 0.7 - 0.2
    want = 1.5 * z * 0.5 * (1.0 + math.erf(z / math.sqrt(2.0))) + 0.3
    s, _ = L.forward(x, p)
    assert s[0] == pytest.approx(want, rel=1e-14)


def test_bce_matches_definition_and_is_stable():
    s = np.array([-2.0, -0.1, 0.0, 0.4, 3.0])
    y = np.array([0.0, 1.0, 1.0, 0.0, 1.0])
    sg = 1.0 / (1.0 + np.exp(-s))
    want = np.mean(-(y * np.log(sg) + (1 - y) * np.log(1 - sg)))
    assert L.bce_loss(s, y) == pytest.approx(want, rel=1e-13)
    big = L.bce_loss(np.array([800.0, -800.0]), np.array([0.0, 1.0]))
    assert big == pytest.approx(800.0, rel=1e-12)
    assert L.bce_loss(np.array([800.0, -800.0]), np.array([1.0, 0.0])) == pytest.approx(0.0,
                                                                                        abs=1e-300)


def _fd_check(backward_fn, pos_weight=1.0, seed=3):
    rng = np.random.default_rng(seed)
    n, F, H = 11, 7, 5
    X = rng.standard_normal((n, F))
    y = (rng.random(n) < 0.4).astype(float)
    p = L.init_params(F, H, seed=seed)
    p["b1"] = rng.standard_normal(H) * 0.3
    p["b2"] = 0.1
    g = backward_fn(X, y, p, pos_weight)
    h = 1e-6
    worst = 0.0
    for key in ("W1", "b1", "w2", "b2"):
        arr = np.atleast_1d(np.asarray(p[key], dtype=np.float64))
        for idx in np.ndindex(arr.shape):
            def loss_at(delta):
                q = {k: (np.array(v, dtype=np.float64, copy=True) if k == key else v)
                     for k, v in p.items()}
                if key == "b2":
                    q["b2"] = float(p["b2"]) + delta
                else:
                    q[key][idx] += delta
                return L.bce_loss(L.forward(X, q)[0], y, pos_weight)
            fd = (loss_at(h) - loss_at(-h)) / (2 * h)
            an = float(np.atleast_1d(np.asarray(g[key]))[idx])
            worst = max(worst, abs(an - fd) / max(1e-8, abs(fd)))
    return worst


@pytest.mark.parametrize("pos_weight", [1.0, 4.0])
def test_backward_matches_finite_differences(pos_weight):
    assert _fd_check(L.backward, pos_weight) < 1e-6


def test_planted_wrong_derivative_is_caught(monkeypatch):
    # the GELU's value in place of its derivative: the finite-difference pin fails
    monkeypatch.setattr(L, "gelu_grad", L.gelu)
    assert _fd_check(L.backward) > 1e-2


def test_feature_rows_by_brute_force():
    grid = (16, 12, 16)
    rows = L.feature_rows(grid)
    nx, ny, nz = grid
    want = [((0 * ny + j) * nz + kz) * nx + i
            for j in range(ny) for kz in range(nz) for i in range(nx)
            if i % 8 == 0 and j % 6 == 0 and kz % 8 == 0]
    assert rows.tolist() == want
    assert len(L.feature_rows((128, 96, 128))) == 4096
    A = np.arange(3 * nx * ny * nz * 2, dtype=np.float64).reshape(-1, 2)
    X = L.column_features(A, grid, scale=2.0)
    assert X.shape == (2, len(want))
    assert np.array_equal(X, 2.0 * A[want, :].T)


def test_propose_order_and_ties():
    s = np.array([0.5, 2.0, 2.0, -1.0, 3.0, 0.5])
    assert L.propose(s, 3).tolist() == [1, 2, 4]
    assert L.propose(s, 5).tolist() == [0, 1, 2, 4, 5]   # tie at 0.5: both taken
    assert L.propose(s, 4).tolist() == [0, 1, 2, 4]      # tie at 0.5: lower index


def test_restricted_id_with_every_column_is_the_plain_id():
    rng = np.random.default_rng(5)
    B = rng.standard_normal((30, 80))
    J0, P0, k0, margin = oracle.column_id(B, 12)
    assert margin > 1e-6
    J, P, k = L.restricted_id(B, np.arange(80), 12)
    assert k == k0 and J.tolist() == J0[:k0].tolist()
    # least squares on B(:, J) reproduces R11^-1 R12 (Sec. 2.4)
    assert np.max(np.abs(P - P0[:k0])) <= 1e-9 * max(1.0, np.abs(P0).max())
    assert np.array_equal(P[:, J], np.eye(k))


def test_restricted_id_recovers_rank_k_from_a_superset_of_candidates():
    import torch
    A = low_rank_matrix(400, 60, 6, seed=2, dtype=torch.float64).numpy()
    J0, _, k0, _ = oracle.column_id(A, 6)
    rng = np.random.default_rng(1)
    others = rng.choice(np.setdiff1d(np.arange(60), J0[:k0]), 6, replace=False)
    cand = np.sort(np.concatenate([J0[:k0], others]))
    J, P, k = L.restricted_id(A, cand, 6)
    assert k == 6
    assert set(J.tolist()) <= set(cand.tolist())
    fro, _ = oracle.recon_error(A, J, P)
    assert fro <= 1e-12


def test_fallback_takes_the_plain_id_when_the_proposal_is_worse():
    import torch
    A = low_rank_matrix(300, 40, 12, seed=4, dtype=torch.float64, decay=0.5).numpy()
    Jp, Pp, kp, _ = oracle.column_id(A, 5)
    plain = (Jp[:kp], Pp[:kp])
    good = L.restricted_id(A, np.arange(40), 5)[:2]
    chosen, used, el, ep = L.choose_with_fallback(A, good, plain)
    assert used and el <= 1.05 * ep
    # a skeleton of five near-duplicate columns: far worse than the plain ID
    A2 = A.copy()
    A2[:, 1:5] = A2[:, [0]] * np.array([1.0, 1.0 + 1e-9, 1.0 - 1e-9, 1.0 + 2e-9])
    Jp2, Pp2, kp2, _ = oracle.column_id(A2, 5)
    plain2 = (Jp2[:kp2], Pp2[:kp2])
    bad_J = np.array([0, 1, 2, 3, 4])
    bad = (bad_J, np.linalg.lstsq(A2[:, bad_J], A2, rcond=None)[0])
    chosen, used, el, ep = L.choose_with_fallback(A2, bad, plain2)
    assert el > 1.05 * ep
    assert not used and chosen[0] is plain2[0]


def test_training_fits_a_separable_toy_problem():
    rng = np.random.default_rng(0)
    n, F, H = 200, 16, 12
    X = rng.standard_normal((n, F))
    y = (X[:, 0] + 0.5 * X[:, 1] > 0.8).astype(float)
    p = L.init_params(F, H, seed=1)
    first = L.bce_loss(L.forward(X, p)[0], y)
    for _ in range(400):
        p = L.sgd_step(p, L.backward(X, y, p), lr=0.5)
    last = L.bce_loss(L.forward(X, p)[0], y)
    assert last < 0.5 * first
    acc = np.mean((L.forward(X, p)[0] > 0) == (y > 0))
    assert acc > 0.9


def test_bf16_products_round_exactly_the_two_products_operands():
    """product_round=bf16_operands: the forward pass equals the plain one on
    bfloat16-rounded X and W1, the W1 gradient differs from the unrounded one
    by no more than the rounding of its two operands allows (|x y - x' y'|
    <= 2^-8 (|x| |y| + |x'| |y'|) per term, bfloat16 relative rounding <= 2^-9
    each), and every other gradient is that of the rounded forward pass."""
    rng = np.random.default_rng(4)
    n, F, H = 24, 40, 16
    X = rng.standard_normal((n, F))
    y = (rng.random(n) < 0.3).astype(float)
    p = L.init_params(F, H, seed=2)
    p["b1"] = rng.standard_normal(H) * 0.3
    r = L.bf16_operands
    Xb = r(X)
    # every rounded value is a bfloat16: 8 significant bits
    m, e = np.frexp(Xb[Xb != 0])
    assert np.all(m * 256 == np.round(m * 256))
    assert np.max(np.abs(Xb - X) / np.abs(X)) <= 2.0 ** -8
    s_r, (Z_r, _) = L.forward(X, p, product_round=r)
    pb = dict(p, W1=r(p["W1"]))
    s_p, (Z_p, _) = L.forward(Xb, pb)
    assert np.array_equal(Z_r, Z_p) and np.array_equal(s_r, s_p)
    g_r = L.backward(X, y, p, product_round=r)
    g_p = L.backward(Xb, y, pb)
    for key in ("b1", "w2", "b2"):
        assert np.allclose(g_r[key], g_p[key], rtol=0, atol=0)
    # gW1 from rounded X and rounded dZ against the unrounded product
    _, (Z, G) = L.forward(Xb, pb)
    bound = 2.0 ** -8 * 2 * (np.abs(Xb).T @ np.abs(np.outer(np.ones(n), p["w2"]))) * \
        np.max(np.abs(L.gelu_grad(Z))) / n
    assert np.all(np.abs(g_r["W1"] - g_p["W1"]) <= bound + 1e-15)
    assert not np.array_equal(g_r["W1"], g_p["W1"])


def test_propose_stratified_by_brute_force():
    """Each stratum contributes its `per` best columns (ties to the lower
    index), checked by sorting each stratum by hand; one stratum reduces to
    propose()."""
    rng = np.random.default_rng(3)
    for n, strata, per in [(100, 7, 2), (512, 50, 2), (9, 3, 3), (50, 50, 1)]:
        sc = np.round(rng.standard_normal(n) * 3) / 3     # ties
        got = L.propose_stratified(sc, strata, per)
        want = []
        for q in range(strata):
            lo, hi = q * n // strata, (q + 1) * n // strata
            idx = sorted(range(lo, hi), key=lambda j: (-sc[j], j))[:per]
            want += idx
        assert got.tolist() == sorted(want)
    sc = rng.standard_normal(40)
    assert L.propose_stratified(sc, 1, 8).tolist() == L.propose(sc, 8).tolist()
