"""Pins for the oracle's interpolative decomposition (Sec. 2.4-2.5).

Each check ties the oracle to something outside itself: LAPACK's pivoted QR
(dgeqp3 via scipy, a library special case), exact recovery of exactly rank-k
matrices, P(:,J) = I, the least-squares identity of the deterministic ID,
the Eckart-Young lower bound and the ID upper bound of eq. ``eqn:id_bound_orig``,
brute force on tiny matrices, Theorem 2.1 for the sub-sampled ID, and explicit
loops for the sketch definitions.  The planted-mistake tests at the end show
that a plausible slip in the oracle breaks at least one of these pins.
"""
import itertools

import numpy as np
import pytest
import scipy.linalg as sla
import torch

import oracle
from oracle import interp_decomp as idm
from synthetic import channel_field, low_rank_matrix


def _rand(m, n, seed, decay=None):
    g = np.random.default_rng(seed)
    A = g.normal(size=(m, n))
    if decay is not None:
        U, s, Vt = np.linalg.svd(A, full_matrices=False)
        A = (U * (decay ** np.arange(len(s)))) @ Vt
    return A


# ---------------------------------------------------------------- Householder

def test_householder_reflects_onto_e1():
    g = np.random.default_rng(0)
    for n in (1, 2, 5, 17):
        x = g.normal(size=n)
        v, tau, beta = oracle.householder(x)
        H = np.eye(n) - tau * np.outer(v, v)
        y = H @ x
        assert abs(y[0] - beta) < 1e-12 * np.linalg.norm(x)
        assert np.allclose(y[1:], 0, atol=1e-12 * np.linalg.norm(x))
        assert np.allclose(H @ H.T, np.eye(n), atol=1e-12)
        if n > 1:
            assert np.sign(beta) == -np.sign(x[0])  # LAPACK sign convention


def test_householder_trivial_vector():
    v, tau, beta = oracle.householder(np.array([-3.0, 0.0, 0.0]))
    assert tau == 0.0 and beta == -3.0


# ----------------------------------------------------------------------- CPQR

@pytest.mark.parametrize("shape,k,seed", [((30, 200), 20, 1), ((60, 120), 50, 2),
                                          ((40, 40), 40, 3), ((300, 25), 25, 4)])
def test_cpqr_matches_lapack_pivots(shape, k, seed):
    A = _rand(*shape, seed, decay=0.9)
    J, R, k_out, margin = oracle.cpqr(A, k)
    assert margin > 1e-6
    Q, Rl, piv = sla.qr(A, pivoting=True, mode="economic")
    kk = min(k, *shape)
    assert k_out == kk
    assert list(J) == list(piv[:kk])
    # R agrees up to the sign of each row
    R11 = R[:, J]
    Rl11 = Rl[:kk, :kk]
    sgn = np.sign(np.diag(R11)) * np.sign(np.diag(Rl11))
    assert np.allclose(R11 * sgn[:, None], Rl11, rtol=1e-9, atol=1e-11 * abs(Rl11).max())
    Rl12 = Rl[:kk, kk:]
    mask = np.ones(shape[1], bool)
    mask[J] = False
    # order of the remaining columns differs (LAPACK swaps); compare per column
    lap_rest = {int(c): Rl12[:, i] for i, c in enumerate(piv[kk:])}
    for j in np.nonzero(mask)[0][:20]:
        assert np.allclose(R[:, j] * sgn, lap_rest[int(j)], rtol=1e-9,
                           atol=1e-11 * abs(Rl11).max())


def test_cpqr_reconstructs_permuted_matrix():
    A = _rand(25, 40, 5)
    J, R, k_out, _ = oracle.cpqr(A, 25)
    # full CPQR: A(:,J) = Q R11 with Q orthogonal -> R11^T R11 = A_J^T A_J
    AJ = A[:, J]
    R11 = R[:, J]
    assert np.allclose(R11.T @ R11, AJ.T @ AJ, atol=1e-10)
    assert np.allclose(np.tril(R11, -1), 0)


def test_back_substitution_against_explicit_inverse():
    g = np.random.default_rng(3)
    U = np.triu(g.normal(size=(12, 12))) + 5 * np.eye(12)
    B = g.normal(size=(12, 7))
    X = oracle.back_substitute(U, B)
    assert np.allclose(U @ X, B, atol=1e-12)
    assert np.allclose(X, np.linalg.inv(U) @ B, atol=1e-11)


# ------------------------------------------------------------------ ID proper

@pytest.mark.parametrize("m,n,k,seed", [(200, 60, 7, 0), (98, 40, 12, 1), (500, 300, 20, 2)])
def test_exact_rank_k_recovery(m, n, k, seed):
    A = low_rank_matrix(m, n, k, seed).numpy()
    J, P, k_out, _ = oracle.deterministic_id(A, k)
    assert k_out == k
    fro, _ = oracle.recon_error(A, J, P)
    assert fro <= 1e-12
    J2, P2, k2, _, _ = oracle.randomized_id(A, k, k + 10, seed=seed)
    fro2, _ = oracle.recon_error(A, J2, P2)
    assert k2 == k and fro2 <= 1e-11


def test_interpolation_matrix_identity_on_skeleton():
    A = _rand(80, 50, 9, decay=0.8)
    J, P, k_out, _ = oracle.deterministic_id(A, 10)
    assert np.array_equal(P[:, J], np.eye(10))  # bit-exact (eq. ``eqn:id``)


def test_deterministic_id_is_least_squares():
    # A(:,J) = Q1 R11 => R11^{-1} R12 = A(:,J)^+ A(:,Jc)
    A = _rand(120, 45, 11, decay=0.85)
    J, P, k_out, _ = oracle.deterministic_id(A, 9)
    mask = np.ones(45, bool)
    mask[J] = False
    X, *_ = np.linalg.lstsq(A[:, J], A[:, mask], rcond=None)
    assert np.allclose(P[:, mask], X, rtol=1e-9, atol=1e-10)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_error_between_eckart_young_and_id_bound(seed):
    A = _rand(150, 70, seed, decay=0.8)
    s = np.linalg.svd(A, compute_uv=False)
    n = A.shape[1]
    for k in (3, 10, 25):
        J, P, _, _ = oracle.deterministic_id(A, k)
        err2 = oracle.spectral_norm(A - A[:, J] @ P)
        assert err2 >= s[k] * (1 - 1e-10)                        # sigma_{k+1} lower bound
        assert err2 <= np.sqrt(1 + k * (n - k)) * s[k]           # eq. eqn:id_bound_orig
        fro = np.linalg.norm(A - A[:, J] @ P)
        assert fro >= np.sqrt(np.sum(s[k:] ** 2)) * (1 - 1e-10)  # Frobenius Eckart-Young


def test_bound_on_channel_field():
    A = channel_field((8, 8, 8), 3, 60, seed=4, dtype=torch.float64).numpy()
    s = np.linalg.svd(A, compute_uv=False)
    for k in (5, 15, 30):
        J, P, _, _ = oracle.deterministic_id(A, k)
        e2 = oracle.spectral_norm(A - A[:, J] @ P)
        assert s[k] * (1 - 1e-10) <= e2 <= np.sqrt(1 + k * (60 - k)) * s[k]


def _residual_norms_by_projection(A, chosen):
    if not chosen:
        return np.linalg.norm(A, axis=0)
    Q, _ = np.linalg.qr(A[:, chosen])
    Rm = A - Q @ (Q.T @ A)
    return np.linalg.norm(Rm, axis=0)


@pytest.mark.parametrize("seed", range(6))
def test_brute_force_greedy_and_best_subset(seed):
    g = np.random.default_rng(100 + seed)
    m, n, k = int(g.integers(4, 13)), int(g.integers(3, 9)), int(g.integers(1, 4))
    A = g.normal(size=(m, n))
    J, P, k_out, _ = oracle.deterministic_id(A, k)
    k = k_out
    # (i) each pivot maximises the residual norm after projecting out the previous ones
    for s in range(k):
        nu = _residual_norms_by_projection(A, list(J[:s]))
        nu[list(J[:s])] = -1
        assert abs(nu[J[s]] - nu.max()) <= 1e-12 * nu.max()
    # (ii) best subset <= ID error <= bound
    err = np.linalg.norm(A - A[:, J] @ P, 2)
    best = min(np.linalg.norm(A - A[:, list(c)] @ np.linalg.lstsq(A[:, list(c)], A, rcond=None)[0], 2)
               for c in itertools.combinations(range(n), k))
    s = np.linalg.svd(A, compute_uv=False)
    assert best <= err * (1 + 1e-12)
    assert err <= np.sqrt(1 + k * (n - k)) * s[k] * (1 + 1e-12) if k < min(m, n) else True


def test_rank_deficient_stops_early():
    A = low_rank_matrix(60, 30, 4, 2).numpy()
    J, P, k_out, _ = oracle.deterministic_id(A, 10)
    assert k_out == 4
    fro, _ = oracle.recon_error(A, J, P)
    assert fro < 1e-12
    Z = np.zeros((20, 10))
    J, P, k_out, _ = oracle.deterministic_id(Z, 3)
    assert k_out == 0 and P.shape == (0, 10)


def test_zero_columns_are_never_pivoted_first():
    A = _rand(30, 12, 1)
    A[:, [2, 7]] = 0.0
    J, P, k_out, _ = oracle.deterministic_id(A, 10)
    assert 2 not in J and 7 not in J
    assert np.allclose(P[:, [2, 7]], 0.0)


def test_tie_break_lowest_index():
    A = np.zeros((4, 5))
    A[0, 1] = A[1, 3] = A[2, 4] = 2.0
    J, R, k_out, _ = oracle.cpqr(A, 3)
    assert list(J) == [1, 3, 4]


# ------------------------------------------------------------------- sketches

def test_sketch_definitions_by_loops():
    g = np.random.default_rng(2)
    A = g.normal(size=(9, 7)).astype(np.float32)
    Psi = oracle.psi(5, 9, seed=1)
    Om = oracle.omega(7, 5, seed=1)
    W, Y = oracle.sketch(A, Psi, Om)
    for s in range(5):
        for j in range(7):
            assert abs(W[s, j] - sum(Psi[s, i] * float(A[i, j]) for i in range(9))) < 1e-12
    for i in range(9):
        for s in range(5):
            assert abs(Y[i, s] - sum(float(A[i, j]) * Om[j, s] for j in range(7))) < 1e-12


def test_randomized_id_statistics():
    """Randomized ID error is comparable to the deterministic one (Sec. 2.4)."""
    A = channel_field((8, 8, 8), 3, 80, seed=7, dtype=torch.float64).numpy()
    k, l = 10, 20
    Jd, Pd, _, _ = oracle.deterministic_id(A, k)
    ed = np.linalg.norm(A - A[:, Jd] @ Pd)
    errs = []
    for seed in range(20):
        J, P, _, _, _ = oracle.randomized_id(A, k, l, seed=seed)
        errs.append(np.linalg.norm(A - A[:, J] @ P))
    assert np.median(errs) <= 2.0 * ed
    s = np.linalg.svd(A, compute_uv=False)
    assert min(errs) >= np.sqrt(np.sum(s[k:] ** 2)) * (1 - 1e-10)


# ------------------------------------------------------------ sub-sampled ID

def test_coarse_rows_brute_force():
    grid, nc, st = (8, 6, 4), 3, (2, 3, 2)
    rows = oracle.coarse_rows(grid, nc, st)
    nx, ny, nz = grid
    expect = [r for r in range(nc * nx * ny * nz)
              if (r % nx) % 2 == 0 and ((r // (nx * nz)) % ny) % 3 == 0 and ((r // nx) % nz) % 2 == 0]
    assert rows.tolist() == expect


def test_subsampled_id_theorem21_bound():
    grid, nc, st, n, k = (12, 10, 12), 3, (2, 2, 2), 40, 6
    A = channel_field(grid, nc, n, seed=2, dtype=torch.float64).numpy()
    Jc, Pc, k_out, _, Ac = oracle.subsampled_id(A, k, grid, nc, st)
    assert k_out == k
    err = oracle.spectral_norm(A - A[:, Jc] @ Pc)
    ac_err = oracle.spectral_norm(Ac - Ac[:, Jc] @ Pc)
    taus = np.concatenate([np.linspace(0, 16, 33), [A.shape[0] / Ac.shape[0]]])
    rho = min(oracle.theorem21_rho(A, Ac, Pc, ac_err, k, t) for t in taus)
    assert err <= rho
    # lifting reproduces the coarse ID on the coarse rows
    rows = oracle.coarse_rows(grid, nc, st)
    assert np.allclose((A[:, Jc] @ Pc)[rows], Ac[:, Jc] @ Pc)


def test_theorem21_rho_hand_computed_values():
    """rho_k(tau) of Theorem 2.1 on a 4 x 2 example worked by hand (two-sided
    pin: a dropped factor, a swapped sigma index or a norm in place of its
    square changes these values).

    A_c = [[2, 1], [0, 1]] and A = [A_c; A_c], so A^T A = 2 A_c^T A_c.
    A_c^T A_c = [[4, 2], [2, 2]] has eigenvalues 3 +- sqrt(5), so
    sigma_1^2 = 3 + sqrt(5), sigma_2^2 = 3 - sqrt(5), and
    eps(tau) = lambda_max((2 - tau) A_c^T A_c) = (2 - tau)(3 + sqrt 5) for
    tau <= 2 and (2 - tau)(3 - sqrt 5) above.  The k = 1 ID of A_c pivots
    column 0 (norm 2 > sqrt 2); its R row is (-2, -1), so P_c = [1, 1/2],
    ||P_c||_2 = sqrt(5)/2, and A_c - A_c(:, 0) P_c = [[0, 0], [0, 1]] has
    2-norm 1.
    """
    Ac = np.array([[2.0, 1.0], [0.0, 1.0]])
    A = np.vstack([Ac, Ac])
    J, P, k_out, _ = oracle.column_id(Ac, 1)
    assert list(J) == [0] and np.allclose(P, [[1.0, 0.5]], rtol=0, atol=1e-15)
    ac_err = oracle.spectral_norm(Ac - Ac[:, J] @ P)
    assert abs(ac_err - 1.0) < 1e-14
    r5 = np.sqrt(5.0)
    s1, s2 = 3.0 + r5, 3.0 - r5                    # sigma_1^2, sigma_2^2
    pn = r5 / 2.0

    def rho(tau):
        eps = (2.0 - tau) * (s1 if tau <= 2.0 else s2)
        return (1.0 + pn) * np.sqrt(tau * s2 + eps) + 1.0 * np.sqrt(tau + eps / s1)

    for tau, closed in [(2.0, (1.0 + pn) * np.sqrt(2.0 * s2) + np.sqrt(2.0)),
                        (1.0, (1.0 + pn) * np.sqrt(6.0) + np.sqrt(2.0)),
                        (0.0, (1.0 + pn) * np.sqrt(2.0 * s1) + np.sqrt(2.0)),
                        (3.0, None)]:
        got = oracle.theorem21_rho(A, Ac, P, ac_err, 1, tau)
        assert abs(got - rho(tau)) <= 1e-12 * rho(tau)
        if closed is not None:
            assert abs(got - closed) <= 1e-12 * closed
    assert abs(oracle.theorem21_rho(A, Ac, P, ac_err, 1, 2.0) - 4.032247551) < 1e-8
    # the theorem's statement on this example: ||A - A_hat||_2 = sqrt(2)
    err = oracle.spectral_norm(A - A[:, J] @ P)
    assert abs(err - np.sqrt(2.0)) < 1e-14
    assert err <= min(oracle.theorem21_rho(A, Ac, P, ac_err, 1, t) for t in (0.0, 1.0, 2.0, 3.0))


# --------------------------------------------------------------- error metric

def test_recon_error_small_example():
    A = np.array([[1.0, 2.0, 3.0], [0.0, 1.0, 1.0]])
    J = np.array([0])
    P = np.array([[1.0, 2.0, 2.0]])
    fro, mx = oracle.recon_error(A, J, P)
    R = np.array([[0, 0, 1.0], [0, 1.0, 1.0]])
    assert fro == pytest.approx(np.sqrt(3.0) / np.sqrt(16.0))
    assert mx == pytest.approx(1.0)   # the zero entry A[1,0] is skipped


# ------------------------------------------------------------ planted mistakes

def test_planted_householder_sign_slip_is_caught(monkeypatch):
    real = idm.householder

    def wrong(x):
        v, tau, beta = real(x)
        return v, tau, -beta          # wrong sign on the R diagonal
    monkeypatch.setattr(idm, "householder", wrong)
    A = _rand(40, 30, 3, decay=0.85)
    J, P, _, _ = oracle.deterministic_id(A, 8)
    mask = np.ones(30, bool)
    mask[J] = False
    X, *_ = np.linalg.lstsq(A[:, J], A[:, mask], rcond=None)
    assert not np.allclose(P[:, mask], X, rtol=1e-6, atol=1e-8)


def test_planted_dropped_term_in_back_substitution_is_caught(monkeypatch):
    def wrong(U, Bm):
        X = np.array(Bm, dtype=np.float64, copy=True)
        for t in range(U.shape[0] - 1, -1, -1):
            X[t] /= U[t, t]           # forgets to subtract the solved rows
        return X
    monkeypatch.setattr(idm, "back_substitute", wrong)
    A = low_rank_matrix(100, 40, 6, 5).numpy()
    J, P, _, _ = oracle.deterministic_id(A, 6)
    fro, _ = oracle.recon_error(A, J, P)
    assert fro > 1e-6


def test_planted_stale_norms_are_caught(monkeypatch):
    """Pivoting on the initial norms (no update) violates the greedy pin."""
    def wrong_cpqr(B, k, rank_tol_factor=idm.RANK_TOL_FACTOR):
        B = np.asarray(B, dtype=np.float64)
        order = np.argsort(-np.linalg.norm(B, axis=0), kind="stable")[:k]
        J = np.array(order)
        Q, Rq = np.linalg.qr(B[:, J])
        return J, Q.T @ B, len(J), 1.0
    monkeypatch.setattr(idm, "cpqr", wrong_cpqr)
    g = np.random.default_rng(8)
    A = g.normal(size=(10, 6))
    A[:, 1] = A[:, 0] * 1.01 + 1e-3 * g.normal(size=10)   # near-duplicate of col 0
    J, P, _, _ = oracle.deterministic_id(A, 2)
    nu = _residual_norms_by_projection(A, [int(J[0])])
    nu[int(J[0])] = -1
    assert abs(nu[J[1]] - nu.max()) > 1e-6 * nu.max()
