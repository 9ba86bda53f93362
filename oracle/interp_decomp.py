"""Plain FP64 interpolative decomposition (ID), step by step.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the CUDA library
never calls it and shares no code with it.

Orientation.  The paper stores snapshots as ROWS of A and computes a row ID
A ~ P A(I,:) (Sec. 2.4, eq. ``eqn:id``).  Here A is (grid points x components)
x snapshots, i.e. the paper's A transposed, and the decomposition is the column
ID  A ~ A(:,J) P  with P (k x n), P(:,J) = I.  Remark 2.1 notes that row and
column IDs are the same construction on A^T; J plays the paper's I and
P here is the paper's P transposed.

Everything is FP64; FP32 inputs are converted exactly.
"""
from __future__ import annotations

import numpy as np

EPS64 = np.finfo(np.float64).eps
# Rank tolerance: pivoting stops once every residual column norm is at most
# RANK_TOL_FACTOR * eps * ||B||_F (the paper's pseudo-inverse in Algorithm 3
# step 4 only matters once R11 becomes singular; this is where that happens).
RANK_TOL_FACTOR = 64.0


def sketch(A, Psi, Omega):
    """Both randomized sketches by their definition (FP64 products).

    W = Psi A (l x n) is the paper's sketch Y = A Omega of Algorithm 4 step 3
    written for the transposed orientation; Y = A Omega (m x l) is the range
    sketch of the same data (Sec. 2.2, eq. ``eq:sampmatrix``).
    """
    A64 = np.asarray(A, dtype=np.float64)
    W = np.asarray(Psi, dtype=np.float64) @ A64
    Y = A64 @ np.asarray(Omega, dtype=np.float64)
    return W, Y


def householder(x):
    """Householder reflector of Golub & Van Loan Sec. 5.1 in the LAPACK sign
    convention: H = I - tau v v^T, v[0] = 1, H x = beta e_1, beta = -sign(x0)||x||.
    Returns (v, tau, beta).  A vector with x[1:] == 0 gives tau = 0, beta = x0.
    """
    x = np.asarray(x, dtype=np.float64)
    alpha = x[0]
    sigma = float(x[1:] @ x[1:])
    v = np.zeros_like(x)
    v[0] = 1.0
    if sigma == 0.0:
        return v, 0.0, alpha
    norm = np.sqrt(alpha * alpha + sigma)
    beta = -norm if alpha >= 0.0 else norm
    tau = (beta - alpha) / beta
    v[1:] = x[1:] / (alpha - beta)
    return v, tau, beta


def cpqr(B, k, rank_tol_factor=RANK_TOL_FACTOR):
    """k steps of column-pivoted Householder QR of B (Algorithm 3 step 3).

    The paper uses pivoted modified Gram-Schmidt (mgsqr); in exact arithmetic
    Householder QR with the same pivot rule gives the same pivots and R.
    Pivot rule: at step s take the non-pivoted column whose residual norm
    ||B^(s)(s:, j)||, recomputed afresh at every step, is largest; among equal
    norms the lowest column index wins.  Columns stay in place (no swaps).

    Returns (J, R, k_out, margin):
      J      pivot column indices, in pivot order (length k_out)
      R      k_out x n; R[s, j] is row s of the triangular factor for original
             column j, so R[:, J] is upper triangular (R11) and R[:, Jc] is R12
      k_out  number of pivots taken (< k when the residual fell below the
             rank tolerance)
      margin min over steps of (nu1 - nu2) / nu1, the gap between the two
             largest residual norms; pivot parity is only meaningful when it is
             comfortably above rounding level
    """
    from scipy.linalg.blas import dger
    M = np.array(B, dtype=np.float64, order="F", copy=True)   # columns contiguous
    rows, n = M.shape
    kmax = min(int(k), rows, n)
    pivoted = np.zeros(n, dtype=bool)
    J = []
    R = np.zeros((kmax, n))
    tol = rank_tol_factor * EPS64 * np.sqrt(float(np.einsum("ij,ij->", M, M)))
    margin = np.inf
    vfull = np.zeros(rows)
    for s in range(kmax):
        Ms = M[s:, :]
        nu = np.sqrt(np.einsum("ij,ij->j", Ms, Ms))   # ||B^(s)(s:, j)||, afresh
        nu[pivoted] = -1.0
        p = int(np.argmax(nu))          # first maximum = lowest index
        if not nu[p] > tol:
            break
        rest = np.sort(nu)[::-1]
        if n - s > 1 and rest[0] > 0:
            margin = min(margin, (rest[0] - max(rest[1], 0.0)) / rest[0])
        v, tau, beta = householder(M[s:, p])
        pivoted[p] = True
        J.append(p)
        if tau != 0.0:
            # H = I - tau v v^T on rows s.. of the non-pivoted columns: the
            # rank-one update B(s:, j) -= tau v (v^T B(s:, j)) (BLAS dger on
            # the whole matrix, v zero above row s; pivoted columns get w = 0)
            w = v @ Ms
            w[pivoted] = 0.0
            vfull[:] = 0.0
            vfull[s:] = v
            M = dger(-tau, vfull, w, a=M, overwrite_a=True)
        M[s, p] = beta
        M[s + 1:, p] = 0.0
        R[s, :] = M[s, :]
    k_out = len(J)
    return np.array(J, dtype=np.int64), R[:k_out].copy(), k_out, margin


def back_substitute(U, Bm):
    """Solve U X = Bm for upper-triangular U by back-substitution, row by row."""
    U = np.asarray(U, dtype=np.float64)
    X = np.array(Bm, dtype=np.float64, copy=True)
    k = U.shape[0]
    for t in range(k - 1, -1, -1):
        if t + 1 < k:
            X[t] -= U[t, t + 1:] @ X[t + 1:]
        X[t] /= U[t, t]
    return X


def interpolation_matrix(J, R, n):
    """P from the CPQR factors (Algorithm 3 steps 4-6, transposed).

    C = R11^{-1} R12 (the paper's pseudo-inverse is the inverse while R11 is
    non-singular, which the rank tolerance guarantees); P(:,J) = I_k and
    P(:,Jc) = C, so that A ~ A(:,J) P.
    """
    J = np.asarray(J, dtype=np.int64)
    k = len(J)
    P = np.zeros((k, n))
    if k == 0:
        return P
    mask = np.ones(n, dtype=bool)
    mask[J] = False
    Jc = np.nonzero(mask)[0]
    R11 = R[:, J]
    C = back_substitute(R11, R[:, Jc])
    P[:, Jc] = C
    P[np.arange(k), J] = 1.0
    return P


def column_id(B, k, rank_tol_factor=RANK_TOL_FACTOR):
    """Column ID of B: returns (J, P, k_out, margin) with B ~ B(:,J) P."""
    J, R, k_out, margin = cpqr(B, k, rank_tol_factor)
    return J, interpolation_matrix(J, R, np.asarray(B).shape[1]), k_out, margin


def deterministic_id(A, k):
    """Algorithm 3 (row ID of A^T = column ID of A)."""
    return column_id(A, k)


def randomized_id(A, k, l, seed, Psi=None):
    """Algorithm 4 transposed: ID of the sketch W = Psi A, applied to A.

    Returns (J, P, k_out, margin, W).
    """
    from .rng import psi as _psi
    A64 = np.asarray(A, dtype=np.float64)
    if Psi is None:
        Psi = _psi(l, A64.shape[0], seed)
    W = Psi @ A64
    J, P, k_out, margin = column_id(W, k)
    return J, P, k_out, margin, W


def coarse_rows(grid, ncomp, stride):
    """Row indices of the coarse grid (direct injection, Sec. 2.5 eq. ``eq:A_c``).

    Row layout of A: r = ((c*ny + j)*nz + kz)*nx + i (component slowest, then
    y, then z, x fastest).  The coarse grid keeps every stride-th index in each
    direction starting at 0, for every component, in increasing row order.
    """
    nx, ny, nz = grid
    sx, sy, sz = stride
    out = []
    for c in range(ncomp):
        for j in range(0, ny, sy):
            for kz in range(0, nz, sz):
                for i in range(0, nx, sx):
                    out.append(((c * ny + j) * nz + kz) * nx + i)
    return np.array(out, dtype=np.int64)


def subsampled_id(A, k, grid, ncomp, stride):
    """Algorithm 5 transposed: deterministic ID of A_c = A(rows_c, :).

    The pair (J_c, P_c) then induces the lifted ID A ~ A(:, J_c) P_c
    (eq. ``eq:coarseregA``).  Returns (J_c, P_c, k_out, margin, A_c).
    """
    rows = coarse_rows(grid, ncomp, stride)
    Ac = np.asarray(A, dtype=np.float64)[rows, :]
    J, P, k_out, margin = column_id(Ac, k)
    return J, P, k_out, margin, Ac


def recon_error(A, J, P):
    """Errors of the reconstruction A_hat = A(:,J) P.

    rel_fro: ||A - A_hat||_F / ||A||_F (the Frobenius metric of Sec. 3.3).
    rel_max: max_{ij} |A_ij - A_hat_ij| / |A_ij| (the entry-wise metric of
             Sec. 3.1); entries with A_ij == 0, where the ratio is undefined,
             are skipped.
    """
    A64 = np.asarray(A, dtype=np.float64)
    Ahat = A64[:, np.asarray(J, dtype=np.int64)] @ np.asarray(P, dtype=np.float64)
    Rm = A64 - Ahat
    rel_fro = np.sqrt(np.sum(Rm * Rm)) / np.sqrt(np.sum(A64 * A64))
    nz = A64 != 0.0
    rel_max = float(np.max(np.abs(Rm[nz]) / np.abs(A64[nz]))) if np.any(nz) else 0.0
    return float(rel_fro), rel_max


def spectral_norm(M):
    """Largest singular value (dense SVD; small matrices only)."""
    M = np.asarray(M, dtype=np.float64)
    if M.size == 0:
        return 0.0
    return float(np.linalg.svd(M, compute_uv=False)[0])


def theorem21_rho(A, Ac, Pc, Ac_err2, k, tau):
    """rho_k(tau) of Theorem 2.1, in the transposed orientation.

    The paper's Gramians A A^T and A_c A_c^T (snapshot x snapshot) are A^T A
    and A_c^T A_c here; sigma_k, sigma_{k+1} are singular values of A_c;
    ||P_c||_2 and ||A_c - A_c_hat||_2 are spectral norms.
    """
    A64 = np.asarray(A, dtype=np.float64)
    Ac64 = np.asarray(Ac, dtype=np.float64)
    G = A64.T @ A64 - tau * (Ac64.T @ Ac64)
    eps_tau = float(np.linalg.eigvalsh(G)[-1])
    sv = np.linalg.svd(Ac64, compute_uv=False)
    s_k = sv[k - 1]
    s_k1 = sv[k] if k < len(sv) else 0.0
    pn = spectral_norm(Pc)
    term1 = (1.0 + pn) * np.sqrt(max(tau * s_k1 * s_k1 + eps_tau, 0.0))
    term2 = Ac_err2 * np.sqrt(max(tau + eps_tau / (s_k * s_k), 0.0))
    return float(term1 + term2)
