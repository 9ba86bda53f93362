"""Learned skeleton proposal, FP64, step by step: the oracle of a small MLP
that scores snapshot columns from coarse-grid features and proposes a
candidate skeleton, refined by the exact pivoted QR restricted to the
candidates, with the plain randomized ID as fallback and judge.

TEST INFRASTRUCTURE ONLY (see the package header).

The paper has no learned component; its concluding section motivates the ID
as the selection of the most important snapshots (Sec. 4).  Readings taken
here:

* features of a column: the u-component (component 0) of the snapshot on a
  16 x 16 x 16 direct-injection sub-grid of the 128 x 96 x 128 channel grid
  (x and z every 8th index, y every 6th, from 0; the row order of
  ``coarse_rows``), 4096 values, multiplied by one global scale (the inverse
  RMS of the training features) so that the inputs are O(1);
* network: s = w2 . gelu(x W1 + b1) + b2 with 256 hidden units and the exact
  GELU, gelu(z) = z Phi(z) (Phi the standard normal CDF); its two dense
  products (x W1 and the W1 gradient X^T dZ) take bfloat16 operands with
  exact accumulation here (``product_round=bf16_operands``), the precision
  of the GPU's tensor-core products (which accumulate in FP32);
* training target: y_j = 1 when column j is in the skeleton the plain
  randomized ID picked on that window, else 0; loss: the mean binary cross
  entropy of sigmoid(s) against y, positives optionally weighted;
* proposal: the 2k columns of highest score (ties to the lower index), or,
  stratified, the 2 highest in each of k consecutive ranges of snapshots (the
  skeleton of a window spreads over its time span); the
  pivoted QR of W restricted to them gives J, and P over all columns is the
  least-squares fit of W on W(:, J), which for a pivoted QR equals
  R11^-1 R12 (Sec. 2.4), with P(:, J) = I exactly;
* fallback: the proposal is used when its reconstruction error is at most
  1.05 times the plain randomized ID's, else the plain ID is.
"""
from __future__ import annotations

import math

import numpy as np

from .interp_decomp import coarse_rows, column_id, recon_error

FEATURE_STRIDE = (8, 6, 8)
HIDDEN = 256


# ------------------------------------------------------------------ features

def feature_rows(grid, stride=FEATURE_STRIDE):
    """Rows of A that form a column's features: component 0 on the sub-grid."""
    return coarse_rows(grid, 1, stride)


def column_features(A, grid, stride=FEATURE_STRIDE, scale=1.0):
    """X (n x F): row j holds the features of snapshot column j, times scale."""
    A64 = np.asarray(A, dtype=np.float64)
    return scale * A64[feature_rows(grid, stride), :].T


def feature_scale(X):
    """One global scale: the inverse RMS of the feature values (1 if all zero)."""
    rms = math.sqrt(float(np.mean(np.asarray(X, dtype=np.float64) ** 2)))
    return 1.0 / rms if rms > 0.0 else 1.0


# ------------------------------------------------------------------- network

def _phi(z):
    return np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def _Phi(z):
    from scipy.special import ndtr
    return ndtr(z)


def gelu(z):
    """Exact GELU, z Phi(z)."""
    z = np.asarray(z, dtype=np.float64)
    return z * _Phi(z)


def gelu_grad(z):
    """d gelu / dz = Phi(z) + z phi(z)."""
    z = np.asarray(z, dtype=np.float64)
    return _Phi(z) + z * _phi(z)


def init_params(F, H=HIDDEN, seed=0):
    """W1 (F x H), b1 (H), w2 (H), b2: scaled Gaussian weights, zero biases."""
    rng = np.random.default_rng(seed)
    return {"W1": rng.standard_normal((F, H)) / math.sqrt(F),
            "b1": np.zeros(H),
            "w2": rng.standard_normal(H) / math.sqrt(H),
            "b2": 0.0}


def bf16_operands(M):
    """Every value rounded to the nearest bfloat16 (ties to even): the
    operand precision of the network's two dense products on the GPU."""
    from .rng import bf16_round_f64
    return bf16_round_f64(np.asarray(M, dtype=np.float64))[0]


def forward(X, p, product_round=None):
    """Scores s (n) and the cache (Z, G) of the hidden layer.

    product_round (e.g. bf16_operands) is applied to both operands of the
    product X W1 (bfloat16 weights and features, exact FP64 accumulation);
    None keeps them as they are."""
    X = np.asarray(X, dtype=np.float64)
    r = (lambda M: M) if product_round is None else product_round
    Z = r(X) @ r(p["W1"]) + p["b1"]
    G = gelu(Z)
    s = G @ p["w2"] + p["b2"]
    return s, (Z, G)


def sigmoid(s):
    s = np.asarray(s, dtype=np.float64)
    out = np.empty_like(s)
    pos = s >= 0
    out[pos] = 1.0 / (1.0 + np.exp(-s[pos]))
    e = np.exp(s[~pos])
    out[~pos] = e / (1.0 + e)
    return out


def bce_loss(s, y, pos_weight=1.0):
    """Mean binary cross entropy of sigmoid(s) against y in {0, 1}, the
    positive terms weighted by pos_weight; stable for large |s|:
    -log sigmoid(s) = softplus(-s), -log(1 - sigmoid(s)) = softplus(s)."""
    s = np.asarray(s, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    softplus = lambda t: np.maximum(t, 0.0) + np.log1p(np.exp(-np.abs(t)))   # noqa: E731
    return float(np.mean(pos_weight * y * softplus(-s) + (1.0 - y) * softplus(s)))


def backward(X, y, p, pos_weight=1.0, product_round=None):
    """Gradients of bce_loss(forward(X, p), y) with respect to every parameter.

    product_round, as in forward, also rounds both operands of the product
    X^T dZ that gives the W1 gradient."""
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    r = (lambda M: M) if product_round is None else product_round
    s, (Z, G) = forward(X, p, product_round)
    n = X.shape[0]
    sg = sigmoid(s)
    # d/ds of w y softplus(-s) + (1 - y) softplus(s) = -w y (1 - sg) + (1 - y) sg
    ds = (-pos_weight * y * (1.0 - sg) + (1.0 - y) * sg) / n
    gw2 = G.T @ ds
    gb2 = float(np.sum(ds))
    dZ = np.outer(ds, p["w2"]) * gelu_grad(Z)
    gW1 = r(X).T @ r(dZ)
    gb1 = np.sum(dZ, axis=0)
    return {"W1": gW1, "b1": gb1, "w2": gw2, "b2": gb2}


def sgd_step(p, g, lr):
    """Plain gradient descent: p - lr g, parameter by parameter."""
    return {key: p[key] - lr * g[key] for key in p}


def skeleton_labels(n, J):
    """y_j = 1 for the columns of the skeleton J (entries < 0 ignored)."""
    y = np.zeros(n)
    J = np.asarray(J)
    y[J[J >= 0]] = 1.0
    return y


# ------------------------------------------------------------------ proposal

def propose(scores, count):
    """The count columns of highest score (ties to the lower index), sorted."""
    scores = np.asarray(scores, dtype=np.float64)
    order = np.lexsort((np.arange(len(scores)), -scores))
    return np.sort(order[:count])


def propose_stratified(scores, strata, per):
    """The per highest scores (ties to the lower index) in each of strata
    consecutive column ranges [floor(q n / strata), floor((q + 1) n / strata)),
    all sorted: candidates spread over the window's snapshots in time."""
    scores = np.asarray(scores, dtype=np.float64)
    n = len(scores)
    out = []
    for q in range(strata):
        lo, hi = (q * n) // strata, ((q + 1) * n) // strata
        out.extend((lo + propose(scores[lo:hi], min(per, hi - lo))).tolist())
    return np.sort(np.array(out, dtype=np.int64))


def restricted_id(B, cand, k):
    """ID of B (l x n) whose skeleton is chosen by the pivoted QR of B(:, cand).

    Returns (J, P, k_out): J in pivot order (indices of B's columns), P
    (k_out x n) the least-squares fit of every column of B on B(:, J) with
    P(:, J) = I set exactly."""
    B = np.asarray(B, dtype=np.float64)
    cand = np.asarray(cand, dtype=np.int64)
    Jc, _, kout, _ = column_id(B[:, cand], k)
    J = cand[Jc[:kout]]
    P = np.linalg.lstsq(B[:, J], B, rcond=None)[0]
    P[:, J] = np.eye(kout)
    return J, P, kout


def choose_with_fallback(A, learned, plain, factor=1.05):
    """The learned ID (J, P) when its reconstruction error of A is at most
    factor times the plain one's, else the plain ID.  Returns
    ((J, P), used_learned, err_learned, err_plain)."""
    el, _ = recon_error(A, learned[0], learned[1])
    ep, _ = recon_error(A, plain[0], plain[1])
    if el <= factor * ep:
        return learned, True, el, ep
    return plain, False, el, ep
