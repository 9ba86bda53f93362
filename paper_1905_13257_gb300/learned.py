"""The learned skeleton proposal on the GPU: a small network scores snapshot
columns from coarse-grid features, its 2k best columns are refined by the
exact pivoted QR restricted to them, and the plain randomized ID is the
fallback and the judge of its error.

No counterpart in the paper, whose conclusion motivates the ID as the choice
of the most important snapshots (Sec. 4).  Every arithmetic step runs in the
library's kernels (id_mlp_features, id_mlp_forward / _backward / _sgd with
tensor-core products in bfloat16 and FP32 accumulation, id_mlp_propose,
id_factor_restricted, id_reconstruct_error); this module orders the calls.

Training data are the skeletons the plain randomized ID picked on earlier
windows of the same snapshot stream: label 1 for a column in the skeleton,
0 otherwise, mean binary cross entropy with the positives weighted by
(n - k) / k, plain SGD one window at a time.
"""
from __future__ import annotations

import math
import time

import numpy as np
import torch

from .api import IdSketch, Mlp, mlp_features
from . import _binding as B

FEATURE_STRIDE = (8, 6, 8)
HIDDEN = 256


def feature_rows(grid, stride=FEATURE_STRIDE):
    """Rows of A holding the u-component (component 0) on the direct-injection
    sub-grid of the channel grid (every stride-th index from 0 in x, y, z),
    in increasing row order (row r = (j nz + kz) nx + i of component 0)."""
    nx, ny, nz = grid
    sx, sy, sz = stride
    j = np.arange(0, ny, sy)[:, None, None]
    kz = np.arange(0, nz, sz)[None, :, None]
    i = np.arange(0, nx, sx)[None, None, :]
    return ((j * nz + kz) * nx + i).reshape(-1).astype(np.int64)


def init_params(F, H=HIDDEN, seed=0):
    """Scaled Gaussian weights (W1 ~ N(0, 1/F), w2 ~ N(0, 1/H)), zero biases."""
    rng = np.random.default_rng(seed)
    return {"W1": rng.standard_normal((F, H)) / math.sqrt(F), "b1": np.zeros(H),
            "w2": rng.standard_normal(H) / math.sqrt(H), "b2": 0.0}


class LearnedProposal:
    """Network, feature gather and proposal of the learned skeleton choice."""

    def __init__(self, grid, k, hidden=HIDDEN, stride=FEATURE_STRIDE, seed=0, stream=None):
        self.grid, self.k = tuple(grid), int(k)
        self.rows = torch.as_tensor(feature_rows(grid, stride), device="cuda")
        self.F = int(self.rows.numel())
        self.net = Mlp(init_params(self.F, hidden, seed), stream=stream)
        self.scale = None
        self.lib = B.load()

    def features(self, A):
        """X (n x F) of the columns of A, times the global feature scale (set
        from the first call: the inverse RMS of its features)."""
        if self.scale is None:   # a host-side statistic of the first window
            X = mlp_features(A, self.rows, 1.0, stream=self.net.stream).cpu().numpy()
            rms = math.sqrt(float(np.mean(X.astype(np.float64) ** 2)))
            self.scale = 1.0 / rms if rms > 0 else 1.0
        return mlp_features(A, self.rows, self.scale, stream=self.net.stream)

    def train_step(self, X, y, lr, pos_weight):
        """One SGD step of the mean binary cross entropy on (X, y); returns
        the scores of the forward pass (before the step)."""
        s = self.net.forward(X).clone()
        self.net.step(self.net.backward(X, y, pos_weight), lr)
        return s

    def propose(self, X, count=None, stratified=True):
        """2k candidate columns (a CUDA int32 tensor, increasing order): by
        default the 2 highest scores in each of k consecutive ranges of the
        window's snapshots (id_mlp_propose_stratified); stratified=False takes
        the count (default 2k) highest scores overall (id_mlp_propose)."""
        return propose_from_scores(self.lib, self.net.forward(X), self.k, count, stratified,
                                   self.net._sh)


def propose_from_scores(lib, s, k, count=None, stratified=True, sh=None):
    """Candidates from scores s (CUDA FP32) by the library's proposal kernels."""
    sh = B.C.c_void_p(torch.cuda.current_stream().cuda_stream) if sh is None else sh
    n = s.numel()
    if stratified:
        cand = torch.empty(2 * k, dtype=torch.int32, device=s.device)
        cnt = torch.zeros(1, dtype=torch.int32, device=s.device)
        B.check(lib.id_mlp_propose_stratified(B.C.c_void_p(s.data_ptr()), n, k, 2,
                                              B.C.c_void_p(cand.data_ptr()),
                                              B.C.c_void_p(cnt.data_ptr()), sh),
                "id_mlp_propose_stratified")
        return cand[: int(cnt.item())]
    count = 2 * k if count is None else int(count)
    cand = torch.empty(count, dtype=torch.int32, device=s.device)
    B.check(lib.id_mlp_propose(B.C.c_void_p(s.data_ptr()), n, count,
                               B.C.c_void_p(cand.data_ptr()), sh), "id_mlp_propose")
    return cand


def bce(s, y, pos_weight):
    """Mean weighted binary cross entropy of sigmoid(s) (a host-side report)."""
    s = np.asarray(s, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    sp = lambda t: np.maximum(t, 0.0) + np.log1p(np.exp(-np.abs(t)))   # noqa: E731
    return float(np.mean(pos_weight * y * sp(-s) + (1.0 - y) * sp(s)))


def plain_skeleton(sk, A, chunk=32):
    """The plain randomized ID of the columns of A (reset handle sk): J, P."""
    sk.reset()
    n = A.shape[1]
    for j0 in range(0, n, chunk):
        sk.stream_columns(A[:, j0:j0 + chunk])
    J, P, kout = sk.factor()
    return J[:kout], P[:kout]


def compare_on_window(prop, sk, A, rng, untrained=None):
    """Plain randomized ID against the learned proposal on one window (and
    against the same proposal rule fed by an untrained network and by random
    scores): reconstruction errors, the fallback decision (proposal used when
    its error is within 1.05x the plain one's), recall of the plain skeleton
    by the candidates, and the time of the pivoted QR over all n columns
    against scoring + proposal + the QR restricted to the candidates."""
    k = prop.k
    n = A.shape[1]
    sk.reset()
    for j0 in range(0, n, 32):
        sk.stream_columns(A[:, j0:j0 + 32])
    sk.flush()
    X = prop.features(A)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Jp, Pp, kp = sk.factor()
    torch.cuda.synchronize()
    t_plain = time.perf_counter() - t0
    t0 = time.perf_counter()
    cand = prop.propose(X)
    Jl, Pl, kl = sk.factor_restricted(cand)
    torch.cuda.synchronize()
    t_learned = time.perf_counter() - t0
    jp = set(Jp[:kp].cpu().tolist())
    ep, _ = sk.reconstruct_error(A, Jp[:kp], Pp[:kp])
    el, _ = sk.reconstruct_error(A, Jl[:kl], Pl[:kl])
    out = {"err_plain": ep, "err_learned": el, "use_learned": el <= 1.05 * ep,
           "recall_learned": len(jp & set(cand.cpu().tolist())) / max(kp, 1),
           "qr_plain_s": t_plain, "proposal_and_qr_s": t_learned}
    others = {"random": torch.as_tensor(rng.random(n), dtype=torch.float32, device="cuda")}
    if untrained is not None:
        others["untrained"] = untrained.net.forward(X)
    for name, sc in others.items():
        c = propose_from_scores(prop.lib, sc, k)
        Jo, Po, ko = sk.factor_restricted(c)
        out[f"err_{name}"] = sk.reconstruct_error(A, Jo[:ko], Po[:ko])[0]
        out[f"recall_{name}"] = len(jp & set(c.cpu().tolist())) / max(kp, 1)
    return out
