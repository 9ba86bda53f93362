"""The learned skeleton proposal trained on the GPU and judged against the
plain randomized ID (paper_1905_13257_gb300.learned).

A reduced stream of the channel generator: 32 x 32 x 32 x 3 = 98,304 rows,
windows of 512 snapshots (k = 50, l = 60), 4096 features (the u-component
on the 16 x 16 x 16 sub-grid of stride 2).  The network is trained by the
library's kernels on the plain ID's skeletons of 24 earlier windows and
judged on 6 later ones.  What the test establishes:
  * training lowers the loss (the forward, backward and SGD kernels learn);
  * on the training windows the trained network's candidates (2 in each of
    k consecutive ranges of snapshots) hold more of the plain skeleton than
    the same network's before training (it fits what it was shown);
  * on every held-out window the chosen ID (the proposal when its error is
    within 1.05x the plain one's, else the plain ID) meets the equal-error
    bar, and the numbers of the comparison with the untrained network and
    with random scores under the same rule (recall, error ratios, fallback
    rate, time of the pivoted QR) are printed.
"""
import numpy as np
import pytest
import torch

from synthetic.channel import channel_field, snapshot_step

pytestmark = pytest.mark.gpu

GRID, N, K, L = (32, 32, 32), 512, 50, 60
STRIDE = (2, 2, 2)


def window(w):
    return channel_field(GRID, 3, N, seed=0, dtype=torch.float32, device="cuda",
                         first=w * N, dt=snapshot_step(1000))


def test_learned_proposal_trains_and_meets_the_equal_error_bar():
    from paper_1905_13257_gb300 import IdSketch
    from paper_1905_13257_gb300.learned import (LearnedProposal, bce, compare_on_window,
                                                plain_skeleton)
    m = 3 * GRID[0] * GRID[1] * GRID[2]
    sk = IdSketch(m, N, K, L, seed=0, dtype=torch.float32, want_Y=False)
    prop = LearnedProposal(GRID, K, stride=STRIDE, seed=1)
    untrained = LearnedProposal(GRID, K, stride=STRIDE, seed=1)   # the same network, untrained
    assert prop.F == 4096
    train, held = range(0, 24), range(24, 30)
    data = []
    for w in train:
        A = window(w)
        J, _ = plain_skeleton(sk, A)
        y = torch.zeros(N, dtype=torch.float32, device="cuda")
        y[J.long()] = 1.0
        data.append((prop.features(A), y))
    pw = (N - K) / K
    losses = []
    for epoch in range(6):
        tot = 0.0
        for X, y in data:
            s = prop.train_step(X, y, lr=0.05, pos_weight=pw)
            tot += bce(s.cpu().numpy(), y.cpu().numpy(), pw)
        losses.append(tot / len(data))
    prop.net.check()
    print("training loss per epoch", [round(v, 4) for v in losses])
    assert losses[-1] < 0.9 * losses[0]
    # fit on the training windows: recall of the plain skeleton by the 2k
    # candidates of the trained network against the untrained one's
    untrained.scale = prop.scale
    rec_t, rec_u = [], []
    for X, y in data:
        rec_t.append(float(y[prop.propose(X).long()].sum().item()) / K)
        rec_u.append(float(y[untrained.propose(X).long()].sum().item()) / K)
    print(f"training windows: candidate recall trained {np.mean(rec_t):.3f}, "
          f"untrained {np.mean(rec_u):.3f}")
    assert np.mean(rec_t) > np.mean(rec_u)
    rng = np.random.default_rng(7)
    rows = []
    for w in held:
        r = compare_on_window(prop, sk, window(w), rng, untrained=untrained)
        rows.append(r)
        chosen = r["err_learned"] if r["use_learned"] else r["err_plain"]
        assert chosen <= 1.05 * r["err_plain"]
        assert r["use_learned"] == (r["err_learned"] <= 1.05 * r["err_plain"])
    ratio = {key: [r[f"err_{key}"] / r["err_plain"] for r in rows]
             for key in ("learned", "untrained", "random")}
    recall = {key: float(np.mean([r[f"recall_{key}"] for r in rows]))
              for key in ("learned", "untrained", "random")}
    print("held-out windows (2 candidates in each of k ranges of snapshots): error / plain "
          f"error: trained {np.round(ratio['learned'], 3).tolist()}, untrained "
          f"{np.round(ratio['untrained'], 3).tolist()}, random scores "
          f"{np.round(ratio['random'], 3).tolist()}; recall {recall}; proposal used "
          f"{sum(r['use_learned'] for r in rows)}/{len(rows)}; QR over n "
          f"{1e3 * np.median([r['qr_plain_s'] for r in rows]):.2f} ms, proposal + restricted QR "
          f"{1e3 * np.median([r['proposal_and_qr_s'] for r in rows]):.2f} ms")
    sk.close()
