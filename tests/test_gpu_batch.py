"""GPU parity of the batched form (id_batch_*): every problem of one
graph-launched batch against the oracle's randomized ID (Algorithm 4,
Sec. 2.4) on the same Psi and Omega, and against one handle per problem.

FP32 problems with aligned columns run in the work-list form (one persistent
launch over row ranges of all of them; the CTA that completes a matrix's
last range sums its W and runs its QR and solve); FP64 and unaligned
problems on their own graph branches.

Bars as for the single-handle randomized ID: k_out equal, P(:, J) = I exactly,
J equal where the oracle's pivot margin is >= 1e-4 (below it, the error of
the returned skeleton within 1.05x the oracle's), P within 1e-3 (FP32 data,
FP32-accurate sketch) or 1e-10 (FP64) of the oracle's, relative to max(1,
max|P|).  Against one handle on the same data: J equal where the margin
allows; P within 1e-9 for FP64 data (the same kernels and split), within the
FP32 bar for FP32 data (the work items split the rows of W's sums
differently from one handle's CTAs).
"""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle
from margins import MARGIN, assert_valid_skeleton
from synthetic import channel_field, low_rank_matrix

pytestmark = pytest.mark.gpu

DEV = "cuda"

# grid (nx = nz = 2 ny, 3 components), n, k, l, dtype, sketch precision
CASES = [
    ((8, 4, 8), 40, 6, 16, torch.float32, "exact"),      # m = 768
    ((12, 6, 12), 97, 12, 22, torch.float32, "exact"),   # m = 2,592, ragged n
    ((16, 8, 16), 200, 20, 30, torch.float32, "bf16"),   # m = 6,144, BF16 form
    ((20, 10, 20), 512, 30, 40, torch.float32, "exact"),  # m = 12,000, n at the limit
    ((16, 8, 16), 300, 16, 26, torch.float64, "exact"),  # FP64 data (SIMT sketch)
    ((8, 4, 8), 64, 10, 64, torch.float64, "exact"),     # l at the limit
    ((24, 12, 24), 130, 24, 34, torch.float32, "exact"),  # m = 20,736
    ((16, 8, 16), 200, 70, 80, torch.float32, "exact"),   # wide sketch: two Psi passes
    ((20, 10, 20), 300, 80, 90, torch.float32, "bf16"),   # wide, BF16 form, k = 80
]


def make_problems(seed0):
    probs = []
    for i, (grid, n, k, l, dtype, prec) in enumerate(CASES):
        A = channel_field(grid, 3, n, seed=seed0 + i, gap_k=k, dtype=dtype, device=DEV)
        probs.append(dict(A=A, k=k, l=l, seed=100 + i, prec=prec))
    return probs


def oracle_id(p):
    A = p["A"]
    An = (A.to(torch.bfloat16) if p.get("prec") == "bf16" else A).double().cpu().numpy()
    m, n = An.shape
    Wo, _ = oracle.sketch(An, oracle.psi(p["l"], m, p["seed"]), oracle.omega(n, p["l"], p["seed"]))
    return oracle.column_id(Wo, p["k"])


def check_against_oracle(p, J, P, kout):
    """J equal to the oracle's when its pivot margin is >= 1e-4; below that
    (pivots within rounding of a tie) a valid skeleton whose error on A is
    the oracle's within 1.05x (the equal-error bar).  Returns the margin."""
    Jo, Po, ko, margin = oracle_id(p)
    k = p["k"]
    assert kout == ko == k
    Jg, Pg = J.cpu().numpy(), P.cpu().numpy()
    assert_valid_skeleton(Jg, Pg, k, p["A"].shape[1])
    if margin < MARGIN:
        An = p["A"].double().cpu().numpy()
        fo, _ = oracle.recon_error(An, Jo, Po)
        fg, _ = oracle.recon_error(An, Jg, Pg)
        assert fg <= 1.05 * fo, (margin, fg, fo)
        return margin
    assert Jg.tolist() == Jo.tolist()
    tol = 1e-10 if p["A"].dtype == torch.float64 else 1e-3
    assert np.max(np.abs(Pg - Po)) <= tol * max(1.0, np.max(np.abs(Po)))
    return margin


def test_batch_matches_oracle_and_single_handles():
    from paper_1905_13257_gb300 import IdBatch, IdSketch
    probs = make_problems(seed0=20)
    bt = IdBatch(probs)
    bt.run()
    res = bt.wait()
    assert len(res) == len(probs)
    for p, (J, P, kout) in zip(probs, res):
        margin = check_against_oracle(p, J, P, kout)
        A = p["A"]
        sk = IdSketch(m=A.shape[0], n_max=A.shape[1], k=p["k"], l=p["l"], seed=p["seed"],
                      dtype=A.dtype, prec=p["prec"], want_Y=False)
        sk.stream_columns(A)
        J1, P1, k1 = sk.factor()
        assert k1 == kout
        if margin >= MARGIN:
            assert J1.tolist() == J.tolist()
        P1n = P1.cpu().numpy()
        tol = 1e-9 if A.dtype == torch.float64 else 1e-3
        if J1.tolist() == J.tolist():
            assert np.max(np.abs(P.cpu().numpy() - P1n)) <= tol * max(1.0, np.abs(P1n).max())
        sk.close()
    bt.close()


def test_batch_replay_reads_new_data_and_counts_launches():
    from paper_1905_13257_gb300 import IdBatch, load
    lib = load()
    probs = make_problems(seed0=40)
    bt = IdBatch(probs)
    bt.run()
    bt.wait()
    # the graph is captured: a replay launches the same kernels again
    l0 = lib.id_kernel_launches()
    bt.run()
    bt.wait()
    per_run = lib.id_kernel_launches() - l0
    # the FP32 problems share one persistent launch (sketches, slab sums, QRs
    # and solves); each FP64 problem has its own chain of kernels
    n64 = sum(1 for p in probs if p["A"].dtype == torch.float64)
    assert 1 + 2 * n64 <= per_run <= 1 + 4 * n64
    # overwrite the data in place: the replay must see the new matrices
    for i, p in enumerate(probs):
        grid, n, k = CASES[i][0], CASES[i][1], CASES[i][2]
        p["A"].copy_(channel_field(grid, 3, n, seed=70 + i, gap_k=k, dtype=p["A"].dtype,
                                   device=DEV))
    l1 = lib.id_kernel_launches()
    bt.run()
    res = bt.wait()
    assert lib.id_kernel_launches() - l1 == per_run
    for i in (0, 3, 4):
        check_against_oracle(probs[i], *res[i])
    bt.close()


def test_batch_rank_deficient_problem():
    from paper_1905_13257_gb300 import IdBatch
    A1 = low_rank_matrix(3000, 60, 5, seed=3, dtype=torch.float64, device=DEV)
    A2 = channel_field((8, 4, 8), 3, 50, seed=4, gap_k=8, dtype=torch.float32, device=DEV)
    probs = [dict(A=A1, k=12, l=20, seed=5), dict(A=A2, k=8, l=18, seed=6)]
    bt = IdBatch(probs)
    bt.run()
    (J1, P1, k1), (J2, P2, k2) = bt.wait()
    Jo, Po, ko, _ = oracle.column_id(
        oracle.sketch(A1.cpu().numpy(), oracle.psi(20, 3000, 5), oracle.omega(60, 20, 5))[0], 12)
    assert k1 == ko == 5
    assert J1.cpu().tolist()[5:] == [-1] * 7
    assert k2 == 8
    check_against_oracle(probs[1], J2, P2, k2)
    bt.close()


def test_batch_output_pointers_and_errors():
    from paper_1905_13257_gb300 import IdBatch, IdError, load
    from paper_1905_13257_gb300 import _binding as B
    lib = load()
    probs = make_problems(seed0=60)[:3]
    bt = IdBatch(probs)
    with pytest.raises(IdError) as e:          # no run yet
        bt.wait()
    assert e.value.status == B.ID_ERR_STATE
    bt.run()
    first = [(J.clone(), P.clone(), k) for J, P, k in bt.wait()]
    # host output pointers are rejected
    Jh = torch.empty_like(bt.J, device="cpu")
    Ph = torch.empty_like(bt.P, device="cpu")
    kh = torch.empty_like(bt.kout, device="cpu")
    st = lib.id_batch_run(bt.h, C.c_void_p(Jh.data_ptr()), C.c_void_p(Ph.data_ptr()),
                          C.c_void_p(kh.data_ptr()))
    assert st == B.ID_ERR_INVALID_ARG
    # other device outputs: the batch captures again and writes there
    bt.J, bt.P, bt.kout = torch.zeros_like(bt.J), torch.zeros_like(bt.P), torch.zeros_like(bt.kout)
    bt.run()
    for (J, P, k), (J0, P0, k0) in zip(bt.wait(), first):
        assert k == k0 and torch.equal(J, J0)
        assert torch.allclose(P, P0, rtol=0, atol=1e-12)
    bt.close()


def test_batch_autotuner_keeps_the_results():
    """id_batch_tune times the candidate work splits, keeps the fastest, and
    the batch run with it still matches the oracle problem by problem."""
    from paper_1905_13257_gb300 import IdBatch
    probs = make_problems(seed0=80)
    bt = IdBatch(probs)
    choice, ms = bt.tune()
    assert choice in ms and all(v > 0 for v in ms.values())
    assert ms[choice] == min(ms.values())
    bt.run()
    for p, (J, P, kout) in zip(probs, bt.wait()):
        check_against_oracle(p, J, P, kout)
    bt.close()


def test_batch_mixed_forms_and_item_sizes():
    """An FP32 problem whose leading dimension is not a multiple of 4 leaves
    the work list for its own branch, beside work-list problems and an FP64
    one; every candidate work-item size of the tuner gives the oracle's
    result (the tuner leaves the last result in the outputs), and so does a
    replay with the chosen size."""
    from paper_1905_13257_gb300 import IdBatch
    probs = []
    for i, (grid, n, k, l, dtype, prec) in enumerate(CASES[:5]):
        A = channel_field(grid, 3, n, seed=90 + i, gap_k=k, dtype=dtype, device=DEV)
        probs.append(dict(A=A, k=k, l=l, seed=300 + i, prec=prec))
    m = probs[1]["A"].shape[0]
    buf = torch.zeros(probs[1]["A"].shape[1], m + 1, dtype=torch.float32, device=DEV)
    buf[:, :m] = probs[1]["A"].T
    probs[1]["A"] = buf[:, :m].T            # column-major, lda = m + 1
    assert probs[1]["A"].stride() == (1, m + 1)
    bt = IdBatch(probs)
    choice, ms = bt.tune()
    assert set(ms) == {0, 32, 16, 8, 4} and ms[choice] == min(ms.values())
    for p, (J, P, kout) in zip(probs, bt.wait()):
        check_against_oracle(p, J, P, kout)
    bt.run()
    for p, (J, P, kout) in zip(probs, bt.wait()):
        check_against_oracle(p, J, P, kout)
    bt.close()
