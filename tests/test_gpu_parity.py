"""GPU parity: every step of the hot path through the C ABI against the oracle.

Tolerances (spec bars, and the arithmetic behind the rest):
  sketches W, Y   relative Frobenius <= 1e-5 for FP32 data (FP32-accurate
                  products, FP64 accumulation of W); <= 1e-12 for FP64 data
  skeleton J      identical on gap inputs (their seeds give an oracle pivot
                  margin >= 1e-4); elsewhere identical when the margin is
                  >= 1e-4, otherwise a valid skeleton (P(:, J) = I) with the
                  oracle's error
  P               from the same W: max |dP| <= 1e-9 * max(1, |P|) (FP64 QR on
                  both sides); end to end: bounded by the W error x cond(R11)
  rel. Frobenius  |e - e_oracle| <= 1e-4 * e_oracle for FP32 data (the
  error           spec bar, no absolute term), 1e-10 * e_oracle for FP64
  entry-wise      |e - e_oracle| <= 1e-4 * e_oracle (+ the FP32 rounding of
  error           A_hat at the maximising entry, where A_ij is tiny)
"""
import numpy as np
import pytest
import torch

import oracle
from margins import MARGIN, assert_valid_skeleton, sketch_seed_with_margin
from synthetic import channel_field, low_rank_matrix, gaussian_matrix

pytestmark = pytest.mark.gpu

DEV = "cuda"


def _sk(**kw):
    from paper_1905_13257_gb300 import IdSketch
    return IdSketch(**kw)


def err_tol(fo, dtype):
    """Bar on the relative Frobenius error: 1e-4 relative for FP32 data
    (the benchmark spec), 1e-10 relative for FP64 data."""
    return (1e-4 if dtype == torch.float32 else 1e-10) * fo


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def stream(sk, A, chunks):
    j = 0
    for c in chunks:
        sk.stream_columns(A[:, j:j + c])
        j += c
    assert j == A.shape[1]


# ----------------------------------------------------------------- generator

@pytest.mark.parametrize("which,first,count,width,seed", [
    (1, 0, 1000, 60, 0), (1, 4_718_000, 592, 60, 0), (2, 0, 1000, 60, 0),
    (1, 123, 77, 30, 0xDEADBEEF12345678), (2, 5, 9, 7, 3)])
def test_gaussian_bitwise(which, first, count, width, seed):
    from paper_1905_13257_gb300 import gaussian_fill
    g = gaussian_fill(which, seed, first, count, width).cpu().double().numpy()
    idx = np.arange(first, first + count)
    if which == 1:
        o = oracle.psi(width, 0, seed, rows=idx).T
    else:
        o = oracle.omega(0, width, seed, cols=idx)
    assert np.array_equal(g, o)


# ------------------------------------------------------------------ sketches

@pytest.mark.parametrize("dtype,tol", [(torch.float32, 1e-5), (torch.float64, 1e-12)])
@pytest.mark.parametrize("grid,n,l,chunks,window", [
    ((16, 12, 16), 100, 30, [32, 32, 32, 4], 0),        # ragged n, several launches
    ((10, 7, 9), 37, 16, [37], 0),                      # m not a multiple of 64
    ((16, 8, 16), 333, 60, [32] * 10 + [13], 96),       # borrowed windows of 96
    ((8, 8, 8), 700, 64, [350, 350], 0),                # > one SIMT window (320)
])
def test_sketch_parity(dtype, tol, grid, n, l, chunks, window):
    A = channel_field(grid, 3, n, seed=3, dtype=dtype, device=DEV)
    m = A.shape[0]
    sk = _sk(m=m, n_max=n, k=min(8, l), l=l, seed=11, dtype=dtype, want_Y=True,
             window_cols=window)
    stream(sk, A, chunks)
    W, Y, _ = sk.sketches()
    An = A.cpu().double().numpy()
    Wo, Yo = oracle.sketch(An, oracle.psi(l, m, 11), oracle.omega(n, l, 11))
    assert rel(W.cpu().numpy(), Wo) <= tol
    assert rel(Y.cpu().double().numpy(), Yo) <= tol
    sk.close()


def test_sketch_leading_dimension_and_separate_buffers():
    m, n, l = 3000, 70, 20
    base = gaussian_matrix(m + 17, n, seed=1, dtype=torch.float32, device=DEV)
    A = base[:m]                            # lda = m + 17 > m
    parts = [A[:, :30].clone(), A[:, 30:31].clone(), A[:, 31:]]   # three buffers
    sk = _sk(m=m, n_max=n, k=5, l=l, seed=2, dtype=torch.float32, window_cols=64)
    for p in parts:
        sk.stream_columns(p)
    W, Y, _ = sk.sketches()
    Wo, Yo = oracle.sketch(A.cpu().double().numpy(), oracle.psi(l, m, 2), oracle.omega(n, l, 2))
    assert rel(W.cpu().numpy(), Wo) <= 1e-5
    assert rel(Y.cpu().double().numpy(), Yo) <= 1e-5
    sk.close()


def test_reset_and_restream():
    A = channel_field((8, 8, 8), 3, 50, seed=1, dtype=torch.float32, device=DEV)
    m = A.shape[0]
    sk = _sk(m=m, n_max=50, k=5, l=16, seed=4, dtype=torch.float32)
    sk.stream_columns(A)
    W1 = sk.sketches()[0].cpu().clone()
    sk.reset()
    sk.stream_columns(A[:, :25])
    sk.stream_columns(A[:, 25:])
    W2, Y2, _ = sk.sketches()
    assert rel(W2.cpu().numpy(), W1.numpy()) <= 1e-12
    sk.close()


# ------------------------------------------------------------ randomized ID

@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("grid,n,k,l", [((16, 12, 16), 120, 10, 20), ((8, 8, 8), 64, 20, 30),
                                        ((12, 12, 12), 200, 16, 16), ((12, 12, 12), 200, 16, 26)])
def test_factor_parity_gap_input(dtype, grid, n, k, l):
    """Gap inputs: J identical to the oracle's.  The sketch seed is the first
    one (from 9) whose oracle pivot margin is >= 1e-4, so the comparison
    always runs (the spectral gap makes the skeleton's span unique, the
    margin makes the greedy pivot order unique)."""
    A = channel_field(grid, 3, n, seed=7, gap_k=k, dtype=dtype, device=DEV)
    m = A.shape[0]
    An = A.cpu().double().numpy()
    seed, Wo, (Jo, Po, ko, margin) = sketch_seed_with_margin(An, k, l, range(9, 73))
    sk = _sk(m=m, n_max=n, k=k, l=l, seed=seed, dtype=dtype)
    stream(sk, A, [32] * (n // 32) + ([n % 32] if n % 32 else []))
    J, P, kout = sk.factor()
    W = sk.sketches()[0].cpu().numpy()
    assert kout == ko == k
    Pg = P.cpu().numpy()
    assert np.array_equal(Pg[:, J.cpu().numpy()], np.eye(k))
    assert J.cpu().tolist() == Jo.tolist()
    # same W on both sides: FP64 QR agreement
    Jw, Pw, _, mw = oracle.column_id(W, k)
    assert J.cpu().tolist() == Jw.tolist()
    assert np.max(np.abs(Pg - Pw)) <= 1e-9 * max(1.0, np.max(np.abs(Pw)))
    # end to end against the FP64 oracle
    tolP = 1e-10 if dtype == torch.float64 else 1e-3
    assert np.max(np.abs(Pg - Po)) <= tolP * max(1.0, np.max(np.abs(Po)))
    sk.close()


@pytest.mark.parametrize("prec,form", [("exact", "tma"), ("bf16", "tma"), ("exact", "register")])
def test_wide_sketch_factor(prec, form, monkeypatch):
    """l = 90, k = 80 (FP32 data, W only): the sketch in one pass with 96-wide
    W^T accumulators (TMA feed) or in two passes of Psi rows 0-59, 60-89
    (register feed), the one-CTA pivoted QR of the 90-row W and the solve for
    80 pivots, against the oracle on the same Psi."""
    if form == "register":
        monkeypatch.setenv("IDSKETCH_SKETCH_TMA", "0")
    grid, n, k, l = (16, 12, 16), 240, 80, 90
    A = channel_field(grid, 3, n, seed=7, gap_k=k, dtype=torch.float32, device=DEV)
    m = A.shape[0]
    An = (A.to(torch.bfloat16) if prec == "bf16" else A).double().cpu().numpy()
    seed, Wo, (Jo, Po, ko, margin) = sketch_seed_with_margin(An, k, l, range(9, 41))
    sk = _sk(m=m, n_max=n, k=k, l=l, seed=seed, dtype=torch.float32, want_Y=False, prec=prec)
    stream(sk, A, [32] * (n // 32) + ([n % 32] if n % 32 else []))
    W = sk.sketches()[0].cpu().numpy()
    assert rel(W, Wo) <= 1e-5
    J, P, kout = sk.factor()
    assert kout == ko == k
    Pg, Jg = P.cpu().numpy(), J.cpu().numpy()
    assert_valid_skeleton(Jg, Pg, k, n)
    Jw, Pw, _, mw = oracle.column_id(W, k)      # same W: FP64 QR agreement
    if mw >= MARGIN:
        assert Jg.tolist() == Jw.tolist()
        assert np.max(np.abs(Pg - Pw)) <= 1e-9 * max(1.0, np.max(np.abs(Pw)))
    if margin >= MARGIN:
        assert Jg.tolist() == Jo.tolist()
    else:
        fo, _ = oracle.recon_error(An, Jo, Po)
        fg, _ = oracle.recon_error(An, Jg, Pg)
        assert fg <= 1.05 * fo
    sk.close()


def test_factor_host_outputs_and_edge_ranks():
    A = channel_field((8, 8, 8), 3, 40, seed=2, gap_k=8, dtype=torch.float64, device=DEV)
    m = A.shape[0]
    An = A.cpu().numpy()
    for k, l, n in [(1, 10, 40), (8, 8, 40), (10, 10, 10), (16, 40, 40)]:
        sk = _sk(m=m, n_max=n, k=k, l=l, seed=1, dtype=torch.float64)
        sk.stream_columns(A[:, :n])
        J, P, kout = sk.factor(device="cpu")
        Wo, _ = oracle.sketch(An[:, :n], oracle.psi(l, m, 1), oracle.omega(n, l, 1))
        Jo, Po, ko, margin = oracle.column_id(Wo, k)
        assert kout == ko
        assert_valid_skeleton(J.numpy(), P.numpy(), kout, n)
        if margin >= MARGIN:
            assert J.tolist()[:kout] == Jo.tolist()
            assert np.max(np.abs(P.numpy()[:kout] - Po)) <= 1e-8 * max(1, np.abs(Po).max())
        else:   # pivot order within rounding of a tie: same error as the oracle's ID
            fo, _ = oracle.recon_error(An[:, :n], Jo, Po)
            fg, _ = oracle.recon_error(An[:, :n], J.numpy()[:kout], P.numpy()[:kout])
            assert abs(fg - fo) <= 1e-6 * fo + 1e-14
        sk.close()


def test_rank_deficient_returns_kout():
    from paper_1905_13257_gb300 import _binding as B
    m, n, r = 2000, 60, 5
    A = low_rank_matrix(m, n, r, seed=3, dtype=torch.float64, device=DEV)
    A[:, 7] = 0.0
    sk = _sk(m=m, n_max=n, k=12, l=20, seed=5, dtype=torch.float64)
    sk.stream_columns(A)
    J, P, kout = sk.factor()
    Wo, _ = oracle.sketch(A.cpu().numpy(), oracle.psi(20, m, 5), oracle.omega(n, 20, 5))
    Jo, Po, ko, _ = oracle.column_id(Wo, 12)
    assert kout == ko == r
    assert J.cpu().tolist()[r:] == [-1] * (12 - r)
    assert 7 not in J.cpu().tolist()
    fro, _ = sk.reconstruct_error(A, J[:r], P[:r])
    assert fro <= 1e-12
    sk.close()


def test_zero_matrix():
    m, n = 500, 20
    A = torch.zeros((n, m), dtype=torch.float32, device=DEV).T
    sk = _sk(m=m, n_max=n, k=3, l=8, seed=0, dtype=torch.float32)
    sk.stream_columns(A)
    J, P, kout = sk.factor()
    assert kout == 0 and J.cpu().tolist() == [-1, -1, -1]
    sk.close()


# ---------------------------------------------------------- sub-sampled ID

@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("grid,stride,n,k", [((16, 12, 16), (2, 2, 2), 90, 8),
                                             ((20, 9, 13), (4, 2, 3), 70, 12),
                                             ((8, 8, 8), (1, 1, 1), 40, 40)])
def test_coarse_factor_parity(dtype, grid, stride, n, k):
    """Gap inputs: J_c identical to the oracle's deterministic ID of A_c.  The
    data seed is the first one (from 5) whose coarse matrix has an oracle
    pivot margin >= 1e-4."""
    nc = 3
    rows = oracle.coarse_rows(grid, nc, stride)
    for dseed in range(5, 37):
        A = channel_field(grid, nc, n, seed=dseed, gap_k=k, dtype=dtype, device=DEV)
        An = A.cpu().double().numpy()
        Jo, Po, ko, margin = oracle.column_id(An[rows], k)
        if margin >= MARGIN:
            break
    assert margin >= MARGIN, f"no data seed gives a coarse pivot margin >= {MARGIN}"
    m = A.shape[0]
    sk = _sk(m=m, n_max=n, k=k, l=max(k, 16), seed=1, dtype=dtype, grid=grid, ncomp=nc,
             coarse_stride=stride, want_coarse=True, window_cols=64)
    stream(sk, A, [32] * (n // 32) + ([n % 32] if n % 32 else []))
    Jc, Pc, kout = sk.coarse_factor()
    Ac = sk.sketches()[2].cpu().numpy()
    assert np.array_equal(Ac.astype(np.float64), An[rows])            # exact gather
    assert kout == ko
    assert Jc.cpu().tolist()[:kout] == Jo.tolist()
    assert np.max(np.abs(Pc.cpu().numpy()[:kout] - Po)) <= 1e-8 * max(1, np.abs(Po).max())
    # lifted error (eq. eq:coarseregA) through the fused error pass
    fro, mx = sk.reconstruct_error(A, Jc[:kout], Pc[:kout])
    fo, mo = oracle.recon_error(An, Jo, Po)
    assert abs(fro - fo) <= err_tol(fo, dtype)
    sk.close()


def test_coarse_started_by_factor_and_later_columns():
    """id_factor starts the coarse QR of the columns seen so far on a side
    stream; columns streamed afterwards, or a reset, must not be mixed with
    it: id_coarse_factor then factors all columns seen.  Gap input whose
    coarse matrix has an oracle pivot margin >= 1e-4 (first such data seed)."""
    grid, stride, n, k, nc = (16, 12, 16), (2, 2, 2), 90, 8, 3
    rows = oracle.coarse_rows(grid, nc, stride)
    for dseed in range(5, 37):
        A = channel_field(grid, nc, n, seed=dseed, gap_k=k, dtype=torch.float32, device=DEV)
        An = A.cpu().double().numpy()
        Jo, Po, ko, margin = oracle.column_id(An[rows], k)
        J1, _, _, margin1 = oracle.column_id(An[rows][:, :48], k)
        if margin >= MARGIN and margin1 >= MARGIN:
            break
    assert margin >= MARGIN and margin1 >= MARGIN
    m = A.shape[0]
    sk = _sk(m=m, n_max=n, k=k, l=16, seed=1, dtype=torch.float32, grid=grid, ncomp=nc,
             coarse_stride=stride, want_coarse=True)
    # the started coarse QR is the one id_coarse_factor returns
    sk.stream_columns(A[:, :48])
    sk.factor()
    Jc, Pc, kc = sk.coarse_factor()
    assert Jc.cpu().tolist()[:kc] == J1.tolist()
    # columns after id_factor: the coarse QR covers all of them
    sk.factor()
    sk.stream_columns(A[:, 48:])
    Jc, Pc, kc = sk.coarse_factor()
    assert kc == ko and Jc.cpu().tolist()[:kc] == Jo.tolist()
    assert np.max(np.abs(Pc.cpu().numpy()[:kc] - Po)) <= 1e-8 * max(1, np.abs(Po).max())
    # a reset after id_factor, then the same columns again
    sk.factor()
    sk.reset()
    sk.stream_columns(A)
    sk.factor()
    Jc2, Pc2, kc2 = sk.coarse_factor()
    # started by id_factor on one CTA fewer than id_coarse_factor's own
    # launch: the per-CTA partial sums differ in rounding order only
    assert kc2 == kc and torch.equal(Jc2, Jc)
    assert np.max(np.abs(Pc2.cpu().numpy()[:kc] - Po)) <= 1e-8 * max(1, np.abs(Po).max())
    sk.close()


def test_coarse_rank_deficient():
    grid, nc = (8, 8, 8), 1
    m, n, r = 512, 30, 4
    A = low_rank_matrix(m, n, r, seed=8, dtype=torch.float64, device=DEV)
    sk = _sk(m=m, n_max=n, k=10, l=16, seed=1, dtype=torch.float64, grid=grid, ncomp=nc,
             coarse_stride=(2, 1, 1), want_coarse=True)
    sk.stream_columns(A)
    Jc, Pc, kout = sk.coarse_factor()
    rows = oracle.coarse_rows(grid, nc, (2, 1, 1))
    Jo, Po, ko, _ = oracle.column_id(A.cpu().numpy()[rows], 10)
    assert kout == ko == r
    sk.close()


def test_coarse_rank_deficient_fp32_cooperative():
    """FP32 data on the cooperative coarse QR (m_c a multiple of 4): six
    independent columns and the rest exactly zero.  The zero columns' norms
    stay exactly zero, so the rank tolerance stops both the kernel and the
    oracle after the six (Algorithm 5 with fewer than k pivots)."""
    grid, nc, n, r, k = (8, 8, 8), 3, 40, 6, 10
    m = nc * grid[0] * grid[1] * grid[2]
    g = np.random.default_rng(11)
    An = np.zeros((m, n))
    cols = g.choice(n, size=r, replace=False)
    An[:, cols] = g.normal(size=(m, r))
    A = torch.tensor(An, dtype=torch.float32).T.contiguous().T.to(DEV)
    An = A.cpu().double().numpy()
    sk = _sk(m=m, n_max=n, k=k, l=16, seed=1, dtype=torch.float32, grid=grid, ncomp=nc,
             coarse_stride=(1, 1, 1), want_coarse=True)
    sk.stream_columns(A)
    Jc, Pc, kout = sk.coarse_factor()
    Jo, Po, ko, margin = oracle.column_id(An, k)
    assert ko == r and kout == r
    assert sorted(Jc.cpu().tolist()[:kout]) == sorted(cols.tolist())
    if margin >= MARGIN:
        assert Jc.cpu().tolist()[:kout] == Jo.tolist()
    P = Pc.cpu().numpy()[:kout]
    assert_valid_skeleton(Jc.cpu().numpy()[:kout], P, kout, n)
    zero = np.setdiff1d(np.arange(n), cols)
    assert np.all(P[:, zero] == 0.0)
    assert all(j == -1 for j in Jc.cpu().tolist()[kout:])
    sk.close()


# ------------------------------------------------------------- error pass

@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("m,n,k", [(6000, 100, 10), (4097, 33, 1), (64 * 7 + 5, 250, 64)])
def test_recon_error_parity(dtype, m, n, k):
    A = gaussian_matrix(m, n, seed=m, dtype=dtype, device=DEV)
    A = A + low_rank_matrix(m, n, 4, seed=1, dtype=dtype, device=DEV) * 10
    A[5, 3] = 0.0   # skipped by the entry-wise metric
    g = np.random.default_rng(n)
    J = torch.tensor(g.choice(n, size=k, replace=False), dtype=torch.int32)
    P = torch.tensor(g.normal(size=(k, n)) * 0.3)
    sk = _sk(m=m, n_max=n, k=min(k, 64), l=64, seed=0, dtype=dtype)
    fro, mx = sk.reconstruct_error(A, J, P)
    fo, mo = oracle.recon_error(A.cpu().double().numpy(), J.numpy(), P.numpy())
    assert abs(fro - fo) <= err_tol(fo, dtype)
    assert abs(mx - mo) <= err_tol(mo, dtype)
    # device-resident J and P give the same numbers
    fro2, mx2 = sk.reconstruct_error(A, J.to(DEV), P.to(DEV))
    assert fro2 == fro and mx2 == mx
    sk.close()


@pytest.mark.parametrize("k", [10, 50])
def test_recon_error_small_residual_fp32(k):
    """The spec bar where it is hardest for FP32: a reconstruction
    whose relative error is about 1e-3 (the residual cancels about 10 bits
    of A), skeleton and P from the oracle's ID of the exact data."""
    grid, n = (16, 12, 16), 200
    A = channel_field(grid, 3, n, seed=3, gap_k=k, dtype=torch.float32, device=DEV)
    An = A.cpu().double().numpy()
    Jo, Po, ko, _ = oracle.column_id(An, k)
    fo, mo = oracle.recon_error(An, Jo, Po)
    assert 1e-4 < fo < 1e-2
    sk = _sk(m=A.shape[0], n_max=n, k=k, l=64, seed=0, dtype=torch.float32)
    fro, mx = sk.reconstruct_error(A, torch.as_tensor(Jo, dtype=torch.int32),
                                   torch.as_tensor(Po))
    assert abs(fro - fo) <= 1e-4 * fo
    sk.close()


@pytest.mark.parametrize("m,n,k", [(3000, 120, 12), (64 * 9 + 17, 300, 40)])
def test_recon_error_zero_entries_fp32(m, n, k):
    """Entries with A_ij = 0 are left out of the entry-wise metric (Sec. 3.1):
    about one entry in a hundred set to zero (their residuals are not zero,
    so the kernel's reciprocal of A_ij is infinite there), and a band of
    zero rows (residual zero as well)."""
    A = gaussian_matrix(m, n, seed=m + 7, dtype=torch.float32, device=DEV)
    A = A + low_rank_matrix(m, n, 4, seed=2, dtype=torch.float32, device=DEV) * 10
    g = np.random.default_rng(m)
    mask = torch.as_tensor(g.random((m, n)) < 0.01, device=DEV)
    A[mask] = 0.0
    A[100:140, :] = 0.0
    J = torch.tensor(g.choice(n, size=k, replace=False), dtype=torch.int32)
    P = torch.tensor(g.normal(size=(k, n)) * 0.3)
    sk = _sk(m=m, n_max=n, k=k, l=64, seed=0, dtype=torch.float32)
    fro, mx = sk.reconstruct_error(A, J, P)
    fo, mo = oracle.recon_error(A.cpu().double().numpy(), J.numpy(), P.numpy())
    assert np.isfinite(mx)
    assert abs(fro - fo) <= err_tol(fo, torch.float32)
    assert abs(mx - mo) <= err_tol(mo, torch.float32)
    sk.close()


def test_recon_error_invalid_arguments():
    from paper_1905_13257_gb300 import IdError
    A = gaussian_matrix(100, 10, seed=1, dtype=torch.float32, device=DEV)
    sk = _sk(m=100, n_max=10, k=2, l=4, seed=0, dtype=torch.float32)
    with pytest.raises(IdError):
        sk.reconstruct_error(A, torch.tensor([0, 10], dtype=torch.int32), torch.zeros(2, 10))
    with pytest.raises(IdError):
        sk.stream_columns(gaussian_matrix(100, 11, 1, torch.float32, DEV))   # > n_max
    sk.close()


def test_factor_before_columns_is_state_error():
    from paper_1905_13257_gb300 import IdError
    sk = _sk(m=100, n_max=10, k=2, l=4, seed=0, dtype=torch.float32)
    with pytest.raises(IdError) as e:
        sk.factor()
    assert e.value.status == 2
    with pytest.raises(IdError) as e:
        sk.coarse_factor()
    assert e.value.status == 2
    sk.close()


def test_allocation_cap_injects_oom(monkeypatch):
    from paper_1905_13257_gb300 import IdError
    monkeypatch.setenv("IDSKETCH_ALLOC_CAP_BYTES", "1000")
    with pytest.raises(IdError) as e:
        _sk(m=10000, n_max=100, k=4, l=8, seed=0, dtype=torch.float32)
    assert e.value.status == 3


# ------------------------------------------------------- precision form (BF16)

def test_bf16_sketch_matches_oracle_on_rounded_data():
    A = channel_field((16, 12, 16), 3, 64, seed=2, dtype=torch.float32, device=DEV)
    m, n, l = A.shape[0], 64, 30
    sk = _sk(m=m, n_max=n, k=10, l=l, seed=3, dtype=torch.float32, prec="bf16")
    sk.stream_columns(A)
    W, Y, _ = sk.sketches()
    Ab = A.to(torch.bfloat16).double().cpu().numpy()
    Wo, Yo = oracle.sketch(Ab, oracle.psi(l, m, 3), oracle.omega(n, l, 3))
    assert rel(W.cpu().numpy(), Wo) <= 1e-5
    assert rel(Y.cpu().double().numpy(), Yo) <= 1e-5
    sk.close()


@pytest.mark.parametrize("tma", ["1", "0"])
def test_tensor_core_sketch_feeds(monkeypatch, tma):
    """Both tensor-core feeds of A (TMA boxes for a single-segment window, and
    register loads for a window made of several separate buffers) against
    the oracle, with coarse gather and ragged m and n."""
    monkeypatch.setenv("IDSKETCH_SKETCH_TMA", tma)
    grid, nc, n, l = (20, 13, 12), 3, 300, 60
    A = channel_field(grid, nc, n, seed=4, dtype=torch.float32, device=DEV)
    m = A.shape[0]
    assert m % 4 == 0
    # separate, 16-byte aligned buffers: windows of several segments
    parts = [A[:, j:j + 45].contiguous().T.contiguous().T for j in range(0, n, 45)]
    sk = _sk(m=m, n_max=n, k=10, l=l, seed=6, dtype=torch.float32, grid=grid, ncomp=nc,
             coarse_stride=(2, 3, 2), want_coarse=True, window_cols=256)
    for p in parts:
        sk.stream_columns(p)
    W, Y, Ac = sk.sketches()
    An = A.cpu().double().numpy()
    Wo, Yo = oracle.sketch(An, oracle.psi(l, m, 6), oracle.omega(n, l, 6))
    assert rel(W.cpu().numpy(), Wo) <= 1e-5
    assert rel(Y.cpu().double().numpy(), Yo) <= 1e-5
    rows = oracle.coarse_rows(grid, nc, (2, 3, 2))
    assert np.array_equal(Ac.cpu().numpy(), A.cpu().numpy()[rows])
    sk.close()
    # one resident buffer: single-segment windows
    sk = _sk(m=m, n_max=n, k=10, l=l, seed=6, dtype=torch.float32, grid=grid, ncomp=nc,
             coarse_stride=(2, 3, 2), want_coarse=True, window_cols=n)
    stream(sk, A, [32] * (n // 32) + [n % 32])
    W2, Y2, Ac2 = sk.sketches()
    assert rel(W2.cpu().numpy(), Wo) <= 1e-5
    assert rel(Y2.cpu().double().numpy(), Yo) <= 1e-5
    assert np.array_equal(Ac2.cpu().numpy(), A.cpu().numpy()[rows])
    sk.close()


@pytest.mark.parametrize("drain", ["1", "3", "5", "8", "64"])
def test_sketch_flush_schedules(monkeypatch, drain):
    """W^T partials leave TMEM one 128-column tile at a time, every `drain` row
    blocks with the four tiles offset by drain / 4 row blocks, and the last
    row block flushes them all.  Every schedule (shorter than the four tiles,
    uneven offsets, longer than a CTA's row range) gives the oracle's
    sketches within the FP32 bar."""
    monkeypatch.setenv("IDSKETCH_DRAIN_BLOCKS", drain)
    grid, nc, n, l = (32, 24, 32), 3, 400, 60        # 576 row blocks, 4 column tiles
    A = channel_field(grid, nc, n, seed=12, dtype=torch.float32, device=DEV)
    m = A.shape[0]
    sk = _sk(m=m, n_max=n, k=10, l=l, seed=13, dtype=torch.float32, want_Y=True,
             window_cols=n)
    stream(sk, A, [32] * (n // 32) + [n % 32])
    W, Y, _ = sk.sketches()
    Wo, Yo = oracle.sketch(A.cpu().double().numpy(), oracle.psi(l, m, 13),
                           oracle.omega(n, l, 13))
    assert rel(W.cpu().numpy(), Wo) <= 1e-5
    assert rel(Y.cpu().double().numpy(), Yo) <= 1e-5
    sk.close()


# ------------------------------------------------------------ kernel timing

def test_kernel_timing_counts_launches():
    """id_timing_enable / id_timing_read: one event pair per launch of the
    fused sketch kernel and of the error-pass kernel, reset on read."""
    from paper_1905_13257_gb300 import IdError
    grid, n = (16, 12, 16), 300
    A = channel_field(grid, 3, n, seed=5, dtype=torch.float32, device=DEV)
    sk = _sk(m=A.shape[0], n_max=n, k=8, l=30, seed=1, dtype=torch.float32, window_cols=n)
    with pytest.raises(IdError) as e:
        sk.read_timing("sketch")
    assert e.value.status == 2
    sk.timing(True)
    stream(sk, A, [32] * 9 + [12])
    sk.flush()
    ms, cnt = sk.read_timing("sketch")
    assert cnt == 1 and ms > 0.0          # 300 columns: one tensor-core window
    assert sk.read_timing("sketch") == (0.0, 0)
    J, P, kout = sk.factor()
    sk.reconstruct_error(A, J[:kout], P[:kout])
    ms, cnt = sk.read_timing("recon")
    assert cnt == 1 and ms > 0.0
    sk.timing(False)
    sk.close()
