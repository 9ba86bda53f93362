"""Parity at the full workload sizes, in the launch configuration bench.py times.

* Full FP64 case: 32x32x32 grid x 3 components = 98,304 rows x 200 snapshots,
  k = 20, p = 10, seed 0, chunks of 32, coarse grid 4x: every output against
  the oracle.
* Streamed FP32 case: 128x96x128 x 3 = 4,718,592 rows x 1000 snapshots
  (18.9 GB), chunks of 32 aggregated into one window, l = 60, k = 50, coarse
  4x: sampled columns of W and rows of Y against the oracle's one-by-one
  products, the exact coarse gather, the pivoted QRs against the oracle on
  the same (validated) inputs, and the reconstruction errors of the
  sub-sampled and the single-pass ID against the oracle's exact sums taken
  over row chunks.
"""
import numpy as np
import pytest
import torch

import oracle
from synthetic import channel_field

pytestmark = pytest.mark.gpu


def _sk(**kw):
    from paper_1905_13257_gb300 import IdSketch
    return IdSketch(**kw)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - np.asarray(b, np.float64)) /
                 np.linalg.norm(np.asarray(b, np.float64)))


def test_full_fp64_case_end_to_end():
    grid, nc, n, k, l, seed = (32, 32, 32), 3, 200, 20, 30, 0
    A = channel_field(grid, nc, n, seed=seed, dtype=torch.float64, device="cuda")
    m = A.shape[0]
    sk = _sk(m=m, n_max=n, k=k, l=l, seed=seed, dtype=torch.float64, grid=grid, ncomp=nc,
             coarse_stride=(4, 4, 4), want_Y=True, want_coarse=True)
    for j0 in range(0, n, 32):
        sk.stream_columns(A[:, j0:j0 + 32])
    J, P, kout = sk.factor()
    Jc, Pc, kc = sk.coarse_factor()
    fro, mx = sk.reconstruct_error(A, J, P)
    W, Y, Ac = sk.sketches()
    An = A.cpu().numpy()
    Wo, Yo = oracle.sketch(An, oracle.psi(l, m, seed), oracle.omega(n, l, seed))
    assert rel(W.cpu().numpy(), Wo) <= 1e-12
    assert rel(Y.cpu().numpy(), Yo) <= 1e-12
    Jo, Po, ko, margin = oracle.column_id(Wo, k)
    assert kout == ko == k
    assert margin >= 1e-4
    assert J.cpu().tolist() == Jo.tolist()
    assert np.max(np.abs(P.cpu().numpy() - Po)) <= 1e-9 * max(1.0, np.abs(Po).max())
    fo, mo = oracle.recon_error(An, Jo, Po)
    assert abs(fro - fo) <= 1e-4 * fo + 1e-12
    assert abs(mx - mo) <= 1e-4 * mo + 1e-12
    rows = oracle.coarse_rows(grid, nc, (4, 4, 4))
    assert np.array_equal(Ac.cpu().numpy(), An[rows])
    Jco, Pco, kco, mco = oracle.column_id(An[rows], k)
    assert kc == kco
    if mco >= 1e-4:
        assert Jc.cpu().tolist() == Jco.tolist()
        assert np.max(np.abs(Pc.cpu().numpy() - Pco)) <= 1e-8 * max(1.0, np.abs(Pco).max())
    sk.close()


@pytest.fixture(scope="module")
def streamed_case():
    grid, nc, n, k, l, seed = (128, 96, 128), 3, 1000, 50, 60, 0
    A = channel_field(grid, nc, n, seed=seed, dtype=torch.float32, device="cuda")
    m = A.shape[0]
    sk = _sk(m=m, n_max=n, k=k, l=l, seed=seed, dtype=torch.float32, grid=grid, ncomp=nc,
             coarse_stride=(4, 4, 4), want_Y=True, want_coarse=True, window_cols=n)
    for j0 in range(0, n, 32):
        sk.stream_columns(A[:, j0:j0 + 32])
    sk.flush()
    J, P, kout = sk.factor()
    Jc, Pc, kc = sk.coarse_factor()
    fro, mx = sk.reconstruct_error(A, J[:kout], P[:kout])
    W, Y, Ac = sk.sketches()
    out = dict(sk=sk, A=A, grid=grid, nc=nc, n=n, k=k, l=l, seed=seed, m=m, J=J.cpu().numpy(),
               P=P.cpu().numpy(), kout=kout, Jc=Jc.cpu().numpy(), Pc=Pc.cpu().numpy(), kc=kc,
               fro=fro, mx=mx, W=W.cpu().numpy().copy(), Y=Y, Ac=Ac.cpu().numpy().copy())
    yield out
    sk.close()


def test_streamed_sketch_sampled_outputs(streamed_case):
    c = streamed_case
    A, m, n, l, seed = c["A"], c["m"], c["n"], c["l"], c["seed"]
    cols = np.array([0, 511, 512, 999])            # both windows and their edges
    Psi = oracle.psi(l, m, seed)                   # l x m, FP64
    Acols = A[:, cols].cpu().double().numpy()
    Wo = Psi @ Acols
    assert rel(c["W"][:, cols], Wo) <= 1e-5
    del Psi
    rows = np.array([0, 127, 128, 2_359_295, m - 1])
    Om = oracle.omega(n, l, seed)
    Yo = A[rows, :].cpu().double().numpy() @ Om
    assert rel(c["Y"][rows, :].cpu().double().numpy(), Yo) <= 1e-5


def test_streamed_coarse_gather_exact(streamed_case):
    c = streamed_case
    rows = torch.as_tensor(oracle.coarse_rows(c["grid"], c["nc"], (4, 4, 4)), device="cuda")
    assert torch.equal(torch.as_tensor(c["Ac"], device="cuda"), c["A"][rows, :])


def test_streamed_factor_against_oracle_qr(streamed_case):
    c = streamed_case
    Jo, Po, ko, margin = oracle.column_id(c["W"], c["k"])
    assert c["kout"] == ko == c["k"]
    assert np.array_equal(c["P"][:, c["J"]], np.eye(c["k"]))
    if margin >= 1e-4:
        assert c["J"].tolist() == Jo.tolist()
        assert np.max(np.abs(c["P"] - Po)) <= 1e-9 * max(1.0, np.abs(Po).max())


def test_streamed_coarse_factor_against_oracle_qr(streamed_case):
    c = streamed_case
    Jo, Po, ko, margin = oracle.column_id(c["Ac"].astype(np.float64), c["k"])
    assert c["kc"] == ko
    assert np.array_equal(c["Pc"][:, c["Jc"]], np.eye(c["kc"]))
    if margin >= 1e-4:
        assert c["Jc"].tolist() == Jo.tolist()
        assert np.max(np.abs(c["Pc"] - Po)) <= 1e-8 * max(1.0, np.abs(Po).max())


def test_streamed_reconstruction_error_exact_sum(streamed_case):
    """The oracle's reconstruction error over all 4.7M rows, summed in row
    chunks (each chunk an exact FP64 residual of the oracle)."""
    c = streamed_case
    A, J, P = c["A"], c["J"][: c["kout"]], c["P"][: c["kout"]]
    ss_res = ss_a = 0.0
    rmax = 0.0
    for r0 in range(0, c["m"], 262_144):
        blk = A[r0:r0 + 262_144].cpu().double().numpy()
        R = blk - blk[:, J] @ P
        ss_res += float(np.sum(R * R))
        ss_a += float(np.sum(blk * blk))
        nz = blk != 0
        if np.any(nz):
            rmax = max(rmax, float(np.max(np.abs(R[nz]) / np.abs(blk[nz]))))
    fo = np.sqrt(ss_res / ss_a)
    assert abs(c["fro"] - fo) <= 1e-4 * fo + 2e-6
    assert abs(c["mx"] - rmax) <= 1e-3 * rmax


def test_streamed_single_pass_id(streamed_case):
    """Algorithm 6 at full size: the lifted skeleton M A_c(:, J_c) and the
    single-pass error against the oracle's operator M (all 4.7M rows)."""
    import oracle.single_pass as osp
    from synthetic.channel import LX, LZ, wall_normal_points
    c = streamed_case
    sk, A, grid, kc = c["sk"], c["A"], c["grid"], c["kc"]
    nx, ny, nz = grid
    coords = (np.arange(nx) * (LX / nx), wall_normal_points(ny), np.arange(nz) * (LZ / nz))
    per = (LX, 0.0, LZ)
    sk.set_mesh(*coords, per)
    Jc = torch.as_tensor(c["Jc"][:kc])
    Pc = torch.as_tensor(c["Pc"][:kc])
    S = sk.single_pass_lift(Jc, kc).cpu().double().numpy()
    fro, mx = sk.single_pass_error(A, Jc, Pc)
    M = osp.coarse_to_fine(grid, c["nc"], (4, 4, 4), coords, per)
    So = M @ c["Ac"].astype(np.float64)[:, c["Jc"][:kc]]
    assert rel(S, So) <= 1e-6
    ss_res = ss_a = 0.0
    rmax = 0.0
    Pn = c["Pc"][:kc]
    for r0 in range(0, c["m"], 262_144):
        blk = A[r0:r0 + 262_144].cpu().double().numpy()
        R = blk - So[r0:r0 + 262_144] @ Pn
        ss_res += float(np.sum(R * R))
        ss_a += float(np.sum(blk * blk))
        nzm = blk != 0
        if np.any(nzm):
            rmax = max(rmax, float(np.max(np.abs(R[nzm]) / np.abs(blk[nzm]))))
    fo = np.sqrt(ss_res / ss_a)
    assert abs(fro - fo) <= 1e-4 * fo + 2e-6
    assert abs(mx - rmax) <= 1e-3 * rmax
