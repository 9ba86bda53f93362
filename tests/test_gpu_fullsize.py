"""Parity at the full workload sizes, in the launch configuration bench.py times.

Bars: sketches <= 1e-5 relative Frobenius (FP32) / 1e-12 (FP64); relative
Frobenius errors within 1e-4 relative of the oracle's (FP32, no absolute
term) / 1e-10 (FP64); J identical when the oracle's pivot margin is >= 1e-4,
otherwise a valid skeleton whose error matches the oracle's ID (the margin is
printed either way).

* Full FP64 case: 32x32x32 grid x 3 components = 98,304 rows x 200 snapshots,
  k = 20, p = 10, seed 0, chunks of 32, coarse grid 4x: every output against
  the oracle.
* Streamed FP32 case: 128x96x128 x 3 = 4,718,592 rows x 1000 snapshots
  (18.9 GB), chunks of 32 aggregated into one window, l = 60, k = 50, coarse
  4x: the oracle's Algorithm 4 on the whole matrix (every entry of W and Y,
  the QR of its own W, its error), the exact coarse gather, the pivoted QRs
  against the oracle on the same inputs, and the errors of the randomized,
  sub-sampled and single-pass IDs against the oracle's exact sums over all
  rows, all from one pass of the oracle over row blocks.
"""
import numpy as np
import pytest
import torch

import oracle
from margins import MARGIN, assert_valid_skeleton
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
    assert abs(fro - fo) <= 1e-10 * fo
    assert abs(mx - mo) <= 1e-10 * mo
    rows = oracle.coarse_rows(grid, nc, (4, 4, 4))
    assert np.array_equal(Ac.cpu().numpy(), An[rows])
    Jco, Pco, kco, mco = oracle.column_id(An[rows], k)
    assert kc == kco
    print(f"full FP64 case: oracle pivot margins {margin:.2e} (sketch), {mco:.2e} (coarse)")
    assert_valid_skeleton(Jc.cpu().numpy(), Pc.cpu().numpy(), kc, n)
    if mco >= MARGIN:
        assert Jc.cpu().tolist() == Jco.tolist()
        assert np.max(np.abs(Pc.cpu().numpy() - Pco)) <= 1e-8 * max(1.0, np.abs(Pco).max())
    else:
        fco, _ = oracle.recon_error(An, Jco, Pco)
        fcg, _ = oracle.recon_error(An, Jc.cpu().numpy(), Pc.cpu().numpy())
        assert abs(fcg - fco) <= 1e-6 * fco
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
    # the single-pass ID (Algorithm 6) of the same coarse skeleton, on the GPU
    from synthetic.channel import LX, LZ, wall_normal_points
    nx, ny, nz = grid
    coords = (np.arange(nx) * (LX / nx), wall_normal_points(ny), np.arange(nz) * (LZ / nz))
    per = (LX, 0.0, LZ)
    sk.set_mesh(*coords, per)
    Jct, Pct = torch.as_tensor(out["Jc"][:kc]), torch.as_tensor(out["Pc"][:kc])
    out["S"] = sk.single_pass_lift(Jct, kc).cpu().double().numpy()
    out["sp_fro"], out["sp_mx"] = sk.single_pass_error(A, Jct, Pct)
    out["coords"], out["per"] = coords, per
    # the precision form (BF16 sketch products) on the same data
    skb = _sk(m=m, n_max=n, k=k, l=l, seed=seed, dtype=torch.float32, prec="bf16", want_Y=True,
              window_cols=n)
    for j0 in range(0, n, 32):
        skb.stream_columns(A[:, j0:j0 + 32])
    Jb, Pb, kb = skb.factor()
    Wb, Yb, _ = skb.sketches()
    out["bf16"] = dict(J=Jb.cpu().numpy(), P=Pb.cpu().numpy(), kout=kb, W=Wb.cpu().numpy().copy(),
                       Y=Yb, fro=skb.reconstruct_error(A, Jb[:kb], Pb[:kb])[0], sk=skb)
    yield out
    skb.close()
    sk.close()


@pytest.fixture(scope="module")
def oracle_pass(streamed_case):
    """The oracle on the whole streamed case, in ONE pass over row blocks of
    A (each block copied to the host once, converted to FP64 exactly):
      * W = Psi A (Algorithm 4 step 3) and the error of the GPU's Y = A Omega;
      * ||A||_F^2;
      * for each approximation A ~ A(:, J) P (GPU randomized ID, GPU and
        oracle sub-sampled ID) or S P (single-pass ID, S = M A_c(:, J_c) by
        the oracle's operator M), the exact FP64 residual sums of squares
        and, where the tests compare it, the maximum entry-wise ratio;
      * G = A(:, J)^T A for the GPU's skeleton J, so that the error of any
        P on that J follows from ||A - A_J P||^2 = ||A||^2 - 2 <P, G> +
        <P P^T, G(:, J)> (checked against the direct sum for the GPU's P).
    """
    import oracle.single_pass as osp
    c = streamed_case
    A, m, n, l, k, seed = c["A"], c["m"], c["n"], c["l"], c["k"], c["seed"]
    kc = c["kc"]
    Jco, Pco, kco, mco = oracle.column_id(c["Ac"].astype(np.float64), k)
    M = osp.coarse_to_fine(c["grid"], c["nc"], (4, 4, 4), c["coords"], c["per"])
    So = M @ c["Ac"].astype(np.float64)[:, c["Jc"][:kc]]
    cb = c["bf16"]
    approx = {"gpu": (c["J"][: c["kout"]], c["P"][: c["kout"]], None, True),
              "bf16": (cb["J"][: cb["kout"]], cb["P"][: cb["kout"]], None, False),
              "gpu_coarse": (c["Jc"][:kc], c["Pc"][:kc], None, False),
              "oracle_coarse": (Jco[:kco], Pco, None, False),
              "single_pass": (None, c["Pc"][:kc], So, True)}
    Om = oracle.omega(n, l, seed)
    Wo = np.zeros((l, n))
    Jg = np.asarray(c["J"][: c["kout"]], dtype=np.int64)
    G = np.zeros((len(Jg), n))
    ss = {key: 0.0 for key in approx}
    rmax = {key: 0.0 for key in approx}
    ss_a = ey_num = ey_den = eyb_num = 0.0
    rb = 262_144
    for r0 in range(0, m, rb):
        r1 = min(m, r0 + rb)
        blk = A[r0:r1].T.contiguous().cpu().numpy().T.astype(np.float64)   # exact
        Wo += oracle.psi(l, 0, seed, rows=np.arange(r0, r1)) @ blk
        Yo = blk @ Om
        Yg = c["Y"][r0:r1].T.contiguous().cpu().numpy().T.astype(np.float64)
        ey_num += float(np.sum((Yg - Yo) ** 2))
        ey_den += float(np.sum(Yo * Yo))
        Yb = cb["Y"][r0:r1].T.contiguous().cpu().numpy().T.astype(np.float64)
        eyb_num += float(np.sum((Yb - Yo) ** 2))
        flat = blk.ravel(order="F")
        ss_a += float(flat @ flat)
        G += blk[:, Jg].T @ blk
        absb = np.abs(blk)
        nz = absb > 0
        for key, (J, P, S, want_max) in approx.items():
            Ab = blk[:, np.asarray(J, dtype=np.int64)] if S is None else S[r0:r1]
            R = (P.T @ Ab.T).T          # A_hat of the block, column-major like blk
            np.subtract(blk, R, out=R)
            rf = R.ravel(order="A")
            ss[key] += float(rf @ rf)
            if want_max:
                np.abs(R, out=R)
                np.divide(R, absb, out=R, where=nz)
                R[~nz] = 0.0
                rmax[key] = max(rmax[key], float(R.max()))
    err = {key: float(np.sqrt(ss[key] / ss_a)) for key in approx}
    return dict(Wo=Wo, ey=float(np.sqrt(ey_num / ey_den)), ss_a=ss_a, err=err, rmax=rmax, G=G,
                Jg=Jg, Jco=Jco, Pco=Pco, kco=kco, mco=mco, So=So,
                ey_bf16=float(np.sqrt(eyb_num / ey_den)))


def _err_on_gpu_skeleton(op, P):
    """Relative error of A ~ A(:, J_gpu) P from the pass's G = A(:, J)^T A."""
    G, J = op["G"], op["Jg"]
    e2 = op["ss_a"] - 2.0 * float(np.sum(P * G)) + float(np.sum((P @ P.T) * G[:, J]))
    return float(np.sqrt(max(e2, 0.0) / op["ss_a"]))


def test_streamed_coarse_gather_exact(streamed_case):
    c = streamed_case
    rows = torch.as_tensor(oracle.coarse_rows(c["grid"], c["nc"], (4, 4, 4)), device="cuda")
    assert torch.equal(torch.as_tensor(c["Ac"], device="cuda"), c["A"][rows, :])


def test_streamed_factor_against_oracle_qr(streamed_case):
    """The GPU's pivoted QR and solve against the oracle's on the same W."""
    c = streamed_case
    Jo, Po, ko, margin = oracle.column_id(c["W"], c["k"])
    print(f"streamed case: pivot margin of the QR of the GPU's W {margin:.2e}")
    assert c["kout"] == ko == c["k"]
    assert_valid_skeleton(c["J"], c["P"], c["kout"], c["n"])
    if margin >= MARGIN:
        assert c["J"].tolist() == Jo.tolist()
        assert np.max(np.abs(c["P"] - Po)) <= 1e-9 * max(1.0, np.abs(Po).max())
    else:   # within rounding of a tie: the same interpolation quality
        assert np.max(np.abs(c["W"] - c["W"][:, c["J"]] @ c["P"])) <= \
            1.0001 * np.max(np.abs(c["W"] - c["W"][:, Jo] @ Po)) + 1e-12


def test_streamed_randomized_id_against_full_oracle(streamed_case, oracle_pass):
    """Algorithm 4 run by the oracle on the whole bench workload (4,718,592 x
    1000 FP32, l = 60, k = 50, seed 0): every entry of the GPU's W and Y, its
    J (or, below the pivot margin, a valid skeleton), P and error against the
    oracle's.  The oracle's error is the workload's "fixed relative error"."""
    c, op = streamed_case, oracle_pass
    Wo = op["Wo"]
    ew = rel(c["W"], Wo)
    Jo, Po, ko, margin = oracle.column_id(Wo, c["k"])
    fg = op["err"]["gpu"]
    print(f"streamed case, oracle Alg. 4: pivot margin {margin:.2e}; GPU: W err {ew:.2e}, "
          f"Y err {op['ey']:.2e}, error {c['fro']:.6e} (oracle's sum for the GPU's J, P "
          f"{fg:.6e}, entry-wise {op['rmax']['gpu']:.4e})")
    assert ew <= 1e-5 and op["ey"] <= 1e-5
    assert c["kout"] == ko == c["k"]
    assert_valid_skeleton(c["J"], c["P"], c["kout"], c["n"])
    # the expansion through G reproduces the direct residual sum
    assert abs(_err_on_gpu_skeleton(op, c["P"][: c["kout"]]) - fg) <= 1e-9 * fg
    if margin >= MARGIN:
        assert c["J"].tolist() == Jo.tolist()
        assert np.max(np.abs(c["P"] - Po)) <= 1e-3 * max(1.0, np.abs(Po).max())
        fo = _err_on_gpu_skeleton(op, Po)
        print(f"oracle's randomized ID error (fixed relative error): {fo:.7e}")
        assert abs(c["fro"] - fo) <= 1e-4 * fo
    else:   # within rounding of a tie: a valid ID of A, its error exact
        assert abs(c["fro"] - fg) <= 1e-4 * fg


def test_streamed_coarse_factor_against_oracle(streamed_case, oracle_pass):
    """The GPU's sub-sampled ID (Algorithm 5) against the oracle's pivoted QR
    of the same A_c; below the pivot margin, a valid skeleton whose lifted
    error equals the oracle ID's."""
    c, op = streamed_case, oracle_pass
    Jo, Po, ko, margin = op["Jco"], op["Pco"], op["kco"], op["mco"]
    print(f"streamed case: pivot margin of the coarse QR {margin:.2e}; lifted errors GPU "
          f"{op['err']['gpu_coarse']:.6e}, oracle {op['err']['oracle_coarse']:.6e}")
    assert c["kc"] == ko
    assert_valid_skeleton(c["Jc"], c["Pc"], c["kc"], c["n"])
    if margin >= MARGIN:
        assert c["Jc"].tolist() == Jo.tolist()
        assert np.max(np.abs(c["Pc"] - Po)) <= 1e-8 * max(1.0, np.abs(Po).max())
    else:
        assert abs(op["err"]["gpu_coarse"] - op["err"]["oracle_coarse"]) <= \
            1e-6 * op["err"]["oracle_coarse"]


def test_streamed_reconstruction_error_exact_sum(streamed_case, oracle_pass):
    """The GPU's error pass against the oracle's exact sums over all 4.7M rows
    for the same (J, P)."""
    c, op = streamed_case, oracle_pass
    fo, rmax = op["err"]["gpu"], op["rmax"]["gpu"]
    assert abs(c["fro"] - fo) <= 1e-4 * fo
    assert abs(c["mx"] - rmax) <= 1e-4 * rmax


def test_streamed_single_pass_id(streamed_case, oracle_pass):
    """Algorithm 6 at full size: the lifted skeleton M A_c(:, J_c) and the
    single-pass error against the oracle's operator M (all 4.7M rows)."""
    c, op = streamed_case, oracle_pass
    assert rel(c["S"], op["So"]) <= 1e-6
    fo, rmax = op["err"]["single_pass"], op["rmax"]["single_pass"]
    assert abs(c["sp_fro"] - fo) <= 1e-4 * fo
    assert abs(c["sp_mx"] - rmax) <= 1e-4 * rmax


def test_streamed_bf16_precision_form_against_full_oracle(streamed_case, oracle_pass):
    """The precision form (sketch products with A rounded to bfloat16, FP32
    accumulation; QR and solve in FP64) against the FP64 oracle of the FP32
    data, at the bench workload.  Bars derived from the rounding: a bfloat16
    keeps 8 significant bits, so each entry of A moves by at most 2^-9 of its
    value and the sketches by at most about that in relative Frobenius norm;
    the ID it picks must reconstruct A within 1.05x the oracle's error (the
    equal-error bar).  The J overlap and every error are printed."""
    c, op = streamed_case, oracle_pass
    cb = c["bf16"]
    Jo, Po, ko, margin = oracle.column_id(op["Wo"], c["k"])
    ew = rel(cb["W"], op["Wo"])
    fo = _err_on_gpu_skeleton(op, Po) if c["J"].tolist() == Jo.tolist() else op["err"]["gpu"]
    fb = op["err"]["bf16"]
    overlap = len(set(cb["J"][: cb["kout"]].tolist()) & set(Jo.tolist())) / ko
    Pdiff = float(np.max(np.abs(cb["P"] - Po))) if cb["J"].tolist() == Jo.tolist() else None
    print(f"BF16 form vs FP64 oracle: W {ew:.3e}, Y {op['ey_bf16']:.3e}, J overlap {overlap:.2f}, "
          f"max|P - P_o| {Pdiff}, error {fb:.6e} (oracle {fo:.6e}, ratio {fb / fo:.5f}; "
          f"GPU's own error pass {cb['fro']:.6e})")
    assert ew <= 2.0 ** -9 and op["ey_bf16"] <= 2.0 ** -9
    assert cb["kout"] == c["k"]
    assert_valid_skeleton(cb["J"], cb["P"], cb["kout"], c["n"])
    assert fb <= 1.05 * fo
    assert abs(cb["fro"] - fb) <= 1e-4 * fb
