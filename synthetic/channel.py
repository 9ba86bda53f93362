"""Seeded synthetic channel-flow snapshot matrices.

This module only makes inputs.  It holds none of the method's arithmetic
(no sketch, no QR, no interpolation) and is the one module that both the CUDA
path's tests/bench and the oracle read.

It stands in for the paper's Re_tau = 180 channel DNS (Sec. 3), which is not
available: same domain 4*pi x 2 x 4*pi/3 (in units of the half height), periodic
in x and z, wall-normal grid stretched toward the walls (Sec. 3, DNS set-up),
spatial dimension far larger than the temporal one (Test case 2, Sec. 3.2).

Field
  y_j = tanh(g (2j/(ny-1) - 1)) / tanh(g), g = 2 (the paper gives only the
        wall resolution range; g is this generator's choice)
  64 modes (kx, kz) in {1..8}^2, wavenumbers kappa_x = 2 pi kx / Lx,
  kappa_z = 2 pi kz / Lz, amplitude |kappa|^(-5/3)
  wall-normal profile (1 - y^2) T_q(y) for u and w, (1 - y^2)^2 T_q(y) for v,
  T_q Chebyshev, q = (kx + kz) mod 4
  value cos(kappa_x x + kappa_z z - omega t + phi_{mode,comp}), omega =
  kappa_x U_mode, t_s = s * SPAN * Lx / (U_c n) with SPAN = 8 flow-through
  times (a band-limited signal over a window of B cycles has numerical rank
  about 2B, so a single flow-through would cap the rank near 30), U_c = 0.8;
  each mode convects at its
  own speed U_mode = U_c (0.75 + 0.5 h_mode), h_mode = frac(0.618034 (mode+1)),
  so that the 64 temporal frequencies are distinct (a single U_c would make
  every mode with the same kx share one frequency and cap the rank at 16);
  phases uniform from ``seed``
  field scaled to unit RMS, plus i.i.d. Gaussian noise of standard deviation
  ``noise`` (default 1e-6)

Structure: the clean field is exactly S T with S (m x 128) and T (128 x n),
so its rank is at most 128.  ``gap_k`` keeps the gap_k/2 largest modes at full
amplitude and scales the others by 1e-3, which makes a clear gap after the
gap_k-th singular value, and gives every mode a slow amplitude envelope
1 + 0.5 sin(2 pi (h_mode + t / t_window)) over the window (still two rows of
T per mode): on a periodic grid the snapshots of a pure travelling wave all
have the same norm, which would make the first pivot of a deterministic ID a
tie; with the envelope the skeleton is unambiguous.

Layout: row r = ((c*ny + j)*nz + kz)*nx + i (component slowest, then y, then
z, x fastest); A is column-major (each snapshot contiguous), returned as a
torch view of shape (m, n) with strides (1, m).
"""
from __future__ import annotations

import math

import numpy as np
import torch

LX = 4.0 * math.pi
LZ = 4.0 * math.pi / 3.0
GAMMA = 2.0
U_C = 0.8
SPAN = 8.0
NMODE_X = 8
NMODE_Z = 8


def wall_normal_points(ny, gamma=GAMMA):
    j = np.arange(ny, dtype=np.float64)
    if ny == 1:
        return np.zeros(1)
    return np.tanh(gamma * (2.0 * j / (ny - 1) - 1.0)) / np.tanh(gamma)


def modes(gap_k=None):
    """List of (kappa_x, kappa_z, amplitude, q) for the 64 modes."""
    out = []
    for kx in range(1, NMODE_X + 1):
        for kz in range(1, NMODE_Z + 1):
            ax = 2.0 * math.pi * kx / LX
            az = 2.0 * math.pi * kz / LZ
            amp = math.hypot(ax, az) ** (-5.0 / 3.0)
            out.append([ax, az, amp, (kx + kz) % 4])
    if gap_k is not None:
        order = sorted(range(len(out)), key=lambda i: (-out[i][2], i))
        keep = set(order[: max(int(gap_k) // 2, 0)])
        for i in range(len(out)):
            if i not in keep:
                out[i][2] *= 1e-3
    return out


def _chebyshev(q, y):
    return np.cos(q * np.arccos(np.clip(y, -1.0, 1.0)))


def snapshot_step(n):
    """Time between snapshots when n snapshots span SPAN flow-through times."""
    return SPAN * LX / (U_C * max(n, 1))


def factors(grid, ncomp, n, seed, gap_k=None, device="cpu", first=0, dt=None):
    """FP64 factors S (m x 128) and T (128 x n) with A_clean = S @ T (unit RMS).

    Snapshot s is taken at time (first + s) * dt, dt = snapshot_step(n) by
    default; a later window of one flow (same seed) takes first > 0 and the
    dt of the whole stream.  The RMS scale is that of the window."""
    nx, ny, nz = (int(g) for g in grid)
    if not 1 <= ncomp <= 3:
        raise ValueError("ncomp must be 1, 2 or 3")
    rng = np.random.default_rng(int(seed))
    md = modes(gap_k)
    phases = rng.uniform(0.0, 2.0 * math.pi, size=(len(md), ncomp))
    dev = torch.device(device)
    f64 = torch.float64
    x = torch.arange(nx, dtype=f64, device=dev) * (LX / nx)
    z = torch.arange(nz, dtype=f64, device=dev) * (LZ / nz)
    y = wall_normal_points(ny)
    m = ncomp * ny * nz * nx
    S = torch.empty((m, 2 * len(md)), dtype=f64, device=dev)
    step = snapshot_step(n) if dt is None else float(dt)
    t = (float(first) + torch.arange(n, dtype=f64, device=dev)) * step
    T = torch.empty((2 * len(md), n), dtype=f64, device=dev)
    plane = ny * nz * nx
    for mi, (ax, az, amp, q) in enumerate(md):
        # spatial phase on the (z, x) plane, same for every y
        th = (az * z)[:, None] + (ax * x)[None, :]
        cheb = _chebyshev(q, y)
        for c in range(ncomp):
            wall = (1.0 - y * y) ** (2 if c == 1 else 1)
            prof = torch.as_tensor(amp * wall * cheb, dtype=f64, device=dev)
            ang = th + phases[mi, c]
            cs = (prof[:, None, None] * torch.cos(ang)[None]).reshape(-1)
            sn = (prof[:, None, None] * torch.sin(ang)[None]).reshape(-1)
            S[c * plane:(c + 1) * plane, 2 * mi] = cs
            S[c * plane:(c + 1) * plane, 2 * mi + 1] = sn
        h = (0.618034 * (mi + 1)) % 1.0
        om = ax * U_C * (0.75 + 0.5 * h)
        env = 1.0
        if gap_k is not None:   # slow amplitude envelope: snapshot norms differ
            env = 1.0 + 0.5 * torch.sin(2.0 * math.pi * (h + t / (step * max(n, 1))))
        T[2 * mi] = env * torch.cos(om * t)
        T[2 * mi + 1] = env * torch.sin(om * t)
    # unit RMS: ||S T||_F^2 = trace((S^T S)(T T^T))
    fro2 = torch.sum((S.T @ S) * (T @ T.T)).item()
    S *= 1.0 / math.sqrt(fro2 / (m * max(n, 1)))
    return S, T


def channel_field(grid, ncomp, n, seed, noise=1e-6, gap_k=None, dtype=torch.float32,
                  device="cpu", col_chunk=64, first=0, dt=None):
    """Snapshot matrix A (m x n, column-major torch view) on ``device``.

    first / dt select a window of a longer stream of the same flow (see
    ``factors``); each window draws its own noise."""
    S, T = factors(grid, ncomp, n, seed, gap_k=gap_k, device=device, first=first, dt=dt)
    m = S.shape[0]
    At = torch.empty((n, m), dtype=dtype, device=S.device)
    gen = torch.Generator(device=S.device)
    gen.manual_seed(int(seed) * 7919 + 3 + 1_000_003 * int(first))
    St = S.T.contiguous()
    for j0 in range(0, n, col_chunk):
        j1 = min(n, j0 + col_chunk)
        blk = T[:, j0:j1].T @ St
        if noise:
            blk += noise * torch.randn(blk.shape, dtype=torch.float64, device=S.device,
                                       generator=gen)
        At[j0:j1] = blk.to(dtype)
        del blk
    return At.T


def gaussian_matrix(m, n, seed, dtype=torch.float64, device="cpu"):
    """Plain seeded Gaussian matrix (column-major view), for generic tests."""
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    return torch.randn((n, m), dtype=torch.float64, device=device, generator=gen).to(dtype).T


def low_rank_matrix(m, n, rank, seed, dtype=torch.float64, device="cpu", decay=None):
    """Exactly rank-``rank`` product B C (column-major view); optional
    geometric singular-value decay ``decay`` per index."""
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    B = torch.randn((m, rank), dtype=torch.float64, device=device, generator=gen)
    C = torch.randn((rank, n), dtype=torch.float64, device=device, generator=gen)
    if decay is not None:
        B = B * (decay ** torch.arange(rank, dtype=torch.float64, device=device))[None, :]
    At = (C.T @ B.T).to(dtype).contiguous()
    return At.T
