"""Python front end of the C ABI, with PyTorch tensors for device memory and
streams.  Argument marshalling only: every step runs in libidsketch.so.

Layout conventions (as in include/idsketch.h): a snapshot matrix is an m x n
column-major torch view (strides (1, ld)), e.g. ``At.T`` for a contiguous
(n, m) tensor; J is int32 in pivot order; P is a row-major (k, n) FP64 tensor.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _binding as B


def _stream_handle(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream), stream


def _colmajor(A, m):
    if A.dim() != 2 or A.shape[0] != m:
        raise ValueError(f"expected an ({m}, n) column-major tensor, got {tuple(A.shape)}")
    if A.shape[1] > 1 and A.stride(0) != 1:
        raise ValueError("columns must be contiguous (stride(0) == 1)")
    ld = A.stride(1) if A.shape[1] > 1 else max(A.stride(1), m)
    return ld


class _DeviceView:
    """Zero-copy torch view of library-owned device memory."""

    def __init__(self, ptr, shape, strides_bytes, typestr):
        self.__cuda_array_interface__ = {
            "shape": tuple(shape), "strides": tuple(strides_bytes), "typestr": typestr,
            "data": (int(ptr), False), "version": 2,
        }


class IdSketch:
    """One stream of snapshot columns compressed by the pass-efficient ID."""

    def __init__(self, m, n_max, k, l, seed=0, dtype=torch.float32, prec="exact",
                 grid=None, ncomp=0, coarse_stride=None, want_Y=True, want_coarse=False,
                 window_cols=0, stream=None):
        self.lib = B.load()
        cfg = B.IdConfig()
        cfg.m, cfg.n_max, cfg.k, cfg.l, cfg.seed = m, n_max, k, l, seed
        cfg.dtype = B.ID_F64 if dtype == torch.float64 else B.ID_F32
        cfg.prec = {"exact": B.ID_SKETCH_EXACT, "bf16": B.ID_SKETCH_BF16,
                    "fp8": B.ID_SKETCH_FP8E4M3}[prec]
        if grid is not None:
            cfg.grid[:] = list(grid)
        cfg.ncomp = ncomp
        if coarse_stride is not None:
            cfg.coarse_stride[:] = list(coarse_stride)
        cfg.want_Y = int(bool(want_Y))
        cfg.want_coarse = int(bool(want_coarse))
        cfg.window_cols = int(window_cols)
        self.cfg = cfg
        self.m, self.n_max, self.k, self.l = m, n_max, k, l
        self.dtype = dtype
        self._sh, self.stream = _stream_handle(stream)
        h = C.c_void_p()
        B.check(self.lib.id_sketch_create(C.byref(cfg), self._sh, C.byref(h)), "id_sketch_create")
        self.h = h
        self._keep = []   # borrowed chunks stay referenced until launched

    def close(self):
        if getattr(self, "h", None):
            self.lib.id_sketch_destroy(self.h)
            self.h = None
            self._keep = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def stream_columns(self, cols):
        ld = _colmajor(cols, self.m)
        if cols.dtype != self.dtype or not cols.is_cuda:
            raise ValueError("columns must be CUDA tensors of the sketch dtype")
        B.check(self.lib.id_sketch_stream_columns(self.h, C.c_void_p(cols.data_ptr()), ld,
                                                  cols.shape[1]), "id_sketch_stream_columns")
        if self.cfg.window_cols:
            self._keep.append(cols)

    def flush(self):
        B.check(self.lib.id_sketch_flush(self.h), "id_sketch_flush")
        self._keep = []

    def reset(self):
        B.check(self.lib.id_sketch_reset(self.h), "id_sketch_reset")
        self._keep = []

    def timing(self, on=True):
        """Record CUDA events around each launch of the fused sketch kernel and
        of the error-pass kernel (id_timing_enable)."""
        B.check(self.lib.id_timing_enable(self.h, 1 if on else 0), "id_timing_enable")

    def read_timing(self, which):
        """(total ms, launches) of 'sketch' or 'recon' since the last read."""
        ms, cnt = C.c_double(), C.c_int64()
        B.check(self.lib.id_timing_read(self.h, {"sketch": 0, "recon": 1}[which], C.byref(ms),
                                        C.byref(cnt)), "id_timing_read")
        return ms.value, cnt.value

    def n_seen(self):
        n = C.c_int64()
        B.check(self.lib.id_sketch_get(self.h, None, None, None, C.byref(n), None), "id_sketch_get")
        return n.value

    def _factor(self, fn, name, device):
        n = self.n_seen()
        dev = self.stream.device if device == "cuda" else torch.device("cpu")
        J = torch.empty(self.k, dtype=torch.int32, device=dev)
        P = torch.empty((self.k, n), dtype=torch.float64, device=dev)
        kout = C.c_int32()
        st = fn(self.h, C.c_void_p(J.data_ptr()), C.c_void_p(P.data_ptr()), C.byref(kout))
        B.check(st, name, allow=(B.ID_ERR_RANK_DEFICIENT,))
        self._keep = []
        return J, P, kout.value

    def factor(self, device="cuda"):
        """Randomized ID from W = Psi A: returns (J, P, k_out)."""
        return self._factor(self.lib.id_factor, "id_factor", device)

    def factor_restricted(self, cand, device="cuda"):
        """ID with the skeleton chosen among the candidate columns cand (host
        or CUDA int32 indices; id_factor_restricted): returns (J, P, k_out)."""
        if not (torch.is_tensor(cand) and cand.is_cuda):
            cand = torch.as_tensor(cand, dtype=torch.int32).cpu()
        cand = cand.to(torch.int32).contiguous()
        n = self.n_seen()
        dev = self.stream.device if device == "cuda" else torch.device("cpu")
        J = torch.empty(self.k, dtype=torch.int32, device=dev)
        P = torch.empty((self.k, n), dtype=torch.float64, device=dev)
        kout = C.c_int32()
        st = self.lib.id_factor_restricted(self.h, C.c_void_p(cand.data_ptr()), cand.numel(),
                                           C.c_void_p(J.data_ptr()), C.c_void_p(P.data_ptr()),
                                           C.byref(kout))
        B.check(st, "id_factor_restricted", allow=(B.ID_ERR_RANK_DEFICIENT,))
        self._keep = []
        return J, P, kout.value

    def coarse_factor(self, device="cuda"):
        """Sub-sampled ID from the coarse rows: returns (J_c, P_c, k_out)."""
        return self._factor(self.lib.id_coarse_factor, "id_coarse_factor", device)

    def reconstruct_error(self, A, J, P, k=None):
        ld = _colmajor(A, self.m)
        k = int(J.numel()) if k is None else int(k)
        J = J.to(torch.int32).contiguous()
        P = P.to(torch.float64).contiguous()
        fro, mx = C.c_double(), C.c_double()
        B.check(self.lib.id_reconstruct_error(self.h, C.c_void_p(A.data_ptr()), ld, A.shape[1],
                                              C.c_void_p(J.data_ptr()), C.c_void_p(P.data_ptr()),
                                              k, C.byref(fro), C.byref(mx)),
                "id_reconstruct_error")
        return fro.value, mx.value

    def set_mesh(self, x, y, z, periods=(0.0, 0.0, 0.0)):
        """Grid coordinates for the single-pass ID's interpolation (id_set_mesh)."""
        import numpy as np
        arrs = [np.ascontiguousarray(v, dtype=np.float64) for v in (x, y, z)]
        per = np.ascontiguousarray(periods, dtype=np.float64)
        B.check(self.lib.id_set_mesh(self.h, *[C.c_void_p(a.ctypes.data) for a in arrs],
                                     C.c_void_p(per.ctypes.data)), "id_set_mesh")

    def single_pass_lift(self, Jc, k=None):
        """S = M A_c(:, J_c) (m x k, device, column-major): the single-pass ID's
        fine skeleton (id_single_pass_lift)."""
        k = int(Jc.numel()) if k is None else int(k)
        Jc = Jc.to(torch.int32).contiguous()
        S = torch.empty((k, self.m), dtype=self.dtype, device=self.stream.device)
        B.check(self.lib.id_single_pass_lift(self.h, C.c_void_p(Jc.data_ptr()), k,
                                             C.c_void_p(S.data_ptr())), "id_single_pass_lift")
        return S.T

    def single_pass_error(self, A, Jc, Pc, k=None):
        """(rel_fro, rel_max) of A_hat = M A_c(:, J_c) P_c (id_single_pass_error)."""
        ld = _colmajor(A, self.m)
        k = int(Jc.numel()) if k is None else int(k)
        Jc = Jc.to(torch.int32).contiguous()
        Pc = Pc.to(torch.float64).contiguous()
        fro, mx = C.c_double(), C.c_double()
        B.check(self.lib.id_single_pass_error(self.h, C.c_void_p(A.data_ptr()), ld, A.shape[1],
                                              C.c_void_p(Jc.data_ptr()),
                                              C.c_void_p(Pc.data_ptr()), k, C.byref(fro),
                                              C.byref(mx)), "id_single_pass_error")
        return fro.value, mx.value

    def sketches(self):
        """Zero-copy views (W (l, n) FP64, Y (m, l) or None, A_c (m_c, n) or None)."""
        w, y, ac = C.c_void_p(), C.c_void_p(), C.c_void_p()
        n, mc = C.c_int64(), C.c_int64()
        B.check(self.lib.id_sketch_get(self.h, C.byref(w), C.byref(y), C.byref(ac), C.byref(n),
                                       C.byref(mc)), "id_sketch_get")
        n = n.value
        es = 8 if self.dtype == torch.float64 else 4
        ts = "<f8" if self.dtype == torch.float64 else "<f4"
        dev = self.stream.device
        W = torch.as_tensor(_DeviceView(w.value, (self.l, n), (8 * self.n_max, 8), "<f8"),
                            device=dev)
        Y = None
        if y.value:
            Y = torch.as_tensor(_DeviceView(y.value, (self.m, self.l), (es, es * self.m), ts),
                                device=dev)
        Ac = None
        if ac.value and n > 0:
            Ac = torch.as_tensor(_DeviceView(ac.value, (mc.value, n), (es, es * mc.value), ts),
                                 device=dev)
        return W, Y, Ac


class IdBatch:
    """Many independent snapshot matrices through the randomized ID in one
    CUDA-graph launch (id_batch_*).

    problems: a list of dicts with ``A`` (an m x n column-major CUDA tensor,
    FP32 or FP64, n <= 512), ``k``, ``l``, ``seed`` and optionally ``prec``
    ("exact" or "bf16").  The tensors are read at every run and stay
    referenced by the batch.
    """

    def __init__(self, problems, stream=None):
        self.lib = B.load()
        self._sh, self.stream = _stream_handle(stream)
        arr = (B.IdBatchProblem * len(problems))()
        self._A = []
        self.shapes = []
        for i, p in enumerate(problems):
            A = p["A"]
            m = A.shape[0]
            ld = _colmajor(A, m)
            if not A.is_cuda or A.dtype not in (torch.float32, torch.float64):
                raise ValueError("A must be an FP32 or FP64 CUDA tensor")
            q = arr[i]
            q.d_A, q.lda, q.m, q.n = A.data_ptr(), ld, m, A.shape[1]
            q.k, q.l, q.seed = int(p["k"]), int(p["l"]), int(p["seed"])
            q.dtype = B.ID_F64 if A.dtype == torch.float64 else B.ID_F32
            q.prec = B.ID_SKETCH_BF16 if p.get("prec", "exact") == "bf16" else B.ID_SKETCH_EXACT
            self._A.append(A)
            self.shapes.append((int(p["k"]), A.shape[1]))
        self.count = len(problems)
        h = C.c_void_p()
        B.check(self.lib.id_batch_create(arr, self.count, self._sh, C.byref(h)),
                "id_batch_create")
        self.h = h
        dev = self.stream.device
        nk = sum(k for k, _ in self.shapes)
        nkn = sum(k * n for k, n in self.shapes)
        self.J = torch.empty(nk, dtype=torch.int32, device=dev)
        self.P = torch.empty(nkn, dtype=torch.float64, device=dev)
        self.kout = torch.empty(self.count, dtype=torch.int32, device=dev)

    def run(self):
        """Enqueue the whole batch (one graph launch after the first run)."""
        B.check(self.lib.id_batch_run(self.h, C.c_void_p(self.J.data_ptr()),
                                      C.c_void_p(self.P.data_ptr()),
                                      C.c_void_p(self.kout.data_ptr())), "id_batch_run")

    def tune(self):
        """Autotune the work split of the batch's sketches (id_batch_tune):
        returns (the chosen candidate, {candidate: ms per graph launch}); a
        candidate is the work-item size in MB of A (0: automatic) for a batch
        with a work list, else the row blocks per CTA of each sketch."""
        choice = C.c_int32()
        ms = (C.c_float * 5)()
        B.check(self.lib.id_batch_tune(self.h, C.c_void_p(self.J.data_ptr()),
                                       C.c_void_p(self.P.data_ptr()),
                                       C.c_void_p(self.kout.data_ptr()), C.byref(choice), ms),
                "id_batch_tune")
        return choice.value, dict(zip((0, 32, 16, 8, 4), [float(x) for x in ms]))

    def wait(self):
        """Wait for the last run: a list of (J_b, P_b, k_out_b), device views."""
        ko = (C.c_int32 * self.count)()
        B.check(self.lib.id_batch_wait(self.h, ko), "id_batch_wait",
                allow=(B.ID_ERR_RANK_DEFICIENT,))
        out, jo, po = [], 0, 0
        for b, (k, n) in enumerate(self.shapes):
            out.append((self.J[jo:jo + k], self.P[po:po + k * n].view(k, n), int(ko[b])))
            jo += k
            po += k * n
        return out

    def close(self):
        if getattr(self, "h", None):
            self.lib.id_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mlp_features(A, rows, scale=1.0, stream=None):
    """X (n x F, FP32): row j holds scale * A(rows, j) (id_mlp_features).
    A: m x n column-major CUDA tensor (FP32 or FP64); rows: int64 indices."""
    lib = B.load()
    sh, stream = _stream_handle(stream)
    m = A.shape[0]
    ld = _colmajor(A, m)
    rows = torch.as_tensor(rows, dtype=torch.int64, device=A.device).contiguous()
    X = torch.empty((A.shape[1], rows.numel()), dtype=torch.float32, device=A.device)
    dt = B.ID_F64 if A.dtype == torch.float64 else B.ID_F32
    B.check(lib.id_mlp_features(C.c_void_p(A.data_ptr()), ld, m, A.shape[1], dt,
                                C.c_void_p(rows.data_ptr()), rows.numel(), C.c_float(scale),
                                C.c_void_p(X.data_ptr()), sh), "id_mlp_features")
    return X


class Mlp:
    """The learned proposal's network on the GPU (id_mlp_*): s = w2 .
    gelu(x W1 + b1) + b2, parameters as FP32 CUDA tensors (W1: F x H; the
    products use them rounded to bfloat16, with FP32 accumulation)."""

    def __init__(self, params, device="cuda", stream=None):
        self.lib = B.load()
        self._sh, self.stream = _stream_handle(stream)
        f32 = dict(dtype=torch.float32, device=device)
        self.W1 = torch.as_tensor(params["W1"], **f32).contiguous()
        self.b1 = torch.as_tensor(params["b1"], **f32).contiguous()
        self.w2 = torch.as_tensor(params["w2"], **f32).contiguous()
        self.b2 = torch.as_tensor(params["b2"], **f32).reshape(1).contiguous()
        self.F, self.H = self.W1.shape

    def forward(self, X):
        """Scores s (n); keeps Z and G for backward."""
        X = X.to(torch.float32).contiguous()
        n = X.shape[0]
        self.Z = torch.empty((n, self.H), dtype=torch.float32, device=X.device)
        self.G = torch.empty_like(self.Z)
        self.s = torch.empty(n, dtype=torch.float32, device=X.device)
        p = lambda t: C.c_void_p(t.data_ptr())   # noqa: E731
        B.check(self.lib.id_mlp_forward(p(X), n, self.F, self.H, p(self.W1), p(self.b1),
                                        p(self.w2), p(self.b2), p(self.Z), p(self.G), p(self.s),
                                        self._sh), "id_mlp_forward")
        return self.s

    def backward(self, X, y, pos_weight=1.0):
        """Gradients {W1, b1, w2, b2} of the loss at the last forward pass."""
        X = X.to(torch.float32).contiguous()
        y = torch.as_tensor(y, dtype=torch.float32, device=X.device).contiguous()
        n = X.shape[0]
        g = {"W1": torch.empty_like(self.W1), "b1": torch.empty_like(self.b1),
             "w2": torch.empty_like(self.w2), "b2": torch.empty_like(self.b2)}
        ds = torch.empty(n, dtype=torch.float32, device=X.device)
        dZ = torch.empty_like(self.Z)
        p = lambda t: C.c_void_p(t.data_ptr())   # noqa: E731
        B.check(self.lib.id_mlp_backward(p(X), n, self.F, self.H, p(self.Z), p(self.G),
                                         p(self.w2), p(self.s), p(y), C.c_float(pos_weight),
                                         p(g["W1"]), p(g["b1"]), p(g["w2"]), p(g["b2"]), p(ds),
                                         p(dZ), self._sh), "id_mlp_backward")
        return g

    def check(self):
        """Synchronise the stream and raise if a tensor-core product's bounded
        wait gave up since the last check (id_mlp_check)."""
        B.check(self.lib.id_mlp_check(self._sh), "id_mlp_check")

    def step(self, grads, lr):
        """SGD: every parameter -= lr * its gradient."""
        for name in ("W1", "b1", "w2", "b2"):
            t = getattr(self, name)
            B.check(self.lib.id_mlp_sgd(C.c_void_p(t.data_ptr()),
                                        C.c_void_p(grads[name].data_ptr()), t.numel(),
                                        C.c_float(lr), self._sh), "id_mlp_sgd")


def gaussian_fill(which, seed, first, count, width, device=None, stream=None):
    """The counter-based Gaussian entries (which=1 Psi, 2 Omega) as a (count, width)
    FP32 CUDA tensor: row i holds G(first + i, 0:width)."""
    lib = B.load()
    sh, stream = _stream_handle(stream)
    out = torch.empty((count, width), dtype=torch.float32, device=stream.device)
    B.check(lib.id_gaussian_fill(which, seed, first, count, width, C.c_void_p(out.data_ptr()), sh),
            "id_gaussian_fill")
    return out


def gaussian_table_bits():
    lib = B.load()
    buf = (C.c_uint16 * 4096)()
    B.check(lib.id_gaussian_table(buf), "id_gaussian_table")
    return [int(x) for x in buf]


def check_wait(mode, device=0):
    """Self-check of the device-side bounded waits (id_check_wait): returns the
    status code (ID_OK = 0, ID_ERR_TIMEOUT = 6); raises IdError on any other."""
    lib = B.load()
    st = lib.id_check_wait(int(device), int(mode))
    if st not in (0, 6):
        B.check(st, "id_check_wait")
    return st
