"""The C ABI without a GPU: the library loads, exports every symbol declared
in include/idsketch.h, and its host-only logic behaves (no GPU compute)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "idsketch.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1905_13257_gb300 import _binding, build
    if not os.path.exists(_binding.LIB_PATH):
        build.build()
    return _binding.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(id_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 13, names
    for name in names:
        assert hasattr(lib, name), name
    from paper_1905_13257_gb300 import _binding
    assert sorted(_binding.SIGNATURES) == names


def test_config_struct_layout(lib):
    from paper_1905_13257_gb300 import _binding
    assert C.sizeof(_binding.IdConfig) == 96


def test_gaussian_table_matches_oracle_bitwise(lib):
    buf = (C.c_uint16 * 4096)()
    assert lib.id_gaussian_table(buf) == 0
    assert np.array_equal(np.array(buf[:], dtype=np.uint16), oracle.gaussian_table_bits())


def test_status_strings_and_version(lib):
    assert lib.id_status_str(0) == b"ok"
    assert b"rank" in lib.id_status_str(5)
    assert lib.id_version() >= 100


def _cfg(**kw):
    from paper_1905_13257_gb300 import _binding
    c = _binding.IdConfig()
    c.m, c.n_max, c.k, c.l, c.seed = 1000, 64, 4, 8, 1
    for key, v in kw.items():
        if key in ("grid", "coarse_stride"):
            getattr(c, key)[:] = v
        else:
            setattr(c, key, v)
    return c


@pytest.mark.parametrize("bad", [dict(m=0), dict(n_max=0), dict(k=0), dict(k=9, l=8),
                                 dict(l=97, k=4), dict(dtype=3), dict(prec=7),
                                 dict(prec=1, dtype=1), dict(prec=2, dtype=1),
                                 dict(prec=3), dict(window_cols=-1),
                                 dict(want_coarse=1, ncomp=3, grid=(10, 10, 10),
                                      coarse_stride=(2, 2, 2)),  # 3000 != m
                                 dict(want_coarse=1, ncomp=1, grid=(10, 10, 10),
                                      coarse_stride=(0, 1, 1)),
                                 dict(n_max=1 << 20)])
def test_invalid_config_rejected_before_any_gpu_call(lib, bad):
    h = C.c_void_p(123)
    cfg = _cfg(**bad)
    assert lib.id_sketch_create(C.byref(cfg), None, C.byref(h)) == 1
    assert h.value is None


@pytest.mark.parametrize("bad", [dict(l=65, k=4, want_Y=1), dict(l=90, k=80, dtype=1),
                                 dict(want_coarse=1, ncomp=1, grid=(10, 10, 10),
                                      coarse_stride=(1, 1, 1), k=65, l=70)])
def test_wide_sketch_limits_rejected_before_any_gpu_call(lib, bad):
    """l > 64 serves FP32 data without Y, and the coarse QR keeps k <= 64:
    the other requests are unsupported (not invalid), before any GPU call."""
    h = C.c_void_p(123)
    cfg = _cfg(**bad)
    assert lib.id_sketch_create(C.byref(cfg), None, C.byref(h)) == 7
    assert h.value is None


def test_null_arguments_rejected(lib):
    assert lib.id_sketch_create(None, None, None) == 1
    assert lib.id_sketch_stream_columns(None, None, 0, 0) == 1
    assert lib.id_factor(None, None, None, None) == 1
    assert lib.id_gaussian_fill(3, 0, 0, 1, 1, None, None) == 1
    lib.id_sketch_destroy(None)


def test_batch_problem_struct_layout(lib):
    from paper_1905_13257_gb300 import _binding
    assert C.sizeof(_binding.IdBatchProblem) == 56
    assert _binding.IdBatchProblem.seed.offset == 48


def _prob(**kw):
    from paper_1905_13257_gb300 import _binding
    p = _binding.IdBatchProblem()
    p.d_A, p.lda, p.m, p.n, p.k, p.l, p.seed = 4096, 1000, 1000, 64, 4, 8, 1
    for key, v in kw.items():
        setattr(p, key, v)
    return p


@pytest.mark.parametrize("bad", [dict(d_A=None), dict(m=0), dict(lda=999), dict(n=0),
                                 dict(n=513), dict(k=0), dict(k=9, l=8), dict(l=97),
                                 dict(l=65, dtype=1),
                                 dict(k=65, l=64, n=64),
                                 dict(dtype=2), dict(prec=2), dict(prec=1, dtype=1),
                                 dict(reserved=1)])
def test_invalid_batch_rejected_before_any_gpu_call(lib, bad):
    from paper_1905_13257_gb300 import _binding
    arr = (_binding.IdBatchProblem * 2)(_prob(), _prob(**bad))
    h = C.c_void_p(123)
    assert lib.id_batch_create(arr, 2, None, C.byref(h)) == 1
    assert h.value is None


def test_batch_count_limits(lib):
    from paper_1905_13257_gb300 import _binding
    arr = (_binding.IdBatchProblem * 1)(_prob())
    h = C.c_void_p()
    assert lib.id_batch_create(arr, 0, None, C.byref(h)) == 1
    assert lib.id_batch_create(arr, _binding.ID_BATCH_MAX_PROBLEMS + 1, None, C.byref(h)) == 1
    assert lib.id_batch_create(None, 1, None, C.byref(h)) == 1
    assert lib.id_batch_run(None, None, None, None) == 1
    assert lib.id_batch_wait(None, None) == 1
    lib.id_batch_destroy(None)


def test_network_calls_reject_bad_arguments_before_any_gpu_call(lib):
    p = C.c_void_p(4096)
    assert lib.id_mlp_forward(None, 10, 10, 8, p, p, p, p, p, p, p, None) == 1
    assert lib.id_mlp_forward(p, 0, 10, 8, p, p, p, p, p, p, p, None) == 1
    assert lib.id_mlp_forward(p, 10, 10, 0, p, p, p, p, p, p, p, None) == 1
    assert lib.id_mlp_backward(p, 10, 10, 8, p, p, p, p, p, C.c_float(-1.0), p, p, p, p, p, p,
                               None) == 1
    assert lib.id_mlp_sgd(p, p, 0, C.c_float(0.1), None) == 1
    assert lib.id_mlp_sgd(p, p, 10, C.c_float(float("nan")), None) == 1
    assert lib.id_mlp_features(p, 100, 100, 10, 7, p, 5, C.c_float(1.0), p, None) == 1
    assert lib.id_mlp_features(p, 99, 100, 10, 0, p, 5, C.c_float(1.0), p, None) == 1
