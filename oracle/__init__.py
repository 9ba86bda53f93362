"""Oracle: a plain, slow FP64 CPU implementation of the pass-efficient ID.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` leg (and
``--impl reference`` arm) of ``bench.py`` may use it.  It shares no code,
tables or helpers with the CUDA library in ``paper_1905_13257_gb300``.

Modules
  rng            Philox4x32-10 counter generator and the bfloat16 quantile
                 table that give Psi and Omega (Sec. 2.2; Algorithm 4 step 3)
  interp_decomp  sketches, column-pivoted Householder QR, interpolation
                 matrix, deterministic / randomized / sub-sampled ID, error
                 metrics and the Theorem 2.1 bound (Sec. 2.4-2.5)
  single_pass    the single-pass ID of Algorithm 6 (Sec. 2.6): the
                 coarse-to-fine interpolation operator M on the mesh, the
                 interpolated skeleton, its error and the Theorem 2.2 bound
  learned        the learned skeleton proposal (no counterpart in the paper):
                 column features on a coarse sub-grid, a 2-layer GELU MLP
                 with its loss, gradients and SGD step, the top-2k proposal,
                 the pivoted QR restricted to it and the fallback rule
                 (import as ``oracle.learned``)
  fp8            the FP8-E4M3 precision form of the sketch products:
                 E4M3 rounding, per-column power-of-two scales, the
                 dequantised matrix (import as ``oracle.fp8``)

Parity status of each function is pinned by ``tests/test_oracle_*.py``; none
is unpinned.
"""
from .rng import (philox4x32_10, twelve_bit_fields, bf16_round_f64, gaussian_table,
                  gaussian_table_bits, psi, omega, STREAM_PSI, STREAM_OMEGA)
from .interp_decomp import (sketch, householder, cpqr, back_substitute,
                            interpolation_matrix, column_id, deterministic_id,
                            randomized_id, coarse_rows, subsampled_id, recon_error,
                            spectral_norm, theorem21_rho, RANK_TOL_FACTOR)
from .single_pass import (axis_weights, coarse_to_fine, single_pass_id, single_pass_error,
                          theorem22_bound)

__all__ = [
    "philox4x32_10", "twelve_bit_fields", "bf16_round_f64", "gaussian_table",
    "gaussian_table_bits", "psi", "omega", "STREAM_PSI", "STREAM_OMEGA",
    "sketch", "householder", "cpqr", "back_substitute", "interpolation_matrix",
    "column_id", "deterministic_id", "randomized_id", "coarse_rows",
    "subsampled_id", "recon_error", "spectral_norm", "theorem21_rho",
    "RANK_TOL_FACTOR", "axis_weights", "coarse_to_fine", "single_pass_id",
    "single_pass_error", "theorem22_bound",
]
