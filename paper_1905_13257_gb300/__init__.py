"""Pass-efficient interpolative decomposition for one GB300 (sm_103a).

The method (Dunton, Jofre, Iaccarino, Doostan, arXiv:1905.13257) compresses a
snapshot matrix A by a column ID A ~ A(:,J) P.  The library forms both
randomized sketches W = Psi A and Y = A Omega in one read of A, selects J by a
column-pivoted QR of W, solves for P, offers the coarse-grid (sub-sampled)
variant and the single-pass ID, measures the reconstruction error in one more
read, and runs batches of independent matrices in one graph launch.  The C ABI
is include/idsketch.h; ``api`` wraps it for PyTorch tensors.
"""
from .api import (IdBatch, IdSketch, Mlp, check_wait, gaussian_fill, gaussian_table_bits,
                  mlp_features)
from ._binding import load, IdError

__all__ = ["IdBatch", "IdSketch", "Mlp", "check_wait", "gaussian_fill",
           "gaussian_table_bits", "mlp_features", "load", "IdError"]
