"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle."""
from .channel import (channel_field, factors, modes, wall_normal_points, gaussian_matrix,
                      low_rank_matrix)

__all__ = ["channel_field", "factors", "modes", "wall_normal_points", "gaussian_matrix",
           "low_rank_matrix"]
