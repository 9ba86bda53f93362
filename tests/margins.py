"""Seed choice and skeleton checks for the pivot-margin rule.

A skeleton J is unique only when the greedy pivot choice is not within
rounding of a tie: the oracle reports the margin min_s (nu1 - nu2) / nu1 over
its steps, and J equality is asserted when it is at least MARGIN.  Gap
inputs pick their seed so that this holds (the seed scan runs the oracle
only); every other comparison asserts either J equality or, below the
margin, that the returned skeleton is a valid one.
"""
import numpy as np

import oracle

MARGIN = 1e-4


def sketch_seed_with_margin(An, k, l, seeds):
    """First sketch seed whose oracle randomized ID of An has pivot margin
    >= MARGIN; returns (seed, Wo, (J, P, k_out, margin))."""
    m, n = An.shape
    for s in seeds:
        Wo, _ = oracle.sketch(An, oracle.psi(l, m, s), np.zeros((n, 1)))
        res = oracle.column_id(Wo, k)
        if res[3] >= MARGIN:
            return s, Wo, res
    raise AssertionError(f"no sketch seed in {list(seeds)} gives a pivot margin >= {MARGIN}")


def assert_valid_skeleton(J, P, kout, n):
    """k_out distinct in-range pivots and P(:, J) = I exactly."""
    J = np.asarray(J)[:kout]
    P = np.asarray(P)[:kout]
    assert len(set(J.tolist())) == kout
    assert np.all((J >= 0) & (J < n))
    assert np.array_equal(P[:, J], np.eye(kout))
