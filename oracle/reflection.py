"""Weights for arbitrary real reflection coefficients (Section 5), FP64.

TEST INFRASTRUCTURE ONLY.  Nothing in the product may import this module.

The four basic runs of one axis are ordered as in Section 5,
p = [p_(1,1), p_(1,-1), p_(-1,1), p_(-1,-1)] = [NN, ND, DN, DD].  Each column
of the image-source polarity matrix M is one basic run; with the image-source
amplitudes r = [R_L, 1, R_R, R_L R_R] the weights are w = (1/4) M^T r, and the
field with reflection coefficients (R_L, R_R) is w^T p, valid for t < 2L/c0
(t < 3L/c0 when both are zero).  In d dimensions the weights of the 4^d runs
are the tensor product of the per-axis weights (the "same idea" of Section 5).
"""
from __future__ import annotations

import itertools

import numpy as np

BASIC_RUNS = (("N", "N"), ("N", "D"), ("D", "N"), ("D", "D"))

POLARITY = np.array([[1, 1, -1, -1],
                     [1, 1, 1, 1],
                     [1, -1, 1, -1],
                     [1, -1, -1, 1]], dtype=np.float64)


def axis_weights(r_left: float, r_right: float) -> np.ndarray:
    """w = (1/4) M^T r for one axis."""
    r = np.array([r_left, 1.0, r_right, r_left * r_right], dtype=np.float64)
    return 0.25 * POLARITY.T @ r


def combination_weights(refl) -> list:
    """All 4^d (bc tuple, weight) pairs for per-axis (R_L, R_R) pairs ``refl``."""
    per_axis = [axis_weights(rl, rr) for rl, rr in refl]
    out = []
    for idx in itertools.product(range(4), repeat=len(refl)):
        w = 1.0
        for a, i in enumerate(idx):
            w *= per_axis[a][i]
        out.append((tuple(BASIC_RUNS[i] for i in idx), w))
    return out
