"""Discrete trigonometric transforms, types I-IV, as direct O(n^2) sums (FP64).

TEST INFRASTRUCTURE ONLY.  Nothing in the product (the CUDA library, its
Python binding or the benchmark's timed path) may import this module; only the
tests, the smoke check and the benchmark's CPU-baseline leg use it.

The paper (Section 3.2) adopts the unnormalised forward transforms of FFTW and
does not restate them; the eight definitions below are the standard ones
(REDFT00/10/01/11 and RODFT00/10/01/11).  With j, k = 0..n-1:

  C1: Y_k = X_0 + (-1)^k X_{n-1} + 2 sum_{j=1}^{n-2} X_j cos(pi j k / (n-1))
  C2: Y_k = 2 sum_j X_j cos(pi (j+1/2) k / n)
  C3: Y_k = X_0 + 2 sum_{j>=1} X_j cos(pi j (k+1/2) / n)
  C4: Y_k = 2 sum_j X_j cos(pi (j+1/2)(k+1/2) / n)
  S1: Y_k = 2 sum_j X_j sin(pi (j+1)(k+1) / (n+1))
  S2: Y_k = 2 sum_j X_j sin(pi (j+1/2)(k+1) / n)
  S3: Y_k = (-1)^k X_{n-1} + 2 sum_{j<=n-2} X_j sin(pi (j+1)(k+1/2) / n)
  S4: Y_k = 2 sum_j X_j sin(pi (j+1/2)(k+1/2) / n)

Each transform is applied as an explicit n x n matrix (the matrix product is
the only library primitive used).  The implied period M of each type
(Table 1) and the inverse identities of Eq. (inverse_transforms) are given by
``implied_period`` and ``inverse``.
"""
from __future__ import annotations

import numpy as np

KINDS = ("C1", "C2", "C3", "C4", "S1", "S2", "S3", "S4")


def dtt_matrix(kind: str, n: int) -> np.ndarray:
    """The n x n matrix T with Y = T @ X for the unnormalised transform ``kind``."""
    if kind not in KINDS:
        raise ValueError(f"unknown transform {kind!r}")
    if n < 1 or (kind == "C1" and n < 2):
        raise ValueError(f"{kind} needs a longer input than n={n}")
    j = np.arange(n, dtype=np.float64)[None, :]   # input index (columns)
    k = np.arange(n, dtype=np.float64)[:, None]   # output index (rows)
    pi = np.pi
    if kind == "C1":
        T = 2.0 * np.cos(pi * j * k / (n - 1))
        T[:, 0] = 1.0
        T[:, n - 1] = (-1.0) ** np.arange(n)
    elif kind == "C2":
        T = 2.0 * np.cos(pi * (j + 0.5) * k / n)
    elif kind == "C3":
        T = 2.0 * np.cos(pi * j * (k + 0.5) / n)
        T[:, 0] = 1.0
    elif kind == "C4":
        T = 2.0 * np.cos(pi * (j + 0.5) * (k + 0.5) / n)
    elif kind == "S1":
        T = 2.0 * np.sin(pi * (j + 1) * (k + 1) / (n + 1))
    elif kind == "S2":
        T = 2.0 * np.sin(pi * (j + 0.5) * (k + 1) / n)
    elif kind == "S3":
        T = 2.0 * np.sin(pi * (j + 1) * (k + 0.5) / n)
        T[:, n - 1] = (-1.0) ** np.arange(n)
    else:  # S4
        T = 2.0 * np.sin(pi * (j + 0.5) * (k + 0.5) / n)
    return T


def implied_period(kind: str, n: int) -> int:
    """Implied period M of the symmetric-periodic sequence (Table 1, groups I and II)."""
    if kind == "C1":
        return 2 * (n - 1)
    if kind == "S1":
        return 2 * (n + 1)
    return 2 * n


# Eq. (inverse_transforms): T_j^{-1} = (1/M) T_{j-1} for j = 3, (1/M) T_j for
# j = 1, 4 and (1/M) T_{j+1} for j = 2 (types I-IV only).
_INVERSE_PARTNER = {"C1": "C1", "C2": "C3", "C3": "C2", "C4": "C4",
                    "S1": "S1", "S2": "S3", "S3": "S2", "S4": "S4"}


def inverse_partner(kind: str) -> str:
    """The transform whose (1/M)-scaled form inverts ``kind`` (Eq. inverse_transforms)."""
    return _INVERSE_PARTNER[kind]


def apply(kind: str, x: np.ndarray, axis: int = -1) -> np.ndarray:
    """Forward transform ``kind`` of ``x`` along ``axis`` (FP64)."""
    x = np.asarray(x, dtype=np.float64)
    xm = np.moveaxis(x, axis, -1)
    T = dtt_matrix(kind, xm.shape[-1])
    y = xm @ T.T
    return np.moveaxis(y, -1, axis)


def inverse(kind: str, y: np.ndarray, axis: int = -1) -> np.ndarray:
    """Inverse of transform ``kind`` via Eq. (inverse_transforms): (1/M) T_partner."""
    y = np.asarray(y, dtype=np.float64)
    n = y.shape[axis]
    M = implied_period(kind, n)
    return apply(inverse_partner(kind), y, axis) / M
