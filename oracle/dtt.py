"""Discrete trigonometric transforms, types I-VIII, as direct O(n^2) sums (FP64).

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

Types V-VIII (groups III and IV of Table 1, odd period M) are not in FFTW
and the paper does not print them.  They are built from what Section 3.2 and
Fig. 3 say a DTT is: the transform of a symmetric-periodic sequence (SPS).
Place the n representative samples at their coordinates t (in units of dx,
the left point of symmetry at t = 0: whole-sample W at t = 0, 1, ...,
half-sample H at t = 1/2, 3/2, ...; an antisymmetric W point holds a zero
and is not a sample), extend them by both symmetries, and sum over one
period M:

    Y_k = sum_j w_j x_j cos(2 pi nu_k t_j / M)   (symmetric left point, DCT)
    Y_k = sum_j w_j x_j sin(2 pi nu_k t_j / M)   (antisymmetric left point, DST)

with w_j = 1 for a sample on a point of symmetry and 2 otherwise, and the
wavenumber index nu_k = k (periodic SPS, cosines), k + 1 (periodic, sines) or
k + 1/2 (antiperiodic).  The same sum reproduces the eight FFTW types above
exactly (a pin), so types V-VIII follow the same conventions.

Each transform is applied as an explicit n x n matrix (the matrix product is
the only library primitive used).  The implied period M of each type
(Table 1) and the inverse identities of Eq. (inverse_transforms) are given by
``implied_period`` and ``inverse``.
"""
from __future__ import annotations

import numpy as np

KINDS = ("C1", "C2", "C3", "C4", "S1", "S2", "S3", "S4")
KINDS_III_IV = ("C5", "C6", "C7", "C8", "S5", "S6", "S7", "S8")

# Table 1: the SPS of each transform (left point, right point).
SPS = {"C1": "WSWS", "C2": "HSHS", "C3": "WSWA", "C4": "HSHA",
       "S1": "WAWA", "S2": "HAHA", "S3": "WAWS", "S4": "HAHS",
       "C5": "WSHS", "C6": "HSWS", "C7": "WSHA", "C8": "HSWA",
       "S5": "WAHA", "S6": "HAWA", "S7": "WAHS", "S8": "HAWS"}


def sps_geometry(sym: str, n: int):
    """(t, w, M, nu): sample coordinates, multiplicities, implied period and
    output wavenumber indices of n representative samples of SPS ``sym``."""
    left_h, left_a, right_h, right_a = sym[0] == "H", sym[1] == "A", sym[2] == "H", sym[3] == "A"
    t0 = 0.5 if left_h else (1.0 if left_a else 0.0)
    t = t0 + np.arange(n, dtype=np.float64)
    # right point of symmetry R: half a sample past the last one (H), on it
    # (symmetric W) or one sample past it (antisymmetric W: a zero)
    R = t[-1] + (0.5 if right_h else (1.0 if right_a else 0.0))
    M = int(round(2 * R))
    w = np.where((t == 0.0) | (t == R), 1.0, 2.0)
    k = np.arange(n, dtype=np.float64)
    if left_a != right_a:
        nu = k + 0.5
    else:
        nu = k + 1.0 if left_a else k
    return t, w, M, nu


def sps_matrix(sym: str, n: int) -> np.ndarray:
    """The n x n transform of SPS ``sym`` by the one-period sum above."""
    t, w, M, nu = sps_geometry(sym, n)
    ang = 2.0 * np.pi * np.outer(nu, t) / M
    return w[None, :] * (np.sin(ang) if sym[1] == "A" else np.cos(ang))


def dtt_matrix(kind: str, n: int) -> np.ndarray:
    """The n x n matrix T with Y = T @ X for the unnormalised transform ``kind``."""
    if kind in KINDS_III_IV:
        if n < 1:
            raise ValueError(f"{kind} needs a longer input than n={n}")
        return sps_matrix(SPS[kind], n)
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
    """Implied period M of the symmetric-periodic sequence (Table 1)."""
    if kind in KINDS_III_IV:
        return 2 * n - 1 if kind in ("C5", "C6", "C7", "S8") else 2 * n + 1
    if kind == "C1":
        return 2 * (n - 1)
    if kind == "S1":
        return 2 * (n + 1)
    return 2 * n


# Eq. (inverse_transforms): T_j^{-1} = (1/M) T_{j-1} for j = 3, 7,
# (1/M) T_j for j = 1, 4, 5, 8 and (1/M) T_{j+1} for j = 2, 6.
_INVERSE_PARTNER = {"C1": "C1", "C2": "C3", "C3": "C2", "C4": "C4",
                    "S1": "S1", "S2": "S3", "S3": "S2", "S4": "S4",
                    "C5": "C5", "C6": "C7", "C7": "C6", "C8": "C8",
                    "S5": "S5", "S6": "S7", "S7": "S6", "S8": "S8"}


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
