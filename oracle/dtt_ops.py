"""Plain differentiation and staggered-grid interpolation with DTTs (FP64).

TEST INFRASTRUCTURE ONLY.  Nothing in the product may import this module.

Section 3.3 and Appendix Tables A1 / A4 (differentiation) and A2 / A5
(interpolation between staggered grids) give, for each symmetric-periodic
sequence (SPS), a forward DTT, an operation on the k-space array and an
inverse DTT.  This module covers the eight SPS types of groups I and II
(types I-IV, even period M = 2N, N = cells):

    symmetry   grid   samples (x = j dx, or (m + 1/2) dx on half-nodes)   forward
    WSWS       nodes  j = 0..N                                            C1
    WAWA       nodes  j = 1..N-1                                          S1
    WSWA       nodes  j = 0..N-1                                          C3
    WAWS       nodes  j = 1..N                                            S3
    HSHS       half   m = 0..N-1                                          C2
    HAHA       half   m = 0..N-1                                          S2
    HSHA       half   m = 0..N-1                                          C4
    HAHS       half   m = 0..N-1                                          S4

and the eight of groups III and IV (types V-VIII, odd period M = 2N - 1):
an axis with a node wall at x = 0 and a mid-cell wall at x = (N - 1/2) dx,
pressure-like nodes j = 0..N-1 and half-nodes m = 0..N-1 (m = N-1 lies on
the mid-cell wall):

    WSHS  nodes j = 0..N-1  C5      HSWS  half m = 0..N-1  C6
    WAHA  nodes j = 1..N-1  S5      HAWA  half m = 0..N-2  S6
    WSHA  nodes j = 0..N-1  C7      HSWA  half m = 0..N-2  C8
    WAHS  nodes j = 1..N-1  S7      HAWS  half m = 0..N-1  S8

Differentiation keeps the grid and swaps S <-> A at both walls; the k-space
operation is -k (cosine -> sine) or +k (sine -> cosine).  Interpolation
keeps the symmetry and swaps the grid (W <-> H); the k-space operation is the
identity.  The inverse is (1/M) times the partner transform of the output
symmetry's forward transform (Eq. inverse_transforms).

The tables state the drop / pad bookkeeping entry by entry.  It is read here
as one rule: every DTT output index is a wavenumber index n (C1, C2: n = k;
S1, S2: n = k + 1; group II: n + 1/2 with n = k), the k-space operation
multiplies wavenumber n, wavenumbers the output transform does not carry are
dropped, and wavenumbers the input does not carry enter as zero.  Two entries
of the printed tables do not follow it and are read through it:
  * Table A2, HSHS -> WSWS lists {u_1, ..., u_{M/2-1}, 0} (M/2 values, no
    wavenumber 0); C1^{-1} takes M/2 + 1 values and a constant must
    interpolate to itself, so it is read as {u_0, ..., u_{M/2-1}, 0};
  * Table A5, WAWS -> HAHS names DST-IV as the forward transform; the forward
    transform of WAWS is DST-III (Table 1 and Table A4), which is used.
"""
from __future__ import annotations

import numpy as np

from . import dtt

# symmetry -> (half-node grid, forward transform, sine family, antiperiodic)
SYMMETRY = {
    "WSWS": (False, "C1", False, False),
    "WAWA": (False, "S1", True, False),
    "WSWA": (False, "C3", False, True),
    "WAWS": (False, "S3", True, True),
    "HSHS": (True, "C2", False, False),
    "HAHA": (True, "S2", True, False),
    "HSHA": (True, "C4", False, True),
    "HAHS": (True, "S4", True, True),
    "WSHS": (False, "C5", False, False),
    "WAHA": (False, "S5", True, False),
    "WSHA": (False, "C7", False, True),
    "WAHS": (False, "S7", True, True),
    "HSWS": (True, "C6", False, False),
    "HAWA": (True, "S6", True, False),
    "HSWA": (True, "C8", False, True),
    "HAWS": (True, "S8", True, True),
}


def mid_wall(sym: str) -> bool:
    """Groups III and IV: one wall at a node, the other at mid-cell."""
    return sym[0] != sym[2]


def period(sym: str, n: int) -> int:
    """M = 2N (groups I, II) or 2N - 1 (groups III, IV)."""
    return 2 * n - 1 if mid_wall(sym) else 2 * n


def sample_length(sym: str, n: int) -> int:
    """Representative samples of a symmetry on an axis of n cells (groups
    III / IV: n nodes, the mid-cell wall at (n - 1/2) dx)."""
    if mid_wall(sym):
        return n - 1 if sym in ("WAHA", "WAHS", "HAWA", "HSWA") else n
    return {"WSWS": n + 1, "WAWA": n - 1}.get(sym, n)


def positions(sym: str, n: int, dx: float) -> np.ndarray:
    """Coordinates of the representative samples."""
    half = SYMMETRY[sym][0]
    if half:
        return (np.arange(sample_length(sym, n)) + 0.5) * dx
    first = 0 if sym[1] == "S" else 1
    return (np.arange(sample_length(sym, n)) + first) * dx


def wavenumber_index(sym: str, n: int) -> np.ndarray:
    """Wavenumber index of each output of the symmetry's forward transform
    (Table 1: k = 2 pi n / (M dx), group II with n + 1/2)."""
    _, T, sine, anti = SYMMETRY[sym]
    length = sample_length(sym, n)
    k = np.arange(length, dtype=np.float64)
    if anti:
        return k + 0.5
    return k + 1.0 if sine else k


def diff_symmetry(sym: str) -> str:
    flip = {"S": "A", "A": "S"}
    return sym[0] + flip[sym[1]] + sym[2] + flip[sym[3]]


def interp_symmetry(sym: str) -> str:
    swap = {"W": "H", "H": "W"}
    return swap[sym[0]] + sym[1] + swap[sym[2]] + sym[3]


def _apply(sym_in: str, sym_out: str, f: np.ndarray, n: int, dx: float, deriv: bool) -> np.ndarray:
    f = np.asarray(f, np.float64)
    if f.shape[-1] != sample_length(sym_in, n):
        raise ValueError(f"{sym_in} on {n} cells has {sample_length(sym_in, n)} samples")
    M = period(sym_in, n)
    _, T_in, sine_in, _ = SYMMETRY[sym_in]
    _, T_out, _, _ = SYMMETRY[sym_out]
    U = dtt.apply(T_in, f, -1)
    n_in = wavenumber_index(sym_in, n)
    n_out = wavenumber_index(sym_out, n)
    V = np.zeros(f.shape[:-1] + (len(n_out),))
    where = {v: i for i, v in enumerate(n_in)}
    for o, nv in enumerate(n_out):
        i = where.get(nv)
        if i is None:
            continue                      # wavenumber absent from the input: zero
        factor = 1.0
        if deriv:
            k = 2.0 * np.pi * nv / (M * dx)
            factor = k if sine_in else -k
        V[..., o] = factor * U[..., i]
    return dtt.apply(dtt.inverse_partner(T_out), V, -1) / M


def diff(sym: str, f: np.ndarray, n: int, dx: float):
    """(derivative on the same grid, its symmetry): Tables A1 and A4."""
    out = diff_symmetry(sym)
    return _apply(sym, out, f, n, dx, True), out


def interp(sym: str, f: np.ndarray, n: int, dx: float):
    """(values on the other grid, their symmetry): Tables A2 and A5."""
    out = interp_symmetry(sym)
    return _apply(sym, out, f, n, dx, False), out


def stagger(sym: str, f: np.ndarray, n: int, dx: float):
    """(derivative on the other grid, its symmetry): differentiation and
    interpolation in one k-space operation (Tables A3 and A6), the staggered
    derivative of the PSTD step."""
    out = interp_symmetry(diff_symmetry(sym))
    return _apply(sym, out, f, n, dx, True), out
