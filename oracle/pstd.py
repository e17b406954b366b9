"""Plain FP64 DTT-based PSTD stepper (Section 4), the oracle for the GPU path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product may import this module; only
the tests, the smoke check and the benchmark's CPU-baseline leg use it.

What it computes, in the paper's notation:

* Table 2 maps the boundary conditions (left, right) of one axis to the
  pressure symmetry and the transform pair (T1, T2) with k-space
  coefficients (a1, a2):
      Neumann-Neumann     WSWS / HAHA   C1 / S2   -k / +k
      Neumann-Dirichlet   WSWA / HAHS   C3 / S4   -k / +k
      Dirichlet-Neumann   WAWS / HSHA   S3 / C4   +k / -k
      Dirichlet-Dirichlet WAWA / HSHS   S1 / C2   +k / -k
* Tables A3 and A6 give the index bookkeeping of each staggered derivative:
  the wavenumber vector of Table 1 (k_n = 2 pi n / (M dx) for groups I,
  k_n = 2 pi (n + 1/2) / (M dx) for group II) and which entries are dropped
  (NN: n = 0 of C1; DD: n = 0 of C2) or padded with a zero (NN: H_0 before
  C1^{-1}; DD: G_0 before C3^{-1}) before the inverse.
* Eq. (dtt_pstd_solution) and its 2-D form (Section 4.3) give the leapfrog:
      u_i^{n+1/2} = u_i^{n-1/2} - (dt/rho0) T_{i,2}^{-1}{ a_{i,1} T_{i,1}{ p^n } }
      p^{n+1}     = p^n - dt rho0 c0^2 sum_i T_{i,1}^{-1}{ a_{i,2} T_{i,2}{ u_i^{n+1/2} } }
  Each T_{i,.} is the 1-D transform along axis i (the untouched axes'
  transform and inverse cancel exactly).

Readings where the paper is silent (each listed in the design notes):

* N is the number of cells per axis, L = N dx, M = 2N; pressure lives on the
  nodes x_j = j dx with walls at j = 0 and j = N, velocity on the N half-nodes
  (m + 1/2) dx.  Only the pressure nodes that are not on a Dirichlet wall are
  stored (Dirichlet wall pressure is identically zero).
* Groups III and IV of Table 1 (types V-VIII, odd period M = 2N - 1) describe
  an axis whose right wall lies half a cell past the last node, at
  x = (N - 1/2) dx, with nodes j = 0..N-1 (bc "Nm" or "Dm" on the right).
  The pressure symmetry is W?H? (WSHS, WSHA, WAHS, WAHA: C5, C7, S7, S5) and
  the velocity's H?W? (HAWA, HAWS, HSWA, HSWS: S6, S8, C8, C6); the staggered
  derivatives apply the same rule as Tables A3/A6 (``dtt_ops.stagger``).  The
  velocity half-node on the mid-cell wall is stored only where u is symmetric
  about it (Dirichlet), so u has N - 1 (Neumann) or N (Dirichlet) samples.
* The initial half-step velocity either equals the given u0
  (``uinit="as_given"``) or is u^{-1/2} = u0 + (dt / (2 rho0)) D_p p^0
  (``uinit="halfstep"``), which makes the time-centred velocity equal u0 at
  t = 0 ("zero initial velocity, accounting for the staggered grid",
  Section 4.2).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Sequence

import numpy as np

from . import dtt, dtt_ops

NEUMANN = "N"
DIRICHLET = "D"
PERIODIC = "P"      # Table 2's periodic row: the Fourier PSTD method of Section 2
NEUMANN_MID = "Nm"  # right wall at mid-cell, x = (N - 1/2) dx (Table 1 groups III / IV)
DIRICHLET_MID = "Dm"

# Table 2: (left, right) -> (T1, T2, sign of a1, sign of a2)
TABLE2 = {
    ("N", "N"): ("C1", "S2", -1.0, +1.0),
    ("N", "D"): ("C3", "S4", -1.0, +1.0),
    ("D", "N"): ("S3", "C4", +1.0, -1.0),
    ("D", "D"): ("S1", "C2", +1.0, -1.0),
}


@dataclass
class Desc:
    """Problem statement: cells per axis, spacing, walls, medium and time step."""
    ncells: Sequence[int]
    dx: Sequence[float]
    bc: Sequence[tuple]          # per axis: (left, right), each "N" or "D"
    c0: float = 1500.0
    rho0: float = 1000.0
    dt: float = 0.0
    ndim: int = field(init=False)

    def __post_init__(self):
        self.ncells = tuple(int(n) for n in self.ncells)
        self.ndim = len(self.ncells)
        if len(self.dx) == 1 and self.ndim > 1:
            self.dx = tuple(float(self.dx[0]) for _ in range(self.ndim))
        self.dx = tuple(float(d) for d in self.dx)
        self.bc = tuple((str(l), str(r)) for l, r in self.bc)
        if not (len(self.dx) == len(self.bc) == self.ndim):
            raise ValueError("ncells, dx and bc must have one entry per axis")


def mid_wall(bc: tuple) -> bool:
    """The right wall lies half a cell past node N - 1 (types V-VIII)."""
    return bc[1] in (NEUMANN_MID, DIRICHLET_MID)


def symmetries(bc: tuple):
    """(pressure SPS, velocity SPS) of a walled axis (Table 2; groups III / IV
    for a mid-cell right wall)."""
    left = "S" if bc[0] == NEUMANN else "A"
    if mid_wall(bc):
        sym_p = "W" + left + "H" + ("S" if bc[1] == NEUMANN_MID else "A")
    else:
        sym_p = "W" + left + "W" + ("S" if bc[1] == NEUMANN else "A")
    return sym_p, dtt_ops.interp_symmetry(dtt_ops.diff_symmetry(sym_p))


def t1_of(bc: tuple) -> str:
    """The pressure transform T1 of a walled axis."""
    if mid_wall(bc):
        return dtt_ops.SYMMETRY[symmetries(bc)[0]][1]
    return TABLE2[bc][0]


def p_nodes(n: int, bc: tuple) -> np.ndarray:
    """Indices j of the stored pressure nodes x_j = j dx (Dirichlet walls dropped).

    A periodic axis stores the N nodes j = 0..N-1 (node N is node 0); an axis
    with a mid-cell right wall the nodes up to N - 1."""
    if bc == (PERIODIC, PERIODIC):
        return np.arange(0, n)
    lo = 1 if bc[0] == DIRICHLET else 0
    hi = n - 1 if (bc[1] == DIRICHLET or mid_wall(bc)) else n
    return np.arange(lo, hi + 1)


def u_len(n: int, bc: tuple) -> int:
    """Stored velocity half-nodes along the axis (N, or N - 1 next to a
    Neumann mid-cell wall, where u vanishes on the wall)."""
    if mid_wall(bc):
        return dtt_ops.sample_length(symmetries(bc)[1], n)
    return n


def p_len(n: int, bc: tuple) -> int:
    return len(p_nodes(n, bc))


def field_shapes(desc: Desc):
    """Shapes of p and u_1..u_d (C order, axis 0 slowest)."""
    plen = [p_len(n, b) for n, b in zip(desc.ncells, desc.bc)]
    shapes = [tuple(plen)]
    for i in range(desc.ndim):
        s = list(plen)
        s[i] = u_len(desc.ncells[i], desc.bc[i])
        shapes.append(tuple(s))
    return shapes


def wavenumbers(n: int, bc: tuple, dx: float):
    """Table 1 wavenumbers for the transform pair of this wall pair (M = 2N)."""
    M = 2 * n
    periodic = bc[0] == bc[1]          # groups I (NN, DD) are periodic, II antiperiodic
    if periodic:
        # index n = 0..N (C1 range); S1 / C2 / S2 use sub-ranges of the same vector
        return 2.0 * np.pi * np.arange(0, n + 1) / (M * dx)
    return 2.0 * np.pi * (np.arange(0, n) + 0.5) / (M * dx)


def fourier_wavenumbers(n: int, dx: float) -> np.ndarray:
    """k_n = 2 pi n / (N dx) in DFT order, n in [-N/2, N/2 - 1] (even N) or
    [-(N-1)/2, (N-1)/2] (odd N), Section 2."""
    idx = np.arange(n)
    nn = np.where(idx < (n + 1) // 2, idx, idx - n)
    if n % 2 == 0:
        nn[n // 2] = -n // 2
    return 2.0 * np.pi * nn / (n * dx)


def dft_matrix(n: int) -> np.ndarray:
    """F[k, j] = exp(-2 pi i j k / N), the discrete Fourier transform."""
    j = np.arange(n)
    return np.exp(-2j * np.pi * np.outer(j, j) / n)


def fourier_grad(x: np.ndarray, axis: int, n: int, dx: float, shift: float) -> np.ndarray:
    """F^{-1}{ i k e^{i k shift} F{x} } along ``axis`` (Eq. fourier_pstd_solution)."""
    k = fourier_wavenumbers(n, dx)
    F = dft_matrix(n)
    xm = np.moveaxis(np.asarray(x, np.float64), axis, -1)
    X = xm @ F.T
    Y = X * (1j * k * np.exp(1j * k * shift))
    y = (Y @ np.conj(F).T) / n
    return np.moveaxis(y.real, -1, axis)


def grad_p(p: np.ndarray, axis: int, n: int, bc: tuple, dx: float) -> np.ndarray:
    """T2^{-1}{ a1 T1{p} } along ``axis``: pressure nodes -> velocity half-nodes."""
    if bc == (PERIODIC, PERIODIC):
        return fourier_grad(p, axis, n, dx, +0.5 * dx)
    if mid_wall(bc):
        pm = np.moveaxis(np.asarray(p, np.float64), axis, -1)
        return np.moveaxis(dtt_ops.stagger(symmetries(bc)[0], pm, n, dx)[0], -1, axis)
    T1, T2, s1, _ = TABLE2[bc]
    M = 2 * n
    k = wavenumbers(n, bc, dx)
    P = dtt.apply(T1, p, axis)
    P = np.moveaxis(P, axis, -1)
    if bc == ("N", "N"):
        # Table A3, WSWS: C1 output n = 0..N; drop n = 0, keep n = 1..N
        G = s1 * k[1:] * P[..., 1:]
    elif bc == ("D", "D"):
        # Table A3, WAWA: S1 output n = 1..N-1; prepend G_0 = 0
        G = np.concatenate([np.zeros(P.shape[:-1] + (1,)),
                            s1 * k[1:n] * P], axis=-1)
    else:
        # Table A6: same index range n = 0..N-1 before and after
        G = s1 * k * P
    G = np.moveaxis(G, -1, axis)
    # T2^{-1} = (1/M) partner(T2), Eq. (inverse_transforms)
    return dtt.apply(dtt.inverse_partner(T2), G, axis) / M


def grad_u(u: np.ndarray, axis: int, n: int, bc: tuple, dx: float) -> np.ndarray:
    """T1^{-1}{ a2 T2{u} } along ``axis``: velocity half-nodes -> pressure nodes."""
    if bc == (PERIODIC, PERIODIC):
        return fourier_grad(u, axis, n, dx, -0.5 * dx)
    if mid_wall(bc):
        um = np.moveaxis(np.asarray(u, np.float64), axis, -1)
        return np.moveaxis(dtt_ops.stagger(symmetries(bc)[1], um, n, dx)[0], -1, axis)
    T1, T2, _, s2 = TABLE2[bc]
    M = 2 * n
    k = wavenumbers(n, bc, dx)
    U = dtt.apply(T2, u, axis)
    U = np.moveaxis(U, axis, -1)
    if bc == ("N", "N"):
        # Table A3, HAHA: S2 output n = 1..N; prepend H_0 = 0 for C1^{-1}
        H = np.concatenate([np.zeros(U.shape[:-1] + (1,)),
                            s2 * k[1:] * U], axis=-1)
    elif bc == ("D", "D"):
        # Table A3, HSHS: C2 output n = 0..N-1; drop n = 0 for S1^{-1}
        H = s2 * k[1:n] * U[..., 1:]
    else:
        H = s2 * k * U
    H = np.moveaxis(H, -1, axis)
    # T1^{-1} = (1/M) partner(T1), Eq. (inverse_transforms)
    return dtt.apply(dtt.inverse_partner(T1), H, axis) / M


def dt_from_cfl(cfl: float, dx: float, c0: float) -> float:
    """dt = CFL dx / c0 (Section 4.2)."""
    return cfl * dx / c0


class State:
    """p^n and u_i^{n-1/2}, FP64."""

    def __init__(self, p, us):
        self.p = np.array(p, dtype=np.float64)
        self.u = [np.array(u, dtype=np.float64) for u in us]

    def copy(self):
        return State(self.p, self.u)


def grad_p_axis(desc: Desc, p: np.ndarray, i: int) -> np.ndarray:
    return grad_p(p, i, desc.ncells[i], desc.bc[i], desc.dx[i])


def grad_u_axis(desc: Desc, u: np.ndarray, i: int) -> np.ndarray:
    return grad_u(u, i, desc.ncells[i], desc.bc[i], desc.dx[i])


def init_velocity(desc: Desc, p0, u0=None, uinit: str = "halfstep"):
    """u^{-1/2} from the given u0 (zero when None) per the chosen reading."""
    shapes = field_shapes(desc)
    us = []
    for i in range(desc.ndim):
        u = np.zeros(shapes[1 + i]) if u0 is None else np.array(u0[i], dtype=np.float64)
        if uinit == "halfstep":
            u = u + (desc.dt / (2.0 * desc.rho0)) * grad_p_axis(desc, np.asarray(p0, np.float64), i)
        elif uinit != "as_given":
            raise ValueError(uinit)
        us.append(u)
    return us


def step(desc: Desc, s: State) -> State:
    """One leapfrog step of Eq. (dtt_pstd_solution) (and its n-D form)."""
    p = s.p
    u_new = [s.u[i] - (desc.dt / desc.rho0) * grad_p_axis(desc, p, i)
             for i in range(desc.ndim)]
    div = np.zeros_like(p)
    for i in range(desc.ndim):
        div += grad_u_axis(desc, u_new[i], i)
    p_new = p - desc.dt * desc.rho0 * desc.c0 ** 2 * div
    return State(p_new, u_new)


def run(desc: Desc, s: State, nsteps: int) -> State:
    for _ in range(nsteps):
        s = step(desc, s)
    return s


def stable_cfl_limit(ndim: int) -> float:
    """CFL bound 2/(pi sqrt(d)): 2/pi in 1-D (Section 4.2), same as Fourier PSTD (Section 4.4)."""
    return 2.0 / (np.pi * np.sqrt(ndim))
