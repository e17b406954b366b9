"""Closed-form discrete solution and discrete energy of the DTT-PSTD leapfrog (FP64).

TEST INFRASTRUCTURE ONLY.  Nothing in the product may import this module.

Both facts below are derived from Eq. (dtt_pstd_solution) and Table 2; the
paper does not print them.  They give references that do not time-step.

Modal solution.  The T1 basis functions of each axis (cosines for a Neumann
left wall, sines for Dirichlet) diagonalise D_u D_p with eigenvalue -k^2,
using the wavenumber attached to each T1 output entry (Table 1).  Eliminating
u from the leapfrog gives p^{n+1} - 2 p^n + p^{n-1} = -(c0 |k| dt)^2 p^n per
mode, so with sin(Omega dt / 2) = c0 |k| dt / 2:

  * half-step start (u^{-1/2} = (dt / 2 rho0) D_p p^0):  P^n = P^0 cos(n Omega dt)
  * u^{-1/2} = 0:  P^n = P^0 cos((n + 1/2) Omega dt) / cos(Omega dt / 2)

Discrete energy.  With the quadrature weight w = 1/2 on a stored pressure node
that lies on a Neumann wall (1 elsewhere) the staggered operators satisfy
D_u = -W^{-1} D_p^T, so the leapfrog conserves
    E^n = sum_j w_j (p_j^n)^2 / (2 rho0 c0^2)
          + (rho0 / 2) sum_i sum w^{(i)} u_i^{n-1/2} u_i^{n+1/2}
exactly (up to rounding); u_i carries the pressure-node weights of the other
axes and weight 1 along its own axis.
"""
from __future__ import annotations

import numpy as np

from . import dtt, dtt_ops
from .pstd import Desc, mid_wall, p_nodes, symmetries, t1_of, u_len


def mode_wavenumbers(n: int, bc: tuple, dx: float) -> np.ndarray:
    """Wavenumber of each T1 output entry of one axis (Table 1, M = 2N).

    A periodic axis uses the DFT and the wavenumbers of Section 2."""
    if bc == ("P", "P"):
        from .pstd import fourier_wavenumbers
        return fourier_wavenumbers(n, dx)
    if mid_wall(bc):    # groups III / IV: M = 2N - 1
        sym = symmetries(bc)[0]
        return 2.0 * np.pi * dtt_ops.wavenumber_index(sym, n) / (dtt_ops.period(sym, n) * dx)
    L = n * dx
    T1 = t1_of(bc)
    if T1 == "C1":      # n = 0..N
        return np.pi * np.arange(0, n + 1) / L
    if T1 == "S1":      # n = 1..N-1
        return np.pi * np.arange(1, n) / L
    return np.pi * (np.arange(0, n) + 0.5) / L   # C3, S3: antiperiodic


def _omega_dt(desc: Desc) -> np.ndarray:
    k2 = np.zeros([len(p_nodes(n, b)) for n, b in zip(desc.ncells, desc.bc)])
    for i in range(desc.ndim):
        k = mode_wavenumbers(desc.ncells[i], desc.bc[i], desc.dx[i])
        shape = [1] * desc.ndim
        shape[i] = len(k)
        k2 = k2 + (k ** 2).reshape(shape)
    s = desc.c0 * desc.dt * np.sqrt(k2) / 2.0
    if np.any(s > 1.0):
        raise ValueError("time step beyond the stability limit")
    return 2.0 * np.arcsin(s)


def _forward(bc, P, axis):
    if bc == ("P", "P"):
        from .pstd import dft_matrix
        n = P.shape[axis]
        return np.moveaxis(np.moveaxis(P, axis, -1) @ dft_matrix(n).T, -1, axis)
    if np.iscomplexobj(P):      # a periodic axis was transformed already
        return dtt.apply(t1_of(bc), P.real, axis) + 1j * dtt.apply(t1_of(bc), P.imag, axis)
    return dtt.apply(t1_of(bc), P, axis)


def _inverse(bc, P, axis):
    if bc == ("P", "P"):
        from .pstd import dft_matrix
        n = P.shape[axis]
        return np.moveaxis((np.moveaxis(P, axis, -1) @ np.conj(dft_matrix(n)).T) / n, -1, axis)
    if np.iscomplexobj(P):
        return dtt.inverse(t1_of(bc), P.real, axis) + 1j * dtt.inverse(t1_of(bc), P.imag, axis)
    return dtt.inverse(t1_of(bc), P, axis)


def modal_pressure(desc: Desc, p0: np.ndarray, nsteps: int, uinit: str = "halfstep") -> np.ndarray:
    """p after ``nsteps`` leapfrog steps from p0 with zero initial velocity."""
    P = np.asarray(p0, dtype=np.float64)
    for i in range(desc.ndim):
        P = _forward(desc.bc[i], P, i)
    wdt = _omega_dt(desc)
    if uinit == "halfstep":
        P = P * np.cos(nsteps * wdt)
    elif uinit == "as_given":
        P = P * np.cos((nsteps + 0.5) * wdt) / np.cos(0.5 * wdt)
    else:
        raise ValueError(uinit)
    for i in range(desc.ndim):
        P = _inverse(desc.bc[i], P, i)
    return P.real if np.iscomplexobj(P) else P


def separable_modal_pressure(desc: Desc, factors: list, nsteps: int,
                             uinit: str = "halfstep", out_index=None) -> np.ndarray:
    """Modal solution for p0 = sum_b prod_i factors[b][i](axis i), at full size.

    ``factors[b][i]`` is the 1-D profile of term b along axis i on the stored
    pressure nodes.  The forward transform of a separable term is the outer
    product of 1-D transforms, so the d-D spectrum costs O(B N^d) and the
    inverse O(d N^{d+1}).  ``out_index`` optionally restricts the result to a
    sub-block (a tuple of index arrays / slices) to bound memory at 3-D sizes.
    """
    wdt = _omega_dt(desc)
    spec = None
    for term in factors:
        t = None
        for i in range(desc.ndim):
            f = dtt.apply(t1_of(desc.bc[i]), np.asarray(term[i], np.float64))
            t = f if t is None else np.multiply.outer(t, f)
        spec = t if spec is None else spec + t
    if uinit == "halfstep":
        spec = spec * np.cos(nsteps * wdt)
    else:
        spec = spec * np.cos((nsteps + 0.5) * wdt) / np.cos(0.5 * wdt)
    for i in range(desc.ndim):
        T1 = t1_of(desc.bc[i])
        n = spec.shape[i]
        Minv = dtt.dtt_matrix(dtt.inverse_partner(T1), n) / dtt.implied_period(T1, n)
        if out_index is not None and out_index[i] is not None:
            Minv = Minv[out_index[i]]
        spec = np.moveaxis(np.tensordot(Minv, spec, axes=([1], [i])), 0, i)
    return spec


def node_weights(n: int, bc: tuple) -> np.ndarray:
    """Quadrature weight of each stored pressure node: 1/2 on a Neumann wall node."""
    j = p_nodes(n, bc)
    w = np.ones(len(j))
    if bc == ("P", "P"):
        return w
    if bc[0] == "N":
        w[0] = 0.5
    if bc[1] == "N":
        w[-1] = 0.5
    return w


def half_weights(n: int, bc: tuple) -> np.ndarray:
    """Weight of each stored velocity half-node: 1/2 on the one a Dirichlet
    mid-cell wall passes through (u symmetric there), 1 elsewhere."""
    w = np.ones(u_len(n, bc))
    if mid_wall(bc) and bc[1] == "Dm":
        w[-1] = 0.5
    return w


def _weights(desc: Desc, field: int) -> np.ndarray:
    """Tensor-product weights of p (field 0) or u_i (field i+1)."""
    w = None
    for a in range(desc.ndim):
        if field == a + 1:
            wa = half_weights(desc.ncells[a], desc.bc[a])
        else:
            wa = node_weights(desc.ncells[a], desc.bc[a])
        w = wa if w is None else np.multiply.outer(w, wa)
    return w


def energy(desc: Desc, p: np.ndarray, u_prev: list, u_next: list) -> float:
    """Discrete energy E^n from p^n, u^{n-1/2} and u^{n+1/2}."""
    e = float(np.sum(_weights(desc, 0) * p * p)) / (2.0 * desc.rho0 * desc.c0 ** 2)
    for i in range(desc.ndim):
        e += 0.5 * desc.rho0 * float(np.sum(_weights(desc, i + 1) * u_prev[i] * u_next[i]))
    return e
