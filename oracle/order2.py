"""Plain FP64 second-order pressure-only form of the DTT-PSTD leapfrog, the
oracle for the GPU path's p-only stepper.

TEST INFRASTRUCTURE ONLY.  Nothing in the product may import this module; only
the tests, the smoke check and the benchmark's CPU legs use it.

The coupled leapfrog of Eq. (dtt_pstd_solution) (Section 4, and its n-D form
in Section 4.3) updates

    u_i^{n+1/2} = u_i^{n-1/2} - (dt/rho0) D_{p,i} p^n
    p^{n+1}     = p^n - dt rho0 c0^2 sum_i D_{u,i} u_i^{n+1/2}

with D_{p,i} = T_{i,2}^{-1} a_{i,1} T_{i,1} and D_{u,i} = T_{i,1}^{-1} a_{i,2}
T_{i,2} the staggered derivatives of Table 2.  Writing the pressure update at
steps n and n-1 and subtracting removes the velocity:

    p^{n+1} - 2 p^n + p^{n-1} = -dt rho0 c0^2 sum_i D_{u,i} (u_i^{n+1/2} - u_i^{n-1/2})
                              = c0^2 dt^2 sum_i D_{u,i} D_{p,i} p^n,

a two-level recurrence in p alone.  It is the coupled scheme exactly when
p^{n-1} is the pressure the coupled scheme had one step earlier.  The paper
states only the coupled form; this module is that elimination, evaluated with
the same D_{u,i} and D_{p,i} as ``oracle.pstd``.

Start (readings, listed in the design notes): zero initial velocity.  With
``uinit="as_given"`` (u^{-1/2} = 0) the coupled step gives p^{-1} = p^0.  With
``uinit="halfstep"`` (u^{-1/2} = (dt / (2 rho0)) D_p p^0, Section 4.2's "zero
initial velocity, accounting for the staggered grid") it gives
p^{-1} = p^0 + (c0^2 dt^2 / 2) sum_i D_{u,i} D_{p,i} p^0, the usual start of a
second-order scheme with zero initial time derivative (p^{-1} = p^1).
"""
from __future__ import annotations

import numpy as np

from . import pstd


def laplacian(desc: pstd.Desc, p: np.ndarray) -> np.ndarray:
    """sum_i D_{u,i} D_{p,i} p: the staggered derivatives composed on each axis."""
    p = np.asarray(p, np.float64)
    out = np.zeros_like(p)
    for i in range(desc.ndim):
        out += pstd.grad_u_axis(desc, pstd.grad_p_axis(desc, p, i), i)
    return out


def init_prev(desc: pstd.Desc, p0: np.ndarray, uinit: str = "halfstep") -> np.ndarray:
    """p^{-1} of a run that starts from p^0 with zero initial velocity."""
    p0 = np.asarray(p0, np.float64)
    if uinit == "as_given":
        return p0.copy()
    if uinit != "halfstep":
        raise ValueError(uinit)
    return p0 + 0.5 * desc.c0 ** 2 * desc.dt ** 2 * laplacian(desc, p0)


def step(desc: pstd.Desc, p: np.ndarray, p_prev: np.ndarray):
    """(p^{n+1}, p^n) from (p^n, p^{n-1})."""
    p = np.asarray(p, np.float64)
    p_new = 2.0 * p - np.asarray(p_prev, np.float64) + desc.c0 ** 2 * desc.dt ** 2 * laplacian(desc, p)
    return p_new, p


def run(desc: pstd.Desc, p: np.ndarray, p_prev: np.ndarray, nsteps: int):
    """(p^{n+nsteps}, p^{n+nsteps-1}) from (p^n, p^{n-1})."""
    p = np.asarray(p, np.float64)
    p_prev = np.asarray(p_prev, np.float64)
    for _ in range(nsteps):
        p, p_prev = step(desc, p, p_prev)
    return p, p_prev
