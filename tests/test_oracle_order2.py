"""Pins of the second-order pressure-only oracle (oracle/order2.py).

The form is the coupled leapfrog of Eq. (dtt_pstd_solution) with the velocity
eliminated, so it is pinned to facts that do not come from its own code:

* the coupled FP64 stepper (a different algorithm: two fields per axis, the
  velocity stepped explicitly), which it must reproduce step by step from the
  matching start, for every wall pair of Table 2, the periodic row, 1-D to 3-D;
* single modes written out by hand: cos(k x) (Neumann left wall) or sin(k x)
  (Dirichlet left wall) with a wavenumber of Table 1 is an eigenfunction of
  D_u D_p with eigenvalue -k^2, so from the zero-velocity start the recurrence
  p^{n+1} = (2 - (c0 k dt)^2) p^n - p^{n-1} gives p^n = cos(n theta) p^0 with
  cos(theta) = 1 - (c0 k dt)^2 / 2 (half-step start) and
  p^n = cos((n + 1/2) theta) / cos(theta / 2) p^0 (u^{-1/2} = 0);
* planted mistakes (a dropped c0^2, a wrong sign, a wrong start) fail.
"""
import numpy as np
import pytest

from oracle import order2, pstd

DX = 1e-4
C0 = 1500.0


def _desc(ncells, bcs, cfl=0.3):
    return pstd.Desc(ncells, (DX,), bcs, c0=C0, rho0=1000.0, dt=pstd.dt_from_cfl(cfl, DX, C0))


def _field(desc, seed):
    shape = pstd.field_shapes(desc)[0]
    return np.random.default_rng(seed).standard_normal(shape)


CASES = [
    ((16,), [("N", "N")]), ((16,), [("N", "D")]), ((16,), [("D", "N")]), ((16,), [("D", "D")]),
    ((12,), [("P", "P")]), ((9,), [("P", "P")]),
    ((10, 7), [("D", "N"), ("N", "N")]), ((6, 9), [("P", "P"), ("D", "D")]),
    ((5, 6, 4), [("N", "D"), ("D", "D"), ("N", "N")]),
]


@pytest.mark.parametrize("ncells,bcs", CASES)
@pytest.mark.parametrize("uinit", ["halfstep", "as_given"])
def test_matches_coupled_leapfrog(ncells, bcs, uinit):
    """The two-level recurrence reproduces the coupled scheme's pressure at every step."""
    d = _desc(ncells, bcs, cfl=0.2)
    p0 = _field(d, 3)
    s = pstd.State(p0, pstd.init_velocity(d, p0, None, uinit))
    p, pm = p0.copy(), order2.init_prev(d, p0, uinit)
    scale = np.abs(p0).max()
    for _ in range(25):
        s = pstd.step(d, s)
        p, pm = order2.step(d, p, pm)
        assert np.abs(p - s.p).max() < 1e-11 * scale


def _mode(n, bc, m):
    """(stored node values, wavenumber) of mode m of one axis."""
    x = pstd.p_nodes(n, bc) * DX
    L = n * DX
    if bc == ("P", "P"):
        k = 2 * np.pi * m / L
        return np.cos(k * x + 0.3), k
    k = np.pi * (m + (0.5 if bc[0] != bc[1] else 0.0)) / L
    return (np.cos(k * x) if bc[0] == "N" else np.sin(k * x)), k


@pytest.mark.parametrize("bc,n,m", [(("N", "N"), 20, 3), (("N", "N"), 20, 20), (("D", "D"), 20, 7),
                                    (("N", "D"), 15, 4), (("D", "N"), 15, 14), (("P", "P"), 16, 5)])
@pytest.mark.parametrize("uinit", ["halfstep", "as_given"])
def test_single_mode_closed_form(bc, n, m, uinit):
    """A Table 1 mode oscillates at the discrete frequency theta (written out by hand)."""
    d = _desc((n,), [bc], cfl=0.5)
    p0, k = _mode(n, bc, m)
    theta = np.arccos(1.0 - (C0 * k * d.dt) ** 2 / 2.0)
    p, pm = p0, order2.init_prev(d, p0, uinit)
    for step in range(1, 60):
        p, pm = order2.step(d, p, pm)
        if uinit == "halfstep":
            ref = np.cos(step * theta) * p0
        else:
            ref = np.cos((step + 0.5) * theta) / np.cos(theta / 2) * p0
        assert np.abs(p - ref).max() < 1e-10


def test_separable_mode_2d():
    """cos(kx x) sin(ky y) on NN x DD: theta from kx^2 + ky^2."""
    d = _desc((12, 10), [("N", "N"), ("D", "D")], cfl=0.4)
    fx, kx = _mode(12, ("N", "N"), 5)
    fy, ky = _mode(10, ("D", "D"), 3)
    p0 = np.outer(fx, fy)
    theta = np.arccos(1.0 - (C0 * d.dt) ** 2 * (kx ** 2 + ky ** 2) / 2.0)
    p, pm = order2.run(d, p0, order2.init_prev(d, p0), 40)
    assert np.abs(p - np.cos(40 * theta) * p0).max() < 1e-10


def test_run_returns_last_two_levels():
    d = _desc((8, 6), [("N", "D"), ("P", "P")])
    p0 = _field(d, 5)
    pm0 = order2.init_prev(d, p0)
    p, pm = order2.run(d, p0, pm0, 7)
    q, qm = order2.run(d, p0, pm0, 6)
    assert np.array_equal(pm, q)
    p1, _ = order2.step(d, q, qm)
    assert np.array_equal(p, p1)


@pytest.mark.parametrize("mistake", ["no_c0sq", "sign", "start"])
def test_planted_mistakes_are_caught(monkeypatch, mistake):
    """A dropped c0^2, a flipped sign or the wrong start breaks the closed form."""
    d = _desc((20,), [("N", "N")], cfl=0.5)
    p0, k = _mode(20, ("N", "N"), 3)
    theta = np.arccos(1.0 - (C0 * k * d.dt) ** 2 / 2.0)
    real_lap = order2.laplacian
    if mistake == "no_c0sq":
        monkeypatch.setattr(order2, "laplacian", lambda desc, p: real_lap(desc, p) / desc.c0 ** 2)
    elif mistake == "sign":
        monkeypatch.setattr(order2, "laplacian", lambda desc, p: -real_lap(desc, p))
    pm = p0.copy() if mistake == "start" else order2.init_prev(d, p0)
    p, _ = order2.run(d, p0, pm, 30)
    assert np.abs(p - np.cos(30 * theta) * p0).max() > 1e-3
