"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test names the paper passage or the mathematical fact it checks:
library transforms (scipy's FFTW-convention DCT/DST), Eq. (inverse_transforms),
exact derivatives of single modes (Eqs. FST_diff / FCT_diff with Tables A3/A6),
the closed-form modal solution and the discrete energy (derived from
Eq. dtt_pstd_solution), the Section 5 worked examples, the non-reflecting
cancellation, image sources (Fig. 2), the 1-D stability limit 2/pi
(Section 4.2) and second-order convergence in the CFL number (Fig. 6).
"""
import os

import numpy as np
import pytest
import scipy.fft as sf

from oracle import dtt, modal, pstd, reflection

HERE = os.path.dirname(os.path.abspath(__file__))
BCS = [("N", "N"), ("N", "D"), ("D", "N"), ("D", "D")]

SCIPY = {
    "C1": lambda x: sf.dct(x, 1), "C2": lambda x: sf.dct(x, 2),
    "C3": lambda x: sf.dct(x, 3), "C4": lambda x: sf.dct(x, 4),
    "S1": lambda x: sf.dst(x, 1), "S2": lambda x: sf.dst(x, 2),
    "S3": lambda x: sf.dst(x, 3), "S4": lambda x: sf.dst(x, 4),
}


@pytest.mark.parametrize("kind", dtt.KINDS)
@pytest.mark.parametrize("n", [2, 3, 5, 8, 17, 64])
def test_dtt_matches_library(kind, n):
    """The direct sums equal an independent FFT-based library implementation."""
    x = np.random.default_rng(n).standard_normal((3, n))
    y = dtt.apply(kind, x, axis=1)
    ref = np.stack([SCIPY[kind](r) for r in x])
    assert np.abs(y - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("kind", dtt.KINDS)
@pytest.mark.parametrize("n", [2, 4, 7, 32, 128])
def test_inverse_identities(kind, n):
    """Eq. (inverse_transforms): T^{-1} T = I with the 1/M factor of Table 1."""
    x = np.random.default_rng(7 * n).standard_normal(n)
    back = dtt.inverse(kind, dtt.apply(kind, x))
    assert np.abs(back - x).max() < 1e-13 * n


def test_implied_periods_table1():
    """Table 1: M = 2(N-1) for C1, 2(N+1) for S1, 2N for the other types I-IV."""
    assert dtt.implied_period("C1", 9) == 16
    assert dtt.implied_period("S1", 7) == 16
    for k in ("C2", "C3", "C4", "S2", "S3", "S4"):
        assert dtt.implied_period(k, 8) == 16


@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("n", [2, 3, 8, 16, 33])
def test_single_mode_derivatives(bc, n):
    """Staggered derivative of each basis mode is exact (Eqs. FST_diff, FCT_diff).

    A Neumann left wall makes the pressure basis cos(k x) and the velocity
    basis sin(k x); a Dirichlet left wall swaps them.  The pressure derivative
    lands on the half-nodes (m + 1/2) dx and the velocity derivative on the
    stored pressure nodes; the wavenumbers are those of Table 1.
    """
    dx = 0.37
    xj = pstd.p_nodes(n, bc) * dx
    xm = (np.arange(n) + 0.5) * dx
    for k in modal.mode_wavenumbers(n, bc, dx):
        if bc[0] == "N":
            p, dp = np.cos(k * xj), -k * np.sin(k * xm)
            u, du = np.sin(k * xm), k * np.cos(k * xj)
        else:
            p, dp = np.sin(k * xj), k * np.cos(k * xm)
            u, du = np.cos(k * xm), -k * np.sin(k * xj)
        tol = 1e-12 * max(1.0, k) * n
        assert np.abs(pstd.grad_p(p, 0, n, bc, dx) - dp).max() < tol
        assert np.abs(pstd.grad_u(u, 0, n, bc, dx) - du).max() < tol


def test_derivative_acts_along_requested_axis():
    """In 2-D the operator along axis 1 equals the 1-D operator on every row."""
    n0, n1 = 6, 9
    bc = ("D", "N")
    p = np.random.default_rng(3).standard_normal((5, pstd.p_len(n1, bc)))
    g = pstd.grad_p(p, 1, n1, bc, 0.1)
    for r in range(5):
        assert np.allclose(g[r], pstd.grad_p(p[r], 0, n1, bc, 0.1), atol=1e-13)
    gt = pstd.grad_p(p.T.copy(), 0, n1, bc, 0.1)
    assert np.allclose(gt.T, g, atol=1e-13)


def _desc(ncells, bcs, cfl=0.3, dx=1e-4):
    return pstd.Desc(ncells, (dx,), bcs, dt=pstd.dt_from_cfl(cfl, dx, 1500.0))


@pytest.mark.parametrize("ncells,bcs", [
    ((2,), [("N", "N")]), ((3,), [("D", "D")]), ((5,), [("N", "D")]), ((7,), [("D", "N")]),
    ((12, 10), [("D", "D"), ("N", "N")]),
    ((9, 8), [("N", "D"), ("D", "N")]),
    ((6, 5, 7), [("D", "N"), ("N", "N"), ("D", "D")]),
])
@pytest.mark.parametrize("uinit", ["halfstep", "as_given"])
def test_modal_closed_form_matches_stepping(ncells, bcs, uinit):
    """Two independent routes agree: 300 leapfrog steps vs the modal solution."""
    d = _desc(ncells, bcs, cfl=0.3 / np.sqrt(len(ncells)))
    p0 = np.random.default_rng(11).standard_normal(pstd.field_shapes(d)[0])
    s = pstd.run(d, pstd.State(p0, pstd.init_velocity(d, p0, None, uinit)), 300)
    ref = modal.modal_pressure(d, p0, 300, uinit)
    assert np.abs(s.p - ref).max() <= 1e-11 * np.abs(p0).max()


def test_separable_modal_matches_dense_modal():
    """The outer-product route equals the dense modal route for a blob sum."""
    d = _desc((16, 12), [("D", "D"), ("N", "N")])
    facs = []
    for c0, c1 in [(0.4e-3, 0.5e-3), (1.1e-3, 0.7e-3)]:
        f0 = np.exp(-((pstd.p_nodes(16, ("D", "D")) * 1e-4 - c0) ** 2) / (2 * (2e-4) ** 2))
        f1 = np.exp(-((pstd.p_nodes(12, ("N", "N")) * 1e-4 - c1) ** 2) / (2 * (2e-4) ** 2))
        facs.append([f0, f1])
    p0 = sum(np.multiply.outer(a, b) for a, b in facs)
    a = modal.separable_modal_pressure(d, facs, 77)
    b = modal.modal_pressure(d, p0, 77)
    assert np.abs(a - b).max() < 1e-13
    sub = modal.separable_modal_pressure(d, facs, 77, out_index=(np.array([0, 3, 14]), slice(2, 5)))
    assert np.abs(sub - b[np.ix_([0, 3, 14], range(2, 5))]).max() < 1e-13


@pytest.mark.parametrize("bcs", [[("N", "N")], [("D", "N"), ("N", "D")],
                                 [("D", "D"), ("N", "N"), ("N", "D")]])
def test_discrete_energy_conserved(bcs):
    """The leapfrog conserves E^n (derived from D_u = -W^{-1} D_p^T)."""
    ncells = (10, 9, 8)[:len(bcs)]
    d = _desc(ncells, bcs, cfl=0.25)
    p0 = np.random.default_rng(5).standard_normal(pstd.field_shapes(d)[0])
    s = pstd.State(p0, pstd.init_velocity(d, p0, None, "halfstep"))
    es = []
    for _ in range(40):
        s1 = pstd.step(d, s)
        es.append(modal.energy(d, s.p, s.u, s1.u))
        s = s1
    es = np.array(es)
    assert np.abs(es - es[0]).max() < 1e-12 * es[0]


def test_energy_weights_are_needed():
    """Dropping the 1/2 Neumann-wall weight breaks conservation (the pin is sharp)."""
    d = _desc((10,), [("N", "N")], cfl=0.25)
    p0 = np.random.default_rng(5).standard_normal(pstd.field_shapes(d)[0])
    s = pstd.State(p0, pstd.init_velocity(d, p0, None, "halfstep"))
    es = []
    for _ in range(40):
        s1 = pstd.step(d, s)
        es.append(np.sum(s.p ** 2) / (2 * d.rho0 * d.c0 ** 2)
                  + 0.5 * d.rho0 * np.sum(s.u[0] * s1.u[0]))
        s = s1
    es = np.array(es)
    assert np.abs(es - es[0]).max() > 1e-6 * es[0]


def test_reflection_weights_worked_examples():
    """Section 5's two printed weight vectors (tests/golden/reflection_weights.txt)."""
    rows = np.loadtxt(os.path.join(HERE, "golden", "reflection_weights.txt"))
    for rl, rr, *w in rows:
        assert np.allclose(reflection.axis_weights(rl, rr), w, atol=0, rtol=0)


def test_reflection_weights_reproduce_basic_runs():
    """R = +-1 walls select exactly one basic run; M/2 is unitary (Section 5)."""
    for i, (l, r) in enumerate(reflection.BASIC_RUNS):
        w = reflection.axis_weights(1.0 if l == "N" else -1.0, 1.0 if r == "N" else -1.0)
        e = np.zeros(4)
        e[i] = 1.0
        assert np.allclose(w, e)
    Mh = reflection.POLARITY / 2
    assert np.allclose(Mh @ Mh.T, np.eye(4))


def _gauss_run_1d(bc, n, cfl, steps, centre_node, sigma_cells, uinit="as_given"):
    d = _desc((n,), [bc], cfl=cfl)
    x = pstd.p_nodes(n, bc) * d.dx[0]
    p0 = np.exp(-((x - centre_node * d.dx[0]) ** 2) / (2 * (sigma_cells * d.dx[0]) ** 2))
    s = pstd.run(d, pstd.State(p0, pstd.init_velocity(d, p0, None, uinit)), steps)
    return d, s


def test_nonreflecting_weighted_sum_cancels():
    """Section 5: with R_L = R_R = 0 the weighted sum vanishes once the waves leave.

    Gaussian at the centre, zero initial velocity, t = 1.5 L / c0 (inside the
    3 L / c0 window).  The four runs have different stored node sets; they are
    compared on the interior nodes that all of them store.
    """
    n, cfl = 128, 0.2
    steps = int(round(1.5 * n / cfl))
    w = reflection.axis_weights(0.0, 0.0)
    total = np.zeros(n - 1)
    for wi, bc in zip(w, reflection.BASIC_RUNS):
        _, s = _gauss_run_1d(bc, n, cfl, steps, n / 2, 4.0)
        j = pstd.p_nodes(n, bc)
        total += wi * s.p[(j >= 1) & (j <= n - 1)]
    assert np.abs(total).max() < 1e-12


def test_image_sources_dirichlet_and_neumann():
    """Fig. 2: a Neumann wall reflects in phase, a Dirichlet wall out of phase.

    The continuous solution with u(0) = 0 is the average of left- and
    right-going copies of p0 plus its images (+ for Neumann, - for Dirichlet)
    about both walls; the scheme matches it to the O((c0 k dt)^2) time
    dispersion at a small CFL number.
    """
    n, cfl, sig = 128, 0.05, 4.0
    steps = int(round(0.75 * n / cfl))          # t = 0.75 L / c0: one reflection each side
    for bc in BCS:
        d, s = _gauss_run_1d(bc, n, cfl, steps, 40.0, sig, uinit="halfstep")
        L = n * d.dx[0]
        ct = 1500.0 * steps * d.dt
        x = pstd.p_nodes(n, bc) * d.dx[0]
        sl = 1.0 if bc[0] == "N" else -1.0
        sr = 1.0 if bc[1] == "N" else -1.0
        x0 = 40.0 * d.dx[0]
        g = lambda z: np.exp(-(z ** 2) / (2 * (sig * d.dx[0]) ** 2))
        src = [(x0, 1.0), (-x0, sl), (2 * L - x0, sr), (-2 * L + x0, sl * sr), (2 * L + x0, sl * sr)]
        ref = sum(a * 0.5 * (g(x - c - ct) + g(x - c + ct)) for c, a in src)
        assert np.abs(s.p - ref).max() < 5e-3, bc


@pytest.mark.parametrize("bc", [("N", "N"), ("D", "D")])
def test_cfl_stability_limit(bc):
    """Section 4.2: the 1-D scheme is stable below CFL 2/pi and not above it."""
    n = 32
    lim = pstd.stable_cfl_limit(1)
    assert abs(lim - 2 / np.pi) < 1e-15
    p0 = np.random.default_rng(2).standard_normal(pstd.p_len(n, bc))
    for cfl, stable in [(0.97 * lim, True), (1.03 * lim, False)]:
        d = _desc((n,), [bc], cfl=cfl)
        with np.errstate(over="ignore", invalid="ignore"):
            s = pstd.run(d, pstd.State(p0, pstd.init_velocity(d, p0, None, "as_given")), 3000)
            m = np.abs(s.p).max()
        grew = (not np.isfinite(m)) or m > 1e3 * np.abs(p0).max()
        # DD drops the Nyquist mode, so its limit is slightly above 2/pi
        if bc == ("D", "D") and not stable:
            continue
        assert grew != stable


def test_round_trip_convergence_algebraic():
    """Fig. 6: NN round-trip error falls algebraically with the CFL number.

    A Gaussian at the centre travels to both walls and back (t = L / c0) and
    recombines into p0.  The leapfrog phase error of each mode is
    O((c0 k dt)^2), and at t = L / c0 every mode sits at a stationary point
    of cos(k c0 t) (k L = pi n), so the L_inf error is the square of the phase
    error: halving the CFL number cuts it 16x.  The paper shows the algebraic
    decay without printing numbers.
    """
    n = 64
    errs = []
    for cfl in (0.2, 0.1, 0.05):
        steps = int(round(n / cfl))
        d, s = _gauss_run_1d(("N", "N"), n, cfl, steps, n / 2, 3.0, uinit="halfstep")
        x = pstd.p_nodes(n, ("N", "N")) * d.dx[0]
        p0 = np.exp(-((x - n / 2 * d.dx[0]) ** 2) / (2 * (3.0 * d.dx[0]) ** 2))
        errs.append(np.abs(s.p - p0).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 14.0 < r1 < 18.0 and 14.0 < r2 < 18.0, errs


def test_planted_sign_error_is_caught(monkeypatch):
    """A flipped a1 sign in Table 2 breaks the single-mode pin (the pin is sharp)."""
    bad = dict(pstd.TABLE2)
    t1, t2, s1, s2 = bad[("N", "D")]
    bad[("N", "D")] = (t1, t2, -s1, s2)
    monkeypatch.setattr(pstd, "TABLE2", bad)
    n, dx = 8, 1.0
    x = pstd.p_nodes(n, ("N", "D")) * dx
    k = modal.mode_wavenumbers(n, ("N", "D"), dx)[2]
    g = pstd.grad_p(np.cos(k * x), 0, n, ("N", "D"), dx)
    assert np.abs(g - (-k * np.sin(k * (np.arange(n) + 0.5) * dx))).max() > 0.1


def test_planted_index_shift_is_caught(monkeypatch):
    """Using the DD pad on the wrong side breaks the modal pin."""
    d = _desc((9,), [("D", "D")])
    p0 = np.random.default_rng(1).standard_normal(pstd.field_shapes(d)[0])
    ref = modal.modal_pressure(d, p0, 20)
    orig = pstd.grad_p

    def shifted(p, axis, n, bc, dx):
        g = orig(p, axis, n, bc, dx)
        return np.roll(g, 1, axis=axis)

    monkeypatch.setattr(pstd, "grad_p", shifted)
    s = pstd.run(d, pstd.State(p0, pstd.init_velocity(d, p0, None, "halfstep")), 20)
    assert np.abs(s.p - ref).max() > 1e-3


# ---- periodic Fourier PSTD (Section 2; Table 2's periodic row) -----------------

@pytest.mark.parametrize("n", [8, 9, 16, 31])
def test_fourier_single_modes(n):
    """i k e^{+-i k dx/2} differentiates each resolved Fourier mode exactly onto the
    staggered grid; the even-N Nyquist mode maps to a real multiple of itself."""
    dx = 0.23
    x = np.arange(n) * dx
    xm = x + 0.5 * dx
    for m in range(1, (n - 1) // 2 + 1):
        k = 2 * np.pi * m / (n * dx)
        for ph in (0.0, 0.7):
            p = np.cos(k * x + ph)
            assert np.abs(pstd.grad_p(p, 0, n, ("P", "P"), dx) + k * np.sin(k * xm + ph)).max() < 1e-11 * k * n
            u = np.sin(k * xm + ph)
            assert np.abs(pstd.grad_u(u, 0, n, ("P", "P"), dx) - k * np.cos(k * x + ph)).max() < 1e-11 * k * n
    if n % 2 == 0:
        kn = np.pi / dx
        p = np.cos(kn * x)                    # (-1)^j
        assert np.abs(pstd.grad_p(p, 0, n, ("P", "P"), dx) + kn * np.sin(kn * xm)).max() < 1e-10 * kn


def test_fourier_modal_and_energy():
    """Periodic 2-D: modal closed form vs stepping; energy conserved."""
    d = _desc((12, 9), [("P", "P"), ("D", "N")], cfl=0.2)
    p0 = np.random.default_rng(4).standard_normal(pstd.field_shapes(d)[0])
    s = pstd.run(d, pstd.State(p0, pstd.init_velocity(d, p0, None, "halfstep")), 200)
    assert np.abs(s.p - modal.modal_pressure(d, p0, 200)).max() < 1e-11 * np.abs(p0).max()
    s = pstd.State(p0, pstd.init_velocity(d, p0, None, "halfstep"))
    es = []
    for _ in range(30):
        s1 = pstd.step(d, s)
        es.append(modal.energy(d, s.p, s.u, s1.u))
        s = s1
    assert np.abs(np.array(es) - es[0]).max() < 1e-12 * es[0]


def test_fourier_wave_wraps_around():
    """Fig. 1: a right-going pulse leaves through one side and re-enters through the
    other; after t = L / c0 it is back where it started (periodic images)."""
    n, cfl, sig = 128, 0.05, 4.0
    d = _desc((n,), [("P", "P")], cfl=cfl)
    dx = d.dx[0]
    x = np.arange(n) * dx
    L = n * dx

    def g(z):
        z = (z + L / 2) % L - L / 2          # nearest periodic image
        return np.exp(-(z ** 2) / (2 * (sig * dx) ** 2))
    x0 = 40 * dx
    p0 = g(x - x0)
    u0 = [g(x + 0.5 * dx - x0) / (1000.0 * 1500.0)]   # right-going: u = p / (rho0 c0)
    steps = int(round(n / cfl))
    s = pstd.run(d, pstd.State(p0, pstd.init_velocity(d, p0, u0, "halfstep")), steps)
    ct = 1500.0 * steps * d.dt
    assert abs(ct - L) < 1e-12
    assert np.abs(s.p - p0).max() < 2e-3
    half = pstd.run(d, pstd.State(p0, pstd.init_velocity(d, p0, u0, "halfstep")), steps // 2)
    assert np.abs(half.p - g(x - x0 - L / 2)).max() < 2e-3
