"""Pins of the DTT differentiation and interpolation oracle (Tables A1, A2,
A4, A5), for the sixteen symmetries of Table 1 (groups I-IV): single modes
map exactly to their derivative / their values on the other grid, and
interpolation after differentiation is the staggered derivative of Table 2."""
import numpy as np
import pytest

from oracle import dtt_ops, pstd

DX = 1e-4


def _mode(sym, nv, n, x):
    k = 2.0 * np.pi * nv / (dtt_ops.period(sym, n) * DX)
    sine = dtt_ops.SYMMETRY[sym][2]
    return (np.sin(k * x) if sine else np.cos(k * x)), k, sine


@pytest.mark.parametrize("sym", sorted(dtt_ops.SYMMETRY))
@pytest.mark.parametrize("n", [6, 9])
def test_single_modes_differentiate_exactly(sym, n):
    for nv in dtt_ops.wavenumber_index(sym, n):
        f, k, sine = _mode(sym, nv, n, dtt_ops.positions(sym, n, DX))
        g, out = dtt_ops.diff(sym, f, n, DX)
        xo = dtt_ops.positions(out, n, DX)
        want = k * np.cos(k * xo) if sine else -k * np.sin(k * xo)
        assert out[0] == sym[0] and out[1] != sym[1] and out[3] != sym[3]
        # rounding leaks into every wavenumber, scaled by up to k_max = pi / dx
        assert np.abs(g - want).max() <= 1e-12 * np.pi / DX, (sym, nv)


@pytest.mark.parametrize("sym", sorted(dtt_ops.SYMMETRY))
@pytest.mark.parametrize("n", [6, 9])
def test_single_modes_interpolate_exactly(sym, n):
    for nv in dtt_ops.wavenumber_index(sym, n):
        f, k, sine = _mode(sym, nv, n, dtt_ops.positions(sym, n, DX))
        g, out = dtt_ops.interp(sym, f, n, DX)
        xo = dtt_ops.positions(out, n, DX)
        want = np.sin(k * xo) if sine else np.cos(k * xo)
        assert out[0] != sym[0] and out[1] == sym[1] and out[3] == sym[3]
        assert np.abs(g - want).max() <= 1e-12, (sym, nv)


@pytest.mark.parametrize("bc,sym", [(("N", "N"), "WSWS"), (("N", "D"), "WSWA"),
                                    (("D", "N"), "WAWS"), (("D", "D"), "WAWA")])
def test_interpolated_derivative_is_the_staggered_derivative(bc, sym):
    """Table A3/A6's derivative onto the staggered grid equals differentiation
    (Table A1/A4) followed by interpolation (Table A2/A5)."""
    n = 11
    # a random combination of the symmetry's modes below Nyquist: plain
    # differentiation on the nodes loses the Nyquist mode of WSWS (its
    # derivative vanishes at every node), the staggered derivative keeps it
    x = dtt_ops.positions(sym, n, DX)
    sine = dtt_ops.SYMMETRY[sym][2]
    rng = np.random.default_rng(3)
    p = np.zeros(len(x))
    for nv in dtt_ops.wavenumber_index(sym, n):
        if nv < n:
            k = 2.0 * np.pi * nv / (2 * n * DX)
            p += rng.standard_normal() * (np.sin(k * x) if sine else np.cos(k * x))
    d, s1 = dtt_ops.diff(sym, p, n, DX)
    g, s2 = dtt_ops.interp(s1, d, n, DX)
    ref = pstd.grad_p(p, 0, n, bc, DX)
    assert s2 == dtt_ops.interp_symmetry(dtt_ops.diff_symmetry(sym))
    np.testing.assert_allclose(g, ref, atol=1e-9 * np.abs(ref).max())


def test_planted_errors_are_caught():
    """A sign or an index shift in the bookkeeping breaks the mode pins."""
    n, sym = 8, "HSHS"
    nv = 3
    f, k, _ = _mode(sym, nv, n, dtt_ops.positions(sym, n, DX))
    g, out = dtt_ops.interp(sym, f, n, DX)
    xo = dtt_ops.positions(out, n, DX)
    shifted = np.cos(k * (xo + DX / 2))            # a half-cell offset error
    assert np.abs(g - shifted).max() > 1e-2
    d, out = dtt_ops.diff(sym, f, n, DX)
    flipped = k * np.sin(k * dtt_ops.positions(out, n, DX))   # a sign error
    assert np.abs(d - flipped).max() > 1e-2 * k
