"""Pins of the oracle's types V-VIII (groups III and IV of Table 1): the
transforms themselves and the PSTD step on an axis with a mid-cell wall.

The transforms are built from one sum over a period of the symmetric-periodic
sequence (oracle/dtt.py).  They are pinned to:
* the FFTW types I-IV, which the same sum must reproduce (those are pinned to
  scipy in test_oracle.py);
* Eq. (inverse_transforms) for j = 5..8 and the implied periods of Table 1;
* the DFT (numpy's FFT) of the explicitly built extension, sample by sample.

The stepper with a right wall at x = (N - 1/2) dx ("Nm", "Dm") is pinned to:
* exact staggered derivatives of single modes (the group III / IV wavenumbers);
* the modal closed form against stepping, and discrete energy conservation;
* image sources about a wall at (N - 1/2) dx (Fig. 2's construction), with a
  planted wall position off by half a cell failing.
"""
import numpy as np
import pytest

from oracle import dtt, dtt_ops, modal, order2, pstd

DX = 1e-4
MID = [("N", "Nm"), ("N", "Dm"), ("D", "Nm"), ("D", "Dm")]


def _desc(ncells, bcs, cfl=0.3):
    return pstd.Desc(ncells, (DX,), bcs, dt=pstd.dt_from_cfl(cfl, DX, 1500.0))


@pytest.mark.parametrize("kind", dtt.KINDS)
@pytest.mark.parametrize("n", [2, 3, 6, 11])
def test_period_sum_reproduces_fftw_types(kind, n):
    assert np.abs(dtt.sps_matrix(dtt.SPS[kind], n) - dtt.dtt_matrix(kind, n)).max() < 1e-12
    assert dtt.sps_geometry(dtt.SPS[kind], n)[2] == dtt.implied_period(kind, n)


@pytest.mark.parametrize("kind", dtt.KINDS_III_IV)
@pytest.mark.parametrize("n", [1, 2, 5, 12, 31])
def test_inverse_identities_types_v_viii(kind, n):
    """Eq. (inverse_transforms): T5, T8 invert themselves, T6 and T7 each other."""
    x = np.random.default_rng(n).standard_normal(n)
    assert np.abs(dtt.inverse(kind, dtt.apply(kind, x)) - x).max() < 1e-13 * n


def test_implied_periods_table1_groups_iii_iv():
    """Table 1: M = 2N - 1 for C5, C6, C7, S8 and 2N + 1 for C8, S5, S6, S7."""
    for kind in dtt.KINDS_III_IV:
        M = dtt.sps_geometry(dtt.SPS[kind], 7)[2]
        assert M == (13 if kind in ("C5", "C6", "C7", "S8") else 15), kind
        assert M == dtt.implied_period(kind, 7)


@pytest.mark.parametrize("kind", dtt.KINDS_III_IV + dtt.KINDS)
def test_transform_is_dft_of_the_extension(kind):
    """Y_k = the DFT of the SPS at wavenumber index nu_k (cosine or -sine part),
    from numpy's FFT of the extension written out over two periods."""
    n = 7
    sym = dtt.SPS[kind]
    x = np.random.default_rng(1).standard_normal(n)
    t, _, M, nu = dtt.sps_geometry(sym, n)
    # reflections alone: x(-t) = sl x(t), x(2R - t) = sr x(t); (anti)periodic with
    # period 2R (sign sl * sr); sample the half-integer lattice over [0, 2M)
    sl, sr = (-1.0 if sym[1] == "A" else 1.0), (-1.0 if sym[3] == "A" else 1.0)
    per = sl * sr
    lattice = np.zeros(4 * M)
    for tj, xj in zip(t, x):
        for m in range(-3, 4):
            for pos, sg in [(tj, 1.0), (-tj, sl)]:
                p = pos + m * M
                if 0 <= p < 2 * M:
                    lattice[int(round(2 * p))] = sg * xj * per ** abs(m)
    # DFT over two periods on the half-integer lattice (4M points, spacing 1/2)
    F = np.fft.fft(lattice)                       # bin b <-> wavenumber index b / 2
    Y = dtt.apply(kind, x)
    for k, v in enumerate(nu):
        b = int(round(2 * v))
        z = F[b] / 2.0                            # two periods summed
        want = -z.imag if sym[1] == "A" else z.real
        assert abs(Y[k] - want) < 1e-10, (kind, k)


@pytest.mark.parametrize("bc", MID)
@pytest.mark.parametrize("n", [6, 9])
def test_single_mode_staggered_derivatives(bc, n):
    """Each mode of the pressure SPS maps to its exact derivative on the half-nodes
    (and back): wavenumbers 2 pi nu / ((2N - 1) dx)."""
    sym_p, sym_u = pstd.symmetries(bc)
    M = 2 * n - 1
    xp = pstd.p_nodes(n, bc) * DX
    xu = (np.arange(pstd.u_len(n, bc)) + 0.5) * DX
    for nv in dtt_ops.wavenumber_index(sym_p, n):
        k = 2 * np.pi * nv / (M * DX)
        sine = sym_p[1] == "A"
        f = np.sin(k * xp) if sine else np.cos(k * xp)
        want = k * np.cos(k * xu) if sine else -k * np.sin(k * xu)
        g = pstd.grad_p(f, 0, n, bc, DX)
        assert np.abs(g - want).max() < 1e-9 * np.pi / DX, (bc, nv)
    for nv in dtt_ops.wavenumber_index(sym_u, n):
        k = 2 * np.pi * nv / (M * DX)
        sine = sym_u[1] == "A"
        f = np.sin(k * xu) if sine else np.cos(k * xu)
        want = k * np.cos(k * xp) if sine else -k * np.sin(k * xp)
        g = pstd.grad_u(f, 0, n, bc, DX)
        assert np.abs(g - want).max() < 1e-9 * np.pi / DX, (bc, nv)


def test_field_shapes_mid_walls():
    d = _desc((7, 5), [("N", "Nm"), ("D", "Dm")])
    assert pstd.field_shapes(d) == [(7, 4), (6, 4), (7, 5)]


@pytest.mark.parametrize("ncells,bcs", [((9,), [("N", "Nm")]), ((9,), [("D", "Dm")]),
                                        ((10, 7), [("N", "Dm"), ("D", "N")]),
                                        ((6, 7, 5), [("D", "Nm"), ("N", "N"), ("P", "P")])])
@pytest.mark.parametrize("uinit", ["halfstep", "as_given"])
def test_modal_closed_form_matches_stepping(ncells, bcs, uinit):
    d = _desc(ncells, bcs, cfl=0.3 / np.sqrt(len(ncells)))
    p0 = np.random.default_rng(11).standard_normal(pstd.field_shapes(d)[0])
    s = pstd.run(d, pstd.State(p0, pstd.init_velocity(d, p0, None, uinit)), 200)
    ref = modal.modal_pressure(d, p0, 200, uinit)
    assert np.abs(s.p - ref).max() <= 1e-11 * np.abs(p0).max()


@pytest.mark.parametrize("bcs", [[("N", "Nm")], [("D", "Dm")], [("N", "Dm"), ("D", "Nm")]])
def test_discrete_energy_conserved(bcs):
    """E^n is conserved with the 1/2 weight on a Neumann node wall and on the
    velocity half-node a Dirichlet mid-cell wall passes through."""
    ncells = (10, 9)[:len(bcs)]
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


def _image_reference(bc, n, x, ct, x0, sig, wall):
    g = lambda z: np.exp(-(z ** 2) / (2 * (sig * DX) ** 2))
    sl = 1.0 if bc[0] == "N" else -1.0
    sr = 1.0 if bc[1] == "Nm" else -1.0
    src = [(x0, 1.0), (-x0, sl), (2 * wall - x0, sr), (-2 * wall + x0, sl * sr), (2 * wall + x0, sl * sr)]
    return sum(a * 0.5 * (g(x - c - ct) + g(x - c + ct)) for c, a in src)


@pytest.mark.parametrize("bc", MID)
def test_image_sources_about_a_mid_cell_wall(bc):
    """A Gaussian reflects from the right wall as from one at (N - 1/2) dx:
    in phase for Neumann, out of phase for Dirichlet (Fig. 2's images)."""
    n, cfl, sig = 128, 0.05, 4.0
    d = _desc((n,), [bc], cfl=cfl)
    steps = int(round(0.75 * n / cfl))
    x = pstd.p_nodes(n, bc) * DX
    x0 = 88.0 * DX
    p0 = np.exp(-((x - x0) ** 2) / (2 * (sig * DX) ** 2))
    s = pstd.run(d, pstd.State(p0, pstd.init_velocity(d, p0, None, "halfstep")), steps)
    ct = 1500.0 * steps * d.dt
    ref = _image_reference(bc, n, x, ct, x0, sig, (n - 0.5) * DX)
    assert np.abs(s.p - ref).max() < 5e-3, bc
    # the same images about a wall at N dx (a planted half-cell error) do not match
    wrong = _image_reference(bc, n, x, ct, x0, sig, n * DX)
    assert np.abs(s.p - wrong).max() > 5e-2, bc


@pytest.mark.parametrize("bc", MID)
def test_second_order_form_with_mid_walls(bc):
    d = _desc((12, 6), [bc, ("N", "D")], cfl=0.2)
    p0 = np.random.default_rng(2).standard_normal(pstd.field_shapes(d)[0])
    s = pstd.State(p0, pstd.init_velocity(d, p0, None, "halfstep"))
    p, pm = p0, order2.init_prev(d, p0)
    for _ in range(20):
        s = pstd.step(d, s)
        p, pm = order2.step(d, p, pm)
    assert np.abs(p - s.p).max() < 1e-11 * np.abs(p0).max()
