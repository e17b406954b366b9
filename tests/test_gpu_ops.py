"""GPU parity of pstd_apply: plain spectral differentiation and staggered-grid
interpolation (Section 3.3, Tables A1, A2, A4, A5) against the FP64 oracle,
for every field kind on the FFT, convolution and dense routes and on periodic
axes."""
import numpy as np
import pytest
import torch

from oracle import dtt_ops, pstd
from paper_2005_00322_gb300 import inputs

pytestmark = pytest.mark.gpu

DX = 1e-4
KINDS = ("nodes_p", "half_u", "nodes_u", "half_p")


def _symmetry(kind, bc):
    grid = "H" if kind.startswith("half") else "W"
    ppar = kind.endswith("_p")
    par = lambda wall: "S" if ppar == (wall == "N") else "A"
    return grid + par(bc[0]) + grid + par(bc[1])


def _periodic(x, n, op, kind):
    k = pstd.fourier_wavenumbers(n, DX)
    F = pstd.dft_matrix(n)
    if op == "diff":
        m = 1j * k
    else:
        m = np.exp(1j * k * (-0.5 if kind.startswith("half") else 0.5) * DX)
    return ((x @ F.T) * m @ np.conj(F).T / n).real


def _reference(x, axis, n, bc, op, kind):
    xm = np.moveaxis(x.astype(np.float64), axis, -1)
    if bc == ("P", "P"):
        ref = _periodic(xm, n, op, kind)
    else:
        ref = (dtt_ops.diff if op == "diff" else dtt_ops.interp)(_symmetry(kind, bc), xm, n, DX)[0]
    return np.moveaxis(ref, -1, axis)


@pytest.mark.parametrize("ncells,bcs", [
    ((40,), [("N", "N")]), ((40,), [("N", "D")]), ((40,), [("D", "N")]), ((40,), [("D", "D")]),
    ((512,), [("D", "D")]),                                   # FFT length 1024
    ((67,), [("N", "D")]), ((97,), [("D", "D")]),              # convolution route
    ((7,), [("D", "D")]), ((11,), [("N", "N")]),               # dense route
    ((64,), [("P", "P")]), ((9,), [("P", "P")]),               # periodic
    ((6, 48), [("D", "N"), ("D", "D")]), ((33, 20, 5), [("N", "D"), ("D", "D"), ("N", "N")]),
])
@pytest.mark.parametrize("op", ["diff", "interp"])
def test_apply_matches_oracle(ncells, bcs, op):
    from paper_2005_00322_gb300 import Solver
    s = Solver(ncells, DX, bcs, cfl=0.1)
    for axis in range(len(ncells)):
        bc = tuple(bcs[axis])
        for i, kind in enumerate(KINDS):
            okind = s.OUT_KIND[(op, kind)]
            try:
                shape = s.apply_shape(axis, kind)
                s.apply_shape(axis, okind)
            except Exception:
                continue                     # a kind with no stored node on this axis
            x = inputs.random_field(shape, 50 + 7 * axis + i).astype(np.float32)
            y = s.apply(axis, op, torch.tensor(x, device="cuda"), kind).cpu().numpy()
            ref = _reference(x, axis, ncells[axis], bc, op, kind)
            assert y.shape == ref.shape
            err = np.abs(y - ref).max() / np.abs(ref).max()
            assert err < 2e-5, (axis, kind, err)
    assert s.last_launch_count() == 1
    s.close()


def test_apply_of_a_gaussian_is_its_derivative_and_shift():
    """A smooth field (a Gaussian away from the walls) on 256 cells: the plain
    derivative matches the analytic derivative and interpolation matches the
    Gaussian at the half-nodes (spectral accuracy)."""
    from paper_2005_00322_gb300 import Solver
    n, sig, x0 = 256, 8 * DX, 130.3 * DX
    s = Solver((n,), DX, [("N", "D")], cfl=0.1)
    x = np.arange(n) * DX                              # ND stores nodes 0..N-1
    g = np.exp(-((x - x0) ** 2) / (2 * sig ** 2))
    d = s.apply(0, "diff", torch.tensor(g.astype(np.float32), device="cuda"), "nodes_p").cpu().numpy()
    assert d.shape == (n,)                             # nodes 1..N (velocity-like parity)
    xs = np.arange(1, n + 1) * DX
    dref = -(xs - x0) / sig ** 2 * np.exp(-((xs - x0) ** 2) / (2 * sig ** 2))
    assert np.abs(d - dref).max() < 1e-4 * np.abs(dref).max()
    h = s.apply(0, "interp", torch.tensor(g.astype(np.float32), device="cuda"), "nodes_p").cpu().numpy()
    xh = (np.arange(n) + 0.5) * DX
    assert np.abs(h - np.exp(-((xh - x0) ** 2) / (2 * sig ** 2))).max() < 1e-5
    s.close()


def test_apply_rejects_bad_arguments():
    from paper_2005_00322_gb300 import Solver, _abi
    s = Solver((16, 8), DX, [("N", "N"), ("D", "D")], cfl=0.1)
    x = torch.zeros(s.apply_shape(0, "nodes_p"), device="cuda")
    with pytest.raises(ValueError):
        s.apply(0, "diff", x, "half_u")                # wrong shape for the kind
    assert s.lib.pstd_apply(s._h, 2, 0, 0, None, None) == -1
    assert s.lib.pstd_apply(s._h, 0, 5, 0, x.data_ptr(), x.data_ptr()) == -1
    with pytest.raises(_abi.PstdError):
        Solver((1,), DX, [("N", "N")], cfl=0.1).apply_shape(0, "nodes_u")   # no stored node
    s.close()
