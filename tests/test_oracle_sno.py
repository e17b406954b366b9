"""Pins of the spectral-neural-operator oracle (oracle/sno.py).

* Every parameter gradient against central finite differences of the loss.
* A one-layer linear network whose mode weights are the discrete modal
  propagator cos(n Omega dt) reproduces the PSTD solution exactly for inputs
  that live in the retained modes (the basis and transform conventions are
  those of Table 2 / Eq. inverse_transforms).
"""
import numpy as np
import pytest

from oracle import modal, pstd, sno


def _setup(C=3, K=3, L=2, nx=8, ny=7, seed=0):
    bcx, bcy = ("N", "N"), ("D", "D")
    Tx, Ix = sno.basis(nx, bcx, K)
    Ty, Iy = sno.basis(ny, bcy, K)
    p = sno.init_params(C, K, L, seed)
    rng = np.random.default_rng(seed + 1)
    for k in p:
        p[k] = p[k] + 0.1 * rng.standard_normal(p[k].shape)
    lpx, lpy = Tx.shape[1], Ty.shape[1]
    x = rng.standard_normal((2, lpx, lpy))
    y = rng.standard_normal((2, lpx, lpy))
    return p, x, y, (Tx, Ix, Ty, Iy)


def test_basis_inverts_on_retained_modes():
    Tx, Ix = sno.basis(16, ("N", "D"), 5)
    assert np.allclose(Tx @ Ix, np.eye(5), atol=1e-12)


@pytest.mark.parametrize("L", [1, 2])
def test_gradients_match_finite_differences(L):
    p, x, y, mats = _setup(L=L)
    loss, g = sno.loss_and_grads(p, x, y, *mats, L)
    rng = np.random.default_rng(3)
    h = 1e-6
    for name, val in p.items():
        for _ in range(4):
            idx = tuple(rng.integers(0, s) for s in val.shape)
            old = val[idx]
            val[idx] = old + h
            lp, _ = sno.loss_and_grads(p, x, y, *mats, L)
            val[idx] = old - h
            lm, _ = sno.loss_and_grads(p, x, y, *mats, L)
            val[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[name][idx]) <= 1e-6 * max(1.0, abs(fd)), (name, idx, fd, g[name][idx])


def test_linear_network_reproduces_modal_propagator():
    n, K, steps = 24, 6, 37
    bcx, bcy = ("N", "N"), ("D", "D")
    d = pstd.Desc((n, n), (1e-4,), [bcx, bcy], dt=pstd.dt_from_cfl(0.25, 1e-4, 1500.0))
    Tx, Ix = sno.basis(n, bcx, K)
    Ty, Iy = sno.basis(n, bcy, K)
    # an input made of the first K x K modes only
    rng = np.random.default_rng(0)
    p0 = Ix @ rng.standard_normal((K, K)) @ Iy.T
    kx = modal.mode_wavenumbers(n, bcx, 1e-4)[:K]
    ky = modal.mode_wavenumbers(n, bcy, 1e-4)[:K]
    kk = np.sqrt(kx[:, None] ** 2 + ky[None, :] ** 2)
    om = 2 * np.arcsin(1500.0 * d.dt * kk / 2)
    params = {"w_lift": np.ones(1), "b_lift": np.zeros(1), "w_proj": np.ones(1), "b_proj": np.zeros(1),
              "R0": np.cos(steps * om)[:, :, None, None], "W0": np.zeros((1, 1)), "b0": np.zeros(1)}
    out, _ = sno.forward(params, p0[None], Tx, Ix, Ty, Iy, 1)
    ref = modal.modal_pressure(d, p0, steps)
    assert np.abs(out[0] - ref).max() < 1e-10 * np.abs(ref).max()
