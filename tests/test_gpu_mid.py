"""GPU parity for axes whose right wall lies at mid-cell, x = (N - 1/2) dx
(Table 1 groups III and IV, DTT types V-VIII), against the FP64 oracle: the
staggered derivatives, the leapfrog, the second-order form and plain
differentiation / interpolation, on the generic FFT (3- and 5-smooth odd
period M = 2N - 1), convolution and dense routes, plus a long run against
the modal closed form.

Tolerances as for the other walls: one derivative or step within 1e-5
relative L2, a run within 1e-4.
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle import dtt_ops, modal, order2, pstd
from paper_2005_00322_gb300 import inputs

pytestmark = pytest.mark.gpu

DX = 1e-4
MID = [("N", "Nm"), ("N", "Dm"), ("D", "Nm"), ("D", "Dm")]


def rel_l2(a, ref):
    a = np.asarray(a, np.float64)
    ref = np.asarray(ref, np.float64)
    return float(np.linalg.norm(a - ref) / np.linalg.norm(ref))


def make(ncells, bcs, cfl=0.3, uinit="halfstep"):
    from paper_2005_00322_gb300 import Solver
    dt = pstd.dt_from_cfl(cfl, DX, 1500.0)
    s = Solver(ncells, DX, bcs, dt=dt, uinit=uinit)
    od = pstd.Desc(ncells, (DX,), bcs, dt=dt)
    assert s.shapes == pstd.field_shapes(od)
    return s, od


def dev(x):
    return torch.tensor(np.asarray(x, np.float32), device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def f32(x):
    return np.asarray(x, np.float32).astype(np.float64)


CASES = (
    # 1-D, every mid-cell wall pair: M = 25 (radix 5), 27 (radix 3), 15, 19 (dense), 139 (convolution)
    [((n,), [bc]) for bc in MID for n in (13, 14, 8, 10, 70)]
    + [((2,), [("N", "Nm")]), ((2,), [("D", "Dm")])]
    # several CTAs per axis and ragged tails, mixed with node and periodic walls
    + [((41, 37), [("D", "Nm"), ("N", "N")]), ((37, 41), [("N", "D"), ("N", "Dm")]),
       ((122, 9), [("N", "Dm"), ("D", "D")]), ((9, 113), [("P", "P"), ("D", "Nm")]),
       ((14, 13, 8), [("N", "Nm"), ("D", "Dm"), ("D", "N")]),
       ((6, 5, 70), [("D", "N"), ("N", "Nm"), ("D", "Dm")])]
)


@pytest.mark.parametrize("ncells,bcs", CASES)
def test_grad_and_step_match_oracle(ncells, bcs):
    s, od = make(ncells, bcs, cfl=0.3 / np.sqrt(len(ncells)))
    for ax in range(len(ncells)):
        p = f32(inputs.random_field(s.shapes[0], 10 + ax))
        g = s.grad(ax, 0, dev(p))
        assert rel_l2(host(g), pstd.grad_p_axis(od, p, ax)) < 1e-5, (ax, "p->u")
        u = f32(inputs.random_field(s.shapes[1 + ax], 20 + ax))
        g = s.grad(ax, 1, dev(u))
        assert rel_l2(host(g), pstd.grad_u_axis(od, u, ax)) < 1e-5, (ax, "u->p")
    p0 = f32(inputs.random_field(s.shapes[0], 3))
    us0 = [f32(inputs.random_field(sh, 30 + i)) * 1e-6 for i, sh in enumerate(s.shapes[1:])]
    p, us = dev(p0), [dev(u) for u in us0]
    s.step(p, us)
    ref = pstd.step(od, pstd.State(p0, us0))
    assert rel_l2(host(p), ref.p) < 1e-5
    for i in range(len(ncells)):
        assert rel_l2(host(us[i]), ref.u[i]) < 1e-5
    s.close()


@pytest.mark.parametrize("ncells,bcs", CASES[::2])
@pytest.mark.parametrize("uinit", ["halfstep", "as_given"])
def test_short_run_matches_oracle(ncells, bcs, uinit):
    """init_velocity + 40 steps (a graph-replayed block of 32 plus a direct tail)."""
    s, od = make(ncells, bcs, cfl=0.3 / np.sqrt(len(ncells)), uinit=uinit)
    p0 = f32(inputs.random_field(s.shapes[0], 4))
    p, us = dev(p0), [torch.zeros(sh, device="cuda") for sh in s.shapes[1:]]
    s.init_velocity(p, us)
    s.run(p, us, 40)
    ref = pstd.run(od, pstd.State(p0, pstd.init_velocity(od, p0, None, uinit)), 40)
    assert rel_l2(host(p), ref.p) < 1e-4
    for i in range(len(ncells)):
        assert rel_l2(host(us[i]), ref.u[i]) < 1e-4
    s.close()


@pytest.mark.parametrize("ncells,bcs", CASES[1::2])
def test_second_order_form_matches_oracle(ncells, bcs):
    s, od = make(ncells, bcs, cfl=0.3 / np.sqrt(len(ncells)))
    p0 = f32(inputs.random_field(s.shapes[0], 5))
    p, pm = dev(p0), torch.empty(s.shapes[0], device="cuda")
    s.init_prev(p, pm)
    s.run2(p, pm, 40)
    ref, _ = order2.run(od, p0, order2.init_prev(od, p0), 40)
    assert rel_l2(host(p), ref) < 1e-4
    s.close()


KIND_SYM = {"nodes_p": lambda sp, su: sp, "half_u": lambda sp, su: su,
            "nodes_u": lambda sp, su: dtt_ops.diff_symmetry(sp),
            "half_p": lambda sp, su: dtt_ops.interp_symmetry(sp)}


@pytest.mark.parametrize("bc", MID)
@pytest.mark.parametrize("n", [13, 10, 70])
@pytest.mark.parametrize("op", ["diff", "interp"])
def test_apply_matches_oracle(bc, n, op):
    """Plain differentiation and interpolation of every field kind (Tables A1,
    A2, A4, A5 rows of groups III and IV)."""
    s, _ = make((n,), [bc])
    sym_p, sym_u = pstd.symmetries(bc)
    for kind, symf in KIND_SYM.items():
        sym = symf(sym_p, sym_u)
        x = inputs.random_field(s.apply_shape(0, kind), 7).astype(np.float32)
        assert x.shape[0] == dtt_ops.sample_length(sym, n)
        y = host(s.apply(0, op, torch.tensor(x, device="cuda"), kind))
        ref = (dtt_ops.diff if op == "diff" else dtt_ops.interp)(sym, x.astype(np.float64), n, DX)[0]
        assert y.shape == ref.shape
        assert np.abs(y - ref).max() / np.abs(ref).max() < 2e-5, (kind, sym)
    s.close()


def test_plane_full_run_vs_modal():
    """2-D 122 x 113 (N / Dm-mid x, D / Nm-mid y: M = 243 and 225 on the generic
    radix-3/5 FFT), 3 blobs, CFL 0.3, 1000 steps vs the modal closed form."""
    ncells, bcs = (122, 113), [("N", "Dm"), ("D", "Nm")]
    s, od = make(ncells, bcs, cfl=0.3)
    w = inputs.small(ncells, bcs, nblobs=3, sigma_cells=3.0)
    p0 = f32(s.restrict(w.p0_full()))
    p, us = dev(p0), [torch.zeros(sh, device="cuda") for sh in s.shapes[1:]]
    s.init_velocity(p, us)
    s.run(p, us, 1000)
    ref = modal.modal_pressure(od, p0, 1000)
    assert rel_l2(host(p), ref) < 1e-4
    pb, pm = dev(p0), torch.empty(s.shapes[0], device="cuda")
    s.init_prev(pb, pm)
    s.run2(pb, pm, 1000)
    assert rel_l2(host(pb), ref) < 1e-4
    s.close()


def test_mid_wall_rejections():
    from paper_2005_00322_gb300 import Solver, _abi
    with pytest.raises(_abi.PstdError):
        Solver((1,), DX, [("N", "Nm")], cfl=0.1)           # N >= 2 next to a mid-cell wall
    with pytest.raises(_abi.PstdError):
        Solver((8,), DX, [("Nm", "N")], cfl=0.1)           # right wall only
    with pytest.raises(_abi.PstdError):
        Solver((8,), DX, [("N", "Dm")], cfl=0.1, form="split")
    with pytest.raises(_abi.PstdError):
        Solver((8,), DX, [("N", "Dm")], cfl=0.7)           # beyond the stability limit
