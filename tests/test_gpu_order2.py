"""GPU parity of the second-order pressure-only form (pstd_init_prev, pstd_run2)
against its FP64 oracle (oracle/order2.py) and the closed-form modal solution.

Tolerances as for the coupled path: one step from the same FP32 input within
1e-5 relative L2, a full run within 1e-4 (the FP32 bar of the path).
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle import modal, order2, pstd
from paper_2005_00322_gb300 import inputs

pytestmark = pytest.mark.gpu

DX = 1e-4


def rel_l2(a, ref):
    a = np.asarray(a, np.float64)
    ref = np.asarray(ref, np.float64)
    return float(np.linalg.norm(a - ref) / np.linalg.norm(ref))


def make(ncells, bcs, cfl=0.3, uinit="halfstep", form="fft"):
    from paper_2005_00322_gb300 import Solver
    dt = pstd.dt_from_cfl(cfl, DX, 1500.0)
    s = Solver(ncells, DX, bcs, dt=dt, uinit=uinit, form=form)
    od = pstd.Desc(ncells, (DX,), bcs, dt=dt)
    return s, od


def dev(x):
    return torch.tensor(np.asarray(x, np.float32), device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def f32(x):
    return np.asarray(x, np.float32).astype(np.float64)


CASES = [
    # register FFT (contiguous and strided), several CTAs and ragged tails
    ((48,), [("N", "N")]), ((48,), [("D", "D")]), ((40,), [("N", "D")]), ((36,), [("D", "N")]),
    ((64, 37), [("D", "D"), ("N", "N")]), ((30, 45), [("N", "D"), ("D", "N")]),
    ((24, 20, 18), [("D", "N"), ("N", "N"), ("D", "D")]),
    ((192, 20), [("D", "N"), ("N", "N")]), ((512, 6), [("N", "N"), ("D", "N")]),
    ((3, 384), [("D", "D"), ("N", "D")]),
    # generic Stockham FFT (2N with no register schedule), convolution and dense routes
    ((40, 9), [("N", "N"), ("D", "D")]), ((67,), [("N", "N")]), ((97,), [("D", "N")]),
    ((6, 101), [("N", "D"), ("D", "D")]), ((7,), [("N", "D")]), ((11,), [("D", "D")]),
    # periodic axes (Fourier PSTD, Section 2)
    ((64,), [("P", "P")]), ((67,), [("P", "P")]), ((7,), [("P", "P")]), ((30, 45), [("P", "P"), ("D", "N")]),
    # tiny edge sizes
    ((1,), [("N", "N")]), ((1,), [("N", "D")]), ((2,), [("D", "D")]), ((2, 3), [("D", "N"), ("N", "D")]),
]


@pytest.mark.parametrize("ncells,bcs", CASES)
def test_one_step_matches_oracle(ncells, bcs):
    s, od = make(ncells, bcs, cfl=0.3 / np.sqrt(len(ncells)))
    p0 = f32(inputs.random_field(s.shapes[0], 11))
    pm = f32(p0 - 0.1 * inputs.random_field(s.shapes[0], 12))
    p, q = dev(p0), dev(pm)
    s.run2(p, q, 1)
    assert s.last_launch_count() == len(ncells) + 2
    ref, ref_prev = order2.step(od, p0, pm)
    assert rel_l2(host(p), ref) < 1e-5
    assert rel_l2(host(q), ref_prev) < 1e-5
    s.close()


@pytest.mark.parametrize("ncells,bcs", CASES)
@pytest.mark.parametrize("uinit", ["halfstep", "as_given"])
def test_init_prev_matches_oracle(ncells, bcs, uinit):
    s, od = make(ncells, bcs, cfl=0.3 / np.sqrt(len(ncells)), uinit=uinit)
    p0 = f32(inputs.random_field(s.shapes[0], 13))
    pm = torch.empty(s.shapes[0], device="cuda")
    s.init_prev(dev(p0), pm)
    assert rel_l2(host(pm), order2.init_prev(od, p0, uinit)) < 1e-5
    s.close()


@pytest.mark.parametrize("ncells,bcs", CASES[:10] + CASES[16:20])
@pytest.mark.parametrize("uinit", ["halfstep", "as_given"])
def test_short_run_matches_oracle(ncells, bcs, uinit):
    """init_prev + 40 steps (a graph-replayed block of 32 plus a direct tail)."""
    s, od = make(ncells, bcs, cfl=0.3 / np.sqrt(len(ncells)), uinit=uinit)
    w = inputs.small(ncells, bcs)
    p0 = s.restrict(w.p0_full()) if w.blobs else inputs.random_field(s.shapes[0], 3)
    p0 = f32(p0)
    p, pm = dev(p0), torch.empty(s.shapes[0], device="cuda")
    s.init_prev(p, pm)
    s.run2(p, pm, 40)
    assert s.last_launch_count() == 40 * len(ncells) + 2
    ref, ref_prev = order2.run(od, p0, order2.init_prev(od, p0, uinit), 40)
    assert rel_l2(host(p), ref) < 1e-4
    assert rel_l2(host(pm), ref_prev) < 1e-4
    s.close()


@pytest.mark.parametrize("ncells,bcs", [((64, 37), [("D", "D"), ("N", "N")]),
                                        ((24, 20, 18), [("D", "N"), ("N", "N"), ("D", "D")]),
                                        ((67,), [("N", "N")]), ((30, 45), [("P", "P"), ("D", "N")])])
def test_equals_coupled_run(ncells, bcs):
    """From the same p^0 with zero initial velocity, the second-order run and the
    coupled leapfrog run on the GPU give the same pressure (up to FP32 rounding)."""
    s, od = make(ncells, bcs, cfl=0.3 / np.sqrt(len(ncells)))
    p0 = dev(inputs.random_field(s.shapes[0], 5))
    pa, us = p0.clone(), [torch.zeros(sh, device="cuda") for sh in s.shapes[1:]]
    s.init_velocity(pa, us)
    s.run(pa, us, 100)
    pb, pm = p0.clone(), torch.empty(s.shapes[0], device="cuda")
    s.init_prev(pb, pm)
    s.run2(pb, pm, 100)
    assert rel_l2(host(pb), host(pa)) < 1e-4
    s.close()


def test_graph_run_equals_direct_launches_bitwise():
    """A graph-replayed run2 (two 32-step graphs and a tail) and the same run
    launched directly (a plan on the legacy stream, no graph) give identical bits,
    and a run split into calls agrees to rounding (each call converts p^{n-1}
    to the increment and back)."""
    from paper_2005_00322_gb300 import _abi
    ncells, bcs = (40, 33), [("D", "N"), ("N", "N")]
    s, _ = make(ncells, bcs)
    p0 = dev(inputs.random_field(s.shapes[0], 4))
    pa, qa = p0.clone(), torch.empty_like(p0)
    s.init_prev(pa, qa)
    pb, qb, pc, qc = pa.clone(), qa.clone(), pa.clone(), qa.clone()
    s.run2(pa, qa, 70)
    assert s.last_launch_count() == 70 * 2 + 2
    lib = _abi.load()
    h = ctypes.c_void_p()
    assert lib.pstd_plan(ctypes.byref(s._desc), None, ctypes.byref(h)) == 0
    torch.cuda.synchronize()
    assert lib.pstd_run2(h, ctypes.c_void_p(pb.data_ptr()), ctypes.c_void_p(qb.data_ptr()), 70) == 0
    assert lib.pstd_sync(h) == 0
    assert lib.pstd_free(h) == 0
    for _ in range(7):
        s.run2(pc, qc, 10)
    torch.cuda.synchronize()
    assert torch.equal(pa, pb) and torch.equal(qa, qb)
    assert rel_l2(host(pc), host(pa)) < 1e-5
    s.close()


def test_other_plan_forms_accept_run2():
    """A plan built for the split-precision form runs the second-order form on the
    FFT passes all the same."""
    ncells, bcs = (64, 37), [("D", "D"), ("N", "N")]
    s, od = make(ncells, bcs, form="split")
    p0 = f32(inputs.random_field(s.shapes[0], 6))
    p, pm = dev(p0), torch.empty(s.shapes[0], device="cuda")
    s.init_prev(p, pm)
    s.run2(p, pm, 20)
    ref, _ = order2.run(od, p0, order2.init_prev(od, p0), 20)
    assert rel_l2(host(p), ref) < 1e-4
    s.close()


def _separable_factors(w):
    facs = []
    for term in w.factors():
        facs.append([term[i][pstd.p_nodes(n, b)] for i, (n, b) in enumerate(zip(w.ncells, w.bc))])
    return facs


def test_plane512_full_run_vs_modal():
    """2-D 512^2 (DD x, NN y), 4 blobs, CFL 0.3, 4000 steps of the second-order
    form vs the modal closed form (the coupled scheme's exact solution)."""
    w = inputs.plane512_dx_ny()
    s, od = make(w.ncells, w.bc, cfl=w.cfl)
    p, pm = dev(s.restrict(w.p0_full())), torch.empty(s.shapes[0], device="cuda")
    s.init_prev(p, pm)
    s.run2(p, pm, w.steps)
    ref = modal.separable_modal_pressure(od, _separable_factors(w), w.steps)
    assert rel_l2(host(p), ref) < 1e-4
    s.close()


def test_cube256_run_vs_modal():
    """3-D 256^3 (D x, N y, D z): 2 steps vs the stepped oracle, 600 vs modal."""
    w = inputs.cube256(steps=600)
    s, od = make(w.ncells, w.bc, cfl=w.cfl)
    p0 = f32(s.restrict(w.p0_full()))
    p, pm = dev(p0), torch.empty(s.shapes[0], device="cuda")
    s.init_prev(p, pm)
    s.run2(p, pm, 2)
    ref, _ = order2.run(od, p0, order2.init_prev(od, p0), 2)
    assert rel_l2(host(p), ref) < 1e-5
    del ref
    s.run2(p, pm, w.steps - 2)
    refm = modal.separable_modal_pressure(od, _separable_factors(w), w.steps)
    assert rel_l2(host(p), refm) < 1e-4
    s.close()


def test_run2_edge_cases_and_errors():
    from paper_2005_00322_gb300 import _abi
    s, _ = make((16, 8), [("N", "N"), ("D", "D")])
    p = dev(inputs.random_field(s.shapes[0], 7))
    q = dev(inputs.random_field(s.shapes[0], 8))
    p1, q1 = p.clone(), q.clone()
    s.run2(p, q, 0)
    assert s.last_launch_count() == 0
    assert torch.equal(p, p1) and torch.equal(q, q1)
    with pytest.raises(_abi.PstdError):
        s.run2(p, p, 1)                                  # the two levels must not alias
    with pytest.raises(_abi.PstdError):
        s.init_prev(p, p)
    with pytest.raises(ValueError):
        s.run2(p, torch.zeros(3, device="cuda"), 1)      # wrong shape
    assert s.lib.pstd_run2(s._h, ctypes.c_void_p(p.data_ptr()), ctypes.c_void_p(q.data_ptr()), -1) == -1
    assert s.lib.pstd_run2(None, None, None, 1) == -1
    s.close()
