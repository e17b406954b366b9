"""GPU parity of the split-precision dense forms: FP16 hi/lo products on the
mma.sync tensor-core path ("split"), TF32 hi/lo products on the tcgen05
tensor cores ("tensor") and the exact BF16 three-way split on the tcgen05
tensor cores ("split-bf16").

Every form is held to the FFT route's tolerances against the FP64 oracle:
1e-5 relative L2 per step from the same state, 1e-4 over a full run.
"""
import numpy as np
import pytest
import torch

from oracle import modal, pstd
from paper_2005_00322_gb300 import inputs

pytestmark = pytest.mark.gpu

DX = 1e-4


def rel_l2(a, ref):
    return float(np.linalg.norm(np.asarray(a, np.float64) - ref) / np.linalg.norm(ref))


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.float64)


CASES = [((48,), [("N", "N")]), ((100,), [("D", "N")]), ((64, 37), [("D", "D"), ("N", "N")]),
         ((30, 45), [("N", "D"), ("D", "N")]), ((24, 20, 18), [("D", "N"), ("N", "N"), ("D", "D")]),
         ((70, 9), [("N", "N"), ("D", "D")]), ((5, 200), [("D", "D"), ("N", "D")])]


STEP_TOL = {"split": 1e-5, "tensor": 1e-5, "split-bf16": 1e-5}


@pytest.mark.parametrize("form", ["split", "split-bf16", "tensor"])
@pytest.mark.parametrize("ncells,bcs", CASES)
def test_split_one_step_matches_oracle(ncells, bcs, form):
    from paper_2005_00322_gb300 import Solver
    cfl = 0.25 / np.sqrt(len(ncells))
    dt = pstd.dt_from_cfl(cfl, DX, 1500.0)
    s = Solver(ncells, DX, bcs, dt=dt, form=form)
    od = pstd.Desc(ncells, (DX,), bcs, dt=dt)
    p0 = inputs.random_field(s.shapes[0], 1).astype(np.float32).astype(np.float64)
    u0 = [inputs.random_field(sh, 2 + i).astype(np.float32).astype(np.float64) * 1e-6
          for i, sh in enumerate(s.shapes[1:])]
    p = torch.tensor(p0, dtype=torch.float32, device="cuda")
    us = [torch.tensor(u, dtype=torch.float32, device="cuda") for u in u0]
    s.step(p, us)
    ref = pstd.step(od, pstd.State(p0, u0))
    tol = STEP_TOL[form]
    assert rel_l2(host(p), ref.p) < tol
    for i in range(len(ncells)):
        assert rel_l2(host(us[i]), ref.u[i]) < tol
    s.close()


RUN_TOL = {"split": 1e-4, "tensor": 1e-4, "split-bf16": 1e-4}


@pytest.mark.parametrize("form", ["split", "split-bf16", "tensor"])
def test_split_plane512_full_run_vs_modal(form):
    """2-D 512^2 DD / NN, 4000 steps of a split form vs the modal closed form."""
    from paper_2005_00322_gb300 import Solver
    w = inputs.plane512_dx_ny()
    s = Solver(w.ncells, w.dx, w.bc, cfl=w.cfl, form=form)
    od = pstd.Desc(w.ncells, (w.dx,), w.bc, dt=s.dt)
    p = torch.tensor(np.asarray(s.restrict(w.p0_full()), np.float32), device="cuda")
    us = [torch.zeros(sh, device="cuda") for sh in s.shapes[1:]]
    s.init_velocity(p, us)
    s.run(p, us, w.steps)
    facs = [[term[i][pstd.p_nodes(n, b)] for i, (n, b) in enumerate(zip(w.ncells, w.bc))]
            for term in w.factors()]
    ref = modal.separable_modal_pressure(od, facs, w.steps)
    assert rel_l2(host(p), ref) < RUN_TOL[form]
    s.close()


@pytest.mark.parametrize("form", ["split", "split-bf16", "tensor"])
def test_split_cube384_full_run_vs_modal(form):
    """3-D 384^3 (D x, N y, D z), 4 blobs, CFL 0.3, 1000 steps of each split
    form vs the modal closed form: every form within 1e-4."""
    from paper_2005_00322_gb300 import Solver
    w = inputs.cube384_dnd()
    s = Solver(w.ncells, w.dx, w.bc, cfl=w.cfl, form=form)
    od = pstd.Desc(w.ncells, (w.dx,), w.bc, dt=s.dt)
    p = torch.tensor(np.asarray(s.restrict(w.p0_full()), np.float32), device="cuda")
    us = [torch.zeros(sh, device="cuda") for sh in s.shapes[1:]]
    s.init_velocity(p, us)
    s.run(p, us, w.steps)
    s.sync()
    facs = [[term[i][pstd.p_nodes(n, b)] for i, (n, b) in enumerate(zip(w.ncells, w.bc))]
            for term in w.factors()]
    ref = modal.separable_modal_pressure(od, facs, w.steps)
    assert rel_l2(host(p), ref) < 1e-4
    s.close()
