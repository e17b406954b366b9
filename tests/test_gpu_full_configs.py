"""GPU parity of the two batched configurations at their full sizes, against
FP64 references that do not time-step:

* 3-D 256^3 with reflection coefficient R = 0.4 on all six faces: the 64
  wall combinations of Section 5 in one batch, 1500 steps at CFL 0.3,
  combined with their weights.  The reference is the weighted sum of each
  combination's modal closed form, evaluated on a sub-lattice of every 4th
  node (`separable_modal_pressure` restricted to those rows).
* 64 independent 2-D runs of seeded sizes in [64, 1024]^2 with random walls
  (most of them on the convolution route), 4000 steps at CFL 0.3, every
  member against its own modal closed form.

The bar is that of a full run: 1e-4 relative L2.
"""
import numpy as np
import pytest
import torch

from oracle import modal, pstd, reflection
from paper_2005_00322_gb300 import inputs

pytestmark = pytest.mark.gpu

DX = 1e-4


def test_cube256_r04_64_combinations_full_run():
    from paper_2005_00322_gb300.batch import ReflectionRun
    w = inputs.cube256_reflect(0.4, steps=1500)
    n = w.ncells[0]
    R = ReflectionRun(w.ncells, w.dx, w.refl, cfl=w.cfl)
    R.set_initial_pressure(w.p0_full())
    R.run(w.steps)
    idx = np.arange(1, n, 4)                      # interior nodes, stored by every combination
    got = R.pressure().cpu().numpy()[np.ix_(idx, idx, idx)].astype(np.float64)
    R.batch.close()
    dt = pstd.dt_from_cfl(w.cfl, w.dx, w.c0)
    ref = np.zeros_like(got)
    for bc, wt in reflection.combination_weights(w.refl):
        od = pstd.Desc(w.ncells, (w.dx,), list(bc), dt=dt)
        facs = [[term[i][pstd.p_nodes(n, bc[i])] for i in range(3)] for term in w.factors()]
        sub = tuple(idx - pstd.p_nodes(n, bc[i])[0] for i in range(3))
        ref += wt * modal.separable_modal_pressure(od, facs, w.steps, out_index=sub)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    print("R = 0.4 combined field rel L2 %.2e" % err)
    assert err < 1e-4, err


def test_plane_batch_64_uneven_members_full_run():
    from paper_2005_00322_gb300.batch import Batch
    from paper_2005_00322_gb300.solver import stored_node_range
    mem = inputs.plane_batch(steps=4000)
    specs = [dict(ncells=m.ncells, dx=m.dx, bc=m.bc, cfl=m.cfl) for m in mem]
    B = Batch(specs)
    fields = B.zeros()
    p0s = []
    for (p, _), m in zip(fields, mem):
        sl = tuple(slice(stored_node_range(n, b)[0], stored_node_range(n, b)[1] + 1)
                   for n, b in zip(m.ncells, m.bc))
        q = np.ascontiguousarray(np.asarray(m.p0_full(), np.float32)[sl])
        p.copy_(torch.tensor(q, device="cuda"))
        p0s.append(q.astype(np.float64))
    B.init_velocity(fields)
    B.run(fields, mem[0].steps)
    torch.cuda.synchronize()
    worst = 0.0
    for (p, _), m, p0 in zip(fields, mem, p0s):
        od = pstd.Desc(m.ncells, (m.dx,), m.bc, dt=pstd.dt_from_cfl(m.cfl, m.dx, m.c0))
        ref = modal.modal_pressure(od, p0, m.steps)
        err = np.linalg.norm(p.cpu().numpy().astype(np.float64) - ref) / np.linalg.norm(ref)
        worst = max(worst, err)
        assert err < 1e-4, (m.ncells, m.bc, err)
    B.close()
    print("worst member rel L2 %.2e" % worst)
