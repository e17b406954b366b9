"""GPU parity of batched runs and of the reflection-coefficient combination (Section 5)."""
import numpy as np
import pytest
import torch

from oracle import pstd, reflection
from paper_2005_00322_gb300 import inputs

pytestmark = pytest.mark.gpu

DX = 1e-4
BCS4 = [("N", "N"), ("N", "D"), ("D", "N"), ("D", "D")]


def _oracle_member(ncells, bc, cfl, p_full, steps):
    d = pstd.Desc(ncells, (DX,), bc, dt=pstd.dt_from_cfl(cfl, DX, 1500.0))
    sl = tuple(slice(j[0], j[-1] + 1) for j in (pstd.p_nodes(n, b) for n, b in zip(ncells, bc)))
    p0 = np.asarray(p_full, np.float32).astype(np.float64)[sl]
    s = pstd.run(d, pstd.State(p0, pstd.init_velocity(d, p0, None, "halfstep")), steps)
    full = np.zeros(tuple(n + 1 for n in ncells))
    full[sl] = s.p
    return full


def test_batch_of_uneven_members_equals_single_runs():
    """Members of one graph launch give the same bits as separate plans."""
    from paper_2005_00322_gb300 import Solver
    from paper_2005_00322_gb300.batch import Batch
    specs = [((64, 48), [("D", "D"), ("N", "N")]), ((40, 96), [("N", "D"), ("D", "N")]),
             ((128,), [("D", "N")]), ((7, 30), [("N", "N"), ("D", "D")]), ((16, 12, 20), [("N", "D"), ("D", "D"), ("N", "N")])]
    members = [dict(ncells=n, dx=DX, bc=b, cfl=0.2) for n, b in specs]
    B = Batch(members)
    fields = B.zeros()
    p0s = [torch.tensor(inputs.random_field(B.shapes[m][0], 40 + m).astype(np.float32), device="cuda")
           for m in range(len(specs))]
    for (p, _), q in zip(fields, p0s):
        p.copy_(q)
    B.init_velocity(fields)
    B.run(fields, 70)                       # 2 graph blocks of 32 + a tail of 6
    steps_launches = B.last_launch_count()
    torch.cuda.synchronize()
    conv = 0
    for m, (n, b) in enumerate(specs):
        s = Solver(n, DX, b, cfl=0.2)
        conv += 2 * sum(1 for sc in s.schedule() if sc[0] >= 0)
        p = p0s[m].clone()
        us = [torch.zeros(sh, device="cuda") for sh in s.shapes[1:]]
        s.init_velocity(p, us)
        s.run(p, us, 70)
        torch.cuda.synchronize()
        assert torch.equal(p, fields[m][0])
        assert all(torch.equal(a, b_) for a, b_ in zip(us, fields[m][1]))
        s.close()
    assert steps_launches == 70 * sum(len(n) for n, _ in specs) + conv
    B.close()


def test_nonreflecting_1d_cancellation():
    """R_L = R_R = 0: the weighted sum vanishes once the waves have left (Section 5)."""
    from paper_2005_00322_gb300.batch import ReflectionRun
    n, cfl = 128, 0.2
    steps = int(round(1.5 * n / cfl))
    x = np.arange(n + 1) * DX
    p_full = np.exp(-((x - n / 2 * DX) ** 2) / (2 * (4 * DX) ** 2))
    R = ReflectionRun((n,), DX, [(0.0, 0.0)], cfl=cfl)
    R.set_initial_pressure(p_full)
    R.run(steps)
    got = R.pressure().cpu().numpy().astype(np.float64)
    ref = sum(w * _oracle_member((n,), [bc], cfl, p_full, steps)
              for bc, w in zip(reflection.BASIC_RUNS, reflection.axis_weights(0.0, 0.0)))
    # the FP32 cast of p0 leaves slow near-Nyquist rounding noise in the box
    assert np.abs(ref).max() < 1e-9
    assert np.abs(got).max() < 1e-5 * p_full.max()
    R.batch.close()


@pytest.mark.parametrize("refl", [[(0.4, 0.4), (0.4, 0.4)], [(0.0, 0.5), (-0.3, 1.0)]])
def test_reflection_2d_matches_oracle(refl):
    """16 wall combinations in one batch, combined, vs the oracle's weighted sum."""
    from paper_2005_00322_gb300.batch import ReflectionRun
    ncells, cfl, steps = (40, 36), 0.2, 90
    w = inputs.small(ncells, [("N", "N")] * 2, nblobs=2, sigma_cells=2.5)
    p_full = w.p0_full()
    R = ReflectionRun(ncells, DX, refl, cfl=cfl)
    R.set_initial_pressure(p_full)
    R.run(steps)
    got = R.pressure().cpu().numpy().astype(np.float64)
    ref = sum(wt * _oracle_member(ncells, list(bc), cfl, p_full, steps)
              for bc, wt in reflection.combination_weights(refl))
    err = np.linalg.norm(got - ref) / np.linalg.norm(p_full)
    assert err < 1e-4, err
    R.batch.close()


def _batch_fields(B, seed):
    fields = B.zeros()
    for m, (p, _) in enumerate(fields):
        p.copy_(torch.tensor(inputs.random_field(B.shapes[m][0], seed + m).astype(np.float32)))
    return fields


def _clone(fields):
    return [(p.clone(), [u.clone() for u in us]) for p, us in fields]


def test_persistent_batch_register_kernel_equals_graph():
    """The 16 wall combinations of one 2-D grid share every register-FFT
    schedule: one cooperative kernel runs all members' passes, bit for bit the
    graph path's result, with one launch per run plus the conversions."""
    from paper_2005_00322_gb300.batch import Batch
    bcs = [(a, b) for a in BCS4 for b in BCS4]
    members = [dict(ncells=(128, 128), dx=DX, bc=list(bc), cfl=0.2) for bc in bcs]
    A, B = Batch(members), Batch(members)
    B.set_persistent()
    assert B.persistent_kind() == "register"
    fa = _batch_fields(A, 60)
    A.init_velocity(fa)
    fb = _clone(fa)
    A.run(fa, 70)
    B.run(fb, 70)
    A.sync()
    B.sync()
    conv = B.last_launch_count() - 1
    assert 0 < conv <= 2 * 2 * len(members)
    for (pa, ua), (pb, ub) in zip(fa, fb):
        assert torch.equal(pa, pb)
        assert all(torch.equal(x, y) for x, y in zip(ua, ub))
    A.close()
    B.close()


def test_persistent_batch_generic_kernel_matches_graph():
    """Uneven members (convolution, dense, generic-FFT and register-FFT axes,
    1-D to 3-D) in one cooperative kernel on the generic CTA program: members
    whose axes all take that program in the graph path too agree bit for bit;
    a register-FFT axis computed by the generic program agrees to rounding."""
    from paper_2005_00322_gb300.batch import Batch
    specs = [((100, 70), [("D", "D"), ("N", "D")]), ((37, 130), [("N", "N"), ("D", "N")]),
             ((128,), [("D", "N")]), ((96, 50), [("N", "D"), ("D", "D")]),
             ((20, 18, 27), [("N", "D"), ("D", "D"), ("N", "N")])]
    members = [dict(ncells=n, dx=DX, bc=b, cfl=0.2) for n, b in specs]
    A, B = Batch(members), Batch(members)
    B.set_persistent()
    assert B.persistent_kind() == "generic"
    fa = _batch_fields(A, 80)
    A.init_velocity(fa)
    fb = _clone(fa)
    A.run(fa, 45)
    B.run(fb, 45)
    A.sync()
    B.sync()
    assert B.last_launch_count() == 1
    from paper_2005_00322_gb300 import Solver
    for m, ((pa, ua), (pb, ub)) in enumerate(zip(fa, fb)):
        s = Solver(specs[m][0], DX, specs[m][1], cfl=0.2)
        register = any(sc[0] >= 0 for sc in s.schedule())
        s.close()
        if not register:
            assert torch.equal(pa, pb), m
            assert all(torch.equal(x, y) for x, y in zip(ua, ub)), m
        else:
            assert ((pa - pb).norm() / pa.norm()).item() < 1e-5, m
            assert all(((x - y).norm() / x.norm()).item() < 1e-5 for x, y in zip(ua, ub)), m
    A.close()
    B.close()


def test_persistent_batch_stalled_barrier_reports_timeout():
    """A barrier that waits for one arrival too many gives up after the poll
    limit: pstd_batch_sync reports PSTD_ETIMEOUT once and the batch runs again."""
    from paper_2005_00322_gb300._abi import PstdError
    from paper_2005_00322_gb300.batch import Batch
    members = [dict(ncells=(100, 70), dx=DX, bc=[("D", "D"), ("N", "D")], cfl=0.2),
               dict(ncells=(64, 48), dx=DX, bc=[("N", "N"), ("D", "D")], cfl=0.2)]
    B = Batch(members)
    B.set_persistent(spin_limit=1000, withhold_arrivals=1)
    f = _batch_fields(B, 90)
    B.run(f, 5)
    with pytest.raises(PstdError, match="ETIMEOUT"):
        B.sync()
    B.sync()
    B.set_persistent(spin_limit=0, withhold_arrivals=0)
    g = _batch_fields(B, 90)
    B.init_velocity(g)
    B.run(g, 5)
    B.sync()
    assert all(torch.isfinite(p).all() for p, _ in g)
    B.close()
