"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances: a single derivative or a single step, from the same FP64 state
cast to FP32, must agree within 1e-5 relative L2; a full run within 1e-4
relative L2 (the FP32 bar stated for this path).  Relative L2 is
||gpu - ref||_2 / ||ref||_2 per field.
"""
import numpy as np
import pytest
import torch

from oracle import modal, pstd
from paper_2005_00322_gb300 import inputs

pytestmark = pytest.mark.gpu

BCS = [("N", "N"), ("N", "D"), ("D", "N"), ("D", "D")]
DX = 1e-4


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


def conversions(s):
    """Launches that move the register-FFT axes' velocities to their spectrum
    form and back around a pstd_step / pstd_run call."""
    return 2 * sum(1 for sc in s.schedule() if sc[0] >= 0)


def dev(x):
    return torch.tensor(np.asarray(x, np.float32), device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


CASES = [
    # (ncells, bcs): FFT route (2N in 2^a 3^b 5^c), several CTAs plus a ragged tail
    ((48,), [("N", "N")]), ((48,), [("D", "D")]), ((40,), [("N", "D")]), ((36,), [("D", "N")]),
    ((64, 37), [("D", "D"), ("N", "N")]),
    ((30, 45), [("N", "D"), ("D", "N")]),
    ((24, 20, 18), [("D", "N"), ("N", "N"), ("D", "D")]),
    ((16, 27, 25), [("N", "N"), ("D", "D"), ("N", "D")]),
    ((192, 20), [("D", "N"), ("N", "N")]), ((8, 96), [("N", "D"), ("D", "D")]),
    ((512, 6), [("N", "N"), ("D", "N")]), ((3, 384), [("D", "D"), ("N", "D")]),
    # convolution route (2N has a prime factor > 5, N > 64): power-of-two linear convolution
    ((67,), [("N", "N")]), ((97,), [("D", "N")]), ((257,), [("N", "D")]), ((130, 9), [("D", "D"), ("N", "N")]),
    ((6, 101), [("N", "D"), ("D", "D")]),
    # periodic axes (Fourier PSTD, Section 2): register FFT, generic, convolution, dense
    ((64,), [("P", "P")]), ((100,), [("P", "P")]), ((67,), [("P", "P")]), ((7,), [("P", "P")]),
    ((30, 45), [("P", "P"), ("D", "N")]), ((17, 96), [("N", "N"), ("P", "P")]),
    # dense route (2N has a factor 7, 11 or 13) and tiny edge sizes
    ((7,), [("N", "D")]), ((11,), [("D", "D")]), ((13, 6), [("N", "N"), ("D", "N")]),
    ((1,), [("N", "N")]), ((1,), [("N", "D")]), ((2,), [("D", "D")]), ((2, 3), [("D", "N"), ("N", "D")]),
]


@pytest.mark.parametrize("ncells,bcs", CASES)
def test_grad_matches_oracle(ncells, bcs):
    s, od = make(ncells, bcs)
    for ax in range(len(ncells)):
        p = inputs.random_field(s.shapes[0], 10 + ax)
        g = s.grad(ax, 0, dev(p))
        ref = pstd.grad_p_axis(od, p.astype(np.float32).astype(np.float64), ax)
        assert rel_l2(host(g), ref) < 1e-5, (ax, "p->u")
        u = inputs.random_field(s.shapes[1 + ax], 20 + ax)
        q = s.grad(ax, 1, dev(u))
        ref = pstd.grad_u_axis(od, u.astype(np.float32).astype(np.float64), ax)
        assert rel_l2(host(q), ref) < 1e-5, (ax, "u->p")
    s.close()


@pytest.mark.parametrize("ncells,bcs", CASES)
def test_one_step_matches_oracle(ncells, bcs):
    s, od = make(ncells, bcs, cfl=0.25 / np.sqrt(len(ncells)))
    p0 = inputs.random_field(s.shapes[0], 1).astype(np.float32).astype(np.float64)
    u0 = [inputs.random_field(sh, 2 + i).astype(np.float32).astype(np.float64) * 1e-6
          for i, sh in enumerate(s.shapes[1:])]
    p, us = dev(p0), [dev(u) for u in u0]
    s.step(p, us)
    ref = pstd.step(od, pstd.State(p0, u0))
    assert rel_l2(host(p), ref.p) < 1e-5
    for i in range(len(ncells)):
        assert rel_l2(host(us[i]), ref.u[i]) < 1e-5
    assert s.last_launch_count() == len(ncells) + conversions(s)
    s.close()


@pytest.mark.parametrize("sched", [
    [(0, 2), (0, 4)], [(1, 1), (1, 2)], [(1, 2), (1, 4)], [(4, 1), (4, 1)], [(4, 2), (4, 4)],
    [(4, 4), (3, 1)], [(1, 4), (4, 2)], [(5, 1), (5, 2)], [(5, 4), (5, 4)], [(4, 2), (5, 1)],
])
def test_every_schedule_matches_oracle(sched):
    """Every register-FFT schedule an axis can take (variant x line pairs per
    CTA) gives the oracle's step: FFT lengths 256 (axis 0) and 512 (axis 1),
    strided tiles with a ragged, odd inner extent (axis 1: 27 lines apart) and
    the phantom partner of the unpaired line."""
    from paper_2005_00322_gb300 import Solver
    ncells, bcs = (128, 256, 27), [("D", "D"), ("N", "N"), ("N", "D")]
    dt = pstd.dt_from_cfl(0.25 / np.sqrt(3), DX, 1500.0)
    s = Solver(ncells, DX, bcs, dt=dt, schedule=sched)
    assert [sc[0] for sc in s.schedule()[:2]] == [v for v, _ in sched]
    assert [sc[2] for sc in s.schedule()[:2]] == [q for _, q in sched]
    od = pstd.Desc(ncells, (DX,), bcs, dt=dt)
    p0 = inputs.random_field(s.shapes[0], 11).astype(np.float32).astype(np.float64)
    u0 = [inputs.random_field(sh, 12 + i).astype(np.float32).astype(np.float64) * 1e-6
          for i, sh in enumerate(s.shapes[1:])]
    p, us = dev(p0), [dev(u) for u in u0]
    s.step(p, us)
    ref = pstd.step(od, pstd.State(p0, u0))
    assert rel_l2(host(p), ref.p) < 1e-5
    for i in range(3):
        assert rel_l2(host(us[i]), ref.u[i]) < 1e-5
    s.close()


def test_unavailable_variant_is_rejected():
    from paper_2005_00322_gb300 import Solver
    from paper_2005_00322_gb300._abi import PstdError
    with pytest.raises(PstdError, match="EINVAL"):
        Solver((96, 64), DX, [("N", "N"), ("D", "D")], cfl=0.2, schedule=[(4, 1), None])   # L = 192
    with pytest.raises(PstdError, match="EINVAL"):
        # the table-in-memory schedules serve walled axes only
        Solver((256, 64), DX, [("P", "P"), ("N", "N")], cfl=0.2, schedule=[(5, 1), None])


@pytest.mark.parametrize("ncells,bcs", CASES[:8])
@pytest.mark.parametrize("uinit", ["halfstep", "as_given"])
def test_short_run_matches_oracle(ncells, bcs, uinit):
    """init_velocity + 40 steps (graph-replayed block plus a direct tail)."""
    s, od = make(ncells, bcs, cfl=0.3 / np.sqrt(len(ncells)), uinit=uinit)
    w = inputs.small(ncells, bcs)
    p0 = s.restrict(w.p0_full()) if w.blobs else inputs.random_field(s.shapes[0], 3)
    p0 = np.asarray(p0, np.float32).astype(np.float64)
    p, us = dev(p0), [torch.zeros(sh, device="cuda") for sh in s.shapes[1:]]
    s.init_velocity(p, us)
    s.run(p, us, 40)
    ref = pstd.run(od, pstd.State(p0, pstd.init_velocity(od, p0, None, uinit)), 40)
    assert rel_l2(host(p), ref.p) < 1e-4
    for i in range(len(ncells)):
        assert rel_l2(host(us[i]), ref.u[i]) < 1e-4
    s.close()


def test_graph_run_equals_direct_launches_bitwise():
    """The graph-replayed run (two 32-step graphs and a tail) and the same run
    launched directly (a plan on the legacy stream, no graph) compute
    identical bits; single steps agree to rounding (each pstd_step converts
    the velocity to its spectrum and back)."""
    import ctypes
    from paper_2005_00322_gb300 import _abi
    ncells, bcs = (40, 33), [("D", "N"), ("N", "N")]
    s, _ = make(ncells, bcs)
    p0 = dev(inputs.random_field(s.shapes[0], 4))
    pa, ua = p0.clone(), [torch.zeros(sh, device="cuda") for sh in s.shapes[1:]]
    pb, ub = p0.clone(), [torch.zeros(sh, device="cuda") for sh in s.shapes[1:]]
    pc, uc = p0.clone(), [torch.zeros(sh, device="cuda") for sh in s.shapes[1:]]
    s.run(pa, ua, 70)
    assert s.last_launch_count() == 70 * 2 + conversions(s)
    lib = _abi.load()
    h = ctypes.c_void_p()
    assert lib.pstd_plan(ctypes.byref(s._desc), None, ctypes.byref(h)) == 0
    U = (ctypes.c_void_p * 3)(*[u.data_ptr() for u in ub])
    torch.cuda.synchronize()
    assert lib.pstd_run(h, ctypes.c_void_p(pb.data_ptr()), U, 70) == 0
    assert lib.pstd_sync(h) == 0
    assert lib.pstd_free(h) == 0
    for _ in range(70):
        s.step(pc, uc)
    torch.cuda.synchronize()
    assert torch.equal(pa, pb) and all(torch.equal(a, b) for a, b in zip(ua, ub))
    assert rel_l2(host(pc), host(pa)) < 1e-5
    assert all(rel_l2(host(a), host(c)) < 1e-5 for a, c in zip(ua, uc))
    s.close()


def test_line256_dd_full_run():
    """1-D N=256 DD Gaussian at node 100, CFL 0.2, 2000 steps vs the stepped oracle."""
    w = inputs.line256_dd()
    s, od = make(w.ncells, w.bc, cfl=w.cfl)
    p0 = np.asarray(s.restrict(w.p0_full()), np.float32).astype(np.float64)
    p, us = dev(p0), [torch.zeros(sh, device="cuda") for sh in s.shapes[1:]]
    s.init_velocity(p, us)
    s.run(p, us, w.steps)
    ref = pstd.run(od, pstd.State(p0, pstd.init_velocity(od, p0, None, "halfstep")), w.steps)
    assert rel_l2(host(p), ref.p) < 1e-4
    assert rel_l2(host(us[0]), ref.u[0]) < 1e-4
    s.close()


def _separable_factors(w, s):
    facs = []
    for term in w.factors():
        f = []
        for i, (n, b) in enumerate(zip(w.ncells, w.bc)):
            j = pstd.p_nodes(n, b)
            f.append(term[i][j])
        facs.append(f)
    return facs


def test_plane512_full_run_vs_modal():
    """2-D 512^2 (DD x, NN y), 4 blobs, CFL 0.3, 4000 steps vs the modal closed form."""
    w = inputs.plane512_dx_ny()
    s, od = make(w.ncells, w.bc, cfl=w.cfl)
    p0 = np.asarray(s.restrict(w.p0_full()), np.float32)
    p, us = dev(p0), [torch.zeros(sh, device="cuda") for sh in s.shapes[1:]]
    s.init_velocity(p, us)
    s.run(p, us, w.steps)
    facs = _separable_factors(w, s)
    ref = modal.separable_modal_pressure(od, facs, w.steps)
    # the FP32 cast of p0 is part of the input: compare against both routes' start
    assert rel_l2(host(p), ref) < 1e-4
    s.close()


def test_cube256_steps_and_modal():
    """3-D 256^3 (D x, N y, D z): 2 steps vs the stepped oracle, 600 steps vs modal."""
    w = inputs.cube256(steps=600)
    s, od = make(w.ncells, w.bc, cfl=w.cfl)
    p0 = np.asarray(s.restrict(w.p0_full()), np.float32)
    p, us = dev(p0), [torch.zeros(sh, device="cuda") for sh in s.shapes[1:]]
    s.init_velocity(p, us)
    s.run(p, us, 2)
    p064 = p0.astype(np.float64)
    ref = pstd.run(od, pstd.State(p064, pstd.init_velocity(od, p064, None, "halfstep")), 2)
    assert rel_l2(host(p), ref.p) < 1e-5
    for i in range(3):
        assert rel_l2(host(us[i]), ref.u[i]) < 1e-5
    del ref
    s.run(p, us, w.steps - 2)
    refm = modal.separable_modal_pressure(od, _separable_factors(w, s), w.steps)
    assert rel_l2(host(p), refm) < 1e-4
    s.close()


def test_periodic_plane_full_run_vs_modal():
    """2-D 128 x 96 periodic in both axes (Fourier PSTD), 1000 steps vs the modal form."""
    ncells, bcs = (128, 96), [("P", "P"), ("P", "P")]
    s, od = make(ncells, bcs, cfl=0.3)
    w = inputs.small(ncells, bcs, nblobs=3, sigma_cells=3.0)
    p0 = np.asarray(s.restrict(w.p0_full()), np.float32)
    p, us = dev(p0), [torch.zeros(sh, device="cuda") for sh in s.shapes[1:]]
    s.init_velocity(p, us)
    s.run(p, us, 1000)
    ref = modal.modal_pressure(od, p0.astype(np.float64), 1000)
    assert rel_l2(host(p), ref) < 1e-4
    s.close()


def test_large_prime_axis_run():
    """N = 1021 (prime): convolution route with a 4096-point FFT, 200 steps vs the oracle."""
    ncells, bcs = (1021,), [("D", "N")]
    s, od = make(ncells, bcs, cfl=0.3)
    w = inputs.small(ncells, bcs, nblobs=3, sigma_cells=6.0)
    p0 = np.asarray(s.restrict(w.p0_full()), np.float32).astype(np.float64)
    p, us = dev(p0), [torch.zeros(sh, device="cuda") for sh in s.shapes[1:]]
    s.init_velocity(p, us)
    s.run(p, us, 200)
    ref = pstd.run(od, pstd.State(p0, pstd.init_velocity(od, p0, None, "halfstep")), 200)
    assert rel_l2(host(p), ref.p) < 1e-4
    s.close()


def test_energy_drift_fp32():
    """The discrete energy of the GPU state stays constant over 1000 steps."""
    ncells, bcs = (60, 50), [("N", "D"), ("N", "N")]
    s, od = make(ncells, bcs)
    w = inputs.small(ncells, bcs, nblobs=3)
    p = dev(s.restrict(w.p0_full()))
    us = [torch.zeros(sh, device="cuda") for sh in s.shapes[1:]]
    s.init_velocity(p, us)
    es = []
    for k in range(5):
        pn = host(p)
        uprev = [host(u) for u in us]
        s.step(p, us)
        es.append(modal.energy(od, pn, uprev, [host(u) for u in us]))
        s.run(p, us, 249)
    es = np.array(es)
    assert np.abs(es - es[0]).max() < 1e-5 * es[0]
    s.close()


def test_errors_surface():
    from paper_2005_00322_gb300 import Solver
    from paper_2005_00322_gb300._abi import PstdError
    with pytest.raises(PstdError, match="EUNSUPPORTED"):
        Solver((4099,), DX, [("N", "N")], cfl=0.2)     # prime N: convolution FFT beyond 8192
    with pytest.raises(PstdError, match="EUNSTABLE"):
        Solver((64,), DX, [("N", "N")], cfl=0.7)
    s, _ = make((16,), [("N", "N")])
    with pytest.raises(ValueError):
        s.step(torch.zeros(5, device="cuda"), [torch.zeros(16, device="cuda")])
    s.close()


ENERGY_CASES = [((60, 50), [("N", "D"), ("N", "N")]), ((48,), [("D", "N")]), ((33, 20, 14), [("N", "N"), ("D", "D"), ("N", "D")]),
                ((40, 30), [("D", "Nm"), ("N", "Dm")]), ((32, 24), [("P", "P"), ("D", "N")])]


@pytest.mark.parametrize("ncells,bcs", ENERGY_CASES)
def test_gpu_energy_matches_oracle(ncells, bcs):
    """pstd_energy (FP64 on the GPU) against oracle.modal.energy on the same fields."""
    s, od = make(ncells, bcs)
    p = dev(inputs.random_field(s.shapes[0], 3))
    up = [dev(inputs.random_field(sh, 4 + i) * 1e-6) for i, sh in enumerate(s.shapes[1:])]
    un = [dev(inputs.random_field(sh, 8 + i) * 1e-6) for i, sh in enumerate(s.shapes[1:])]
    e_gpu = s.energy(p, up, un)
    e_ref = modal.energy(od, host(p), [host(u) for u in up], [host(u) for u in un])
    assert abs(e_gpu - e_ref) <= 1e-12 * abs(e_ref)
    s.close()


def test_gpu_energy_drift_plane512():
    """The FP32 4000-step 512^2 DD / NN run conserves the FP64 energy to 1e-5."""
    from paper_2005_00322_gb300 import Solver
    w = inputs.plane512_dx_ny()
    s = Solver(w.ncells, w.dx, w.bc, cfl=w.cfl)
    p = dev(s.restrict(w.p0_full()))
    us = [torch.zeros(sh, device="cuda") for sh in s.shapes[1:]]
    s.init_velocity(p, us)

    def energy_now():
        pn, uprev = p.clone(), [u.clone() for u in us]
        s.step(p, us)
        return s.energy(pn, uprev, us)
    e0 = energy_now()
    s.run(p, us, w.steps - 2)
    e1 = energy_now()
    assert abs(e1 - e0) < 1e-5 * e0
    s.close()


@pytest.mark.parametrize("ncells,bcs", [((512, 512), [("D", "D"), ("N", "N")]), ((96, 80, 64), [("N", "D"), ("D", "N"), ("D", "D")])])
def test_autotuned_plan(ncells, bcs):
    """pstd_plan_autotune: the tuned schedule is never slower than the default
    by its own measurement, the choice is cached, and a tuned run matches the
    default plan's run to the parity tolerance."""
    from paper_2005_00322_gb300 import Solver
    a = Solver(ncells, 1e-4, bcs, cfl=0.3, autotune=True)
    tuned, default = a.tune_us
    assert 0 < tuned <= default
    b = Solver(ncells, 1e-4, bcs, cfl=0.3, autotune=True)     # cached: same choice, same times
    assert b.tune_us == a.tune_us and [b.schedule()] == [a.schedule()]
    c = Solver(ncells, 1e-4, bcs, cfl=0.3)
    w = inputs.small(ncells, bcs, nblobs=2)
    p0 = np.asarray(c.restrict(w.p0_full()), np.float32)
    outs = []
    for s in (a, c):
        p = torch.tensor(p0, device="cuda")
        us = [torch.zeros(sh, device="cuda") for sh in s.shapes[1:]]
        s.init_velocity(p, us)
        s.run(p, us, 100)
        outs.append(host(p))
    assert rel_l2(outs[0], outs[1]) < 1e-5
    for s in (a, b, c):
        s.close()
