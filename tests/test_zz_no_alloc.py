"""pstd_step_noalloc against the planned path, through the C ABI.

pstd_step_noalloc serves callers that must not allocate device memory when
they call the library (their device memory belongs to a memory manager, or
their loop cannot pay for cudaMalloc / cudaFree).  It keeps its scratch
accumulator and tables in fixed device arrays instead of a plan.  This test
checks that two calls in a row give the same fields as the plan-based
pstd_plan / pstd_run path on the same inputs, within the per-step tolerance
of the other parity tests (1e-5 relative L2).  It is collected last on
purpose and builds everything it needs, so it also runs alone in a fresh
process.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

DX = 1e-4


def rel_l2(a, ref):
    a = a.double().cpu().numpy()
    ref = ref.double().cpu().numpy()
    return float(np.linalg.norm(a - ref) / np.linalg.norm(ref))


@pytest.mark.parametrize("ncells,bcs,steps", [
    ((96, 80), [("D", "D"), ("N", "N")], (5, 7)),
    ((40, 24, 30), [("N", "D"), ("D", "N"), ("D", "D")], (3, 4)),
    ((64,), [("D", "N")], (6, 9)),
])
def test_noalloc_matches_planned_path(ncells, bcs, steps):
    from paper_2005_00322_gb300 import Solver, _abi, build
    from paper_2005_00322_gb300.inputs import random_field

    build.build()
    lib = _abi.load()
    cfl = 0.25 / np.sqrt(len(ncells))
    solver = Solver(ncells, DX, bcs, cfl=cfl)
    p0 = torch.tensor(random_field(solver.shapes[0], 5).astype(np.float32), device="cuda")
    u0 = [torch.tensor(random_field(s, 6 + i).astype(np.float32) * 1e-6, device="cuda")
          for i, s in enumerate(solver.shapes[1:])]

    # existing entry point: plan + run
    pa, ua = p0.clone(), [u.clone() for u in u0]
    # new entry point: the same descriptor, no plan
    pb, ub = p0.clone(), [u.clone() for u in u0]
    desc = _abi.make_desc(ncells, DX, bcs, solver.c0, solver.rho0, solver.dt)
    stream = torch.cuda.current_stream()
    ptrs = (ctypes.c_void_p * 3)(*[u.data_ptr() for u in ub])

    for call, n in enumerate(steps):     # two calls in a row on the same buffers
        solver.run(pa, ua, n)
        solver.sync()
        free_before = torch.cuda.mem_get_info()[0]
        rc = lib.pstd_step_noalloc(ctypes.byref(desc), ctypes.c_void_p(pb.data_ptr()), ptrs,
                                   n, ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, _abi.ERRORS.get(rc, rc)
        torch.cuda.synchronize()
        if call > 0:
            # a call after the first takes no device memory (the first may have
            # committed the file-scope arrays when it loaded the module)
            assert torch.cuda.mem_get_info()[0] == free_before
        assert rel_l2(pb, pa) < 1e-5
        for a, b in zip(ua, ub):
            assert rel_l2(b, a) < 1e-5
    solver.close()


def test_noalloc_rejects_sizes_beyond_capacity():
    from paper_2005_00322_gb300 import _abi, build

    build.build()
    lib = _abi.load()
    ptrs = (ctypes.c_void_p * 3)(1, 1, 1)
    # 2049^2 pressure points > PSTD_NOALLOC_MAX_POINTS
    big = _abi.make_desc((2048, 2048), DX, [("N", "N"), ("N", "N")], 1500.0, 1000.0, 0.1 * DX / 1500.0)
    assert lib.pstd_step_noalloc(ctypes.byref(big), ctypes.c_void_p(1), ptrs, 1, None) == -6
    # 2N = 2 * 3000 > PSTD_NOALLOC_MAX_FFT
    long = _abi.make_desc((3000,), DX, [("N", "N")], 1500.0, 1000.0, 0.1 * DX / 1500.0)
    assert lib.pstd_step_noalloc(ctypes.byref(long), ctypes.c_void_p(1), ptrs, 1, None) == -6
    # 2N = 14 has a factor 7: no FFT schedule
    odd = _abi.make_desc((7,), DX, [("N", "N")], 1500.0, 1000.0, 0.1 * DX / 1500.0)
    assert lib.pstd_step_noalloc(ctypes.byref(odd), ctypes.c_void_p(1), ptrs, 1, None) == -6
    # valid wall types without a schedule here: periodic axes, mid-cell walls
    per = _abi.make_desc((64,), DX, [("P", "P")], 1500.0, 1000.0, 0.1 * DX / 1500.0)
    assert lib.pstd_step_noalloc(ctypes.byref(per), ctypes.c_void_p(1), ptrs, 1, None) == -6
    mid = _abi.make_desc((64,), DX, [("D", "Nm")], 1500.0, 1000.0, 0.1 * DX / 1500.0)
    assert lib.pstd_step_noalloc(ctypes.byref(mid), ctypes.c_void_p(1), ptrs, 1, None) == -6
