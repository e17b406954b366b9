"""The one-kernel (cooperative, persistent) pstd_run and its bounded waits."""
import numpy as np
import pytest
import torch

from paper_2005_00322_gb300 import inputs

pytestmark = pytest.mark.gpu

DX = 1e-4


@pytest.mark.parametrize("ncells,bcs", [
    ((256, 256), [("D", "N"), ("N", "N")]),
    ((512, 512), [("D", "D"), ("N", "N")]),
    ((128, 128, 128), [("N", "D"), ("D", "D"), ("N", "N")]),
])
def test_persistent_run_equals_graph_run(ncells, bcs):
    """The same passes in one cooperative kernel give the graph run's fields
    bit for bit: both inline the same pass code, whose every product, sum and
    fused multiply-add is an explicitly rounded operation (no contraction
    left to the compiler), on the same schedule."""
    from paper_2005_00322_gb300 import Solver
    a = Solver(ncells, DX, bcs, cfl=0.2)
    b = Solver(ncells, DX, bcs, cfl=0.2, persistent=True)
    assert b.persistent()[0], b.schedule()
    p0 = torch.tensor(inputs.random_field(a.shapes[0], 9).astype(np.float32), device="cuda")
    pa, ua = p0.clone(), [torch.zeros(s, device="cuda") for s in a.shapes[1:]]
    pb, ub = p0.clone(), [torch.zeros(s, device="cuda") for s in b.shapes[1:]]
    a.run(pa, ua, 45)
    b.run(pb, ub, 45)
    # one cooperative kernel, plus the velocity conversions around it
    assert b.last_launch_count() == 1 + 2 * sum(1 for sc in b.schedule() if sc[0] >= 0)
    a.sync()
    b.sync()
    assert [sc[:2] for sc in b.schedule()] == [sc[:2] for sc in a.schedule()]
    assert torch.equal(pb, pa)
    assert all(torch.equal(y, x) for x, y in zip(ua, ub))
    a.close()
    b.close()


def test_stalled_barrier_reports_timeout_and_context_survives():
    """A barrier that cannot complete (one arrival withheld) gives up after the
    poll limit: pstd_sync reports PSTD_ETIMEOUT once, and the GPU stays usable."""
    from paper_2005_00322_gb300 import Solver
    from paper_2005_00322_gb300._abi import PstdError
    ncells, bcs = (256, 256), [("D", "N"), ("N", "N")]
    s = Solver(ncells, DX, bcs, cfl=0.2, persistent=True, spin_limit=1000, withhold_arrivals=1)
    assert s.persistent()[0]
    p, us = s.zeros()
    p.copy_(torch.tensor(inputs.random_field(s.shapes[0], 1).astype(np.float32)))
    s.run(p, us, 10)
    with pytest.raises(PstdError, match="ETIMEOUT"):
        s.sync()
    s.sync()                                     # the status was reported once and cleared
    s.step(p, us)                                # the per-axis kernels still run
    s.sync()
    ok = Solver(ncells, DX, bcs, cfl=0.2, persistent=True)
    q, vs = ok.zeros()
    q.copy_(p)
    ok.run(q, vs, 3)
    ok.sync()
    assert torch.isfinite(q).all()
    s.close()
    ok.close()
