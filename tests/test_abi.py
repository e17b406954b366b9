"""The C-ABI library builds, loads and exports every symbol include/pstd.h declares.

These tests make no compute call: only descriptor validation and static
helpers run, which return before any CUDA work.
"""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2005_00322_gb300 import _abi, build as _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pstd.h")


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return _abi.load()


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pstd_[a-z0-9_]+)\s*\(", text)))


def test_header_declarations_have_bindings():
    syms = declared_symbols()
    assert "pstd_plan" in syms and "pstd_step" in syms and "pstd_run" in syms
    assert set(syms) == set(_abi.SIGNATURES), set(syms) ^ set(_abi.SIGNATURES)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_desc_layout_matches_c():
    # int ndim; int64 ncells[3]; double dx[3]; int bc[3][2]; double c0, rho0, dt; int uinit
    assert _abi.PstdDesc.ncells.offset == 8
    assert _abi.PstdDesc.dx.offset == 32
    assert _abi.PstdDesc.bc.offset == 56
    assert _abi.PstdDesc.c0.offset == 80
    assert _abi.PstdDesc.uinit.offset == 104
    assert ctypes.sizeof(_abi.PstdDesc) == 112


def _plan_rc(lib, **kw):
    args = dict(ncells=(16,), dx=1e-4, bc=[("N", "N")], c0=1500.0, rho0=1000.0,
                dt=0.2e-4 / 1500.0, uinit=0)
    args.update(kw)
    d = _abi.make_desc(args["ncells"], args["dx"], args["bc"], args["c0"], args["rho0"],
                       args["dt"], args["uinit"])
    if "ndim" in kw:
        d.ndim = kw["ndim"]
    h = ctypes.c_void_p()
    rc = lib.pstd_plan(ctypes.byref(d), None, ctypes.byref(h))
    assert not h.value
    return rc


def test_invalid_descriptors_rejected_before_device_work(lib):
    assert _plan_rc(lib, ndim=0) == -1
    assert _plan_rc(lib, ndim=4) == -1
    assert _plan_rc(lib, ncells=(0,)) == -1
    assert _plan_rc(lib, dx=-1.0) == -1
    assert _plan_rc(lib, c0=0.0) == -1
    assert _plan_rc(lib, dt=float("nan")) == -1
    assert _plan_rc(lib, uinit=7) == -1
    assert _plan_rc(lib, bc=[(0, 5)]) == -1
    assert _plan_rc(lib, ncells=(1,), bc=[("D", "D")]) == -1   # no pressure node
    assert _plan_rc(lib, bc=[("P", "N")]) == -1                # periodic needs both walls
    assert _plan_rc(lib, ncells=(1,), bc=[("P", "P")]) == -1


def test_stability_limit_enforced(lib):
    """c0 dt |k|_max / 2 <= 1: 1-D NN keeps k = pi/dx, so CFL 2/pi is the limit."""
    import math
    lim = 2.0 / math.pi
    dx = 1e-4
    assert _plan_rc(lib, dt=1.01 * lim * dx / 1500.0) == -2
    assert _plan_rc(lib, ncells=(16, 16), bc=[("N", "N"), ("N", "N")],
                    dt=1.01 * lim / math.sqrt(2) * dx / 1500.0) == -2


def test_static_helpers(lib):
    assert lib.pstd_dt_from_cfl(0.3, 1e-4, 1500.0) == pytest.approx(0.3e-4 / 1500.0, rel=1e-15)
    assert lib.pstd_strerror(-2).decode().startswith("time step")
    assert b"sm_103a" in lib.pstd_version()
    assert lib.pstd_free(None) == 0
    assert lib.pstd_field_numel(None, 0) == 0


def test_library_is_built_for_sm103a():
    """The build passes exactly one -gencode for sm_103a."""
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_reflection_combos_match_oracle(lib):
    """pstd_reflection_combos (host only) reproduces Section 5's weights."""
    from oracle import reflection
    from paper_2005_00322_gb300.batch import reflection_combos
    for refl in [[(0.0, 0.0)], [(0.0, 0.5)], [(0.4, 0.4), (0.4, 0.4)], [(0.4, -0.2), (1.0, 0.0), (0.3, 0.3)]]:
        bcs, w = reflection_combos((8,) * len(refl), 1e-4, refl)
        ref = reflection.combination_weights(refl)
        assert len(bcs) == len(ref)
        for (b, wv), (rb, rw) in zip(zip(bcs, w), ref):
            assert b == rb
            assert abs(wv - rw) < 1e-15
    _, w = reflection_combos((8,), 1e-4, [(0.0, 0.5)])
    assert w == [0.375, 0.125, 0.375, 0.125]


@pytest.mark.parametrize("bc", [("N", "N"), ("N", "D"), ("D", "N"), ("D", "D")])
def test_sno_basis_matches_oracle(lib, bc):
    """pstd_sno_basis (host, from the mode functions) equals the truncated T1
    pair the oracle builds from the transform matrices of Table 2."""
    from oracle import sno as osno
    code = {"N": _abi.NEUMANN, "D": _abi.DIRICHLET}
    N, K = 37, 12
    T_ref, I_ref = osno.basis(N, bc, K)
    lp = T_ref.shape[1]
    T = (ctypes.c_float * (K * lp))()
    I = (ctypes.c_float * (lp * K))()
    assert lib.pstd_sno_basis(N, code[bc[0]], code[bc[1]], K, T, I) == 0
    T = np.frombuffer(T, dtype=np.float32).reshape(K, lp)
    I = np.frombuffer(I, dtype=np.float32).reshape(lp, K)
    np.testing.assert_allclose(T, T_ref, atol=2e-6)
    np.testing.assert_allclose(I, I_ref, atol=2e-7)
    assert lib.pstd_sno_basis(N, code[bc[0]], code[bc[1]], lp + 1, T.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                              I.ctypes.data_as(ctypes.POINTER(ctypes.c_float))) == -1
    assert lib.pstd_sno_basis(N, _abi.PERIODIC, _abi.PERIODIC, K, None, None) == -1
