"""Python binding of libpstd.so for torch device tensors (marshalling only).

Every computation runs in the CUDA library; this module checks tensor
arguments, passes raw device pointers and orders the plan's stream against
torch's current stream.  It raises if the library is not built: there is no
CPU path.
"""
from __future__ import annotations

import ctypes

import torch

from . import _abi

_UINIT = {"halfstep": _abi.U_HALFSTEP, "as_given": _abi.U_AS_GIVEN}


def stored_node_range(n: int, bc) -> tuple:
    """(first, last) stored pressure node of an axis: Dirichlet wall nodes are
    dropped; a periodic axis stores nodes 0..N-1, and so does an axis whose
    right wall is at mid-cell ("Nm" / "Dm", x = (N - 1/2) dx)."""
    if bc[0] in ("P", _abi.PERIODIC):
        return 0, n - 1
    lo = 1 if bc[0] in ("D", _abi.DIRICHLET) else 0
    hi = n - 1 if bc[1] in ("D", _abi.DIRICHLET, "Nm", "Dm", _abi.NEUMANN_MID, _abi.DIRICHLET_MID) else n
    return lo, hi


class Solver:
    """A plan of the DTT-PSTD leapfrog on one GPU (see include/pstd.h).

    ncells: cells per axis (1 to 3 axes); dx: spacing (scalar or per axis);
    bc: per axis a (left, right) pair of "N" / "D" / "P", the right wall also
    "Nm" / "Dm" (at mid-cell, Table 1 groups III / IV); dt or cfl (dt = cfl dx / c0
    with the smallest dx); uinit: "halfstep" or "as_given".
    """

    # derivative forms (pstd_plan_opts.form): FFT passes, FP16 hi/lo split
    # dense GEMMs on mma.sync, TF32 hi/lo and BF16 three-way split dense GEMMs
    # on tcgen05
    FORMS = {"fft": 0, "split": 1, "tensor": 2, "split-bf16": 3}

    def __init__(self, ncells, dx, bc, c0=1500.0, rho0=1000.0, dt=None, cfl=None,
                 uinit="halfstep", device=None, stream=None, schedule=None, form="fft",
                 persistent=False, spin_limit=0, withhold_arrivals=0, autotune=False):
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the PSTD library runs on the GPU only")
        self.lib = _abi.load()
        self.device = torch.device(device or "cuda", torch.cuda.current_device()
                                   if device is None else torch.device(device).index)
        self.ndim = len(ncells)
        dxs = list(dx) if hasattr(dx, "__len__") else [dx] * self.ndim
        if dt is None:
            if cfl is None:
                raise ValueError("give dt or cfl")
            dt = self.lib.pstd_dt_from_cfl(float(cfl), float(min(dxs)), float(c0))
        self.ncells, self.dx, self.bc = tuple(ncells), tuple(dxs), tuple(tuple(b) for b in bc)
        self.c0, self.rho0, self.dt = float(c0), float(rho0), float(dt)
        self._desc = _abi.make_desc(ncells, dxs, bc, c0, rho0, dt, _UINIT[uinit])
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        opts = None
        if form not in self.FORMS:
            raise ValueError("form is one of " + ", ".join(repr(f) for f in self.FORMS))
        if schedule is not None or form != "fft" or persistent or withhold_arrivals:
            # schedule: per axis (variant, seqs_per_cta), None entries automatic
            opts = _abi.PstdPlanOpts()
            for i in range(3):
                v, q = (schedule[i] if schedule and i < len(schedule) and schedule[i] else (None, None))
                opts.variant[i] = -1 if v is None else int(v)
                opts.seqs_per_cta[i] = -1 if q is None else int(q)
            opts.form = self.FORMS[form]
            opts.persistent = 1 if persistent else 0
            opts.spin_limit = int(spin_limit)
            opts.withhold_arrivals = int(withhold_arrivals)
        h = ctypes.c_void_p()
        # autotune: the axis-pass schedules are measured on the device (pstd_plan_autotune)
        self.tune_us = None
        if autotune:
            times = (ctypes.c_double * 2)()
            rc = self.lib.pstd_plan_autotune(ctypes.byref(self._desc), ctypes.c_void_p(self.stream.cuda_stream),
                                             ctypes.byref(opts) if opts is not None else None, ctypes.byref(h),
                                             times)
            _abi.check(self.lib, rc, "pstd_plan_autotune")
            self.tune_us = (times[0], times[1])
        else:
            rc = self.lib.pstd_plan_ex(ctypes.byref(self._desc), ctypes.c_void_p(self.stream.cuda_stream),
                                       ctypes.byref(opts) if opts is not None else None, ctypes.byref(h))
            _abi.check(self.lib, rc, "pstd_plan_ex")
        self._h = h
        self.shapes = [self.field_shape(f) for f in range(self.ndim + 1)]

    # -- bookkeeping ---------------------------------------------------------
    def field_shape(self, field: int) -> tuple:
        s = (ctypes.c_int64 * 3)()
        _abi.check(self.lib, self.lib.pstd_field_shape(self._h, field, s), "pstd_field_shape")
        return tuple(int(s[i]) for i in range(self.ndim))

    def zeros(self):
        """Zero-filled (p, [u_1..u_d]) on the device."""
        p = torch.zeros(self.shapes[0], dtype=torch.float32, device=self.device)
        us = [torch.zeros(s, dtype=torch.float32, device=self.device) for s in self.shapes[1:]]
        return p, us

    def restrict(self, p_full):
        """Stored pressure nodes of a field given on the full node lattice."""
        sl = tuple(slice(*(lambda lo, hi: (lo, hi + 1))(*stored_node_range(n, b)))
                   for n, b in zip(self.ncells, self.bc))
        return p_full[sl]

    def schedule(self):
        """Per axis (variant, lanes per sequence, sequences per CTA, CTAs); -1s on the generic path."""
        out = []
        for a in range(self.ndim):
            v = (ctypes.c_int * 4)()
            _abi.check(self.lib, self.lib.pstd_plan_schedule(self._h, a, v), "pstd_plan_schedule")
            out.append(tuple(v))
        return out

    def persistent(self):
        """(enabled, CTAs, threads) of the one-kernel pstd_run."""
        v = (ctypes.c_int * 3)()
        _abi.check(self.lib, self.lib.pstd_plan_persistent(self._h, v), "pstd_plan_persistent")
        return bool(v[0]), int(v[1]), int(v[2])

    def last_launch_count(self) -> int:
        return int(self.lib.pstd_last_launch_count(self._h))

    # -- argument checks -----------------------------------------------------
    def _t(self, x, field: int, name: str):
        if not isinstance(x, torch.Tensor):
            raise TypeError(f"{name} must be a torch tensor")
        if x.device != self.device or x.dtype != torch.float32 or not x.is_contiguous():
            raise ValueError(f"{name} must be a contiguous float32 tensor on {self.device}")
        if tuple(x.shape) != self.shapes[field]:
            raise ValueError(f"{name} has shape {tuple(x.shape)}, expected {self.shapes[field]}")
        return ctypes.c_void_p(x.data_ptr())

    def _us(self, us):
        if len(us) != self.ndim:
            raise ValueError(f"expected {self.ndim} velocity fields")
        arr = (ctypes.c_void_p * 3)()
        for i, u in enumerate(us):
            arr[i] = self._t(u, i + 1, f"u[{i}]")
        return arr

    def _enter(self):
        self.stream.wait_stream(torch.cuda.current_stream(self.device))

    def _leave(self):
        torch.cuda.current_stream(self.device).wait_stream(self.stream)

    # -- the C ABI -----------------------------------------------------------
    def grad(self, axis: int, direction: int, x, out=None):
        """Staggered derivative along ``axis``: direction 0 p -> u_axis, 1 u_axis -> p."""
        fin, fout = (0, axis + 1) if direction == 0 else (axis + 1, 0)
        if out is None:
            out = torch.empty(self.shapes[fout], dtype=torch.float32, device=self.device)
        a, b = self._t(x, fin, "in"), self._t(out, fout, "out")
        self._enter()
        _abi.check(self.lib, self.lib.pstd_grad(self._h, axis, direction, a, b), "pstd_grad")
        self._leave()
        return out

    # field kinds and operations of pstd_apply (plain differentiation and
    # staggered interpolation, Section 3.3)
    KINDS = {"nodes_p": _abi.NODES_P, "half_u": _abi.HALF_U, "nodes_u": _abi.NODES_U, "half_p": _abi.HALF_P}
    OUT_KIND = {("diff", "nodes_p"): "nodes_u", ("diff", "nodes_u"): "nodes_p", ("diff", "half_u"): "half_p",
                ("diff", "half_p"): "half_u", ("interp", "nodes_p"): "half_p", ("interp", "half_p"): "nodes_p",
                ("interp", "nodes_u"): "half_u", ("interp", "half_u"): "nodes_u"}

    def apply_shape(self, axis: int, kind: str) -> tuple:
        s = (ctypes.c_int64 * 3)()
        _abi.check(self.lib, self.lib.pstd_apply_shape(self._h, axis, self.KINDS[kind], s), "pstd_apply_shape")
        return tuple(int(s[i]) for i in range(self.ndim))

    def apply(self, axis: int, op: str, x, kind: str, out=None):
        """Plain derivative (op "diff") or interpolation to the other grid (op
        "interp") along ``axis`` of a field of ``kind``; returns the output."""
        okind = self.OUT_KIND[(op, kind)]
        if out is None:
            out = torch.empty(self.apply_shape(axis, okind), dtype=torch.float32, device=self.device)
        for t, k, name in ((x, kind, "in"), (out, okind, "out")):
            if (not isinstance(t, torch.Tensor) or t.device != self.device or t.dtype != torch.float32
                    or not t.is_contiguous() or tuple(t.shape) != self.apply_shape(axis, k)):
                raise ValueError(f"{name} must be a contiguous float32 {self.apply_shape(axis, k)} tensor")
        self._enter()
        rc = self.lib.pstd_apply(self._h, axis, _abi.OP_DIFF if op == "diff" else _abi.OP_INTERP,
                                 self.KINDS[kind], ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()))
        _abi.check(self.lib, rc, "pstd_apply")
        self._leave()
        return out

    def init_velocity(self, p0, us):
        a, arr = self._t(p0, 0, "p0"), self._us(us)
        self._enter()
        _abi.check(self.lib, self.lib.pstd_init_velocity(self._h, a, arr), "pstd_init_velocity")
        self._leave()

    def step(self, p, us):
        a, arr = self._t(p, 0, "p"), self._us(us)
        self._enter()
        _abi.check(self.lib, self.lib.pstd_step(self._h, a, arr), "pstd_step")
        self._leave()

    def run(self, p, us, nsteps: int):
        a, arr = self._t(p, 0, "p"), self._us(us)
        self._enter()
        _abi.check(self.lib, self.lib.pstd_run(self._h, a, arr, int(nsteps)), "pstd_run")
        self._leave()

    def init_prev(self, p0, p_prev):
        """p^{-1} into ``p_prev`` for the second-order form, from p^0 with zero
        initial velocity (the plan's uinit reading)."""
        a, b = self._t(p0, 0, "p0"), self._t(p_prev, 0, "p_prev")
        self._enter()
        _abi.check(self.lib, self.lib.pstd_init_prev(self._h, a, b), "pstd_init_prev")
        self._leave()

    def run2(self, p, p_prev, nsteps: int):
        """``nsteps`` steps of the second-order pressure-only form in place:
        (p^n, p^{n-1}) -> (p^{n+nsteps}, p^{n+nsteps-1})."""
        a, b = self._t(p, 0, "p"), self._t(p_prev, 0, "p_prev")
        self._enter()
        _abi.check(self.lib, self.lib.pstd_run2(self._h, a, b, int(nsteps)), "pstd_run2")
        self._leave()

    def energy(self, p, u_prev, u_next):
        """FP64 discrete energy E^n of (p^n, u^{n-1/2}, u^{n+1/2}), computed on
        the GPU (pstd_energy)."""
        a, prev, nxt = self._t(p, 0, "p"), self._us(u_prev), self._us(u_next)
        out = ctypes.c_double()
        self._enter()
        _abi.check(self.lib, self.lib.pstd_energy(self._h, a, prev, nxt, ctypes.byref(out)), "pstd_energy")
        return out.value

    def sync(self):
        _abi.check(self.lib, self.lib.pstd_sync(self._h), "pstd_sync")

    def close(self):
        if getattr(self, "_h", None):
            self.lib.pstd_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
