"""Batched runs and reflection-coefficient combinations (marshalling only).

``Batch`` wraps pstd_batch_*: independent simulations advanced together, one
CUDA graph branch per member.  ``ReflectionRun`` builds the 4^d wall
combinations of Section 5 for given reflection coefficients and returns their
weighted sum on the full node lattice.
"""
from __future__ import annotations

import ctypes

import torch

from . import _abi


def reflection_combos(ncells, dx, refl, c0=1500.0, rho0=1000.0, dt=1.0, uinit=0):
    """(list of per-axis bc tuples, list of weights) of Section 5 (host only).

    refl: per axis (R_left, R_right).  Order: axis 0 slowest, per axis
    NN, ND, DN, DD.
    """
    lib = _abi.load()
    d = len(ncells)
    tmpl = _abi.make_desc(ncells, dx, [("N", "N")] * d, c0, rho0, dt, uinit)
    n = 4 ** d
    descs = (_abi.PstdDesc * n)()
    w = (ctypes.c_double * n)()
    r = (ctypes.c_double * (2 * d))(*[float(x) for pair in refl for x in pair])
    _abi.check(lib, lib.pstd_reflection_combos(ctypes.byref(tmpl), r, descs, w), "pstd_reflection_combos")
    name = {_abi.NEUMANN: "N", _abi.DIRICHLET: "D"}
    bcs = [tuple((name[descs[c].bc[i][0]], name[descs[c].bc[i][1]]) for i in range(d)) for c in range(n)]
    return bcs, [w[c] for c in range(n)]


class Batch:
    """Independent simulations on one GPU, advanced together.

    members: list of dicts with keys ncells, dx, bc and dt (or cfl), optional
    c0, rho0, uinit ("halfstep" / "as_given").
    """

    def __init__(self, members, device=None, stream=None):
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the PSTD library runs on the GPU only")
        self.lib = _abi.load()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None
                                   else torch.device(device).index)
        n = len(members)
        descs = (_abi.PstdDesc * n)()
        self.members = []
        for m, spec in enumerate(members):
            ncells = tuple(spec["ncells"])
            dx = spec["dx"]
            c0 = spec.get("c0", 1500.0)
            dxs = list(dx) if hasattr(dx, "__len__") else [dx] * len(ncells)
            dt = spec.get("dt") or self.lib.pstd_dt_from_cfl(float(spec["cfl"]), float(min(dxs)), float(c0))
            uinit = {"halfstep": _abi.U_HALFSTEP, "as_given": _abi.U_AS_GIVEN}[spec.get("uinit", "halfstep")]
            descs[m] = _abi.make_desc(ncells, dxs, spec["bc"], c0, spec.get("rho0", 1000.0), dt, uinit)
            self.members.append(dict(ncells=ncells, bc=tuple(tuple(b) for b in spec["bc"]), dt=dt))
        self._descs = descs
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        h = ctypes.c_void_p()
        rc = self.lib.pstd_batch_plan(descs, n, ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        _abi.check(self.lib, rc, "pstd_batch_plan")
        self._h = h
        self.n = n
        self.shapes = []
        for m in range(n):
            ph = ctypes.c_void_p()
            _abi.check(self.lib, self.lib.pstd_batch_member(self._h, m, ctypes.byref(ph)), "pstd_batch_member")
            d = len(self.members[m]["ncells"])
            sh = []
            for f in range(d + 1):
                s = (ctypes.c_int64 * 3)()
                _abi.check(self.lib, self.lib.pstd_field_shape(ph, f, s), "pstd_field_shape")
                sh.append(tuple(int(s[i]) for i in range(d)))
            self.shapes.append(sh)

    def zeros(self):
        """Per member (p, [u...]) zero-filled on the device."""
        out = []
        for sh in self.shapes:
            p = torch.zeros(sh[0], dtype=torch.float32, device=self.device)
            out.append((p, [torch.zeros(s, dtype=torch.float32, device=self.device) for s in sh[1:]]))
        return out

    def _ptrs(self, fields):
        if len(fields) != self.n:
            raise ValueError(f"expected {self.n} members")
        P = (ctypes.c_void_p * self.n)()
        U = (ctypes.c_void_p * (3 * self.n))()
        for m, (p, us) in enumerate(fields):
            sh = self.shapes[m]
            for t, want in [(p, sh[0])] + list(zip(us, sh[1:])):
                if (t.device != self.device or t.dtype != torch.float32 or not t.is_contiguous()
                        or tuple(t.shape) != want):
                    raise ValueError(f"member {m}: expected a contiguous float32 {want} tensor on {self.device}")
            P[m] = p.data_ptr()
            for a, u in enumerate(us):
                U[3 * m + a] = u.data_ptr()
        return P, U

    def _enter(self):
        self.stream.wait_stream(torch.cuda.current_stream(self.device))

    def _leave(self):
        torch.cuda.current_stream(self.device).wait_stream(self.stream)

    def init_velocity(self, fields):
        P, U = self._ptrs(fields)
        self._enter()
        _abi.check(self.lib, self.lib.pstd_batch_init_velocity(self._h, P, U), "pstd_batch_init_velocity")
        self._leave()

    def run(self, fields, nsteps: int):
        P, U = self._ptrs(fields)
        self._enter()
        _abi.check(self.lib, self.lib.pstd_batch_run(self._h, P, U, int(nsteps)), "pstd_batch_run")
        self._leave()

    def combine(self, weights, fields, out=None):
        """sum_m w_m p_m on the full node lattice (all members share ncells)."""
        P, _ = self._ptrs(fields)
        full = tuple(n + 1 for n in self.members[0]["ncells"])
        if out is None:
            out = torch.empty(full, dtype=torch.float32, device=self.device)
        w = (ctypes.c_double * self.n)(*[float(x) for x in weights])
        self._enter()
        _abi.check(self.lib, self.lib.pstd_batch_combine(self._h, w, P, ctypes.c_void_p(out.data_ptr())),
                   "pstd_batch_combine")
        self._leave()
        return out

    def last_launch_count(self) -> int:
        return int(self.lib.pstd_batch_last_launch_count(self._h))

    def set_persistent(self, enable=True, spin_limit=0, withhold_arrivals=0):
        """Later runs as one cooperative kernel over all members (pstd_batch_set_persistent)."""
        _abi.check(self.lib, self.lib.pstd_batch_set_persistent(self._h, 1 if enable else 0, int(spin_limit),
                                                                int(withhold_arrivals)),
                   "pstd_batch_set_persistent")

    def persistent_kind(self) -> str:
        """Which cooperative kernel a persistent run uses: "register" or "generic"."""
        k = self.lib.pstd_batch_persistent_kind(self._h)
        return {1: "register", 2: "generic"}.get(k, "none")

    def sync(self):
        """Wait for the batch; raises PstdError (PSTD_ETIMEOUT) if a barrier wait gave up."""
        _abi.check(self.lib, self.lib.pstd_batch_sync(self._h), "pstd_batch_sync")

    def close(self):
        if getattr(self, "_h", None):
            self.lib.pstd_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ReflectionRun:
    """Walls with arbitrary real reflection coefficients (Section 5).

    refl: per axis (R_left, R_right).  Runs the 4^d Neumann/Dirichlet
    combinations as one batch and combines them with the weights of Section 5.
    The combination is valid while t < 2 L / c0 (3 L / c0 when every
    coefficient is zero).
    """

    def __init__(self, ncells, dx, refl, c0=1500.0, rho0=1000.0, dt=None, cfl=None, uinit="halfstep",
                 device=None):
        lib = _abi.load()
        dxs = list(dx) if hasattr(dx, "__len__") else [dx] * len(ncells)
        if dt is None:
            dt = lib.pstd_dt_from_cfl(float(cfl), float(min(dxs)), float(c0))
        self.bcs, self.weights = reflection_combos(ncells, dxs, refl, c0, rho0, dt)
        self.ncells, self.dx, self.c0, self.dt = tuple(ncells), dxs, c0, dt
        zero = all(r == 0.0 for pair in refl for r in pair)
        self.t_valid = (3.0 if zero else 2.0) * min(n * h for n, h in zip(ncells, dxs)) / c0
        self.batch = Batch([dict(ncells=ncells, dx=dxs, bc=b, dt=dt, c0=c0, rho0=rho0, uinit=uinit)
                            for b in self.bcs], device=device)
        self.fields = self.batch.zeros()
        self.steps = 0

    def set_initial_pressure(self, p_full):
        """p0 on the full node lattice (N_i + 1 per axis); velocities start at zero."""
        from .solver import stored_node_range
        p_full = torch.as_tensor(p_full, dtype=torch.float32, device=self.batch.device)
        for (p, us), bc in zip(self.fields, self.bcs):
            sl = tuple(slice(stored_node_range(n, b)[0], stored_node_range(n, b)[1] + 1)
                       for n, b in zip(self.ncells, bc))
            p.copy_(p_full[sl])
            for u in us:
                u.zero_()
        self.batch.init_velocity(self.fields)
        self.steps = 0

    def run(self, nsteps: int):
        if (self.steps + nsteps) * self.dt >= self.t_valid:
            raise ValueError("beyond the validity window of the weighted sum (Section 5)")
        self.batch.run(self.fields, nsteps)
        self.steps += nsteps

    def pressure(self, out=None):
        return self.batch.combine(self.weights, self.fields, out)
