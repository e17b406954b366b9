"""Learned spectral operator for a fixed number of PSTD steps (marshalling only).

Not in the paper: a spectral neural operator that maps an initial pressure on
a 2-D box to the pressure a fixed number of leapfrog steps later, trained on
data the PSTD solver produces.  Its spectral layers work in the truncated T1
basis of each axis (Table 2: C1 for a Neumann pair, S1 for a Dirichlet pair,
C3 / S3 for mixed walls), which already satisfies the walls, and the solver
stays the arbiter: ``Surrogate`` answers with the network only while a held-out
set and sampled per-request audits stay within a relative error tolerance, and
runs PSTD otherwise.

Architecture (channels C, modes K per axis, L layers; field layout
[B][C][X][Y], X and Y the stored pressure nodes of the two axes):
    v_0 = w_lift p + b_lift
    v_l = act_l( Ix [ R_l (Tx v_{l-1} Ty^T) ] Iy^T + W_l v_{l-1} + b_l ),
          R_l mixing channels per mode (kx, ky), act relu except the last layer
    out = w_proj . v_L + b_proj
Every product is one call of the library's strided batched GEMM and every
other step (lift, bias and activation, projection, reductions, loss, Adam) one
of its elementwise kernels; this module only allocates buffers with torch and
passes pointers and strides.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np
import torch

from . import _abi


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class SpectralOperator:
    """The network's parameters and its forward, backward and Adam step on one GPU.

    ncells: (N0, N1) cells; bc: per axis a (left, right) pair of "N" / "D".
    All parameters live in one flat FP32 device buffer (with matching gradient
    and Adam moment buffers); ``params[name]`` are views into it.
    """

    def __init__(self, ncells, bc, channels=32, modes=16, layers=4, seed=0, device=None, normalize=True):
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the learned operator runs on the GPU only")
        if len(ncells) != 2:
            raise ValueError("the learned operator is 2-D")
        self.lib = _abi.load()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None
                                   else torch.device(device).index)
        self.C, self.K, self.L = int(channels), int(modes), int(layers)
        # The propagator is linear: train and predict on p0 / rms(p0) and
        # scale the answer back, so the error does not depend on amplitude.
        self.normalize = bool(normalize)
        self.ncells = tuple(int(n) for n in ncells)
        self.bc = tuple(tuple(b) for b in bc)
        code = {"N": _abi.NEUMANN, "D": _abi.DIRICHLET}
        bases = []
        for n, (l, r) in zip(self.ncells, self.bc):
            lp = n + 1 - (l == "D") - (r == "D")
            T = np.zeros((self.K, lp), np.float32)
            I = np.zeros((lp, self.K), np.float32)
            fp = ctypes.POINTER(ctypes.c_float)
            _abi.check(self.lib, self.lib.pstd_sno_basis(n, code[l], code[r], self.K, T.ctypes.data_as(fp),
                                                         I.ctypes.data_as(fp)), "pstd_sno_basis")
            bases.append((torch.from_numpy(T).to(self.device), torch.from_numpy(I).to(self.device)))
        (self.Tx, self.Ix), (self.Ty, self.Iy) = bases
        self.X, self.Y = self.Tx.shape[1], self.Ty.shape[1]
        C, K = self.C, self.K
        self.shapes = {"w_lift": (C,), "b_lift": (C,), "w_proj": (C,), "b_proj": (1,)}
        for l in range(self.L):
            self.shapes[f"R{l}"] = (K, K, C, C)
            self.shapes[f"W{l}"] = (C, C)
            self.shapes[f"b{l}"] = (C,)
        total = sum(math.prod(s) for s in self.shapes.values())
        z = lambda: torch.zeros(total, dtype=torch.float32, device=self.device)
        self.flat, self.gflat, self.m1, self.m2 = z(), z(), z(), z()
        self.params, self.grads = self._views(self.flat), self._views(self.gflat)
        self.adam_steps = 0
        # tensor-core GEMMs (tcgen05, TF32 operands, FP32 accumulation) when set
        self.tf32 = False
        self._status = torch.zeros(1, dtype=torch.int32, device=self.device)
        self._init(seed)

    # -- parameters ----------------------------------------------------------
    def _views(self, buf):
        out, off = {}, 0
        for name, s in self.shapes.items():
            n = math.prod(s)
            out[name] = buf[off:off + n].view(s)
            off += n
        return out

    def _init(self, seed):
        g = torch.Generator().manual_seed(int(seed))
        C = self.C
        scale = {"w_lift": 0.5, "w_proj": 1.0 / math.sqrt(C)}
        for name, s in self.shapes.items():
            if name[0] == "b":
                continue
            sd = scale.get(name, 1.0 / C if name[0] == "R" else 1.0 / math.sqrt(C))
            self.params[name].copy_(torch.randn(s, generator=g, dtype=torch.float64).float() * sd)

    def set_params(self, values):
        """Copy a {name: array} mapping (the layout of ``shapes``) into the device buffer."""
        for name, s in self.shapes.items():
            self.params[name].copy_(torch.as_tensor(np.asarray(values[name], dtype=np.float32).reshape(s)))
        self.m1.zero_()
        self.m2.zero_()
        self.adam_steps = 0

    def get_params(self):
        return {k: v.detach().cpu().numpy().astype(np.float64) for k, v in self.params.items()}

    def bf16_weights(self):
        """A copy of the parameters rounded to bfloat16 (for inference)."""
        out = torch.empty_like(self.flat)
        self._ck(self.lib.pstd_nn_round_bf16(_ptr(self.flat), _ptr(out), self.flat.numel(), self._s()),
                 "pstd_nn_round_bf16")
        return self._views(out)

    # -- marshalling ---------------------------------------------------------
    def _s(self):
        return ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)

    def _ck(self, rc, what):
        _abi.check(self.lib, rc, what)
        self.launches += 1

    launches = 0

    def _gemm(self, batch, M, N, K, A, sA, B, sB, Cm, sC, beta=0.0, split=None):
        # split: (batch2, sAb2, sBb2, sCb2, K_last) of a chunked reduction
        d = _abi.PstdGemmDesc(batch, M, N, K, A.data_ptr(), *sA, B.data_ptr(), *sB, Cm.data_ptr(), *sC, 1.0, beta,
                              *(split or (1, 0, 0, 0, K)))
        if self.tf32:
            self._ck(self.lib.pstd_nn_gemm_tf32(ctypes.byref(d), _ptr(self._status), self._s()), "pstd_nn_gemm_tf32")
        else:
            self._ck(self.lib.pstd_nn_gemm(ctypes.byref(d), self._s()), "pstd_nn_gemm")

    def tensor_core_status(self) -> int:
        """1 if a bounded wait of a tensor-core GEMM gave up since the last call (reset)."""
        v = int(self._status.item())
        self._status.zero_()
        return v

    def _empty(self, *shape):
        return torch.empty(shape, dtype=torch.float32, device=self.device)

    def _check_field(self, t, name):
        if (not isinstance(t, torch.Tensor) or t.device != self.device or t.dtype != torch.float32
                or not t.is_contiguous() or t.dim() != 3 or tuple(t.shape[1:]) != (self.X, self.Y)):
            raise ValueError(f"{name} must be a contiguous float32 (B, {self.X}, {self.Y}) tensor on {self.device}")

    # -- forward -------------------------------------------------------------
    def forward(self, p0, keep=False, params=None):
        """Network output for p0 (B, X, Y) on the device; with keep=True also the
        activations the backward pass needs."""
        self._check_field(p0, "p0")
        prm = params or self.params
        B, C, K, X, Y = p0.shape[0], self.C, self.K, self.X, self.Y
        P, KK = X * Y, K * K
        if B * C > 65535 or (B * C * X + 127) // 128 > 65535:
            raise ValueError("batch too large for one pass: split it")
        s = self._s()
        v = self._empty(B, C, X, Y)
        self._ck(self.lib.pstd_nn_lift(_ptr(p0), _ptr(prm["w_lift"]), _ptr(prm["b_lift"]), _ptr(v), B, C, P, s),
                 "pstd_nn_lift")
        cache = {"p0": p0, "v": [v], "V": []}
        A1, A2, U = self._empty(B, C, X, K), self._empty(B, C, X, K), self._empty(B, C, K, K)
        Vh = self._empty(B, C, K, K)
        for l in range(self.L):
            if keep:
                Vh = self._empty(B, C, K, K)
            R, W, b = prm[f"R{l}"], prm[f"W{l}"], prm[f"b{l}"]
            # forward transforms: A1 = v Ty^T (rows (b, c, x)), Vh[bc] = Tx A1[bc]
            self._gemm(1, B * C * X, K, Y, v, (0, Y, 1), self.Ty, (0, 1, Y), A1, (0, K, 1))
            self._gemm(B * C, K, K, X, self.Tx, (0, X, 1), A1, (X * K, K, 1), Vh, (KK, K, 1))
            # per-mode channel mixing: U[:, :, q] = R[q] Vh[:, :, q]
            self._gemm(KK, C, B, C, R, (C * C, C, 1), Vh, (1, KK, C * KK), U, (1, KK, C * KK))
            # inverse transforms: A2[bc] = Ix U[bc], pre = A2 Iy^T
            self._gemm(B * C, X, K, K, self.Ix, (0, K, 1), U, (KK, K, 1), A2, (X * K, K, 1))
            vn = self._empty(B, C, X, Y)
            self._gemm(1, B * C * X, Y, K, A2, (0, K, 1), self.Iy, (0, 1, K), vn, (0, Y, 1))
            # pointwise channel mixing, bias, activation
            self._gemm(B, C, P, C, W, (0, C, 1), v, (C * P, P, 1), vn, (C * P, P, 1), beta=1.0)
            act = 1 if l < self.L - 1 else 0
            self._ck(self.lib.pstd_nn_bias_act(_ptr(vn), _ptr(b), _ptr(vn), B, C, P, act, s), "pstd_nn_bias_act")
            if keep:
                cache["V"].append(Vh)
                cache["v"].append(vn)
            v = vn
        out = self._empty(B, X, Y)
        self._ck(self.lib.pstd_nn_proj(_ptr(v), _ptr(prm["w_proj"]), _ptr(prm["b_proj"]), _ptr(out), B, C, P, s),
                 "pstd_nn_proj")
        return (out, cache) if keep else out

    # -- backward ------------------------------------------------------------
    def backward(self, cache, dout):
        """Gradients of sum(dout * out) into ``grads`` (every entry overwritten)."""
        p0 = cache["p0"]
        B, C, K, X, Y = p0.shape[0], self.C, self.K, self.X, self.Y
        P, KK = X * Y, K * K
        s, prm, g = self._s(), self.params, self.grads
        vL = cache["v"][-1]
        self._ck(self.lib.pstd_nn_chan_dot(_ptr(vL), _ptr(dout), 0, _ptr(g["w_proj"]), B, C, P, s), "chan_dot")
        self._ck(self.lib.pstd_nn_chan_dot(_ptr(dout), None, 0, _ptr(g["b_proj"]), B, 1, P, s), "chan_dot")
        dv = self._empty(B, C, X, Y)
        self._ck(self.lib.pstd_nn_proj_bwd(_ptr(dout), _ptr(prm["w_proj"]), _ptr(dv), B, C, P, s), "proj_bwd")
        # chunks of Lc points (a multiple of 16, at most 256) with B * S <= 65535
        Lc = max(-(-P // (65535 // B)), 256 if P >= 4096 else 64)
        Lc = -(-Lc // 16) * 16
        S = -(-P // Lc)
        Wp = self._empty(S, B, C, C)
        dA = self._empty(B, C, X, K)
        dU, dV = self._empty(B, C, K, K), self._empty(B, C, K, K)
        for l in reversed(range(self.L)):
            vin, vout, Vh = cache["v"][l], cache["v"][l + 1], cache["V"][l]
            R, W = prm[f"R{l}"], prm[f"W{l}"]
            if l < self.L - 1:      # relu: pre > 0 exactly where its output is > 0
                self._ck(self.lib.pstd_nn_act_bwd(_ptr(dv), _ptr(vout), _ptr(dv), dv.numel(), 1, s), "act_bwd")
            dpre = dv
            self._ck(self.lib.pstd_nn_chan_dot(_ptr(dpre), None, 0, _ptr(g[f"b{l}"]), B, C, P, s), "chan_dot")
            # dW = sum_b dpre[b] vin[b]^T, its point sum split into S chunks
            # (one GEMM each) so that B * S CTAs share the reduction
            self._gemm(B, C, C, Lc, dpre, (C * P, P, 1), vin, (C * P, 1, P), Wp, (C * C, C, 1),
                       split=(S, Lc, Lc, B * C * C, P - (S - 1) * Lc))
            self._ck(self.lib.pstd_nn_sum_lead(_ptr(Wp), _ptr(g[f"W{l}"]), S * B, C * C, s), "sum_lead")
            dvin = self._empty(B, C, X, Y)
            self._gemm(B, C, P, C, W, (0, 1, C), dpre, (C * P, P, 1), dvin, (C * P, P, 1))
            # adjoint of the inverse transforms: dU[bc] = Ix^T dpre[bc] Iy
            self._gemm(1, B * C * X, K, Y, dpre, (0, Y, 1), self.Iy, (0, K, 1), dA, (0, K, 1))
            self._gemm(B * C, K, K, X, self.Ix, (0, 1, K), dA, (X * K, K, 1), dU, (KK, K, 1))
            # dR[q] = dU[:, :, q] Vh[:, :, q]^T,  dV[:, :, q] = R[q]^T dU[:, :, q]
            self._gemm(KK, C, C, B, dU, (1, KK, C * KK), Vh, (1, C * KK, KK), g[f"R{l}"], (C * C, C, 1))
            self._gemm(KK, C, B, C, R, (C * C, 1, C), dU, (1, KK, C * KK), dV, (1, KK, C * KK))
            # adjoint of the forward transforms: dvin += Tx^T dV[bc] Ty
            self._gemm(B * C, X, K, K, self.Tx, (0, 1, X), dV, (KK, K, 1), dA, (X * K, K, 1))
            self._gemm(1, B * C * X, Y, K, dA, (0, K, 1), self.Ty, (0, Y, 1), dvin, (0, Y, 1), beta=1.0)
            dv = dvin
        self._ck(self.lib.pstd_nn_chan_dot(_ptr(dv), _ptr(p0), 0, _ptr(g["w_lift"]), B, C, P, s), "chan_dot")
        self._ck(self.lib.pstd_nn_chan_dot(_ptr(dv), None, 0, _ptr(g["b_lift"]), B, C, P, s), "chan_dot")
        return g

    def loss_and_grads(self, p0, target):
        """Mean squared error (a 1-element device tensor) and the gradients."""
        self._check_field(target, "target")
        out, cache = self.forward(p0, keep=True)
        dout = torch.empty_like(out)
        loss = self._empty(1)
        self._ck(self.lib.pstd_nn_mse(_ptr(out), _ptr(target), _ptr(dout), _ptr(loss), out.numel(), self._s()),
                 "pstd_nn_mse")
        self.backward(cache, dout)
        return loss, self.grads

    def adam(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.adam_steps += 1
        self._ck(self.lib.pstd_nn_adam(_ptr(self.flat), _ptr(self.gflat), _ptr(self.m1), _ptr(self.m2),
                                       self.flat.numel(), lr, beta1, beta2, eps, self.adam_steps, self._s()),
                 "pstd_nn_adam")

    def _row_scale(self, x, sc, mode, out=None):
        out = torch.empty_like(x) if out is None else out
        self._ck(self.lib.pstd_nn_row_scale(_ptr(x), _ptr(sc), _ptr(out), x.shape[0], x[0].numel(), mode,
                                            self._s()), "pstd_nn_row_scale")
        return out

    def _normalized(self, p0):
        """(p0 / rms per sample, rms)."""
        sc = self._empty(p0.shape[0])
        self._ck(self.lib.pstd_nn_row_rms(_ptr(p0), _ptr(sc), p0.shape[0], p0[0].numel(), self._s()),
                 "pstd_nn_row_rms")
        return self._row_scale(p0, sc, 0), sc

    def train(self, p0s, targets, iters, batch=16, lr=1e-3, seed=0, lr_final=None):
        """Adam on minibatches drawn (seeded) from the device tensors p0s / targets.
        Learning rate decays by cosine from lr to lr_final (default lr / 20).
        Returns the per-iteration losses (host floats)."""
        n = p0s.shape[0]
        rng = np.random.default_rng(seed)
        lr_final = lr / 20 if lr_final is None else lr_final
        losses = torch.empty(iters, dtype=torch.float32, device=self.device)
        for it in range(iters):
            idx = torch.as_tensor(rng.choice(n, size=min(batch, n), replace=False), device=self.device)
            xb, tb = p0s.index_select(0, idx).contiguous(), targets.index_select(0, idx).contiguous()
            if self.normalize:
                xb, sc = self._normalized(xb)
                tb = self._row_scale(tb, sc, 0)
            loss, _ = self.loss_and_grads(xb, tb)
            losses[it:it + 1].copy_(loss)
            a = lr_final + 0.5 * (lr - lr_final) * (1 + math.cos(math.pi * it / max(iters - 1, 1)))
            self.adam(lr=a)
        return losses.cpu().numpy().tolist()

    def predict(self, p0, chunk=256, bf16=False, tf32=None):
        """Network output for any batch size (processed in chunks).  bf16: the
        weights rounded to BF16 (the arithmetic stays FP32); tf32 (default: the
        operator's setting) runs the GEMMs on the tensor cores in TF32."""
        if tf32 is not None and bool(tf32) != self.tf32:
            saved, self.tf32 = self.tf32, bool(tf32)
            try:
                return self.predict(p0, chunk, bf16)
            finally:
                self.tf32 = saved
        prm = self.bf16_weights() if bf16 else None
        outs = []
        for i in range(0, p0.shape[0], chunk):
            x = p0[i:i + chunk].contiguous()
            if self.normalize:
                x, sc = self._normalized(x)
                y = self.forward(x, params=prm)
                outs.append(self._row_scale(y, sc, 1, out=y))
            else:
                outs.append(self.forward(x, params=prm))
        return outs[0] if len(outs) == 1 else torch.cat(outs)

    def high_mode_fraction(self, p0, chunk=256):
        """Per-sample ||p - P_K p|| / ||p|| on the device, P_K = Ix Tx (x) Iy Ty
        the projection onto the first K modes of each axis of the network's
        basis: the part of an input that no K-mode spectral layer carries.  For
        the linear wave propagator it is about the smallest error any such
        network can reach on that input.  Four FP32 GEMMs and a reduction of
        the library per chunk of samples."""
        self._check_field(p0, "p0")
        B, K, X, Y = p0.shape[0], self.K, self.X, self.Y
        out = self._empty(B)
        s = self._s()

        def gemm(batch, M, N, Kd, A, sA, Bm, sB, Cm, sC):
            d = _abi.PstdGemmDesc(batch, M, N, Kd, A.data_ptr(), *sA, Bm.data_ptr(), *sB, Cm.data_ptr(), *sC,
                                  1.0, 0.0, 1, 0, 0, 0, Kd)
            self._ck(self.lib.pstd_nn_gemm(ctypes.byref(d), s), "pstd_nn_gemm")
        for i in range(0, B, chunk):
            x = p0[i:i + chunk].contiguous()
            b = x.shape[0]
            A1, V, A2, low = self._empty(b, X, K), self._empty(b, K, K), self._empty(b, X, K), self._empty(b, X, Y)
            gemm(1, b * X, K, Y, x, (0, Y, 1), self.Ty, (0, 1, Y), A1, (0, K, 1))
            gemm(b, K, K, X, self.Tx, (0, X, 1), A1, (X * K, K, 1), V, (K * K, K, 1))
            gemm(b, X, K, K, self.Ix, (0, K, 1), V, (K * K, K, 1), A2, (X * K, K, 1))
            gemm(1, b * X, Y, K, A2, (0, K, 1), self.Iy, (0, 1, K), low, (0, Y, 1))
            out[i:i + b].copy_(self.rel_err(low, x))
        return out

    def rel_err(self, a, ref):
        """Per-sample ||a - ref|| / ||ref|| on the device (FP64 sums)."""
        err = self._empty(a.shape[0])
        self._ck(self.lib.pstd_nn_rel_err(_ptr(a), _ptr(ref), _ptr(err), a.shape[0], a[0].numel(), self._s()),
                 "pstd_nn_rel_err")
        return err


class PstdRunner:
    """The solver's answers for batches of initial pressures: one batch plan
    of `group` independent members (pstd_batch_*), kept and reused; requests
    run `group` at a time (a short last group is padded with zero fields)."""

    def __init__(self, ncells, bc, dx, cfl, steps, c0=1500.0, rho0=1000.0, group=64, device=None):
        from .batch import Batch
        self.steps, self.group = int(steps), int(group)
        self.batch = Batch([dict(ncells=ncells, dx=dx, bc=bc, cfl=cfl, c0=c0, rho0=rho0)] * self.group,
                           device=device)
        self.fields = self.batch.zeros()

    def __call__(self, p0s):
        out = torch.empty_like(p0s)
        B, n = p0s.shape[0], self.group
        for g0 in range(0, B, n):
            k = min(n, B - g0)
            for m, (p, us) in enumerate(self.fields):
                if m < k:
                    p.copy_(p0s[g0 + m])
                else:
                    p.zero_()
                for u in us:
                    u.zero_()
            self.batch.init_velocity(self.fields)
            self.batch.run(self.fields, self.steps)
            for m in range(k):
                out[g0 + m].copy_(self.fields[m][0])
        return out

    def close(self):
        self.batch.close()


def pstd_reference(ncells, bc, dx, cfl, steps, p0s, c0=1500.0, rho0=1000.0, group=64):
    """The solver's answer for every sample of p0s (B, X, Y): `steps` leapfrog
    steps from zero velocity (half-step rule), `group` samples at a time as one
    batch of independent members."""
    if p0s.shape[0] == 0:
        return torch.empty_like(p0s)
    r = PstdRunner(ncells, bc, dx, cfl, steps, c0, rho0, min(group, p0s.shape[0]), p0s.device)
    try:
        return r(p0s)
    finally:
        r.close()


class Surrogate:
    """The learned operator with the solver as arbiter.

    ``validate`` compares the network with PSTD on a held-out set.  A K-mode
    spectral network cannot carry the part of an input above its K-th mode, so
    each request is gated by that part's share, ``high_mode_fraction`` r: the
    network answers only requests with r below the gate, and PSTD all others.
    The gate is set on the held-out set: walking its samples by increasing r,
    the first whose error exceeds ``safety`` x ``tol`` fixes it at ``margin``
    times that sample's r (no gate if none does), so that the admitted held-out
    samples keep a margin below ``tol``.  The network is trusted while some held-out sample lies below the
    gate.  Every ``audit_every``-th call also runs PSTD on one network-answered
    request and, if its error exceeds ``tol``, answers the call with PSTD and
    stops trusting the network.
    """

    def __init__(self, net: SpectralOperator, dx, cfl, steps, tol=1e-2, audit_every=16, seed=0,
                 c0=1500.0, rho0=1000.0, margin=0.9, safety=0.7):
        self.net, self.dx, self.cfl, self.steps, self.tol = net, dx, cfl, int(steps), float(tol)
        self.c0, self.rho0, self.margin, self.safety = c0, rho0, float(margin), float(safety)
        self._runner = None
        self.audit_every = int(audit_every)
        self.trusted = False
        self.gate = 0.0
        self.routed = 0.0
        self.calls = 0
        self.last_source = None
        self.last_routed = 0
        self.heldout_err = None
        self.audits = []
        self._rng = np.random.default_rng(seed)

    def _pstd(self, p0s):
        if self._runner is None:
            self._runner = PstdRunner(self.net.ncells, self.net.bc, self.dx, self.cfl, self.steps, self.c0,
                                      self.rho0, device=p0s.device)
        return self._runner(p0s)

    def close(self):
        if self._runner is not None:
            self._runner.close()
            self._runner = None

    def validate(self, p0s, targets=None):
        """Held-out check: returns the network's worst relative error on p0s and
        sets the gate and the share of held-out samples it admits."""
        if targets is None:
            targets = self._pstd(p0s)
        err = self.net.rel_err(self.net.predict(p0s), targets).cpu().numpy()
        frac = self.net.high_mode_fraction(p0s).cpu().numpy()
        self.heldout_err = float(err.max())
        bad = frac[err > self.safety * self.tol]
        self.gate = self.margin * float(bad.min()) if bad.size else math.inf
        self.routed = float((frac < self.gate).mean())
        self.trusted = self.routed > 0
        return self.heldout_err

    def __call__(self, p0s):
        self.calls += 1
        if not self.trusted:
            self.last_source, self.last_routed = "pstd", 0
            return self._pstd(p0s)
        if math.isinf(self.gate):
            mask = torch.ones(p0s.shape[0], dtype=torch.bool, device=p0s.device)
        else:
            mask = self.net.high_mode_fraction(p0s) < self.gate
        net_idx = torch.nonzero(mask).flatten()
        n_net = int(net_idx.numel())
        self.last_routed = n_net
        if n_net == 0:
            self.last_source = "pstd"
            return self._pstd(p0s)
        if n_net == p0s.shape[0]:
            out = self.net.predict(p0s)
            net_out, sel = out, net_idx
        else:
            out = torch.empty_like(p0s)
            sel = net_idx
            net_out = self.net.predict(p0s.index_select(0, sel).contiguous())
            out.index_copy_(0, sel, net_out)
            rest = torch.nonzero(~mask).flatten()
            out.index_copy_(0, rest, self._pstd(p0s.index_select(0, rest).contiguous()))
        if self.audit_every > 0 and self.calls % self.audit_every == 0:
            i = int(self._rng.integers(n_net))
            ref = self._pstd(p0s[int(sel[i])].unsqueeze(0).contiguous())
            e = float(self.net.rel_err(net_out[i:i + 1].contiguous(), ref)[0])
            self.audits.append(e)
            if e > self.tol:
                self.trusted = False
                self.last_source, self.last_routed = "pstd", 0
                return self._pstd(p0s)
        self.last_source = "network" if n_net == p0s.shape[0] else "mixed"
        return out
