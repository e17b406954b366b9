"""FP64 reference of the sine/cosine-basis spectral neural operator (forward and backward).

TEST INFRASTRUCTURE ONLY.  Nothing in the product may import this module.

The paper has no learned component; this network is the project's "learned"
form: it maps an initial pressure on a box to the pressure some fixed number
of leapfrog steps later, trained on data the PSTD solver generates.  It works
in the basis that already satisfies the walls -- the T1 transform of each
axis (Table 2: C1 for a Neumann-Neumann axis, S1 for Dirichlet-Dirichlet, ...),
truncated to the first K modes -- so every layer's spectral part keeps the
boundary conditions.

Architecture (channels C, modes K per axis, layers n_layers):
    v_0 = w_lift * p + b_lift                                   (1 -> C per point)
    v_l = relu( S_l(v_{l-1}) + W_l v_{l-1} + b_l ),  l = 1..n_layers
          S_l(v) = Ix @ [ sum_ci R_l[kx, ky, co, ci] (Tx @ v[ci] @ Ty^T)[kx, ky] ] @ Iy^T
    out = w_proj . v_L + b_proj                                 (C -> 1 per point)
Tx (K x nx): the first K rows of the T1 matrix of axis x; Ix (nx x K): the
first K columns of T1^{-1} = (1/M) partner(T1) (Eq. inverse_transforms).
The last layer has no relu.  Loss: mean squared error.
"""
from __future__ import annotations

import numpy as np

from . import dtt
from .pstd import TABLE2


def basis(n: int, bc: tuple, K: int):
    """(T (K x lp), I (lp x K)): truncated forward and inverse T1 of one axis."""
    T1 = TABLE2[bc][0]
    lp = {"C1": n + 1, "S1": n - 1}.get(T1, n)
    F = dtt.dtt_matrix(T1, lp)
    Inv = dtt.dtt_matrix(dtt.inverse_partner(T1), lp) / dtt.implied_period(T1, lp)
    return F[:K, :], Inv[:, :K]


def init_params(C: int, K: int, n_layers: int, seed: int = 0):
    rng = np.random.default_rng(seed)
    p = {"w_lift": rng.standard_normal(C) * 0.5, "b_lift": np.zeros(C),
         "w_proj": rng.standard_normal(C) / np.sqrt(C), "b_proj": np.zeros(1)}
    for l in range(n_layers):
        p[f"R{l}"] = rng.standard_normal((K, K, C, C)) / C
        p[f"W{l}"] = rng.standard_normal((C, C)) / np.sqrt(C)
        p[f"b{l}"] = np.zeros(C)
    return p


def forward(params, p0, Tx, Ix, Ty, Iy, n_layers):
    """p0: (B, nx, ny).  Returns the output (B, nx, ny) and the cache for backward."""
    v = params["w_lift"][None, :, None, None] * p0[:, None] + params["b_lift"][None, :, None, None]
    cache = {"p0": p0, "v": [v], "pre": []}
    for l in range(n_layers):
        V = np.einsum("kx,bcxy,qy->bckq", Tx, v, Ty)                     # B, C, K, K
        U = np.einsum("kqoi,bikq->bokq", params[f"R{l}"], V)
        s = np.einsum("xk,bokq,yq->boxy", Ix, U, Iy)
        w = np.einsum("oi,bixy->boxy", params[f"W{l}"], v)
        pre = s + w + params[f"b{l}"][None, :, None, None]
        v = np.maximum(pre, 0.0) if l < n_layers - 1 else pre
        cache["V" + str(l)] = V
        cache["pre"].append(pre)
        cache["v"].append(v)
    out = np.einsum("c,bcxy->bxy", params["w_proj"], v) + params["b_proj"][0]
    return out, cache


def loss_and_grads(params, p0, target, Tx, Ix, Ty, Iy, n_layers):
    """Mean squared error and its gradient with respect to every parameter."""
    out, cache = forward(params, p0, Tx, Ix, Ty, Iy, n_layers)
    diff = out - target
    loss = float(np.mean(diff ** 2))
    g = {}
    dout = 2.0 * diff / diff.size
    vL = cache["v"][-1]
    g["w_proj"] = np.einsum("bxy,bcxy->c", dout, vL)
    g["b_proj"] = np.array([dout.sum()])
    dv = params["w_proj"][None, :, None, None] * dout[:, None]
    for l in reversed(range(n_layers)):
        pre = cache["pre"][l]
        dpre = dv * (pre > 0) if l < n_layers - 1 else dv
        vin = cache["v"][l]
        g[f"b{l}"] = dpre.sum(axis=(0, 2, 3))
        g[f"W{l}"] = np.einsum("boxy,bixy->oi", dpre, vin)
        dv_in = np.einsum("oi,boxy->bixy", params[f"W{l}"], dpre)
        dU = np.einsum("xk,boxy,yq->bokq", Ix, dpre, Iy)                  # adjoint of the inverse
        g[f"R{l}"] = np.einsum("bokq,bikq->kqoi", dU, cache["V" + str(l)])
        dV = np.einsum("kqoi,bokq->bikq", params[f"R{l}"], dU)
        dv_in += np.einsum("kx,bikq,qy->bixy", Tx, dV, Ty)               # adjoint of the forward
        dv = dv_in
    g["w_lift"] = np.einsum("bcxy,bxy->c", dv, cache["p0"])
    g["b_lift"] = dv.sum(axis=(0, 2, 3))
    return loss, g
