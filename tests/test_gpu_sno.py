"""GPU parity of the learned spectral operator: its kernels against numpy, the
whole network's forward and backward against the FP64 oracle, training, and
the fallback to the solver."""
import ctypes

import numpy as np
import pytest
import torch

from oracle import sno as osno
from paper_2005_00322_gb300 import _abi, inputs

pytestmark = pytest.mark.gpu

DX = 1e-4


def _dev(a):
    return torch.tensor(np.asarray(a, np.float32), device="cuda")


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


@pytest.fixture(scope="module")
def lib():
    return _abi.load()


def _strided(rng, batch, rows, cols, layout):
    """A (batch, rows, cols) operand stored in one of several layouts; returns
    (storage, (s_batch, s_row, s_col), logical array)."""
    X = rng.standard_normal((batch, rows, cols)).astype(np.float32)
    if layout == "row":
        st = X.copy()
        return st.ravel(), (rows * cols, cols, 1), X
    if layout == "col":
        st = np.ascontiguousarray(X.transpose(0, 2, 1))
        return st.ravel(), (rows * cols, 1, rows), X
    # batch innermost: element (b, r, c) at b + r * batch * cols + c * batch
    st = np.ascontiguousarray(X.transpose(1, 2, 0))
    return st.ravel(), (1, cols * batch, batch), X


@pytest.mark.parametrize("M,N,K,batch,la,lb,lc,beta", [
    (70, 130, 37, 3, "row", "row", "row", 0.0),
    (64, 64, 16, 1, "col", "row", "row", 0.0),
    (5, 200, 1, 2, "row", "col", "col", 1.0),
    (129, 16, 127, 4, "row", "col", "row", 0.0),
    (32, 33, 300, 5, "inner", "inner", "inner", 1.0),
    (1, 1, 1, 1, "row", "row", "row", 0.0),
    (17, 9, 0, 2, "row", "row", "row", 1.0),
])
def test_gemm_strided(lib, M, N, K, batch, la, lb, lc, beta):
    rng = np.random.default_rng(M * 1000 + N + K)
    a, sa, A = _strided(rng, batch, M, K, la)
    b, sb, B = _strided(rng, batch, K, N, lb)
    c, sc, C0 = _strided(rng, batch, M, N, lc)
    ta, tb, tc = _dev(a), _dev(b), _dev(c)
    d = _abi.PstdGemmDesc(batch, M, N, K, ta.data_ptr(), *sa, tb.data_ptr(), *sb, tc.data_ptr(), *sc, 0.75, beta)
    assert lib.pstd_nn_gemm(ctypes.byref(d), None) == 0
    torch.cuda.synchronize()
    ref = 0.75 * np.einsum("bmk,bkn->bmn", A.astype(np.float64), B.astype(np.float64)) + beta * C0
    got = tc.cpu().numpy()
    # read back through the same layout
    if lc == "row":
        got = got.reshape(batch, M, N)
    elif lc == "col":
        got = got.reshape(batch, N, M).transpose(0, 2, 1)
    else:
        got = got.reshape(M, N, batch).transpose(2, 0, 1)
    tol = 1e-5 * max(1.0, np.sqrt(K)) * (np.abs(ref).max() + 1)
    np.testing.assert_allclose(got, ref, atol=tol)


@pytest.mark.parametrize("K,Lc", [(300, 112), (1000, 256), (40, 16), (17, 64)])
def test_gemm_split_reduction(lib, K, Lc):
    """Second batch level: chunk c of the reduction into its own output; the
    chunks sum to the whole product, the last one using K_last."""
    rng = np.random.default_rng(K)
    batch, M, N = 3, 33, 20
    A = rng.standard_normal((batch, M, K)).astype(np.float32)
    B = rng.standard_normal((batch, N, K)).astype(np.float32)       # used transposed: B[b]^T
    S = -(-K // Lc)
    ta, tb = _dev(A), _dev(B)
    out = torch.full((S, batch, M, N), float("nan"), device="cuda")
    d = _abi.PstdGemmDesc(batch, M, N, min(Lc, K), ta.data_ptr(), M * K, K, 1, tb.data_ptr(), N * K, 1, K,
                          out.data_ptr(), M * N, N, 1, 1.0, 0.0, S, Lc, Lc, batch * M * N, K - (S - 1) * Lc)
    assert lib.pstd_nn_gemm(ctypes.byref(d), None) == 0
    got = out.cpu().numpy().astype(np.float64)
    for c in range(S):
        ref = np.einsum("bmk,bnk->bmn", A[:, :, c * Lc:(c + 1) * Lc].astype(np.float64),
                        B[:, :, c * Lc:(c + 1) * Lc].astype(np.float64))
        np.testing.assert_allclose(got[c], ref, atol=1e-4 * np.sqrt(Lc))
    if S > 1:                                   # K_last only matters with a second level
        d.K_last = Lc + 1
        assert lib.pstd_nn_gemm(ctypes.byref(d), None) == -1


@pytest.mark.parametrize("M,N,K,batch,la,lb,lc,beta", [
    (70, 130, 37, 3, "row", "row", "row", 0.0),
    (128, 64, 32, 1, "col", "row", "row", 0.0),
    (5, 200, 1, 2, "row", "col", "col", 1.0),
    (129, 16, 127, 4, "row", "col", "row", 0.0),
    (32, 33, 300, 5, "inner", "inner", "inner", 1.0),
    (300, 100, 77, 2, "col", "row", "row", 0.0),
    (17, 9, 0, 2, "row", "row", "row", 1.0),
])
def test_gemm_tf32_tensor_cores(lib, M, N, K, batch, la, lb, lc, beta):
    """The tcgen05 GEMM (TF32 operands, FP32 accumulation in tensor memory)
    against FP64 numpy: each product carries at most 2 x 2^-11 relative error
    from the two roundings to TF32, so the sum of K products is off by at most
    about 2^-10 sqrt(K) max|a b| for random operands."""
    rng = np.random.default_rng(M * 1000 + N + K)
    a, sa, A = _strided(rng, batch, M, K, la)
    b, sb, B = _strided(rng, batch, K, N, lb)
    c, sc, C0 = _strided(rng, batch, M, N, lc)
    ta, tb, tc = _dev(a), _dev(b), _dev(c)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    d = _abi.PstdGemmDesc(batch, M, N, K, ta.data_ptr(), *sa, tb.data_ptr(), *sb, tc.data_ptr(), *sc, 0.75, beta)
    assert lib.pstd_nn_gemm_tf32(ctypes.byref(d), _p(status), None) == 0
    torch.cuda.synchronize()
    assert status.item() == 0
    ref = 0.75 * np.einsum("bmk,bkn->bmn", A.astype(np.float64), B.astype(np.float64)) + beta * C0
    got = tc.cpu().numpy()
    if lc == "row":
        got = got.reshape(batch, M, N)
    elif lc == "col":
        got = got.reshape(batch, N, M).transpose(0, 2, 1)
    else:
        got = got.reshape(M, N, batch).transpose(2, 0, 1)
    amax = np.abs(A).max() if K else 0.0
    bmax = np.abs(B).max() if K else 0.0
    tol = 0.75 * 2.0 ** -10 * 4.0 * np.sqrt(max(K, 1)) * amax * bmax + 1e-6 * (np.abs(ref).max() + 1)
    np.testing.assert_allclose(got, ref, atol=tol)
    d.batch = 0
    assert lib.pstd_nn_gemm_tf32(ctypes.byref(d), None, None) == -1


def test_gemm_rejects_bad_args(lib):
    t = torch.zeros(4, device="cuda")
    d = _abi.PstdGemmDesc(0, 1, 1, 1, t.data_ptr(), 0, 1, 1, t.data_ptr(), 0, 1, 1, t.data_ptr(), 0, 1, 1, 1.0, 0.0)
    assert lib.pstd_nn_gemm(ctypes.byref(d), None) == -1
    d.batch, d.M = 1, -1
    assert lib.pstd_nn_gemm(ctypes.byref(d), None) == -1
    d.M = 1
    d.batch = 70000
    assert lib.pstd_nn_gemm(ctypes.byref(d), None) == -1
    d.batch, d.A = 1, None
    assert lib.pstd_nn_gemm(ctypes.byref(d), None) == -1


def test_elementwise_kernels(lib):
    rng = np.random.default_rng(5)
    B, C, P = 3, 5, 1001
    x = rng.standard_normal((B, C, P))
    y = rng.standard_normal((B, C, P))
    bias = rng.standard_normal(C)
    w = rng.standard_normal(C)
    p = rng.standard_normal((B, P))
    tx, ty, tb, tw, tp = map(_dev, (x, y, bias, w, p))
    o = torch.empty_like(tx)
    assert lib.pstd_nn_bias_act(_p(tx), _p(tb), _p(o), B, C, P, 1, None) == 0
    np.testing.assert_allclose(o.cpu().numpy(), np.maximum(x + bias[None, :, None], 0), atol=1e-6)
    assert lib.pstd_nn_bias_act(_p(tx), None, _p(o), B, C, P, 0, None) == 0
    np.testing.assert_allclose(o.cpu().numpy(), x, atol=0)
    assert lib.pstd_nn_act_bwd(_p(ty), _p(tx), _p(o), B * C * P, 1, None) == 0
    np.testing.assert_allclose(o.cpu().numpy(), y * (x.astype(np.float32) > 0), atol=0)
    assert lib.pstd_nn_lift(_p(tp), _p(tw), _p(tb), _p(o), B, C, P, None) == 0
    np.testing.assert_allclose(o.cpu().numpy(), w[None, :, None] * p[:, None] + bias[None, :, None], atol=1e-5)
    out = torch.empty(B, P, device="cuda")
    b1 = _dev([0.3])
    assert lib.pstd_nn_proj(_p(tx), _p(tw), _p(b1), _p(out), B, C, P, None) == 0
    np.testing.assert_allclose(out.cpu().numpy(), np.einsum("c,bcp->bp", w, x) + 0.3, atol=1e-5)
    assert lib.pstd_nn_proj_bwd(_p(tp), _p(tw), _p(o), B, C, P, None) == 0
    np.testing.assert_allclose(o.cpu().numpy(), w[None, :, None] * p[:, None], atol=1e-6)
    g = torch.empty(C, device="cuda")
    assert lib.pstd_nn_chan_dot(_p(tx), _p(ty), 1, _p(g), B, C, P, None) == 0
    np.testing.assert_allclose(g.cpu().numpy(), np.einsum("bcp,bcp->c", x, y), rtol=1e-5, atol=1e-4)
    assert lib.pstd_nn_chan_dot(_p(tx), _p(tp), 0, _p(g), B, C, P, None) == 0
    np.testing.assert_allclose(g.cpu().numpy(), np.einsum("bcp,bp->c", x, p), rtol=1e-5, atol=1e-4)
    assert lib.pstd_nn_chan_dot(_p(tx), None, 0, _p(g), B, C, P, None) == 0
    np.testing.assert_allclose(g.cpu().numpy(), x.sum(axis=(0, 2)), rtol=1e-5, atol=1e-4)
    s = torch.empty(C * P, device="cuda")
    assert lib.pstd_nn_sum_lead(_p(tx), _p(s), B, C * P, None) == 0
    np.testing.assert_allclose(s.cpu().numpy(), x.reshape(B, -1).sum(0), atol=1e-5)
    # mse and its gradient
    loss = torch.empty(1, device="cuda")
    d = torch.empty_like(tx)
    assert lib.pstd_nn_mse(_p(tx), _p(ty), _p(d), _p(loss), tx.numel(), None) == 0
    x32, y32 = x.astype(np.float32).astype(np.float64), y.astype(np.float32).astype(np.float64)
    np.testing.assert_allclose(loss.item(), np.mean((x32 - y32) ** 2), rtol=1e-6)
    np.testing.assert_allclose(d.cpu().numpy(), 2 * (x32 - y32) / x.size, rtol=1e-5, atol=1e-12)
    # per-sample relative error
    e = torch.empty(B, device="cuda")
    assert lib.pstd_nn_rel_err(_p(tx), _p(ty), _p(e), B, C * P, None) == 0
    ref = np.linalg.norm((x32 - y32).reshape(B, -1), axis=1) / np.linalg.norm(y32.reshape(B, -1), axis=1)
    np.testing.assert_allclose(e.cpu().numpy(), ref, rtol=1e-6)
    # bf16 rounding: nearest representable, ties to even
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -9, -3.14159, 1e-30, 65504.0], np.float32)
    tv = _dev(vals)
    r = torch.empty_like(tv)
    assert lib.pstd_nn_round_bf16(_p(tv), _p(r), vals.size, None) == 0
    np.testing.assert_array_equal(r.cpu().numpy(), tv.to(torch.bfloat16).float().cpu().numpy())
    assert r[1].item() == 1.0 and r[2].item() == 1.0 + 2 ** -6   # ties to even
    # per-sample rms and scaling
    rms = torch.empty(B, device="cuda")
    assert lib.pstd_nn_row_rms(_p(tp), _p(rms), B, P, None) == 0
    p32 = p.astype(np.float32).astype(np.float64)
    np.testing.assert_allclose(rms.cpu().numpy(), np.sqrt((p32 ** 2).mean(1)), rtol=1e-6)
    q = torch.empty_like(tp)
    assert lib.pstd_nn_row_scale(_p(tp), _p(rms), _p(q), B, P, 0, None) == 0
    np.testing.assert_allclose(q.cpu().numpy(), p32 / np.sqrt((p32 ** 2).mean(1))[:, None], rtol=1e-6)
    assert lib.pstd_nn_row_scale(_p(q), _p(rms), _p(q), B, P, 1, None) == 0
    np.testing.assert_allclose(q.cpu().numpy(), p32, rtol=1e-6, atol=1e-7)
    zero = torch.zeros(B, device="cuda")
    assert lib.pstd_nn_row_scale(_p(tp), _p(zero), _p(q), B, P, 0, None) == 0
    assert torch.count_nonzero(q).item() == 0
    assert lib.pstd_nn_bias_act(_p(tx), None, _p(o), B, C, P, 2, None) == -1
    assert lib.pstd_nn_mse(None, _p(ty), None, _p(loss), 4, None) == -1


def test_adam_matches_definition(lib):
    rng = np.random.default_rng(9)
    n = 777
    w, g = rng.standard_normal(n), rng.standard_normal(n)
    m, v = rng.standard_normal(n) * 0.1, np.abs(rng.standard_normal(n)) * 0.01
    tw, tg, tm, tv = map(_dev, (w, g, m, v))
    lr, b1, b2, eps, t = 1e-2, 0.9, 0.999, 1e-8, 3
    assert lib.pstd_nn_adam(_p(tw), _p(tg), _p(tm), _p(tv), n, lr, b1, b2, eps, t, None) == 0
    # the kernel's operands are FP32: take the same rounded inputs and betas
    w, g, m, v = (np.float32(a).astype(np.float64) for a in (w, g, m, v))
    b1, b2 = float(np.float32(b1)), float(np.float32(b2))
    m1 = b1 * m + (1 - b1) * g
    v1 = b2 * v + (1 - b2) * g * g
    w1 = w - lr * (m1 / (1 - b1 ** t)) / (np.sqrt(v1 / (1 - b2 ** t)) + eps)
    np.testing.assert_allclose(tm.cpu().numpy(), m1, rtol=1e-5, atol=1e-7)
    np.testing.assert_allclose(tv.cpu().numpy(), v1, rtol=1e-5, atol=1e-9)
    np.testing.assert_allclose(tw.cpu().numpy(), w1, rtol=1e-5, atol=1e-6)
    assert lib.pstd_nn_adam(_p(tw), _p(tg), _p(tm), _p(tv), n, lr, b1, b2, eps, 0, None) == -1


def _net_and_oracle(ncells, bc, C, K, L, B, seed):
    from paper_2005_00322_gb300.sno import SpectralOperator
    net = SpectralOperator(ncells, bc, channels=C, modes=K, layers=L, seed=seed)
    prm = osno.init_params(C, K, L, seed)
    rng = np.random.default_rng(seed + 1)
    for l in range(L):                         # non-zero biases exercise their gradients
        prm[f"b{l}"] = 0.1 * rng.standard_normal(C)
    prm["b_lift"] = 0.1 * rng.standard_normal(C)
    prm["b_proj"] = np.array([0.05])
    net.set_params(prm)
    prm = {k: np.asarray(v, np.float32).astype(np.float64) for k, v in prm.items()}
    Tx, Ix = osno.basis(ncells[0], bc[0], K)
    Ty, Iy = osno.basis(ncells[1], bc[1], K)
    p0 = rng.standard_normal((B, Tx.shape[1], Ty.shape[1])).astype(np.float32)
    tgt = rng.standard_normal(p0.shape).astype(np.float32)
    return net, prm, (Tx, Ix, Ty, Iy), p0, tgt


@pytest.mark.parametrize("ncells,bc,C,K,L,B", [
    ((24, 20), (("N", "N"), ("D", "D")), 8, 6, 3, 3),
    ((19, 33), (("N", "D"), ("D", "N")), 6, 5, 2, 2),
    ((128, 128), (("N", "N"), ("D", "D")), 32, 16, 4, 2),    # the learned operator's own size
])
def test_forward_backward_match_oracle(ncells, bc, C, K, L, B):
    """Output, loss and every gradient against the FP64 oracle (FP32 path:
    relative 1e-4 of each tensor's largest entry)."""
    net, prm, bases, p0, tgt = _net_and_oracle(ncells, bc, C, K, L, B, seed=3)
    out_ref, _ = osno.forward(prm, p0.astype(np.float64), *bases, L)
    loss_ref, g_ref = osno.loss_and_grads(prm, p0.astype(np.float64), tgt.astype(np.float64), *bases, L)
    tp, tt = _dev(p0), _dev(tgt)
    out = net.forward(tp).cpu().numpy()
    np.testing.assert_allclose(out, out_ref, atol=1e-4 * np.abs(out_ref).max())
    loss, g = net.loss_and_grads(tp, tt)
    assert abs(loss.item() - loss_ref) <= 1e-4 * loss_ref
    for name, ref in g_ref.items():
        got = g[name].cpu().numpy().reshape(ref.shape)
        np.testing.assert_allclose(got, ref, atol=1e-4 * np.abs(ref).max(), err_msg=name)


def test_forward_backward_tf32_tensor_cores_match_oracle():
    """The learned operator with every GEMM on the tensor cores (TF32
    operands) at its own size: output and gradients within 1% of each
    tensor's largest entry of the FP64 oracle."""
    ncells, bc, C, K, L, B = (128, 128), (("N", "N"), ("D", "D")), 32, 16, 4, 2
    net, prm, bases, p0, tgt = _net_and_oracle(ncells, bc, C, K, L, B, seed=3)
    net.tf32 = True
    out_ref, _ = osno.forward(prm, p0.astype(np.float64), *bases, L)
    _, g_ref = osno.loss_and_grads(prm, p0.astype(np.float64), tgt.astype(np.float64), *bases, L)
    tp, tt = _dev(p0), _dev(tgt)
    out = net.forward(tp).cpu().numpy()
    np.testing.assert_allclose(out, out_ref, atol=1e-2 * np.abs(out_ref).max())
    _, g = net.loss_and_grads(tp, tt)
    for name, ref in g_ref.items():
        got = g[name].cpu().numpy().reshape(ref.shape)
        np.testing.assert_allclose(got, ref, atol=1e-2 * np.abs(ref).max(), err_msg=name)
    assert net.tensor_core_status() == 0


def test_bf16_weights_close_to_fp32():
    net, prm, bases, p0, _ = _net_and_oracle((40, 40), (("N", "N"), ("D", "D")), 16, 8, 4, 2, seed=4)
    tp = _dev(p0)
    a = net.predict(tp)
    b = net.predict(tp, bf16=True)
    err = net.rel_err(b, a).max().item()
    assert 0 < err < 3e-2


def _dataset(ncells, bc, steps, n, seed):
    from paper_2005_00322_gb300.sno import pstd_reference
    from paper_2005_00322_gb300.solver import stored_node_range
    full = inputs.sno_initial_pressures(n, seed, ncells=ncells, sigma_cells=(0.1 * min(ncells), 0.12 * min(ncells)))
    sl = tuple(slice(stored_node_range(k, b)[0], stored_node_range(k, b)[1] + 1) for k, b in zip(ncells, bc))
    p0 = _dev(full[(slice(None),) + sl])
    return p0, pstd_reference(ncells, bc, DX, 0.3, steps, p0)


def test_pstd_reference_matches_solver():
    """The batched data generator gives each sample the single-plan answer."""
    from paper_2005_00322_gb300 import Solver
    ncells, bc = (32, 28), (("N", "N"), ("D", "D"))
    p0, ref = _dataset(ncells, bc, 40, 3, seed=11)
    s = Solver(ncells, DX, bc, cfl=0.3)
    for i in range(3):
        p = p0[i].clone()
        _, us = s.zeros()
        s.init_velocity(p, us)
        s.run(p, us, 40)
        torch.cuda.synchronize()
        assert torch.equal(p, ref[i])


def test_training_reduces_loss_and_fallback():
    """Adam on solver-generated data lowers the loss; the surrogate answers with
    PSTD (bit for bit) until the network passes the held-out check, and an
    audit above the tolerance sends it back to PSTD."""
    from paper_2005_00322_gb300.sno import SpectralOperator, Surrogate, pstd_reference
    ncells, bc, steps = (32, 32), (("N", "N"), ("D", "D")), 30
    p0, tgt = _dataset(ncells, bc, steps, 96, seed=21)
    net = SpectralOperator(ncells, bc, channels=8, modes=10, layers=2, seed=0)
    losses = net.train(p0[:80], tgt[:80], iters=300, batch=16, lr=3e-3)
    assert np.mean(losses[-20:]) < 0.2 * np.mean(losses[:5])
    sur = Surrogate(net, DX, 0.3, steps, tol=1e-12, audit_every=1)
    err = sur.validate(p0[80:], tgt[80:])
    assert err > 1e-12 and not sur.trusted
    out = sur(p0[80:88].contiguous())
    assert sur.last_source == "pstd" and torch.equal(out, pstd_reference(ncells, bc, DX, 0.3, steps, p0[80:88].contiguous()))
    sur.tol = 1e9
    assert sur.validate(p0[80:], tgt[80:]) == err and sur.trusted
    out = sur(p0[80:88].contiguous())
    assert sur.last_source == "network" and torch.equal(out, net.predict(p0[80:88].contiguous()))
    sur.tol = 1e-12                              # the next audit fails
    out = sur(p0[80:88].contiguous())
    assert sur.last_source == "pstd" and not sur.trusted and len(sur.audits) == 2
    assert torch.equal(out, tgt[80:88])


def test_learned_operator_on_configured_inputs():
    """The configured workload: 128^2 NN / DD box, 200 steps, inputs of 1-6
    blobs with sigma U[2, 8] dx; trained on 20k PSTD answers (seed 1), gated on
    512 held-out samples (seed 3), scored on the 1k test set (seed 2).

    A 16-mode network cannot carry an input's content above the 16th mode, so
    on this distribution it is within 1e-2 of PSTD only for its smooth end.
    Asserted: the gated pipeline answers every test sample within 1e-2 of PSTD
    (the network where the gate admits the input, PSTD bit for bit elsewhere);
    on the smooth end of the distribution (single blobs of sigma 7.5-8 dx) the
    gate admits at least a quarter of the inputs, every answer is within 1e-2,
    and the network gives at least 3x the predictions/s of 200 batched PSTD
    steps."""
    from paper_2005_00322_gb300.sno import PstdRunner, SpectralOperator, Surrogate
    from paper_2005_00322_gb300.solver import stored_node_range
    w = inputs.plane128_nn_dd()
    ncells, bc = w.ncells, w.bc
    sl = tuple(slice(stored_node_range(k, b)[0], stored_node_range(k, b)[1] + 1) for k, b in zip(ncells, bc))
    runner = PstdRunner(ncells, bc, w.dx, w.cfl, w.steps)

    def dataset(n, seed, **kw):
        p0 = _dev(inputs.sno_initial_pressures(n, seed, ncells=ncells, **kw)[(slice(None),) + sl])
        return p0, runner(p0)
    p_tr, t_tr = dataset(20000, 1)
    p_te, t_te = dataset(1024, 2)
    p_ho, t_ho = dataset(512, 3)
    net = SpectralOperator(ncells, bc, channels=32, modes=16, layers=4, seed=0)
    net.train(p_tr, t_tr, iters=12000, batch=32, lr=2e-3)
    sur = Surrogate(net, w.dx, w.cfl, w.steps, tol=1e-2)
    sur.validate(p_ho, t_ho)

    # the whole configured test set: every answer within the tolerance
    out = torch.cat([sur(p_te[i:i + 256].contiguous()) for i in range(0, 1024, 256)])
    assert net.rel_err(out, t_te).max().item() <= 1e-2
    admitted = (net.high_mode_fraction(p_te) < sur.gate).cpu().numpy()
    rest = np.nonzero(~admitted)[0]
    assert torch.equal(out[rest], t_te[rest])
    net_err = net.rel_err(net.predict(p_te), t_te).cpu().numpy()
    print(f"configured test set: network within 1e-2 for {(net_err <= 1e-2).mean():.3f}, median error "
          f"{np.median(net_err):.3g}; gate {sur.gate:.3g} admits {admitted.mean():.3f}")

    # the smooth end of the configured distribution (single blobs of sigma
    # 7.5-8 dx, whose share above the 16th mode straddles the gate): the
    # network answers a good part of it, every answer within the tolerance
    p_sm, t_sm = dataset(256, 4, sigma_cells=(7.5, 8.0), nblobs=(1, 1))
    out = sur(p_sm)
    assert sur.last_source in ("network", "mixed") and sur.last_routed >= 64
    assert net.rel_err(out, t_sm).max().item() <= 1e-2

    # measured gain on the requests the network answers: predictions/s of the
    # network against the same 200 steps run as batched PSTD (64 members)
    def rate(fn, n, reps=5):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        e1.synchronize()
        return n * reps / (e0.elapsed_time(e1) / 1e3)
    net_rate = rate(lambda: net.predict(p_sm), 256)
    pstd_rate = rate(lambda: runner(p_sm), 256)
    print(f"network {net_rate:.0f}/s, PSTD {pstd_rate:.0f}/s")
    assert net_rate >= 3.0 * pstd_rate
    sur.close()
    runner.close()
