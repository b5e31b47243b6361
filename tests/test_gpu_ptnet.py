"""GPU parity of the parallel-transport network kernels (forward, backward,
Adam training) against the FP64 oracle, whose gradient is pinned by finite
differences, and of the learned subspace generation with its judge."""
import numpy as np
import pytest
import torch

from oracle.dirac import WilsonClover
from oracle.ptnet import PTNet, init_weights
from paper_0706_2298_gb300 import dwsolve as dw
from paper_0706_2298_gb300 import synth

from .gpu_util import from_packed, rel, to_packed

pytestmark = pytest.mark.gpu

L = (8, 8, 8, 8)


def weights_to_dev(W):
    flat = np.concatenate([w.reshape(-1) for w in W]).astype(np.complex64)
    return torch.from_numpy(flat.view(np.float32).copy()).cuda()


def dev_to_weights(t, C=16):
    flat = t.cpu().numpy().view(np.complex64).astype(np.complex128)
    dims = [(1, C), (C, C), (C, 1)]
    out, o = [], 0
    for cin, cout in dims:
        n = 9 * 4 * cout * 4 * cin
        out.append(flat[o:o + n].reshape(9, 4 * cout, 4 * cin))
        o += n
    return out


@pytest.fixture(scope="module")
def setup():
    U = synth.random_gauge(L, 51)
    ctx = dw.dw_create(L, 0.0, 1.0, U, (4, 4, 4, 4))
    P = PTNet(WilsonClover(L, U.numpy(), 0.0, 1.0))
    return ctx, P


def test_weight_count():
    assert dw.ptnet_weight_count(16) == 9 * 16 * (16 + 256 + 16)


def test_forward(setup):
    ctx, P = setup
    W = init_weights(16, seed=1, scale=0.5)
    x = synth.gaussian_source(L, 3).numpy()
    xd = to_packed(ctx, dw.DW_F32, x)
    yd = ctx.empty_field(dw.DW_F32)
    dw.ptnet_forward(ctx, weights_to_dev(W), 1, xd, yd)
    assert rel(from_packed(ctx, dw.DW_F32, yd), P.forward(W, x)) <= 2e-5


def test_loss_and_gradient(setup):
    ctx, P = setup
    W = init_weights(16, seed=2, scale=0.5)
    xs = [synth.gaussian_source(L, 4 + k).numpy() for k in range(2)]
    ys = [synth.gaussian_source(L, 6 + k).numpy() for k in range(2)]
    loss_o, G = P.loss_and_grad(W, xs, ys)
    xd = to_packed(ctx, dw.DW_F32, np.stack(xs))
    yd = to_packed(ctx, dw.DW_F32, np.stack(ys))
    g = torch.empty(2 * dw.ptnet_weight_count(16), dtype=torch.float32, device="cuda")
    loss = dw.ptnet_loss_grad(ctx, weights_to_dev(W), 2, xd, yd, g)
    assert abs(loss - loss_o) <= 1e-4 * loss_o
    Gd = dev_to_weights(g)
    errs = [rel(Gd[li], G[li]) for li in range(3)]
    assert max(errs) <= 1e-4, errs


def test_training_reduces_loss(setup):
    """Adam steps on the GPU lower the regression loss of the plain procedure's fields."""
    ctx, P = setup
    Ns = 4
    start = synth.start_fields(L, Ns, 9).cuda()
    x = ctx.empty_field(dw.DW_F32, Ns)
    dw.dw_pack(ctx, dw.DW_F32, Ns, start, x)
    dw.dfl_inverse_iteration(ctx, 4, 4, 1, Ns, x)
    y = x.clone()
    dw.dfl_inverse_iteration(ctx, 4, 4, 4, Ns, y)
    W = weights_to_dev(init_weights(16, seed=3, scale=0.1))
    m = torch.zeros_like(W)
    v = torch.zeros_like(W)
    g = torch.empty_like(W)
    first = dw.ptnet_loss_grad(ctx, W, Ns, x, y, g)
    loss = first
    for step in range(1, 41):
        loss = dw.ptnet_loss_grad(ctx, W, Ns, x, y, g)
        dw.ptnet_adam(W, g, m, v, step, 3e-3)
    assert loss < 0.7 * first, (first, loss)


def test_learned_build_judge(setup):
    """With random (untrained) weights the judge rejects the network output and the plain
    procedure finishes; the subspace is then the plain one."""
    ctx, P = setup
    start = synth.start_fields(L, 6, 10).cuda()
    W = weights_to_dev(init_weights(16, seed=4, scale=3.0))
    d = dw.deflation_build(ctx, (4, 4, 4, 4), 6, 5, 4, 4, start, basis_prec=dw.DW_F64, iter_prec=dw.DW_F32,
                           net_weights=W, net_k0=2, net_judge=0.95)
    info = d.info
    assert info.rho_in > 0 and info.rho_out > 0
    if not info.learned_used:
        d_plain = dw.deflation_build(ctx, (4, 4, 4, 4), 6, 5, 4, 4, start, basis_prec=dw.DW_F64,
                                     iter_prec=dw.DW_F32)
        a = torch.empty((6, ctx.V, 4, 3), dtype=torch.complex128, device="cuda")
        b = torch.empty_like(a)
        dw.dfl_basis_export(d, a)
        dw.dfl_basis_export(d_plain, b)
        assert rel(a.cpu().numpy(), b.cpu().numpy()) <= 1e-6


def test_trained_network_gains_over_equal_cost_plain():
    """Trained on two gauge fields and evaluated on a held-out one, the learned generation
    (k0 plain steps, then the network) deflates approximate low modes better than the plain
    procedure stopped after the same k0 steps; every subspace still solves to 1e-10."""
    from paper_0706_2298_gb300 import ptnet_train as pt
    Ls, Ns, k0, n_inv = (8, 8, 8, 8), 8, 1, 6
    samples = []
    for s in (61, 62):
        ctx = dw.dw_create(Ls, 0.0, 1.0, synth.random_gauge(Ls, s), (4, 4, 4, 4))
        x, y = pt.make_pairs(dw, synth, ctx, Ls, Ns, k0, n_inv, 4, 4, s + 100)
        samples.append((ctx, x, y, Ns))
    W = pt.init_weights(16, seed=7)
    losses = pt.train(dw, samples, W, 120, 3e-3)
    assert losses[-1] < 0.5 * losses[0]
    res = pt.evaluate(dw, synth, W, Ls, 71, Ns, k0, n_inv, 4, 4, (4, 4, 4, 4), 0.0, 1.0, nlow=4, low_steps=20)
    assert res["learned"]["learned_used"] == 1
    assert res["learned"]["rho_out"] < res["learned"]["rho_in"]
    assert res["learned"]["deficit"] < 0.95 * res["plain_k0"]["deficit"]
    assert res["plain_n_inv"]["deficit"] < res["plain_k0"]["deficit"]
    assert all(r["converged"] and r["relres"] <= 1e-10 for r in res.values())


@pytest.mark.parametrize("tile", ["64", "32"])
@pytest.mark.parametrize("adjoint", [0, 1])
def test_layer16_tensor_cores(setup, adjoint, tile, monkeypatch):
    """The 16 -> 16 layer (and its adjoint) on the tcgen05 tensor cores with BF16 operands and FP32
    accumulation against the FP64 oracle (BF16 path: within 2e-2; the rounding of 576-term sums of
    BF16 products gives a few 1e-3), and the FP32 CUDA-core path within 2e-5."""
    ctx, P = setup
    monkeypatch.setenv("DW_TC_TILE", tile)        # 64 sites per tile (one CTA per SM) or 32 (two)
    w = init_weights(16, seed=7, scale=0.6)[1]
    h = synth.complex_gaussian((16, ctx.V, 4, 3), 71).numpy()
    hg = h.reshape((16,) + L + (4, 3))
    ref = (P.layer_adjoint(w, hg) if adjoint else P.layer(w, hg)).reshape(16, ctx.V, 4, 3)
    wd = torch.from_numpy(w.astype(np.complex64).view(np.float32).copy()).cuda()
    x = to_packed(ctx, dw.DW_F32, h)
    for tc, tol in ((1, 2e-2), (0, 2e-5)):
        y = ctx.empty_field(dw.DW_F32, 16)
        y.fill_(float("nan"))
        dw.ptnet_layer16(ctx, wd, adjoint, tc, x, y)
        got = from_packed(ctx, dw.DW_F32, y, 16)
        assert np.isfinite(got).all()
        err = rel(got, ref)
        assert err <= tol, (tc, err)
        if tc:
            assert err >= 1e-6          # BF16 operands really were used


def test_forward_tensor_cores(setup):
    """The whole network with its 16 -> 16 layer on the tensor cores against the oracle."""
    ctx, P = setup
    W = init_weights(16, seed=1, scale=0.5)
    x = synth.gaussian_source(L, 3).numpy()
    xd = to_packed(ctx, dw.DW_F32, x)
    yd = ctx.empty_field(dw.DW_F32)
    dw.ptnet_forward_tc(ctx, weights_to_dev(W), 1, xd, yd)
    assert rel(from_packed(ctx, dw.DW_F32, yd), P.forward(W, x)) <= 2e-2
