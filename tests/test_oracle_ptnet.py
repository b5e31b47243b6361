"""Pins of the oracle's parallel-transport network: adjoint transports,
gauge covariance, linearity, and the analytic gradient against central finite
differences in FP64."""
import numpy as np
import pytest

from oracle.dirac import WilsonClover
from oracle.ptnet import PTNet, init_weights
from paper_0706_2298_gb300 import synth

L = (4, 4, 4, 4)


@pytest.fixture(scope="module")
def net():
    U = synth.random_gauge(L, 41).numpy()
    D = WilsonClover(L, U, 0.0, 1.0)
    return PTNet(D), U


def _grid(v, C=1):
    return v.reshape((C,) + L + (4, 3))


def test_transport_adjoint(net):
    P, _ = net
    h = _grid(synth.complex_gaussian((2, synth.volume(L), 4, 3), 1).numpy(), 2)
    g = _grid(synth.complex_gaussian((2, synth.volume(L), 4, 3), 2).numpy(), 2)
    for d in range(9):
        lhs = np.vdot(g, P.transport(h, d))
        rhs = np.vdot(P.transport_adj(g, d), h)
        assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_gauge_covariance(net):
    P, U = net
    W = init_weights(C=4, seed=3, scale=0.5)
    V = synth.volume(L)
    Om = synth.random_su3(V, 12).numpy().reshape(L + (3, 3))
    Ug = U.reshape(L + (4, 3, 3))
    Up = np.empty_like(Ug)
    for mu in range(4):
        Up[..., mu, :, :] = Om @ Ug[..., mu, :, :] @ np.conj(np.swapaxes(np.roll(Om, -1, axis=mu), -1, -2))
    Pp = PTNet(WilsonClover(L, Up.reshape(V, 4, 3, 3), 0.0, 1.0))
    x = synth.gaussian_source(L, 4).numpy()
    rot = lambda f: np.einsum("xab,xsb->xsa", Om.reshape(V, 3, 3), f)
    assert np.linalg.norm(Pp.forward(W, rot(x)) - rot(P.forward(W, x))) < 1e-12 * np.linalg.norm(x)


def test_linear_and_identity_at_init(net):
    P, _ = net
    W = init_weights(C=4, seed=5, scale=0.0)
    x = synth.gaussian_source(L, 5).numpy()
    assert np.allclose(P.forward(W, x), x, atol=1e-13)
    W = init_weights(C=4, seed=6, scale=0.4)
    y = synth.gaussian_source(L, 6).numpy()
    a, b = 0.3 - 0.7j, 1.1 + 0.2j
    assert np.allclose(P.forward(W, a * x + b * y), a * P.forward(W, x) + b * P.forward(W, y), atol=1e-12)


def test_gradient_finite_differences(net):
    P, _ = net
    W = init_weights(C=3, seed=7, scale=0.5)
    xs = [synth.gaussian_source(L, 7).numpy()]
    ys = [synth.gaussian_source(L, 8).numpy()]
    loss, G = P.loss_and_grad(W, xs, ys)
    rng = np.random.default_rng(0)
    h = 1e-6
    for li in range(3):
        for _ in range(4):
            idx = tuple(rng.integers(0, n) for n in W[li].shape)
            for part, unit in (("re", 1.0), ("im", 1j)):
                Wp = [w.copy() for w in W]
                Wm = [w.copy() for w in W]
                Wp[li][idx] += h * unit
                Wm[li][idx] -= h * unit
                fd = (P.loss_and_grad(Wp, xs, ys)[0] - P.loss_and_grad(Wm, xs, ys)[0]) / (2 * h)
                an = G[li][idx].real if part == "re" else G[li][idx].imag
                assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (li, idx, part, fd, an)


def test_layer_adjoint_identity():
    """(layer(w, h), g) = (h, layer_adjoint(w, g)) for a 16 -> 16 layer on random fields."""
    from oracle.ptnet import PTNet, init_weights
    L = (4, 2, 2, 2)
    P = PTNet(WilsonClover(L, synth.random_gauge(L, 61).numpy(), 0.0, 1.0))
    w = init_weights(16, seed=5, scale=0.7)[1]
    h = synth.complex_gaussian((16,) + L + (4, 3), 62).numpy()
    g = synth.complex_gaussian((16,) + L + (4, 3), 63).numpy()
    lhs = np.vdot(P.layer(w, h), g)
    rhs = np.vdot(h, P.layer_adjoint(w, g))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
