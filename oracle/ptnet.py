"""Gauge-covariant parallel-transport network (PTNet), FP64 reference.

The learned part of the subspace generation: a small network maps quark
fields after k0 plain inverse-iteration steps (5.1) to approximations of the
fields after n_inv steps, so most Schwarz sweeps of the subspace generation
are replaced by three network layers.  Each layer is

    h'(x)_{c' s'} = sum_{d in {0, +mu, -mu}} sum_{c s} W_d[c' s', c s] (T_d h)(x)_{c s}

with channels c, spin s, colour acting untouched, and the parallel transports
T_0 h(x) = h(x), T_{+mu} h(x) = U_mu(x) h(x+mu), T_{-mu} h(x) = U_mu(x-mu)^dag h(x-mu)
(fermion links: antiperiodic sign across the time boundary, as in D).
Because W acts on (channel, spin) only and T_d is covariant, every layer
maps Omega(x) h(x) to Omega(x) h'(x) under a gauge transformation.  The
network is linear in the field (like the inverse iteration it replaces is
homogeneous of degree one); 3 layers with 1 -> C -> C -> 1 channels.

Directions are ordered d = 0 (site), 1 + 2 mu (forward), 2 + 2 mu (backward).
Fields: h[channel, V, 4, 3] complex128.  Weights: W[layer][9, cout*4, cin*4].

Training loss (regression onto the plain procedure):
    L = sum_l ||N(x_l) - y_l||^2 / sum_l ||y_l||^2.
Gradient returned as G = dL/dRe W + i dL/dIm W.
"""
from __future__ import annotations

import numpy as np

from .dirac import WilsonClover
from .lattice import Lattice


def init_weights(C: int = 16, seed: int = 0, scale: float = 0.3):
    """Near-identity start: the site term carries the input through, hops are small."""
    rng = np.random.default_rng(seed)
    dims = [(1, C), (C, C), (C, 1)]
    W = []
    for cin, cout in dims:
        w = (rng.normal(size=(9, 4 * cout, 4 * cin)) + 1j * rng.normal(size=(9, 4 * cout, 4 * cin)))
        w *= scale / np.sqrt(9 * 4 * cin)
        # identity-like site term: spin preserved, channels mixed evenly
        for s in range(4):
            for co in range(cout):
                for ci in range(cin):
                    w[0, 4 * co + s, 4 * ci + s] += 1.0 / np.sqrt(cin * cout) if cin * cout > 1 else 1.0
        W.append(w)
    return W


class PTNet:
    def __init__(self, D: WilsonClover):
        self.D = D
        self.L = D.L
        self.Uf = D.Uf           # fermion links per direction, (L0..L3, 3, 3)

    # -- transports -------------------------------------------------------------------
    def transport(self, h, d):
        """T_d h for h[C, L0..L3, 4, 3] (grid layout)."""
        if d == 0:
            return h
        mu, back = (d - 1) // 2, (d - 1) % 2
        U = self.Uf[mu][None, ..., None, :, :]              # (1, L.., 1, 3, 3) broadcast over spin
        if not back:
            hs = Lattice.shift(h, mu, 1, lead=1)             # h(x + mu)
            return np.einsum("...ab,...b->...a", U, hs)
        t = np.einsum("...ba,...b->...a", np.conj(U), h)     # U^dag h at y
        return Lattice.shift(t, mu, -1, lead=1)              # taken at y = x - mu

    def transport_adj(self, g, d):
        """Adjoint of T_d: (T_d)^dag g."""
        if d == 0:
            return g
        mu, back = (d - 1) // 2, (d - 1) % 2
        U = self.Uf[mu][None, ..., None, :, :]
        if not back:
            # T h(x) = U(x) h(x+mu)  ->  T^dag g(y) = U(y-mu)^dag g(y-mu)
            t = np.einsum("...ba,...b->...a", np.conj(U), g)
            return Lattice.shift(t, mu, -1, lead=1)
        # T h(x) = U(x-mu)^dag h(x-mu)  ->  T^dag g(y) = U(y) g(y+mu)
        return np.einsum("...ab,...b->...a", U, Lattice.shift(g, mu, 1, lead=1))

    def layer(self, w, h):
        """One layer: h[cin, L.., 4, 3] -> [cout, L.., 4, 3]."""
        cin = h.shape[0]
        cout = w.shape[1] // 4
        out = np.zeros((cout,) + h.shape[1:], dtype=np.complex128)
        for d in range(9):
            th = self.transport(h, d)
            # flatten (channel, spin) of the input, contract with w[d]
            thf = np.moveaxis(th, -2, 1).reshape((cin * 4,) + th.shape[1:-2] + (3,))   # [cin*4, L.., 3]
            o = np.tensordot(w[d], thf, axes=(1, 0))                                     # [cout*4, L.., 3]
            out += np.moveaxis(o.reshape((cout, 4) + o.shape[1:]), 1, -2)
        return out

    def layer_adjoint(self, w, g):
        """The adjoint of `layer`: sum_d T_d^dag (w[d]^dag g), g[cout, L.., 4, 3] -> [cin, L.., 4, 3]
        (the data gradient of back-propagation)."""
        cout = g.shape[0]
        cin = w.shape[2] // 4
        out = np.zeros((cin,) + g.shape[1:], dtype=np.complex128)
        gf = np.moveaxis(g, -2, 1).reshape((cout * 4,) + g.shape[1:-2] + (3,))
        for d in range(9):
            b = np.tensordot(w[d].conj().T, gf, axes=(1, 0))                            # [cin*4, L.., 3]
            out += self.transport_adj(np.moveaxis(b.reshape((cin, 4) + b.shape[1:]), 1, -2), d)
        return out

    def forward(self, W, x, keep=False):
        """x: [V, 4, 3] field -> N(x) [V, 4, 3]; keep=True also returns the layer inputs."""
        h = np.asarray(x, dtype=np.complex128).reshape((1,) + self.L + (4, 3))
        acts = [h]
        for w in W:
            h = self.layer(w, h)
            acts.append(h)
        out = h.reshape(-1, 4, 3)
        return (out, acts) if keep else out

    def backward(self, W, acts, g_out):
        """Gradients of Re <g_out, N(x)> w.r.t. the weights (g_out: [V,4,3]).

        Returns (grads, g_in): grads[l][d] = dF/dRe W + i dF/dIm W for
        F = Re sum conj(g_out) N(x), and g_in = dF/d conj(x)-style adjoint field.
        """
        g = np.asarray(g_out).reshape((1,) + self.L + (4, 3))
        grads = [np.zeros_like(w) for w in W]
        for li in range(len(W) - 1, -1, -1):
            w, h = W[li], acts[li]
            cin = h.shape[0]
            cout = w.shape[1] // 4
            gf = np.moveaxis(g, -2, 1).reshape((cout * 4, -1))                  # [cout*4, V*3]
            g_prev = np.zeros_like(h)
            for d in range(9):
                th = self.transport(h, d)
                thf = np.moveaxis(th, -2, 1).reshape((cin * 4, -1))              # [cin*4, V*3]
                # F = Re sum conj(g) (w th): dF/dRe w + i dF/dIm w = g th^dag
                grads[li][d] = gf @ thf.conj().T
                back = (w[d].conj().T @ gf).reshape((cin, 4) + h.shape[1:5] + (3,))
                back = np.moveaxis(back, 1, -2)                                  # [cin, L.., 4, 3]
                g_prev += self.transport_adj(back, d)
            g = g_prev
        return grads, g.reshape(-1, 4, 3)

    def loss_and_grad(self, W, xs, ys):
        """L = sum ||N(x) - y||^2 / sum ||y||^2 and dL/dRe W + i dL/dIm W."""
        den = sum(float(np.vdot(y, y).real) for y in ys)
        loss = 0.0
        grads = [np.zeros_like(w) for w in W]
        for x, y in zip(xs, ys):
            out, acts = self.forward(W, x, keep=True)
            e = out - y
            loss += float(np.vdot(e, e).real)
            g, _ = self.backward(W, acts, e)
            for li in range(len(W)):
                grads[li] += 2.0 * g[li]
        return loss / den, [gr / den for gr in grads]
