"""ln psi and its log-derivatives O_k(x) = d ln psi(x) / d theta_k (Sec. 2).

Test infrastructure (see package docstring). Plain NumPy, complex128.

The network maps x in {-1,+1}^N to a complex log-amplitude (Sec. 2, first
paragraph). Two architectures, with the flat parameter layouts of
``workloads``:

RBM:   ln psi(x) = sum_i a_i x_i + sum_j lncosh(b_j + sum_i W_ji x_i)
FFNN:  h_0 = x; z_l = W_l h_{l-1} + b_l; h_l = lncosh(z_l) (hidden layers);
       ln psi = W_L h_{L-1} + b_L (one output)
VIT:   the transformer of ``oracle.vit`` (both functions dispatch there)

ln cosh branch (the paper is silent): lncosh(z) = s z - ln 2 + log1p(exp(-2 s z))
with s = sign(Re z) (s = +1 at Re z = 0). It is holomorphic away from the
zeros of cosh, with derivative tanh(z). Parameters enter holomorphically, so
O is the complex derivative.
"""
from __future__ import annotations

import numpy as np

from workloads import FFNN, RBM, VIT, Model

LN2 = np.log(2.0)


def lncosh(z: np.ndarray) -> np.ndarray:
    """Branch-fixed complex ln cosh (see module docstring)."""
    z = np.asarray(z, dtype=np.complex128)
    s = np.where(z.real >= 0, 1.0, -1.0)
    return s * z - LN2 + np.log1p(np.exp(-2.0 * s * z))


def split_ffnn(model: Model, theta: np.ndarray):
    """List of (W_l [out,in], b_l [out]) views of the flat parameter vector."""
    out, p = [], 0
    for (o, i) in model.layer_shapes():
        w = theta[p:p + o * i].reshape(o, i)
        p += o * i
        b = theta[p:p + o]
        p += o
        out.append((w, b))
    assert p == model.n_params
    return out


def split_rbm(model: Model, theta: np.ndarray):
    n, m = model.widths
    a = theta[:n]
    b = theta[n:n + m]
    w = theta[n + m:].reshape(m, n)
    return a, b, w


def log_psi(model: Model, theta: np.ndarray, x: np.ndarray) -> np.ndarray:
    """ln psi for every row of x (int or float, values +-1). complex128 [n_s]."""
    x = np.asarray(x, dtype=np.float64)
    theta = np.asarray(theta, dtype=np.complex128)
    if model.kind == VIT:
        from . import vit
        return vit.log_psi(model, theta, x)
    if model.kind == RBM:
        a, b, w = split_rbm(model, theta)
        th = x @ w.T + b
        return x @ a + lncosh(th).sum(axis=1)
    layers = split_ffnn(model, theta)
    h = x.astype(np.complex128)
    for l, (w, b) in enumerate(layers):
        z = h @ w.T + b
        h = z if l == len(layers) - 1 else lncosh(z)
    return h[:, 0]


def jacobian(model: Model, theta: np.ndarray, x: np.ndarray):
    """(ln psi [n_s], O [n_s, n_p]) with O_k = d ln psi / d theta_k.

    RBM closed form: O(a_i) = x_i, O(b_j) = tanh(theta_j), O(W_ji) = tanh(theta_j) x_i,
    theta_j = b_j + sum_i W_ji x_i.
    FFNN holomorphic back-propagation: output layer O(W_L) = h_{L-1}, O(b_L) = 1,
    g_h = W_L; for each hidden layer l from the top: g_z = g_h * tanh(z_l),
    O(W_l)[j,k] = g_z[j] h_{l-1}[k], O(b_l) = g_z, g_h <- W_l^T g_z (no conjugation).
    """
    x = np.asarray(x, dtype=np.float64)
    theta = np.asarray(theta, dtype=np.complex128)
    if model.kind == VIT:
        from . import vit
        return vit.jacobian(model, theta, x)
    ns = x.shape[0]
    O = np.empty((ns, model.n_params), dtype=np.complex128)
    if model.kind == RBM:
        n, m = model.widths
        a, b, w = split_rbm(model, theta)
        th = x @ w.T + b
        t = np.tanh(th)
        O[:, :n] = x
        O[:, n:n + m] = t
        O[:, n + m:] = (t[:, :, None] * x[:, None, :]).reshape(ns, m * n)
        lp = x @ a + lncosh(th).sum(axis=1)
        return lp, O
    layers = split_ffnn(model, theta)
    hs = [x.astype(np.complex128)]
    zs = []
    for l, (w, b) in enumerate(layers):
        z = hs[-1] @ w.T + b
        zs.append(z)
        hs.append(z if l == len(layers) - 1 else lncosh(z))
    lp = hs[-1][:, 0]
    offs = np.concatenate([[0], np.cumsum([o * i + o for (o, i) in model.layer_shapes()])])
    L = len(layers)
    # output layer
    wL, _ = layers[-1]
    o_, i_ = wL.shape
    O[:, offs[L - 1]:offs[L - 1] + i_] = hs[L - 1]
    O[:, offs[L - 1] + i_] = 1.0
    g_h = np.broadcast_to(wL[0], (ns, i_)).copy()
    for l in range(L - 2, -1, -1):
        w, _ = layers[l]
        o_, i_ = w.shape
        g_z = g_h * np.tanh(zs[l])
        p = offs[l]
        O[:, p:p + o_ * i_] = (g_z[:, :, None] * hs[l][:, None, :]).reshape(ns, o_ * i_)
        O[:, p + o_ * i_:p + o_ * i_ + o_] = g_z
        g_h = g_z @ w
    return lp, O
