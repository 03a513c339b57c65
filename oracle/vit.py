"""ln psi and O = d ln psi / d theta of the transformer wavefunction (the network whose
modules define the block partition of Sec. 2: patching and embedding, encoder layers,
output layer).

Test infrastructure (see package docstring). Plain NumPy, complex128.

The paper names a Vision Transformer with a two-layer encoder but does not specify it; this
is the holomorphic variant the library implements (complex parameters, no layer norm, ln cosh
non-linearities, attention weights that depend only on the token positions):

  patches   x_t = (x_{tp}, ..., x_{tp+p-1}),  t = 0 .. T-1,  T = N / p
  embedding h_t = W_E x_t + b_E                                   (d_model)
  encoder   v_s = W_V h_s;  u_t = h_t + sum_s A_ts v_s            (attention + residual)
  (each)    z_t = W_1 u_t + b_1;  h_t <- u_t + W_2 lncosh(z_t) + b_2   (MLP + residual)
  output    ln psi = w_O . sum_t lncosh(h_t) + b_O

O follows by back-propagating g = d ln psi / d(.) through these formulas in reverse order,
with plain transposes (no conjugation): the map is holomorphic in the parameters.
"""
from __future__ import annotations

import numpy as np

LN2 = np.log(2.0)


def _lncosh(z):
    s = np.where(z.real >= 0, 1.0, -1.0)
    return s * z - LN2 + np.log1p(np.exp(-2.0 * s * z))


def split(model, theta: np.ndarray):
    """(W_E [d,p], b_E [d], encoder layers [dict], w_O [d], b_O) views of theta."""
    _, p, t, d, h = model.vit_dims()
    k = 0

    def take(n, shape=None):
        nonlocal k
        v = theta[k:k + n]
        k += n
        return v.reshape(shape) if shape else v

    we, be = take(d * p, (d, p)), take(d)
    layers = []
    for _ in range(model.n_enc):
        layers.append(dict(A=take(t * t, (t, t)), WV=take(d * d, (d, d)), W1=take(h * d, (h, d)), b1=take(h),
                           W2=take(d * h, (d, h)), b2=take(d)))
    wo, bo = take(d), take(1)[0]
    assert k == model.n_params
    return we, be, layers, wo, bo


def _forward(model, theta, x):
    _, p, t, d, h = model.vit_dims()
    theta = np.asarray(theta, dtype=np.complex128)
    xs = np.asarray(x, dtype=np.float64).reshape(x.shape[0], t, p)
    we, be, layers, wo, bo = split(model, theta)
    hs = [xs @ we.T + be]
    saved = []
    for L in layers:
        hp = hs[-1]
        v = hp @ L["WV"].T
        u = hp + np.einsum("ts,nsk->ntk", L["A"], v)
        z = u @ L["W1"].T + L["b1"]
        a = _lncosh(z)
        hs.append(u + a @ L["W2"].T + L["b2"])
        saved.append(dict(v=v, u=u, z=z, a=a))
    lp = _lncosh(hs[-1]).sum(axis=1) @ wo + bo
    return lp, xs, hs, saved, (we, be, layers, wo, bo)


def log_psi(model, theta, x) -> np.ndarray:
    return _forward(model, theta, x)[0]


def jacobian(model, theta, x):
    """(ln psi [n_s], O [n_s, n_p]) by holomorphic back-propagation."""
    lp, xs, hs, saved, (we, be, layers, wo, bo) = _forward(model, theta, x)
    ns = xs.shape[0]
    blocks_rev = []
    # output layer: O(w_O) = sum_t lncosh(h_t), O(b_O) = 1; g_h = w_O * tanh(h)
    blocks_rev.append(np.concatenate([_lncosh(hs[-1]).sum(axis=1), np.ones((ns, 1))], axis=1))
    gh = wo[None, None, :] * np.tanh(hs[-1])
    for l in range(len(layers) - 1, -1, -1):
        L, S, hp = layers[l], saved[l], hs[l]
        ga = gh @ L["W2"]                                   # W_2^T g_h per token
        gz = ga * np.tanh(S["z"])
        o_w2 = np.einsum("nti,ntk->nik", gh, S["a"])
        o_b2 = gh.sum(axis=1)
        o_w1 = np.einsum("ntk,ntj->nkj", gz, S["u"])
        o_b1 = gz.sum(axis=1)
        gu = gh + gz @ L["W1"]
        o_a = np.einsum("ntk,nsk->nts", gu, S["v"])
        gv = np.einsum("ts,ntk->nsk", L["A"], gu)
        o_wv = np.einsum("nsk,nsj->nkj", gv, hp)
        gh = gu + gv @ L["WV"]
        blocks_rev.append(np.concatenate([o_a.reshape(ns, -1), o_wv.reshape(ns, -1), o_w1.reshape(ns, -1), o_b1,
                                          o_w2.reshape(ns, -1), o_b2], axis=1))
    o_we = np.einsum("ntk,ntj->nkj", gh, xs)
    blocks_rev.append(np.concatenate([o_we.reshape(ns, -1), gh.sum(axis=1)], axis=1))
    O = np.concatenate(blocks_rev[::-1], axis=1).astype(np.complex128)
    return lp, O
