"""Pins of the oracle's transformer wavefunction (the module partition of Sec. 2).

O is pinned against central finite differences of ln psi in the real and imaginary
directions (holomorphy), the network against its reduction to the RBM (one token, no encoder
layer, unit output weights) and the residual structure against encoder layers whose
branches are zero; its local energies against the dense Hamiltonian.
"""
import numpy as np

import workloads as W
from oracle import hamiltonian, nqs, vit


def _small(n_enc=2, widths=(8, 2, 4, 6), seed=0, scale=1.0):
    model = W.Model(W.VIT, widths, n_enc)
    theta = W.init_params(model, np.random.default_rng(seed)) * scale
    return model, theta


def test_block_sizes_and_split_cover_theta():
    model, theta = _small()
    we, be, layers, wo, bo = vit.split(model, theta)
    assert we.shape == (4, 2) and len(layers) == 2 and layers[0]["A"].shape == (4, 4)
    assert list(model.block_sizes()) == [4 * 2 + 4, 16 + 16 + 24 + 6 + 24 + 4, 90, 5]


def test_jacobian_matches_central_differences():
    model, theta = _small(scale=2.0)
    x = W.zero_sz_configs(8, 5, np.random.default_rng(1))
    lp, O = vit.jacobian(model, theta, x)
    np.testing.assert_allclose(lp, vit.log_psi(model, theta, x), rtol=1e-13)
    h = 1e-6
    for k in range(model.n_params):
        e = np.zeros(model.n_params)
        e[k] = h
        fd = (vit.log_psi(model, theta + e, x) - vit.log_psi(model, theta - e, x)) / (2 * h)
        fdi = (vit.log_psi(model, theta + 1j * e, x) - vit.log_psi(model, theta - 1j * e, x)) / (2 * h)
        np.testing.assert_allclose(O[:, k], fd, rtol=1e-6, atol=1e-8)
        np.testing.assert_allclose(1j * O[:, k], fdi, rtol=1e-6, atol=1e-8)


def test_one_token_without_encoder_is_an_rbm():
    n, d = 6, 5
    model = W.Model(W.VIT, (n, n, d, 3), 0)
    rng = np.random.default_rng(2)
    theta = (rng.normal(size=model.n_params) + 1j * rng.normal(size=model.n_params)) * 0.3
    theta[-d - 1:-1] = 1.0   # w_O = 1
    theta[-1] = 0.0          # b_O = 0
    rbm = W.Model(W.RBM, (n, d))
    th_rbm = np.concatenate([np.zeros(n), theta[d * n:d * n + d], theta[:d * n]])  # a = 0, b = b_E, W = W_E
    x = hamiltonian.all_configs(n)
    np.testing.assert_allclose(vit.log_psi(model, theta, x), nqs.log_psi(rbm, th_rbm, x), rtol=1e-13, atol=1e-13)
    _, O = vit.jacobian(model, theta, x)
    _, Or = nqs.jacobian(rbm, th_rbm, x)
    np.testing.assert_allclose(O[:, :d * n], Or[:, n + d:], rtol=1e-12, atol=1e-13)   # W_E <-> W
    np.testing.assert_allclose(O[:, d * n:d * n + d], Or[:, n:n + d], rtol=1e-12, atol=1e-13)


def test_zero_residual_branches_are_the_identity():
    model1, theta1 = _small(n_enc=1, seed=3)
    model0 = W.Model(W.VIT, model1.widths, 0)
    d, h, t = 4, 6, 4
    enc = t * t + d * d + 2 * h * d + h + d
    th = theta1.copy()
    e0 = d * 2 + d                                          # embedding block (patch 2)
    th[e0:e0 + t * t] = 0.0                                 # A = 0
    th[e0 + enc - d - d * h:e0 + enc] = 0.0                 # W_2 = 0, b_2 = 0
    th0 = np.concatenate([th[:e0], th[e0 + enc:]])
    x = hamiltonian.all_configs(8)
    np.testing.assert_allclose(vit.log_psi(model1, th, x), vit.log_psi(model0, th0, x), rtol=1e-13, atol=1e-13)


def test_local_energy_of_the_transformer_matches_dense_hamiltonian():
    model, theta = _small(scale=1.5, seed=4)
    ij, jj = W.chain_bonds(8, 1.0)
    x = hamiltonian.all_configs(8)
    psi = np.exp(nqs.log_psi(model, theta, x))
    H = hamiltonian.dense_hamiltonian(8, ij, jj, 1.0, -1, sparse=True)
    el = hamiltonian.local_energy(model, theta, x, ij, jj, 1.0, -1)
    np.testing.assert_allclose(el, (H @ psi) / psi, rtol=1e-11, atol=1e-11)
