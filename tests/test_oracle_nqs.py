"""Pins of the oracle's ln psi and Jacobian (Sec. 2: O_k = d ln psi / d theta_k).

The Jacobian is pinned by central finite differences of ln psi along the real
and the imaginary axis of each parameter (they agree because ln psi is
holomorphic in theta), and the FFNN by its RBM special case.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from oracle import nqs


def _fd(model, theta, x, k, h, direction):
    tp = theta.copy()
    tm = theta.copy()
    tp[k] += h * direction
    tm[k] -= h * direction
    return (nqs.log_psi(model, tp, x) - nqs.log_psi(model, tm, x)) / (2 * h * direction)


def test_lncosh_is_log_of_cosh_and_has_tanh_derivative():
    rng = np.random.default_rng(0)
    z = rng.normal(size=400) * 3 + 1j * rng.normal(size=400) * 3
    z = np.concatenate([z, [0.0, 1e-12, -1e-12, 30 + 2j, -30 - 2j, 1j]])
    lc = nqs.lncosh(z)
    np.testing.assert_allclose(np.exp(lc), np.cosh(z), rtol=1e-12)
    # branch: the real part is the log-modulus, the imaginary part stays within
    # s*Im z +- pi/2 (continuous in z within each half plane)
    s = np.where(z.real >= 0, 1.0, -1.0)
    assert np.all(np.abs(lc.imag - s * z.imag) <= np.pi / 2 + 1e-12)
    h = 1e-6
    d = (nqs.lncosh(z + h) - nqs.lncosh(z - h)) / (2 * h)
    np.testing.assert_allclose(d, np.tanh(z), rtol=1e-7, atol=1e-8)


@pytest.mark.parametrize("direction", [1.0, 1j])
def test_rbm_jacobian_matches_central_differences(direction):
    model = W.Model(W.RBM, (8, 6))
    rng = np.random.default_rng(1)
    theta = (rng.normal(size=model.n_params) + 1j * rng.normal(size=model.n_params)) * 0.3
    x = W.zero_sz_configs(8, 5, rng)
    lp, O = nqs.jacobian(model, theta, x)
    np.testing.assert_allclose(lp, nqs.log_psi(model, theta, x), rtol=0, atol=1e-13)
    for k in range(model.n_params):
        fd = _fd(model, theta, x, k, 1e-6, direction)
        np.testing.assert_allclose(O[:, k], fd, rtol=1e-7, atol=1e-8)


@pytest.mark.parametrize("direction", [1.0, 1j])
def test_ffnn_jacobian_matches_central_differences(direction):
    model = W.Model(W.FFNN, (6, 5, 4, 3, 1))
    rng = np.random.default_rng(2)
    theta = W.init_params(model, rng) * 2.0
    x = W.zero_sz_configs(6, 7, rng)
    lp, O = nqs.jacobian(model, theta, x)
    np.testing.assert_allclose(lp, nqs.log_psi(model, theta, x), rtol=0, atol=1e-13)
    for k in range(model.n_params):
        fd = _fd(model, theta, x, k, 1e-6, direction)
        np.testing.assert_allclose(O[:, k], fd, rtol=1e-7, atol=1e-8)


def test_ffnn_jacobian_workload_shape_sampled_fd():
    w = W.make_workload("j1j2_6x6_ffnn", 16)
    lp, O = nqs.jacobian(w.model, w.theta, w.configs)
    rng = np.random.default_rng(3)
    for k in rng.choice(w.model.n_params, 25, replace=False):
        fd = _fd(w.model, w.theta, w.configs, int(k), 1e-6, 1.0)
        np.testing.assert_allclose(O[:, k], fd, rtol=1e-6, atol=1e-8)


def test_one_hidden_layer_ffnn_equals_rbm_without_visible_bias():
    n, m = 8, 5
    rng = np.random.default_rng(4)
    wgt = rng.normal(size=(m, n)) * 0.4 + 1j * rng.normal(size=(m, n)) * 0.4
    bias = rng.normal(size=m) * 0.4 + 1j * rng.normal(size=m) * 0.4
    rbm = W.Model(W.RBM, (n, m))
    th_r = np.concatenate([np.zeros(n), bias, wgt.ravel()]).astype(np.complex128)
    ffnn = W.Model(W.FFNN, (n, m, 1))
    th_f = np.concatenate([wgt.ravel(), bias, np.ones(m), [0.0]]).astype(np.complex128)
    x = W.zero_sz_configs(n, 9, rng)
    lr, Or = nqs.jacobian(rbm, th_r, x)
    lf, Of = nqs.jacobian(ffnn, th_f, x)
    np.testing.assert_allclose(lf, lr, rtol=0, atol=1e-13)
    # FFNN first layer [W | b] <-> RBM [W | b] columns
    np.testing.assert_allclose(Of[:, : m * n], Or[:, n + m:], atol=1e-13)
    np.testing.assert_allclose(Of[:, m * n: m * n + m], Or[:, n: n + m], atol=1e-13)


def test_workload_shapes():
    sizes = {name: W.make_workload(name, 4).model.block_sizes() for name in W.WORKLOADS}
    assert sizes["chain10_rbm"] == [10, 10, 100]
    assert sizes["j1j2_6x6_ffnn"] == [2368, 4160, 65]
    assert sizes["j1j2_10x10_ffnn5"] == [6464, 4160, 4160, 4160, 65]
    assert sizes["j1j2_10x10_ffnn256"] == [25856, 65792, 257]
    b = W.make_workload("batch8x8_3", 4)
    assert b.model.n_params == 47937 and min(b.model.block_sizes()) == 65
    assert max(b.model.block_sizes()) == 8320
    x = W.make_workload("j1j2_10x10_ffnn5", 64).configs
    assert x.dtype == np.int8 and np.all(x.sum(axis=1) == 0)
