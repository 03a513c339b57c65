"""Pins of the oracle's QGT, force and solve (Eq. 2, Eq. 3, Sec. 2).

Exact enumeration of all 2^N states replaces sampling (w = |psi|^2/Z). The
QGT is checked against the first form of Eq. 2 built from finite-difference
derivatives of psi itself, the force against the finite-difference gradient
of the exact energy, and the solve against identities and limits.
"""
import numpy as np
import pytest

import workloads as W
from oracle import exact, hamiltonian, nqs, qgt


def _small_rbm(seed=7, n=8, m=4, scale=0.3):
    model = W.Model(W.RBM, (n, m))
    rng = np.random.default_rng(seed)
    theta = (rng.normal(size=model.n_params) + 1j * rng.normal(size=model.n_params)) * scale
    return model, theta


def _small_ffnn(seed=8):
    model = W.Model(W.FFNN, (8, 4, 3, 1))
    return model, W.init_params(model, np.random.default_rng(seed)) * 2


@pytest.mark.parametrize("make", [_small_rbm, _small_ffnn])
def test_energy_and_qgt_match_exact_enumeration(make):
    model, theta = make()
    n = model.n_sites
    ij, jj = W.chain_bonds(n, 1.0)
    x, wts = exact.born_weights(model, theta, n)
    lp, O = nqs.jacobian(model, theta, x)
    el = hamiltonian.local_energy(model, theta, x, ij, jj)
    e_mean, o_mean, dO, e = qgt.center(O, el, wts)
    assert abs(e_mean - exact.energy(model, theta, n, ij, jj)) < 1e-11
    S = qgt.full_qgt(dO, wts)
    _, psi = exact.psi_vector(model, theta, n)
    S1 = exact.qgt_first_form(psi, exact.dpsi_fd(model, theta, n))
    np.testing.assert_allclose(S, S1, rtol=0, atol=1e-8 * np.abs(S).max())


def test_force_is_wirtinger_gradient_of_exact_energy():
    model, theta = _small_rbm(9, 6, 3)
    n = 6
    ij, jj = W.chain_bonds(n, 1.0)
    x, wts = exact.born_weights(model, theta, n)
    _, O = nqs.jacobian(model, theta, x)
    el = hamiltonian.local_energy(model, theta, x, ij, jj)
    _, _, dO, e = qgt.center(O, el, wts)
    F = qgt.force(dO, e, wts)
    h = 1e-6
    for k in range(model.n_params):
        g = []
        for d in (1.0, 1j):
            tp = theta.copy(); tp[k] += h * d
            tm = theta.copy(); tm[k] -= h * d
            g.append((exact.energy(model, tp, n, ij, jj) - exact.energy(model, tm, n, ij, jj)) / (2 * h))
        np.testing.assert_allclose(F[k], 0.5 * (g[0] + 1j * g[1]), rtol=1e-6, atol=1e-8)


def _sampled(name="j1j2_6x6_ffnn", ns=64):
    w = W.make_workload(name, ns)
    _, O = nqs.jacobian(w.model, w.theta, w.configs)
    el = hamiltonian.local_energy(w.model, w.theta, w.configs, w.bond_ij, w.bond_j)
    return w, O, el


def test_block_rule_single_block_and_diagonal_blocks():
    model, theta = _small_ffnn()
    x = W.zero_sz_configs(8, 50, np.random.default_rng(1))
    _, O = nqs.jacobian(model, theta, x)
    el = np.zeros(50)
    _, _, dO, _ = qgt.center(O, el)
    off = model.block_offsets()
    full = qgt.full_qgt(dO)
    one = qgt.block_qgt(dO, [0, model.n_params])[0]
    np.testing.assert_array_equal(full, one)
    for b, Sb in enumerate(qgt.block_qgt(dO, off)):
        np.testing.assert_allclose(Sb, full[off[b]:off[b + 1], off[b]:off[b + 1]], atol=1e-15)


def test_block_qgt_hermitian_psd_and_trace():
    w, O, el = _sampled("chain10_rbm", 100)
    _, _, dO, _ = qgt.center(O, el)
    for b, Sb in enumerate(qgt.block_qgt(dO, w.block_off)):
        np.testing.assert_allclose(Sb, np.conj(Sb).T, atol=1e-15)
        ev = np.linalg.eigvalsh(Sb)
        assert ev.min() >= -1e-12 * np.abs(ev).max()
        blk = dO[:, w.block_off[b]:w.block_off[b + 1]]
        assert abs(np.trace(Sb).real - np.mean(np.sum(np.abs(blk) ** 2, axis=1))) < 1e-12 * np.trace(Sb).real


def test_solve_residual_limits_and_eta():
    w, O, el = _sampled("chain10_rbm", 200)
    _, _, dO, e = qgt.center(O, el)
    F = qgt.force(dO, e)
    S = qgt.block_qgt(dO, w.block_off)
    d, sig, kept = qgt.block_solve(S, F, w.block_off, 1e-3, 1e-12, eta=0.7)
    assert np.all(kept == np.diff(w.block_off))
    for b, Sb in enumerate(S):
        sl = slice(w.block_off[b], w.block_off[b + 1])
        r = (Sb + 1e-3 * np.eye(Sb.shape[0])) @ d[sl] + 0.7 * F[sl]
        assert np.linalg.norm(r) <= 1e-12 * np.linalg.norm(F[sl]) * np.linalg.cond(Sb + 1e-3 * np.eye(Sb.shape[0]))
    big = 1e9
    d2, _, _ = qgt.block_solve(S, F, w.block_off, big, 1e-12)
    np.testing.assert_allclose(d2, -F / big, rtol=1e-6, atol=0)
    d3, _, _ = qgt.block_solve(S, F, w.block_off, 1e-3, 1e-12, eta=1.4)
    np.testing.assert_allclose(d3, 2 * d, rtol=1e-12, atol=1e-300)


def test_single_sample_gives_zero_update():
    w, O, el = _sampled("chain10_rbm", 1)
    r = qgt.sr_step(w.model, w.theta, w.configs, w.bond_ij, w.bond_j, w.block_off, 1e-4, 1e-10)
    assert np.all(r["dtheta"] == 0) and np.all(r["F"] == 0)


def test_active_cutoff_matches_library_pinv():
    rng = np.random.default_rng(11)
    n = 40
    q, _ = np.linalg.qr(rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n)))
    spec = np.logspace(-9, 2, n)
    S = (q * spec) @ np.conj(q).T
    S = 0.5 * (S + np.conj(S).T)
    F = rng.normal(size=n) + 1j * rng.normal(size=n)
    for cut in (1e-12, 1e-6, 1e-3):
        d, sig, kept = qgt.pinv_solve(S, F, 1e-7, cut)
        St = S + 1e-7 * np.eye(n)
        ref = -np.linalg.pinv(St, rcond=cut, hermitian=True) @ F
        np.testing.assert_allclose(d, ref, rtol=1e-7 * np.linalg.norm(ref) / np.abs(ref).min(), atol=1e-9 * np.linalg.norm(ref))
        assert kept == np.sum(sig > cut * sig.max())
    d, sig, kept = qgt.pinv_solve(S, F, 1e-7, 1e-3, absolute=True)
    assert kept == np.sum(sig > 1e-3)


def test_full_qgt_solve_equals_ntk_solve():
    w, O, el = _sampled("j1j2_6x6_ffnn", 48)
    _, _, dO, e = qgt.center(O, el)
    F = qgt.force(dO, e)
    S = qgt.full_qgt(dO)
    lam = 1e-2
    d_full = -np.linalg.solve(S + lam * np.eye(S.shape[0]), F)
    d_ntk = qgt.ntk_solve(dO, e, lam)
    np.testing.assert_allclose(d_ntk, d_full, rtol=0, atol=1e-9 * np.linalg.norm(d_full))


def test_sample_permutation_and_duplication_invariance():
    w, O, el = _sampled("chain10_rbm", 120)
    def run(Ox, ex):
        _, _, dO, e = qgt.center(Ox, ex)
        F = qgt.force(dO, e)
        S = qgt.block_qgt(dO, w.block_off)
        return S, F, qgt.block_solve(S, F, w.block_off, 1e-4, 1e-10)[0]
    S0, F0, d0 = run(O, el)
    p = np.random.default_rng(3).permutation(120)
    for Ox, ex in ((O[p], el[p]), (np.concatenate([O, O]), np.concatenate([el, el]))):
        S1, F1, d1 = run(Ox, ex)
        for a, b in zip(S0, S1):
            np.testing.assert_allclose(a, b, atol=1e-13)
        np.testing.assert_allclose(F1, F0, atol=1e-13)
        np.testing.assert_allclose(d1, d0, rtol=1e-8, atol=1e-9 * np.linalg.norm(d0))


@pytest.mark.parametrize("weighted", [False, True])
def test_block_sample_space_solve_equals_block_solve(weighted):
    """Per-block push-through identity: for every block, the N_s x N_s sample-space solve
    equals the n_b x n_b eigen-decomposition solve when no eigenvalue is cut; blocks both
    wider (408, 200 parameters) and narrower (9) than the 100 samples."""
    model = W.Model(W.FFNN, (16, 24, 8, 1))
    rng = np.random.default_rng(21)
    theta = W.init_params(model, rng)
    x = W.zero_sz_configs(16, 100, rng)
    ij, jj = W.square_j1j2_bonds(4, 4, 1.0, 0.4)
    _, O = nqs.jacobian(model, theta, x)
    el = hamiltonian.local_energy(model, theta, x, ij, jj)
    w = None
    if weighted:
        r = rng.random(100) + 0.05
        w = r / r.sum()
    _, _, dO, e = qgt.center(O, el, w)
    F = qgt.force(dO, e, w)
    off = model.block_offsets()
    S = qgt.block_qgt(dO, off, w)
    lam = 3e-3
    ref, sig, kept = qgt.block_solve(S, F, off, lam, 1e-12, eta=0.7)
    assert all(k == n for k, n in zip(kept, np.diff(off)))
    d = qgt.block_solve_sample_space(dO, e, off, lam, eta=0.7, w=w)
    for b in range(len(off) - 1):
        sl = slice(off[b], off[b + 1])
        np.testing.assert_allclose(d[sl], ref[sl], rtol=0, atol=1e-10 * np.linalg.norm(ref[sl]))
    with pytest.raises(ValueError):
        qgt.block_solve_sample_space(dO, e, off, 0.0)
