"""Pins of the oracle's VMC loop (exchange-move Metropolis sampling of |psi|^2, Sec. 1; the
SR update of Sec. 2).

The sampler is pinned by its stationary distribution against |psi|^2 / Z computed by exact
enumeration of the S^z = 0 sector, the proposal by brute force, and the loop by reaching
the exact ground energy of a small chain (Lanczos) from a random start.
"""
import itertools

import numpy as np

import workloads as W
from oracle import exact, hamiltonian, nqs, vmc


def test_proposal_picks_the_counted_up_and_down_spins():
    rng = np.random.default_rng(0)
    x = W.zero_sz_configs(10, 200, rng)
    u = rng.random((200, 2))
    ii, jj, ok = vmc.propose(x, u[:, 0], u[:, 1])
    assert ok.all()
    for c in range(200):
        ups = [s for s in range(10) if x[c, s] == 1]     # brute force, site order
        dns = [s for s in range(10) if x[c, s] == -1]
        assert ii[c] == ups[int(u[c, 0] * 5)] and jj[c] == dns[int(u[c, 1] * 5)]
    # a fully polarised chain has no exchange move
    _, _, ok1 = vmc.propose(np.ones((3, 4), dtype=np.int8), u[:3, 0], u[:3, 1])
    assert not ok1.any()


def test_sampler_conserves_sz_and_is_reproducible():
    w = W.make_workload("chain10_rbm", 64)
    u = W.metropolis_uniforms(30, 64, 7)
    x1, a1 = vmc.metropolis(w.model, w.theta, w.configs, u)
    x2, a2 = vmc.metropolis(w.model, w.theta, w.configs, u)
    assert np.array_equal(x1, x2) and a1 == a2 and a1 > 0
    assert np.array_equal(x1.sum(axis=1), w.configs.sum(axis=1))


def test_stationary_distribution_is_born_rule():
    """Chains started anywhere in the S^z = 0 sector of a 6-site RBM with strongly varying
    amplitudes end up distributed as |psi|^2 / Z over the 20 states of the sector."""
    n = 6
    model = W.Model(W.RBM, (n, 6))
    rng = np.random.default_rng(3)
    theta = (rng.normal(size=model.n_params) + 1j * rng.normal(size=model.n_params)) * 0.4
    states = []
    for ups in itertools.combinations(range(n), n // 2):
        s = -np.ones(n, dtype=np.int8)
        s[list(ups)] = 1
        states.append(s)
    states = np.array(states)
    p = np.abs(np.exp(nqs.log_psi(model, theta, states))) ** 2
    p /= p.sum()
    n_chains, burn, keep = 3000, 100, 40
    x0 = W.zero_sz_configs(n, n_chains, np.random.default_rng(4))
    x, _ = vmc.metropolis(model, theta, x0, W.metropolis_uniforms(burn, n_chains, 5))
    counts = np.zeros(len(states))
    idx = {tuple(s): k for k, s in enumerate(states)}
    u = W.metropolis_uniforms(keep, n_chains, 6)
    for t in range(keep):
        x, _ = vmc.metropolis(model, theta, x, u[t:t + 1])
        for row in x:
            counts[idx[tuple(row)]] += 1
    q = counts / counts.sum()
    tv = 0.5 * np.abs(q - p).sum()
    assert tv < 0.01, tv
    # the pin discriminates: the distribution of |psi| (a wrong acceptance ratio) is far away
    pa = np.sqrt(p) / np.sqrt(p).sum()
    assert 0.5 * np.abs(pa - p).sum() > 0.1


def test_training_loop_reaches_the_ground_energy():
    """The loop (sampling, block-layer SR step, update) takes an RBM on the 8-site chain from
    its random start to within 1% of the exact ground energy (variational energy of the
    trained state by enumeration), and the sampled <E> agrees with that exact energy."""
    n = 8
    model = W.Model(W.RBM, (n, 16))
    theta = W.init_params(model, np.random.default_rng(11))
    ij, jj = W.chain_bonds(n, 1.0)
    x0 = W.zero_sz_configs(n, 256, np.random.default_rng(12))
    us = [W.metropolis_uniforms(8, 256, 100 + k) for k in range(40)]
    theta1, x1, energies = vmc.train(model, theta, x0, ij, jj, model.block_offsets(), 1e-3, 1e-10, 0.05, us,
                                     1.0, -1)
    e0 = hamiltonian.ground_energy_sz0(n, ij, jj, 1.0)
    # exact energy of the trained state within the S^z = 0 sector (Marshall-rotated H)
    xs = hamiltonian.all_configs(n)
    xs = xs[xs.sum(axis=1) == 0]
    psi = np.exp(nqs.log_psi(model, theta1, xs))
    el = hamiltonian.local_energy(model, theta1, xs, ij, jj, 1.0, -1)
    e_var = float(np.real(np.sum(np.abs(psi) ** 2 * el) / np.sum(np.abs(psi) ** 2)))
    assert e_var >= e0 - 1e-9
    assert (e_var - e0) / abs(e0) < 0.01, (e_var, e0)
    assert abs(np.mean([e.real for e in energies[-10:]]) - e_var) / abs(e0) < 0.01
    assert energies[0].real > energies[-1].real
