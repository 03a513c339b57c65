"""Variational Monte Carlo loop: exchange-move Metropolis sampling of |psi|^2 and the
SR update theta <- theta + dtheta (Sec. 1: samples drawn from the square of the
wavefunction by Markov chain Monte Carlo; Sec. 2, Eq. 1 update with the block-layer QGT).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sampler, in the order of its steps (one step = one proposal per chain):
  1. from the chain's configuration x pick the k1-th up spin i, k1 = floor(u1 n_up), and the
     k2-th down spin j, k2 = floor(u2 n_down), counting sites in increasing order;
  2. x' = x with spins i and j flipped (an exchange: total S^z is conserved);
  3. accept x' when u3 < |psi(x') / psi(x)|^2 = exp(2 Re(ln psi(x') - ln psi(x))).
The proposal is symmetric (n_up and n_down do not change), so this is the Metropolis rule
for the distribution |psi|^2 restricted to the chain's S^z sector. The uniforms (u1, u2, u3)
are inputs, one triple per step and chain. A chain with no up or no down spin stays put.
ln psi is a full forward pass of each configuration (no incremental update).

Parity: the chains are pinned by their stationary distribution against |psi|^2 / Z by
exact enumeration, and the loop by its convergence toward the exact ground energy.
"""
from __future__ import annotations

import numpy as np

from . import nqs, qgt


def propose(x: np.ndarray, u1: np.ndarray, u2: np.ndarray):
    """Exchange pairs (i, j) of every chain and a validity mask (steps 1-2)."""
    n_chains = x.shape[0]
    ii = np.zeros(n_chains, dtype=np.int64)
    jj = np.zeros(n_chains, dtype=np.int64)
    ok = np.zeros(n_chains, dtype=bool)
    for c in range(n_chains):
        ups = np.flatnonzero(x[c] == 1)
        dns = np.flatnonzero(x[c] == -1)
        if len(ups) == 0 or len(dns) == 0:
            continue
        ii[c] = ups[int(np.floor(u1[c] * len(ups)))]
        jj[c] = dns[int(np.floor(u2[c] * len(dns)))]
        ok[c] = True
    return ii, jj, ok


def metropolis(model, theta, x0: np.ndarray, uniforms: np.ndarray):
    """Run uniforms.shape[0] Metropolis steps on every chain. Returns (x, n_accepted)."""
    x = np.array(x0, dtype=np.int8, copy=True)
    n_acc = 0
    rows = np.arange(x.shape[0])
    for t in range(uniforms.shape[0]):
        u = uniforms[t]
        ii, jj, ok = propose(x, u[:, 0], u[:, 1])
        xp = x.copy()
        xp[rows[ok], ii[ok]] *= -1
        xp[rows[ok], jj[ok]] *= -1
        d = nqs.log_psi(model, theta, xp) - nqs.log_psi(model, theta, x)
        acc = ok & (u[:, 2] < np.exp(2.0 * d.real))
        x[acc] = xp[acc]
        n_acc += int(acc.sum())
    return x, n_acc


def train(model, theta0, x0, bond_ij, bond_j, block_off, diag_shift, cutoff, eta, uniforms_per_iter,
          c=1.0, sign_rule=1):
    """VMC loop: for every array of uniforms, sample, take one block-layer SR step on the
    samples and add dtheta to theta. Returns (theta, x, list of <E>)."""
    theta = np.array(theta0, dtype=np.complex128, copy=True)
    x = np.array(x0, dtype=np.int8, copy=True)
    energies = []
    for u in uniforms_per_iter:
        x, _ = metropolis(model, theta, x, u)
        r = qgt.sr_step(model, theta, x, bond_ij, bond_j, block_off, diag_shift, cutoff, eta, c, sign_rule)
        theta = theta + r["dtheta"]
        energies.append(complex(r["e_mean"]))
    return theta, x, energies
