"""Exact expectations by enumeration of all 2^N states (N <= 12).

Test infrastructure (see package docstring). Plain NumPy, complex128.

The Born distribution (Eq. 1) is replaced by its exact weights
w(x) = |psi(x)|^2 / sum_y |psi(y)|^2 over the full Hilbert space, so every
sampled expectation of the method becomes an exact one. Derivatives of psi
itself are taken by central finite differences of psi (never through the
Jacobian O), which gives the first form of Eq. 2 independently of the
second.
"""
from __future__ import annotations

import numpy as np

from . import hamiltonian, nqs


def psi_vector(model, theta, n_sites):
    x = hamiltonian.all_configs(n_sites)
    return x, np.exp(nqs.log_psi(model, theta, x))


def born_weights(model, theta, n_sites):
    x, psi = psi_vector(model, theta, n_sites)
    p = np.abs(psi) ** 2
    return x, p / p.sum()


def energy(model, theta, n_sites, bond_ij, bond_j, c=1.0) -> float:
    """<psi|H|psi>/<psi|psi> with the dense Hamiltonian (left side of Eq. 1)."""
    _, psi = psi_vector(model, theta, n_sites)
    h = hamiltonian.dense_hamiltonian(n_sites, bond_ij, bond_j, c)
    return float(np.real(np.vdot(psi, h @ psi) / np.vdot(psi, psi)))


def dpsi_fd(model, theta, n_sites, h=1e-6):
    """d psi(x) / d theta_k for all x, k by central differences (complex step
    along the real axis; psi is holomorphic in theta)."""
    n_p = theta.shape[0]
    x = hamiltonian.all_configs(n_sites)
    out = np.empty((x.shape[0], n_p), dtype=np.complex128)
    for k in range(n_p):
        tp = theta.copy()
        tm = theta.copy()
        tp[k] += h
        tm[k] -= h
        out[:, k] = (np.exp(nqs.log_psi(model, tp, x)) - np.exp(nqs.log_psi(model, tm, x))) / (2 * h)
    return out


def qgt_first_form(psi: np.ndarray, dpsi: np.ndarray) -> np.ndarray:
    """First form of Eq. 2: <d_i psi|d_j psi>/<psi|psi> - <d_i psi|psi><psi|d_j psi>/<psi|psi>^2."""
    nrm = np.vdot(psi, psi).real
    g = np.conj(dpsi).T @ dpsi / nrm
    v = np.conj(dpsi).T @ psi / nrm
    return g - np.outer(v, np.conj(v))
