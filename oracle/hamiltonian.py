"""Local energies of the Heisenberg / J1-J2 Hamiltonians (Eq. 1, Sec. 3).

Test infrastructure (see package docstring). Plain NumPy / SciPy, float64.

H = c * sum_b J_b (sx_i sx_j + sy_i sy_j + sz_i sz_j) over the bond list, with
Pauli matrices s. c = 1 is the Pauli normalisation that the printed energies
of Table 2 imply (the printed S = sigma/2 operators correspond to c = 1/4).
In the S^z basis the bond term is diagonal c J x_i x_j and, for x_i != x_j,
has off-diagonal element 2 c J to the configuration with spins i and j
exchanged. An optional Marshall sign (sign_rule = -1) flips the sign of the
off-diagonal elements.

E_loc(x) = <x|H|psi> / <x|psi> (Eq. 1) is evaluated here with a FULL forward
pass of every connected configuration (no incremental update).
"""
from __future__ import annotations

import numpy as np

from . import nqs


def connections(configs: np.ndarray, bond_ij: np.ndarray):
    """Brute-force connected elements: list of (sample, bond) with x_i != x_j.

    Returned in sample-major, then bond order, as int64 [n_conn, 2].
    """
    x = np.asarray(configs)
    out = []
    for s in range(x.shape[0]):
        for b in range(bond_ij.shape[0]):
            i, j = bond_ij[b]
            if x[s, i] != x[s, j]:
                out.append((s, b))
    return np.array(out, dtype=np.int64).reshape(-1, 2)


def local_energy(model, theta, configs, bond_ij, bond_j, c: float = 1.0,
                 sign_rule: int = 1) -> np.ndarray:
    """E_loc [n_s] complex128, by full forward passes of flipped configurations."""
    x = np.asarray(configs, dtype=np.float64)
    lp = nqs.log_psi(model, theta, x)
    e = np.zeros(x.shape[0], dtype=np.complex128)
    for b in range(bond_ij.shape[0]):
        i, j = int(bond_ij[b, 0]), int(bond_ij[b, 1])
        jb = float(bond_j[b])
        e += c * jb * x[:, i] * x[:, j]
        anti = x[:, i] != x[:, j]
        if not anti.any():
            continue
        xf = x[anti].copy()
        xf[:, i] *= -1
        xf[:, j] *= -1
        lpf = nqs.log_psi(model, theta, xf)
        e[anti] += 2.0 * c * jb * sign_rule * np.exp(lpf - lp[anti])
    return e


# ---------- dense Hamiltonian for small N (pins only) ----------

_SX = np.array([[0, 1], [1, 0]], dtype=np.complex128)
_SY = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
_SZ = np.array([[1, 0], [0, -1]], dtype=np.complex128)


def _site_op(op, k, n):
    """Sparse op acting on site k of n sites; site 0 is the most significant factor."""
    import scipy.sparse as sp
    m = sp.identity(1, dtype=np.complex128, format="csr")
    for q in range(n):
        m = sp.kron(m, sp.csr_matrix(op) if q == k else sp.identity(2, format="csr"), format="csr")
    return m


def dense_hamiltonian(n_sites, bond_ij, bond_j, c: float = 1.0, sign_rule: int = 1,
                      sparse: bool = False):
    """H = c sum_b J_b (sx sx + sy sy + sz sz), built from Kronecker products of
    Pauli matrices (sign_rule = -1 negates the sx sx + sy sy part).

    Basis index bits: site 0 is the most significant bit; bit 0 means x = +1
    (the +1 eigenvector of sigma^z is the first basis vector).
    """
    dim = 2 ** n_sites
    import scipy.sparse as sp
    h = sp.csr_matrix((dim, dim), dtype=np.complex128)
    for b in range(bond_ij.shape[0]):
        i, j = int(bond_ij[b, 0]), int(bond_ij[b, 1])
        for op, sgn in ((_SX, sign_rule), (_SY, sign_rule), (_SZ, 1)):
            h = h + (c * bond_j[b] * sgn) * (_site_op(op, i, n_sites) @ _site_op(op, j, n_sites))
    return h if sparse else h.toarray()


def all_configs(n_sites: int) -> np.ndarray:
    """All 2^N configurations in the basis order of ``dense_hamiltonian``."""
    idx = np.arange(2 ** n_sites)
    bits = (idx[:, None] >> (n_sites - 1 - np.arange(n_sites))[None, :]) & 1
    return (1 - 2 * bits).astype(np.int8)


def ground_energy_sz0(n_sites, bond_ij, bond_j, c: float = 1.0) -> float:
    """Lowest eigenvalue of H in the S^z = 0 sector, by sparse Lanczos (SciPy)."""
    import itertools
    import scipy.sparse as sp
    import scipy.sparse.linalg as sla
    states = []
    for ups in itertools.combinations(range(n_sites), n_sites // 2):
        v = 0
        for u in ups:
            v |= 1 << u
        states.append(v)
    states = np.array(sorted(states), dtype=np.int64)
    index = {int(v): k for k, v in enumerate(states)}
    rows, cols, vals = [], [], []
    for k, v in enumerate(states):
        v = int(v)
        diag = 0.0
        for b in range(bond_ij.shape[0]):
            i, j = int(bond_ij[b, 0]), int(bond_ij[b, 1])
            si = 1 if (v >> i) & 1 else -1
            sj = 1 if (v >> j) & 1 else -1
            diag += c * bond_j[b] * si * sj
            if si != sj:
                w = v ^ (1 << i) ^ (1 << j)
                rows.append(k)
                cols.append(index[w])
                vals.append(2.0 * c * bond_j[b])
        rows.append(k)
        cols.append(k)
        vals.append(diag)
    h = sp.csr_matrix((vals, (rows, cols)), shape=(len(states), len(states)))
    ev = sla.eigsh(h, k=1, which="SA", tol=1e-12)[0]
    return float(ev[0])
