"""Block-layer QGT and the shifted pseudo-inverse solve (Sec. 2).

Test infrastructure (see package docstring). Plain NumPy, complex128.

Readings of the paper fixed here:
* Expectations are weighted sums sum_s w_s f(x_s) with sum_s w_s = 1;
  w_s = 1/N_s for Born samples (Eq. 1, Eq. 2), w = |psi|^2/Z for enumeration.
* Centring first (second form of Eq. 2): dO = O - <O>, e = E_loc - <E>.
* Force F_k = sum_s w_s conj(dO_sk) e_s (Sec. 2: F is the energy gradient;
  any factor 2 is absorbed into the step size eta).
* Block QGT (Eq. 3): S_b = sum_s w_s dO_sb^H dO_sb for the contiguous block
  [off_b, off_{b+1}) of the flat parameter vector.
* Solve (Sec. 2, block-layer paragraph, and the pseudo-inverse remark after
  Eq. 2): S~_b = S_b + lambda I; S~_b = U diag(sigma) U^H (LAPACK eigh);
  keep sigma_i > cutoff * max_i sigma_i (relative; "absolute" mode keeps
  sigma_i > cutoff); dtheta_b = -eta U diag(keep/sigma) U^H F_b.
"""
from __future__ import annotations

import numpy as np

from . import hamiltonian, nqs


def uniform_weights(n_s: int) -> np.ndarray:
    return np.full(n_s, 1.0 / n_s)


def center(O: np.ndarray, eloc: np.ndarray, w=None):
    """(<E>, <O>, dO, e) with weights w (default uniform)."""
    O = np.asarray(O, dtype=np.complex128)
    eloc = np.asarray(eloc, dtype=np.complex128)
    w = uniform_weights(O.shape[0]) if w is None else np.asarray(w, dtype=np.float64)
    e_mean = np.sum(w * eloc)
    o_mean = w @ O
    return e_mean, o_mean, O - o_mean, eloc - e_mean


def force(dO: np.ndarray, e: np.ndarray, w=None) -> np.ndarray:
    """F_k = sum_s w_s conj(dO_sk) e_s."""
    w = uniform_weights(dO.shape[0]) if w is None else np.asarray(w, dtype=np.float64)
    return np.conj(dO).T @ (w * e)


def block_qgt(dO: np.ndarray, block_off, w=None):
    """List of S_b = dO_b^H diag(w) dO_b (n_b x n_b, complex128)."""
    w = uniform_weights(dO.shape[0]) if w is None else np.asarray(w, dtype=np.float64)
    out = []
    for b in range(len(block_off) - 1):
        x = dO[:, block_off[b]:block_off[b + 1]]
        out.append(np.conj(x).T @ (w[:, None] * x))
    return out


def full_qgt(dO: np.ndarray, w=None) -> np.ndarray:
    return block_qgt(dO, [0, dO.shape[1]], w)[0]


def pinv_solve(S: np.ndarray, F: np.ndarray, diag_shift: float, cutoff: float,
               eta: float = 1.0, absolute: bool = False):
    """(dtheta, sigma ascending, n_kept) for one block."""
    St = S + diag_shift * np.eye(S.shape[0])
    sig, U = np.linalg.eigh(St)
    thr = cutoff if absolute else cutoff * sig.max()
    keep = sig > thr
    inv = np.where(keep, 1.0 / np.where(keep, sig, 1.0), 0.0)
    dth = -eta * (U @ (inv * (np.conj(U).T @ F)))
    return dth, sig, int(keep.sum())


def block_solve(S_blocks, F, block_off, diag_shift, cutoff, eta=1.0, absolute=False):
    """Concatenated dtheta, list of eigenvalues, n_kept per block."""
    dth = np.empty(block_off[-1], dtype=np.complex128)
    sigs, kept = [], []
    for b, S in enumerate(S_blocks):
        lo, hi = block_off[b], block_off[b + 1]
        d, s, k = pinv_solve(S, F[lo:hi], diag_shift, cutoff, eta, absolute)
        dth[lo:hi] = d
        sigs.append(s)
        kept.append(k)
    return dth, sigs, np.array(kept, dtype=np.int32)


def ntk_solve(dO: np.ndarray, e: np.ndarray, diag_shift: float, eta: float = 1.0, w=None):
    """Sample-space solve: dtheta = -eta X^H (X X^H + lambda I)^-1 eps,
    X = sqrt(w) dO, eps = sqrt(w) e (the NTK form the paper compares against)."""
    w = uniform_weights(dO.shape[0]) if w is None else np.asarray(w, dtype=np.float64)
    sw = np.sqrt(w)
    X = sw[:, None] * dO
    eps = sw * e
    T = X @ np.conj(X).T + diag_shift * np.eye(X.shape[0])
    return -eta * (np.conj(X).T @ np.linalg.solve(T, eps))


def block_solve_sample_space(dO: np.ndarray, e: np.ndarray, block_off, diag_shift: float, eta: float = 1.0,
                             w=None) -> np.ndarray:
    """Per-block sample-space form of the block-layer update, for blocks with more
    parameters than samples. With X_b = sqrt(w) dO_b (N_s x n_b) and eps = sqrt(w) e, the
    block update -eta (X_b^H X_b + lambda I)^-1 X_b^H eps equals
        dtheta_b = -eta X_b^H (X_b X_b^H + lambda I)^-1 eps
    (push-through identity), which needs an N_s x N_s solve instead of an n_b x n_b one.
    It is the block solve of Sec. 2 exactly when lambda > 0 and no eigenvalue is cut
    (every eigenvalue of S_b + lambda I is at least lambda)."""
    if not diag_shift > 0:
        raise ValueError("the sample-space form needs a positive diagonal shift")
    w = uniform_weights(dO.shape[0]) if w is None else np.asarray(w, dtype=np.float64)
    sw = np.sqrt(w)
    eps = sw * np.asarray(e, dtype=np.complex128)
    out = np.empty(block_off[-1], dtype=np.complex128)
    for b in range(len(block_off) - 1):
        X = sw[:, None] * dO[:, block_off[b]:block_off[b + 1]]
        T = X @ np.conj(X).T + diag_shift * np.eye(X.shape[0])
        out[block_off[b]:block_off[b + 1]] = -eta * (np.conj(X).T @ np.linalg.solve(T, eps))
    return out


def sr_step(model, theta, configs, bond_ij, bond_j, block_off, diag_shift, cutoff,
            eta=1.0, c=1.0, sign_rule=1, w=None, absolute=False):
    """One block-layer SR step. Returns a dict of every intermediate."""
    lp, O = nqs.jacobian(model, theta, configs)
    eloc = hamiltonian.local_energy(model, theta, configs, bond_ij, bond_j, c, sign_rule)
    e_mean, o_mean, dO, e = center(O, eloc, w)
    F = force(dO, e, w)
    S = block_qgt(dO, block_off, w)
    dth, sig, kept = block_solve(S, F, block_off, diag_shift, cutoff, eta, absolute)
    return dict(log_psi=lp, O=O, eloc=eloc, e_mean=e_mean, o_mean=o_mean, dO=dO, e=e,
                F=F, S=S, dtheta=dth, sigma=sig, n_kept=kept)
