"""Inverse-metric diagnostics (Eq. 4) and the infidelity (Sec. 3).

Test infrastructure (see package docstring). Plain NumPy.

A and B are Hermitian matrices (the inverse block-layer and inverse exact
QGT in the paper). (a) Frobenius overlap Tr[A^H B]/(|A|_F |B|_F);
(b) relative Frobenius error |A-B|_F/|B|_F; (c) condition number
lambda_max/lambda_min; (d) Pearson correlation of the two spectra sorted in
descending order. Infidelity 1 - |<psi|phi>|^2 / (<psi|psi><phi|phi>).
The values of Table 1 need the paper's trained network and are not
reproduced (parity unpinned for those numbers).
"""
from __future__ import annotations

import numpy as np


def frobenius_overlap(A, B) -> float:
    return float(np.real(np.trace(np.conj(A).T @ B)) / (np.linalg.norm(A) * np.linalg.norm(B)))


def frobenius_rel_error(A, B) -> float:
    return float(np.linalg.norm(A - B) / np.linalg.norm(B))


def condition_number(A) -> float:
    ev = np.linalg.eigvalsh(A)
    return float(ev.max() / ev.min())


def spectrum_correlation(A, B) -> float:
    a = np.sort(np.linalg.eigvalsh(A))[::-1]
    b = np.sort(np.linalg.eigvalsh(B))[::-1]
    return float(np.corrcoef(a, b)[0, 1])


def infidelity(psi, phi) -> float:
    ov = np.vdot(psi, phi)
    return float(1.0 - abs(ov) ** 2 / (np.vdot(psi, psi).real * np.vdot(phi, phi).real))
