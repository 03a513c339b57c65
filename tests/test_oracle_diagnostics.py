"""Pins of the inverse-metric diagnostics (Eq. 4) and the infidelity (Sec. 3)."""
import numpy as np

from oracle import diagnostics as D


def _herm(n, seed, lo=-3, hi=1):
    rng = np.random.default_rng(seed)
    q, _ = np.linalg.qr(rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n)))
    return (q * np.logspace(lo, hi, n)) @ np.conj(q).T


def test_identities():
    A = _herm(20, 1)
    B = _herm(20, 2)
    assert abs(D.frobenius_overlap(A, A) - 1) < 1e-12
    assert abs(D.frobenius_overlap(A, 3 * A) - 1) < 1e-12
    assert D.frobenius_rel_error(A, A) == 0
    assert abs(D.frobenius_rel_error(2 * A, A) - 1) < 1e-12
    assert abs(D.condition_number(A) - 1e4) < 1e-6 * 1e4
    assert abs(D.spectrum_correlation(A, 5 * A) - 1) < 1e-12
    assert abs(D.spectrum_correlation(A, B) - 1) < 1e-12  # same spectra
    assert -1 <= D.frobenius_overlap(A, B) <= 1


def test_infidelity():
    rng = np.random.default_rng(3)
    psi = rng.normal(size=64) + 1j * rng.normal(size=64)
    assert abs(D.infidelity(psi, 2.5 * np.exp(0.3j) * psi)) < 1e-14
    phi = rng.normal(size=64) + 1j * rng.normal(size=64)
    phi -= np.vdot(psi, phi) / np.vdot(psi, psi) * psi
    assert abs(D.infidelity(psi, phi) - 1) < 1e-12
