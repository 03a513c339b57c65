"""Inverse-metric diagnostics (Eq. 4) computed by the library against the oracle.

B is the pseudo-inverse of the exact QGT of a state small enough to enumerate (all 2^N
configurations weighted by |psi|^2 / Z; the oracle's exact QGT is pinned against the first
form of Eq. 2); A that of the block-layer restriction of the sampled QGT, of the full
sampled QGT, or of the block-layer restriction of the exact QGT. The paper's own Table 1
values need its trained network and stay unpinned."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from gpu_util import dev_inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _pinv(S, shift, cutoff):
    sig, U = np.linalg.eigh(S + shift * np.eye(S.shape[0]))
    keep = sig > cutoff * sig.max()
    return (U * np.where(keep, 1.0 / np.where(keep, sig, 1.0), 0.0)) @ np.conj(U).T, np.where(keep, 1 / sig, 0.0)


def _oracle_diag(Sa, off, Sb, shift, cutoff):
    Sr = np.zeros_like(Sa)
    for b in range(len(off) - 1):
        sl = slice(off[b], off[b + 1])
        Sr[sl, sl] = Sa[sl, sl]
    A, ea = _pinv(Sr, shift, cutoff)
    B, eb = _pinv(Sb, shift, cutoff)
    D = oracle.diagnostics
    ka = ea[ea > 0].max() / ea[ea > 0].min()
    kb = eb[eb > 0].max() / eb[eb > 0].min()
    return {"F": D.frobenius_overlap(A, B), "eps_F": D.frobenius_rel_error(A, B), "kappa_A": ka, "kappa_B": kb,
            "r_lambda": D.spectrum_correlation(A, B)}


def _oracle_qgts(w):
    x_all = oracle.hamiltonian.all_configs(w.model.n_sites)
    _, O_all = oracle.nqs.jacobian(w.model, w.theta, x_all)
    wts = oracle.exact.born_weights(w.model, w.theta, w.model.n_sites)[1]
    _, _, dO, _ = oracle.qgt.center(O_all, np.zeros(x_all.shape[0]), wts)
    S_exact = oracle.qgt.full_qgt(dO, wts)
    _, O = oracle.nqs.jacobian(w.model, w.theta, w.configs)
    _, _, dOs, _ = oracle.qgt.center(O, np.zeros(w.configs.shape[0]))
    return oracle.qgt.full_qgt(dOs), S_exact


def _small_ffnn():
    model = W.Model(W.FFNN, (12, 10, 6, 1))
    rng = np.random.default_rng(41)
    theta = W.init_params(model, rng) * 1.5
    x = W.zero_sz_configs(12, 300, rng)
    ij, jj = W.square_j1j2_bonds(3, 4, 1.0, 0.5)
    return W.Workload("ffnn3x4", model, theta, x, ij, jj, model.block_offsets(), 1e-3, 1e-10, "fp64")


@pytest.mark.parametrize("make", [lambda: W.make_workload("chain10_rbm", 512), _small_ffnn])
@pytest.mark.parametrize("cutoff", [1e-12, 1e-4])
def test_inverse_metric_study_matches_oracle(make, cutoff):
    import paper_2510_08430_gb300 as nq
    w = make()
    model, theta, x, _ = dev_inputs(w)
    shift = w.diag_shift
    got = nq.inverse_metric_study(model, theta, x, w.block_off, shift, cutoff)
    S_samp, S_exact = _oracle_qgts(w)
    full = np.array([0, w.model.n_params])
    ref = {"block_sampled_vs_exact": _oracle_diag(S_samp, w.block_off, S_exact, shift, cutoff),
           "full_sampled_vs_exact": _oracle_diag(S_samp, full, S_exact, shift, cutoff),
           "block_exact_vs_exact": _oracle_diag(S_exact, w.block_off, S_exact, shift, cutoff)}
    for case, r in ref.items():
        g = got[case]
        for k in ("F", "r_lambda"):
            assert abs(g[k] - r[k]) < 1e-9, (case, k, g[k], r[k])
        for k in ("eps_F", "kappa_A", "kappa_B"):
            assert abs(g[k] - r[k]) <= 1e-7 * abs(r[k]) + 1e-9, (case, k, g[k], r[k])
    # the block-layer inverse of the exact QGT is not the exact inverse; the full one is closer
    assert got["block_exact_vs_exact"]["F"] < 1.0
