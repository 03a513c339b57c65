"""sr_step_batched (several SR instances, one grouped Gram and one eigensolver launch)
against one sr_step call per instance, and against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from gpu_util import dev_inputs, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def nq():
    import paper_2510_08430_gb300 as m
    return m


def _small_ffnn(seed, ns, widths=(16, 24, 8, 1), j2=0.3):
    """A third instance shape: FFNN on a 4x4 J1-J2 lattice (three blocks of unequal size)."""
    model = W.Model(W.FFNN, tuple(widths))
    rng = np.random.default_rng(seed)
    theta = W.init_params(model, rng)
    configs = W.zero_sz_configs(widths[0], ns, rng)
    ij, jj = W.square_j1j2_bonds(4, 4, 1.0, j2)
    return W.Workload(f"ffnn4x4_{seed}", model, theta, configs, ij, jj, model.block_offsets(), 1e-3, 1e-10,
                      "split_bf16_exact")


def _instances():
    return [W.make_workload("chain10_rbm", 200), W.make_workload("j1j2_6x6_ffnn", 300), _small_ffnn(7, 150)]


@pytest.mark.parametrize("prec,solver,tol", [
    ("fp64", "fp64", 1e-12),
    ("split_bf16_exact", "mixed", 1e-9),
    ("split_bf16x3", "mixed", 1e-9),
])
def test_batched_equals_separate_steps(prec, solver, tol):
    ws = _instances()
    ins = [dev_inputs(w) for w in ws]
    dths, em, _, nk = nq().sr_step_batched([i[0] for i in ins], [i[1] for i in ins], [i[2] for i in ins],
                                           [i[3] for i in ins], [w.block_off for w in ws], 1e-3, 1e-10, 1.0,
                                           prec, solver=solver)
    k = 0
    for j, (w, (model, theta, x, ham)) in enumerate(zip(ws, ins)):
        # the batched step forms every S_b in parameter space: compare with the same form
        d1, e1, _, n1 = nq().sr_step(model, theta, x, ham, w.block_off, 1e-3, 1e-10, 1.0, prec, solver=solver,
                                     param_space=True)
        assert rel(dths[j].cpu().numpy(), d1.cpu().numpy()) < tol, w.name
        assert abs(em[j].item() - e1.cpu().numpy()[0]) <= 1e-12 * abs(e1.cpu().numpy()[0])
        nbj = len(w.block_off) - 1
        assert np.array_equal(nk[k:k + nbj].cpu().numpy(), n1.cpu().numpy())
        k += nbj


def test_batched_fp64_matches_oracle():
    ws = _instances()
    ins = [dev_inputs(w) for w in ws]
    dths, em, _, nk = nq().sr_step_batched([i[0] for i in ins], [i[1] for i in ins], [i[2] for i in ins],
                                           [i[3] for i in ins], [w.block_off for w in ws], 1e-3, 1e-10, 1.0,
                                           "fp64", solver="fp64")
    for j, w in enumerate(ws):
        r = oracle.qgt.sr_step(w.model, w.theta, w.configs, w.bond_ij, w.bond_j, w.block_off, 1e-3, 1e-10, 1.0,
                               w.c, w.sign_rule)
        assert rel(dths[j].cpu().numpy(), r["dtheta"]) < 1e-10, w.name
        assert abs(em[j].item() - r["e_mean"]) < 1e-12 * abs(r["e_mean"])


def test_batched_8x8_twelve_layer_split_matches_oracle():
    """Two instances of the batched 8x8 workload (12-layer FFNN with widths cycling 32/64/128,
    blocks of 65 to 8320 parameters; J2/J1 = 0 and 0.28) at 256 samples each, in the five-slice
    split with the mixed solver, against the oracle. Every block but the last is wider than the
    sample count, so the oracle uses its per-block sample-space solve, which equals the block
    solve here (lambda = 1e-3 > 0, the 1e-10 cutoff drops nothing)."""
    ws = [W.make_workload(f"batch8x8_{i}", 256) for i in (0, 7)]
    ins = [dev_inputs(w) for w in ws]
    dths, em, _, nk = nq().sr_step_batched([i[0] for i in ins], [i[1] for i in ins], [i[2] for i in ins],
                                           [i[3] for i in ins], [w.block_off for w in ws], 1e-3, 1e-10, 1.0,
                                           "split_bf16_exact", solver="mixed")
    assert max(np.diff(ws[0].block_off)) == 8320
    k = 0
    for j, w in enumerate(ws):
        _, O = oracle.nqs.jacobian(w.model, w.theta, w.configs)
        el = oracle.hamiltonian.local_energy(w.model, w.theta, w.configs, w.bond_ij, w.bond_j, w.c, w.sign_rule)
        e_mean, _, dO, e = oracle.qgt.center(O, el)
        ref = oracle.qgt.block_solve_sample_space(dO, e, w.block_off, 1e-3)
        assert rel(dths[j].cpu().numpy(), ref) < 1e-6, w.name
        assert abs(em[j].item() - e_mean) < 1e-12 * abs(e_mean)
        nbj = len(w.block_off) - 1
        assert np.array_equal(nk[k:k + nbj].cpu().numpy(), np.diff(w.block_off).astype(np.int32))
        k += nbj


def test_batched_rejects_too_many_blocks():
    ws = [_small_ffnn(s, 64) for s in range(90)]  # 90 instances x 3 blocks > 256
    ins = [dev_inputs(w) for w in ws]
    with pytest.raises(nq().NQSError):
        nq().sr_step_batched([i[0] for i in ins], [i[1] for i in ins], [i[2] for i in ins], [i[3] for i in ins],
                             [w.block_off for w in ws], 1e-3, 1e-10)
