"""ntk_solve (sample-space form of the full-QGT update) against the oracle's NTK solve and,
by the push-through identity, against the full-QGT step (one block of all parameters)."""
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


@pytest.mark.parametrize("name,ns,prec,tol", [
    ("chain10_rbm", 200, "fp64", 1e-10),
    ("j1j2_6x6_ffnn", 300, "fp64", 1e-10),
    ("j1j2_6x6_ffnn", 300, "fp32", 1e-4),
])
def test_ntk_solve(name, ns, prec, tol):
    import paper_2510_08430_gb300 as nq
    w = W.make_workload(name, ns)
    model, theta, x, ham = dev_inputs(w)
    _, O = nq.nqs_jacobian(model, theta, x, "fp64")
    el = nq.nqs_local_energy(model, theta, x, ham, "fp64")
    dth, em = nq.ntk_solve(O, ns, el, w.diag_shift, 1e-10, 1.0, prec)
    # oracle
    _, Oo = oracle.nqs.jacobian(w.model, w.theta, w.configs)
    elo = oracle.hamiltonian.local_energy(w.model, w.theta, w.configs, w.bond_ij, w.bond_j, w.c, w.sign_rule)
    _, _, dO, e = oracle.qgt.center(Oo, elo)
    ref = oracle.qgt.ntk_solve(dO, e, w.diag_shift)
    assert rel(dth.cpu().numpy(), ref) < tol
    if prec == "fp64":
        # push-through: equal to the full-QGT step
        full = np.array([0, int(w.block_off[-1])], dtype=np.int64)
        d_full, _, _, _ = nq.sr_step(model, theta, x, ham, full, w.diag_shift, 1e-10, 1.0, "fp64", solver="fp64")
        assert rel(dth.cpu().numpy(), d_full.cpu().numpy()) < 1e-9
