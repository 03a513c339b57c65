"""Sample-sharded step through the library with ranks simulated on one GPU (shards in turn,
sums on the host) against the unsharded sr_step and the FP64 oracle. In the FP64 path the
two orders of summation agree to rounding; in the split precision each shard forms its own
16-sample exponent groups, so sharded and unsharded are two roundings of the same step and
both are held to the split bar against the oracle."""
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


@pytest.mark.parametrize("name,ns,prec,solver,tol", [
    ("j1j2_6x6_ffnn", 300, "fp64", "fp64", 1e-11),
    ("j1j2_6x6_ffnn", 300, "split_bf16_exact", "mixed", 1e-6),
    ("chain10_rbm", 333, "fp64", "fp64", 1e-11),
])
def test_simulated_ranks_equal_unsharded_step(name, ns, prec, solver, tol):
    import paper_2510_08430_gb300 as nq
    from paper_2510_08430_gb300 import sharded
    w = W.make_workload(name, ns)
    model, theta, x, ham = dev_inputs(w)
    shards = [x[idx] for idx in np.array_split(np.arange(ns), 3)]
    be = sharded.LibraryShardBackend(model, ham, w.block_off, prec, solver)
    dth, em = sharded.step_simulated(be, theta, shards, w.block_off, w.diag_shift, w.cutoff)
    d1, e1, _, _ = nq.sr_step(model, theta, x, ham, w.block_off, w.diag_shift, w.cutoff, 1.0, prec, solver=solver,
                              want_evals=False, param_space=True)
    assert rel(dth.cpu().numpy(), d1.cpu().numpy()) < tol
    r = oracle.qgt.sr_step(w.model, w.theta, w.configs, w.bond_ij, w.bond_j, w.block_off, w.diag_shift, w.cutoff,
                           1.0, w.c, w.sign_rule)
    assert rel(dth.cpu().numpy(), r["dtheta"]) < (1e-10 if prec == "fp64" else 1e-6)
    assert abs(em.cpu().numpy()[0] - e1.cpu().numpy()[0]) <= 1e-12 * abs(e1.cpu().numpy()[0])
