"""FFNN 100-256-256-1 on the 10x10 J1-J2 lattice (blocks of 25856, 65792 and 257 parameters).

* At 512 samples every block but the output layer is wider than the sample count, so the
  step runs the per-block sample-space solve (push-through identity); it must equal the
  oracle (whose wide blocks use its own sample-space form, pinned against its
  eigen-decomposition solve) to the split bar in the five-slice split and to 1e-10 in FP64.
* At the full 32768 samples the Jacobian (a 91905 x 32768 complex128 matrix) is checked on
  sampled entries against central finite differences of ln psi (h = 1e-6, FP64), each
  difference taken by the library's own forward on the sampled configurations.
"""
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


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("split_bf16_exact", 1e-6)])
def test_config5_step_at_512_samples_matches_oracle(prec, tol):
    import paper_2510_08430_gb300 as nq
    w = W.make_workload("j1j2_10x10_ffnn256", 512)
    sizes = np.diff(w.block_off)
    assert list(sizes) == [25856, 65792, 257]
    model, theta, x, ham = dev_inputs(w)
    dth, em, _, nk = nq.sr_step(model, theta, x, ham, w.block_off, w.diag_shift, w.cutoff, 1.0, prec,
                                solver="mixed", want_evals=False)
    _, O = oracle.nqs.jacobian(w.model, w.theta, w.configs)
    el = oracle.hamiltonian.local_energy(w.model, w.theta, w.configs, w.bond_ij, w.bond_j, w.c, w.sign_rule)
    e_mean, _, dO, e = oracle.qgt.center(O, el)
    ref = oracle.qgt.block_solve_sample_space(dO, e, w.block_off, w.diag_shift)
    assert rel(dth.cpu().numpy(), ref) < tol
    assert abs(em.cpu().numpy()[0] - e_mean) < 1e-12 * abs(e_mean)
    assert np.array_equal(nk.cpu().numpy(), sizes.astype(np.int32))


def test_config5_full_size_jacobian_against_finite_differences():
    import paper_2510_08430_gb300 as nq
    w = W.make_workload("j1j2_10x10_ffnn256")
    assert w.n_samples == 32768
    model, theta, x, _ = dev_inputs(w)
    _, O = nq.nqs_jacobian(model, theta, x, "fp64")
    rng = np.random.default_rng(0)
    ks = np.sort(rng.choice(w.model.n_params, size=24, replace=False))
    ss = np.sort(rng.choice(w.n_samples, size=256, replace=False))
    Os = O[torch.as_tensor(ks, device="cuda")][:, torch.as_tensor(ss, device="cuda")].cpu().numpy()
    del O
    torch.cuda.empty_cache()
    xs = x[torch.as_tensor(ss, device="cuda")].contiguous()
    h = 1e-6
    fd = np.empty((len(ks), len(ss)), dtype=np.complex128)
    for i, k in enumerate(ks):
        tp = theta.clone()
        tm = theta.clone()
        tp[int(k)] += h
        tm[int(k)] -= h
        lp, _ = nq.nqs_jacobian(model, tp, xs, "fp64")
        lm, _ = nq.nqs_jacobian(model, tm, xs, "fp64")
        fd[i] = (lp - lm).cpu().numpy() / (2 * h)
    scale = np.maximum(np.abs(Os).max(axis=1, keepdims=True), 1e-3)
    assert np.max(np.abs(Os - fd) / scale) < 1e-6
    # the same entries from the oracle's holomorphic backward on the sampled configurations
    _, Oo = oracle.nqs.jacobian(w.model, w.theta, w.configs[ss])
    assert rel(Os, Oo[:, ks].T) < 1e-12
