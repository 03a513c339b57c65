"""Failure paths of the library, driven from the host without faulting the GPU.

* Non-finite inputs (NaN or Inf written into theta, O, E_loc or S by the test) must come back
  as NQS_ERR_NONFINITE from the device status word.
* Sweep limits lowered by the nqs_set_limits test hook must come back as
  NQS_ERR_NOT_CONVERGED (implicit QL; iterative refinement).
* A device wait budget lowered to 1 ns makes the grid barriers of the persistent solver
  kernels run out: NQS_ERR_TIMEOUT, the kernels return, and the context stays usable.
* A bond index outside [0, N) is NQS_ERR_INVALID_ARG and is never used to index memory.
After every case the defaults are restored and a normal call must still succeed.
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


@pytest.fixture(autouse=True)
def _default_limits():
    import paper_2510_08430_gb300 as nq
    nq.api.set_limits(0, 0)
    yield
    nq.api.set_limits(0, 0)


def _code(fn, *a, **k):
    from paper_2510_08430_gb300._lib import NQSError
    with pytest.raises(NQSError) as ei:
        fn(*a, **k)
        torch.cuda.synchronize()
    return ei.value.code


def _psd_blocks(sizes, seed, spread=1e-2):
    rng = np.random.default_rng(seed)
    blocks = []
    for n in sizes:
        X = rng.normal(size=(2 * n + 3, n)) + 1j * rng.normal(size=(2 * n + 3, n))
        X[:, : n // 2] *= spread
        blocks.append(np.conj(X).T @ X / X.shape[0])
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    F = rng.normal(size=off[-1]) + 1j * rng.normal(size=off[-1])
    return blocks, off, F


def _solve(blocks, off, F, shift, cutoff, solver, want_evals=True):
    import paper_2510_08430_gb300 as nq
    S = torch.as_tensor(np.concatenate([B.ravel() for B in blocks]), device="cuda")
    return nq.qgt_block_solve(S, off, torch.as_tensor(F, device="cuda"), shift, cutoff, 0, 1.0,
                              want_evals=want_evals, solver=solver)


def _ok_step():
    """A normal FP64 step after a failure: the context is usable and the result is right."""
    import paper_2510_08430_gb300 as nq
    w = W.make_workload("chain10_rbm", 64)
    model, theta, x, ham = dev_inputs(w)
    dth, _, _, _ = nq.sr_step(model, theta, x, ham, w.block_off, w.diag_shift, w.cutoff, 1.0, "fp64")
    r = oracle.qgt.sr_step(w.model, w.theta, w.configs, w.bond_ij, w.bond_j, w.block_off, w.diag_shift, w.cutoff)
    assert rel(dth.cpu().numpy(), r["dtheta"]) < 1e-10


@pytest.mark.parametrize("prec", ["fp64", "split_bf16_exact"])
def test_nan_in_theta_is_nonfinite(prec):
    import paper_2510_08430_gb300 as nq
    from paper_2510_08430_gb300._lib import NQS_ERR_NONFINITE
    w = W.make_workload("j1j2_6x6_ffnn", 96)
    model, theta, x, ham = dev_inputs(w)
    theta = theta.clone()
    theta[7] = complex(float("nan"), 0.0)
    assert _code(nq.sr_step, model, theta, x, ham, w.block_off, w.diag_shift, w.cutoff, 1.0, prec,
                 solver="mixed", want_evals=False) == NQS_ERR_NONFINITE
    _ok_step()


@pytest.mark.parametrize("where", ["O", "eloc"])
def test_nonfinite_jacobian_or_local_energy(where):
    import paper_2510_08430_gb300 as nq
    from paper_2510_08430_gb300._lib import NQS_ERR_NONFINITE
    w = W.make_workload("j1j2_6x6_ffnn", 80)
    model, theta, x, ham = dev_inputs(w)
    _, O = nq.nqs_jacobian(model, theta, x, "fp64")
    el = nq.nqs_local_energy(model, theta, x, ham, "fp64")
    if where == "O":
        O[100, 17] = complex(float("inf"), 0.0)
    else:
        el[5] = complex(0.0, float("nan"))
    assert _code(nq.qgt_block_build, O, 80, w.block_off, el, "fp64") == NQS_ERR_NONFINITE
    _ok_step()


@pytest.mark.parametrize("solver", ["fp64", "mixed"])
def test_nan_in_S_is_nonfinite(solver):
    from paper_2510_08430_gb300._lib import NQS_ERR_NONFINITE
    blocks, off, F = _psd_blocks([40, 70], 3)
    blocks[1][5, 3] = np.nan
    assert _code(_solve, blocks, off, F, 1e-4, 1e-10, solver) == NQS_ERR_NONFINITE
    _ok_step()


def test_ql_sweep_limit_is_not_converged():
    """A binding cutoff makes the FP64 path form eigenvectors by implicit QL; one sweep per
    eigenvalue is not enough."""
    import paper_2510_08430_gb300 as nq
    from paper_2510_08430_gb300._lib import NQS_ERR_NOT_CONVERGED
    blocks, off, F = _psd_blocks([60, 33], 5, spread=1e-4)
    nq.api.set_limits(1, 0)
    assert _code(_solve, blocks, off, F, 1e-9, 1e-3, "fp64") == NQS_ERR_NOT_CONVERGED
    nq.api.set_limits(0, 0)
    dth, _, nk = _solve(blocks, off, F, 1e-9, 1e-3, "fp64")
    ref, _, kept = oracle.qgt.block_solve(blocks, F, off, 1e-9, 1e-3)
    assert np.array_equal(nk.cpu().numpy(), kept) and kept.min() < 60
    assert rel(dth.cpu().numpy(), ref) < 1e-9


@pytest.mark.parametrize("want_evals", [True, False])
def test_refinement_sweep_limit_hands_over_to_fp64(want_evals):
    """One refinement sweep of the mixed solvers cannot reach ||r|| <= 1e-14 ||F||: the
    unconverged blocks are handed to the FP64 path, whose result is still the definition."""
    import paper_2510_08430_gb300 as nq
    blocks, off, F = _psd_blocks([300, 129], 8)
    ref, _, _ = oracle.qgt.block_solve(blocks, F, off, 1e-4, 1e-10)
    nq.api.set_limits(1, 0)
    dth, _, _ = _solve(blocks, off, F, 1e-4, 1e-10, "mixed_psd", want_evals)
    assert rel(dth.cpu().numpy(), ref) < 1e-10
    nq.api.set_limits(0, 0)
    dth, _, _ = _solve(blocks, off, F, 1e-4, 1e-10, "mixed_psd", want_evals)
    assert rel(dth.cpu().numpy(), ref) < 1e-10


def test_refinement_sweep_limit_under_capture_is_retry():
    """Under stream capture nothing can fall back on the host: an unconverged refinement is
    recorded as NQS_ERR_RETRY for the caller to retake the step uncaptured."""
    import paper_2510_08430_gb300 as nq
    from paper_2510_08430_gb300._lib import NQS_ERR_RETRY, NQSError
    w = W.make_workload("j1j2_6x6_ffnn", 128)
    model, theta, x, ham = dev_inputs(w)
    st = nq.SRStep(model, 128, ham, w.block_off, "split_bf16_exact", w.diag_shift, w.cutoff, solver="mixed")
    st.capture(theta, x)
    nq.api.set_limits(1, 0)
    g = st.capture(theta, x)  # recaptured: the lowered limit is a kernel argument of the graph
    st.replay()
    with pytest.raises(NQSError) as ei:
        st.ws.sync_status()
    assert ei.value.code == NQS_ERR_RETRY
    nq.api.set_limits(0, 0)
    del g
    _ok_step()


@pytest.mark.parametrize("solver,want_evals", [("fp64", True), ("mixed_psd", False)])
def test_wait_budget_runs_out_is_timeout(solver, want_evals):
    """With a 1 ns budget the grid-wide waits of the persistent kernels give up: the kernels
    record NQS_ERR_TIMEOUT and return (every loop they run is bounded), and the device
    stays usable for the next call."""
    import paper_2510_08430_gb300 as nq
    from paper_2510_08430_gb300._lib import NQS_ERR_TIMEOUT
    blocks, off, F = _psd_blocks([200, 130, 64], 11)
    nq.api.set_limits(0, 1)
    assert _code(_solve, blocks, off, F, 1e-4, 1e-10, solver, want_evals) == NQS_ERR_TIMEOUT
    nq.api.set_limits(0, 0)
    dth, _, _ = _solve(blocks, off, F, 1e-4, 1e-10, solver, want_evals)
    ref, _, _ = oracle.qgt.block_solve(blocks, F, off, 1e-4, 1e-10)
    assert rel(dth.cpu().numpy(), ref) < 1e-10
    _ok_step()


@pytest.mark.parametrize("bad", [(0, 10), (-1, 3), (4, 4)])
def test_bad_bond_is_invalid_argument(bad):
    import paper_2510_08430_gb300 as nq
    from paper_2510_08430_gb300._lib import NQS_ERR_INVALID_ARG
    w = W.make_workload("chain10_rbm", 50)
    model, theta, x, _ = dev_inputs(w)
    ij = np.array(w.bond_ij, dtype=np.int32).copy()
    ij[3] = bad
    ham = nq.Hamiltonian(10, ij, w.bond_j)
    assert _code(nq.nqs_local_energy, model, theta, x, ham, "fp64") == NQS_ERR_INVALID_ARG
    assert _code(nq.nqs_connections, x, ham) == NQS_ERR_INVALID_ARG
    # the other bonds are still evaluated: the result equals the Hamiltonian without bond 3
    keep = np.arange(len(ij)) != 3
    ham_ok = nq.Hamiltonian(10, ij[keep], np.asarray(w.bond_j)[keep])
    el_ok = nq.nqs_local_energy(model, theta, x, ham_ok, "fp64").cpu().numpy()
    ref = oracle.hamiltonian.local_energy(w.model, w.theta, w.configs, np.asarray(w.bond_ij)[keep],
                                          np.asarray(w.bond_j)[keep], w.c, w.sign_rule)
    assert np.max(np.abs(el_ok - ref) / np.maximum(np.abs(ref), 1.0)) < 1e-12
    _ok_step()
