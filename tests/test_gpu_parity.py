"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Sizes span several tiles with ragged tails; tolerances follow the precision of
each path: FP64 path 1e-12 relative on intermediate results and 1e-10 on
dtheta; FP32 path 1e-4 on dtheta; BF16 split path 1e-6 on dtheta.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from gpu_util import ELOC_SPLIT_BAR, dev_inputs, emean_bar, rel, unpack_lower

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def nq():
    import paper_2510_08430_gb300 as m
    return m


def _oracle_all(w):
    return oracle.qgt.sr_step(w.model, w.theta, w.configs, w.bond_ij, w.bond_j, w.block_off, w.diag_shift,
                              w.cutoff, 1.0, w.c, w.sign_rule)


@pytest.mark.parametrize("name,ns,prec,tol", [
    ("chain10_rbm", 77, "fp64", 1e-12),
    ("j1j2_6x6_ffnn", 45, "fp64", 1e-12),
    ("j1j2_6x6_ffnn", 45, "fp32", 1e-5),
    ("j1j2_10x10_ffnn5", 33, "fp32", 1e-5),
])
def test_jacobian_and_logpsi(name, ns, prec, tol):
    w = W.make_workload(name, ns)
    model, theta, x, ham = dev_inputs(w)
    lp, O = nq().nqs_jacobian(model, theta, x, prec, ldo=ns + 5)
    lp_o, O_o = oracle.nqs.jacobian(w.model, w.theta, w.configs)
    Og = O.cpu().numpy()
    assert np.all(Og[:, ns:] == 0)
    assert rel(lp.cpu().numpy(), lp_o) < tol
    assert rel(Og[:, :ns].T, O_o) < tol
    # element-wise relative to the per-parameter scale
    err = np.abs(Og[:, :ns].T - O_o) / (np.abs(O_o).max(axis=0, keepdims=True) + 1e-300)
    assert err.max() < 20 * tol


@pytest.mark.parametrize("name,ns", [("chain10_rbm", 50), ("j1j2_6x6_ffnn", 37), ("j1j2_10x10_ffnn5", 21)])
def test_connections_bit_exact(name, ns):
    w = W.make_workload(name, ns)
    _, _, x, ham = dev_inputs(w)
    cnt, off, bond = nq().nqs_connections(x, ham)
    ref = oracle.hamiltonian.connections(w.configs, w.bond_ij)
    assert np.array_equal(bond.cpu().numpy(), ref[:, 1].astype(np.int32))
    assert np.array_equal(np.repeat(np.arange(ns), cnt.cpu().numpy()), ref[:, 0])
    o = off.cpu().numpy()
    assert o[0] == 0 and o[-1] == len(ref) and np.array_equal(np.diff(o), cnt.cpu().numpy())


@pytest.mark.parametrize("name,ns,prec,tol", [
    ("chain10_rbm", 64, "fp64", 1e-12),
    ("j1j2_6x6_ffnn", 40, "fp64", 1e-12),
    ("j1j2_6x6_ffnn", 40, "fp32", 1e-5),
    ("j1j2_10x10_ffnn5", 12, "fp32", 1e-5),
    ("j1j2_6x6_ffnn", 40, "split_bf16_exact", 1e-12),
    # FP32 difference propagation: FP32 rounding of the differences dz, dh (about 1e-7 of each
    # connection's term), summed over ~200 terms of magnitude <= 2|J| exp(Re d)
    ("j1j2_6x6_ffnn", 40, "split_bf16_exact/diff32", ELOC_SPLIT_BAR),
    ("j1j2_10x10_ffnn5", 24, "split_bf16_exact/diff32", ELOC_SPLIT_BAR),
    ("j1j2_10x10_ffnn256", 8, "split_bf16_exact/diff32", ELOC_SPLIT_BAR),
    ("j1j2_6x6_ffnn", 40, "fp64/diff32", ELOC_SPLIT_BAR),
])
def test_local_energy(name, ns, prec, tol):
    w = W.make_workload(name, ns)
    model, theta, x, ham = dev_inputs(w)
    prec, _, opt = prec.partition("/")
    el = nq().nqs_local_energy(model, theta, x, ham, prec, diff32=opt == "diff32").cpu().numpy()
    ref = oracle.hamiltonian.local_energy(w.model, w.theta, w.configs, w.bond_ij, w.bond_j, w.c, w.sign_rule)
    assert np.max(np.abs(el - ref) / np.maximum(np.abs(ref), 1.0)) < tol


@pytest.mark.parametrize("name,ns", [("j1j2_6x6_ffnn", 64), ("j1j2_10x10_ffnn5", 32)])
def test_local_energy_difference_fallback_path(name, ns):
    """With every connection sent to the FP64-class kernel (test hook), the difference-propagation
    local energies are bit-identical to those of NQS_FP64: the listed connections take exactly
    the FP64 arithmetic and are summed in the same order."""
    w = W.make_workload(name, ns)
    model, theta, x, ham = dev_inputs(w)
    m = nq()
    ref = m.nqs_local_energy(model, theta, x, ham, "fp64")
    try:
        m.set_eloc_fallback_all(True)
        el = m.nqs_local_energy(model, theta, x, ham, "split_bf16_exact", diff32=True)
    finally:
        m.set_eloc_fallback_all(False)
    assert torch.equal(el, ref)
    el_dp = m.nqs_local_energy(model, theta, x, ham, "split_bf16_exact", diff32=True)
    assert not torch.equal(el_dp, ref)  # the FP32 path ran (it rounds differently)


def test_local_energy_marshall_sign_and_units():
    w = W.make_workload("chain10_rbm", 30)
    import paper_2510_08430_gb300 as m
    model, theta, x, _ = dev_inputs(w)
    ham = m.Hamiltonian(10, w.bond_ij, w.bond_j, 0.25, -1)
    el = m.nqs_local_energy(model, theta, x, ham, "fp64").cpu().numpy()
    ref = oracle.hamiltonian.local_energy(w.model, w.theta, w.configs, w.bond_ij, w.bond_j, 0.25, -1)
    assert rel(el, ref) < 1e-12


@pytest.mark.parametrize("name,ns,prec,tol", [
    ("chain10_rbm", 97, "fp64", 1e-12),
    ("j1j2_6x6_ffnn", 70, "fp64", 1e-12),
    ("j1j2_6x6_ffnn", 70, "fp32", 1e-5),
    ("j1j2_6x6_ffnn", 70, "split_bf16", 5e-5),
    ("j1j2_6x6_ffnn", 70, "split_bf16x3", 2e-5),
    ("chain10_rbm", 1100, "split_bf16x3", 2e-6),
    ("j1j2_6x6_ffnn", 70, "split_bf16_exact", 1e-6),
    ("chain10_rbm", 1100, "split_bf16_exact", 1e-7),
    ("j1j2_10x10_ffnn5", 45, "split_bf16_exact", 1e-6),
])
def test_qgt_block_build(name, ns, prec, tol):
    w = W.make_workload(name, ns)
    model, theta, x, ham = dev_inputs(w)
    _, O = nq().nqs_jacobian(model, theta, x, prec)
    el = nq().nqs_local_energy(model, theta, x, ham, prec)
    S, F, Om, Em = nq().qgt_block_build(O, ns, w.block_off, el, prec)
    r = _oracle_all(w)
    Sl = unpack_lower(S.cpu().numpy(), w.block_off)
    for b, Sb in enumerate(r["S"]):
        assert rel(Sl[b], np.tril(Sb)) < tol, b
    assert rel(F.cpu().numpy(), r["F"]) < 10 * tol
    assert rel(Om.cpu().numpy(), r["o_mean"]) < tol
    assert abs(Em.cpu().numpy()[0] - r["e_mean"]) < tol * abs(r["e_mean"])


def _herm_psd(n, seed, spec):
    rng = np.random.default_rng(seed)
    q, _ = np.linalg.qr(rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n)))
    S = (q * spec) @ np.conj(q).T
    return 0.5 * (S + np.conj(S).T)


@pytest.mark.parametrize("sizes", [[1, 2, 3], [17, 65, 130], [64, 129, 5]])
@pytest.mark.parametrize("cutoff,shift", [(1e-12, 1e-3), (1e-3, 1e-7)])
def test_qgt_block_solve_against_definition(sizes, cutoff, shift):
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    blocks = []
    for b, n in enumerate(sizes):
        spec = np.concatenate([np.logspace(-9, 1, n)]) if n > 1 else np.array([0.7])
        blocks.append(_herm_psd(n, 100 + b, spec))
    rng = np.random.default_rng(7)
    F = rng.normal(size=off[-1]) + 1j * rng.normal(size=off[-1])
    packed = np.concatenate([B.ravel() for B in blocks])
    S = torch.as_tensor(packed, device="cuda")
    dth, ev, nk = nq().qgt_block_solve(S, off, torch.as_tensor(F, device="cuda"), shift, cutoff, 0, 0.9)
    ref, sig, kept = oracle.qgt.block_solve(blocks, F, off, shift, cutoff, 0.9)
    assert np.array_equal(nk.cpu().numpy(), kept)
    evg = ev.cpu().numpy()
    for b in range(len(sizes)):
        sl = slice(off[b], off[b + 1])
        np.testing.assert_allclose(evg[sl], sig[b], rtol=0, atol=1e-12 * sig[b].max())
    assert rel(dth.cpu().numpy(), ref) < 1e-9


def test_solve_absolute_cutoff_mode():
    sizes = [40, 9]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    blocks = [_herm_psd(n, 3 + n, np.logspace(-6, 0, n)) for n in sizes]
    F = np.random.default_rng(1).normal(size=off[-1]) + 0j
    S = torch.as_tensor(np.concatenate([B.ravel() for B in blocks]), device="cuda")
    dth, _, nk = nq().qgt_block_solve(S, off, torch.as_tensor(F, device="cuda"), 1e-8, 3e-3, 1, 1.0)
    ref, _, kept = oracle.qgt.block_solve(blocks, F, off, 1e-8, 3e-3, 1.0, absolute=True)
    assert np.array_equal(nk.cpu().numpy(), kept)
    assert rel(dth.cpu().numpy(), ref) < 1e-9


@pytest.mark.parametrize("name,ns,prec,tol", [
    ("chain10_rbm", 512, "fp64", 1e-10),
    ("chain10_rbm", 333, "fp32", 1e-4),
    ("j1j2_6x6_ffnn", 300, "fp64", 1e-10),
    ("j1j2_6x6_ffnn", 300, "fp32", 1e-4),
    # three 8-bit slices keep 24 significant bits per element, as FP32 does: FP32-class bar
    ("j1j2_6x6_ffnn", 300, "split_bf16x3", 1e-4),
    ("j1j2_10x10_ffnn5", 200, "split_bf16x3", 1e-4),
    ("chain10_rbm", 777, "split_bf16_exact", 1e-6),
    ("j1j2_6x6_ffnn", 300, "split_bf16_exact", 1e-6),
    ("j1j2_10x10_ffnn5", 200, "split_bf16_exact", 1e-6),
])
def test_sr_step(name, ns, prec, tol):
    w = W.make_workload(name, ns)
    model, theta, x, ham = dev_inputs(w)
    dth, em, ev, nk = nq().sr_step(model, theta, x, ham, w.block_off, w.diag_shift, w.cutoff, 1.0, prec)
    r = _oracle_all(w)
    assert rel(dth.cpu().numpy(), r["dtheta"]) < tol
    assert abs(em.cpu().numpy()[0] - r["e_mean"]) < max(tol, 1e-12) * abs(r["e_mean"])
    assert np.array_equal(nk.cpu().numpy(), r["n_kept"])


@pytest.mark.parametrize("name,ns", [("chain10_rbm", 777), ("j1j2_6x6_ffnn", 300), ("j1j2_10x10_ffnn5", 200)])
def test_sr_step_two_slice_split(name, ns):
    """NQS_SPLIT_BF16 (hi + lo, three products) is a reduced-accuracy mode: each centred entry
    is held to 2^-17, which the solve amplifies by up to 1/lambda; its stated dtheta bar is
    1e-2 relative (it misses the 1e-6 split bar; the five-slice split is the one that meets it)."""
    w = W.make_workload(name, ns)
    model, theta, x, ham = dev_inputs(w)
    dth, em, _, nk = nq().sr_step(model, theta, x, ham, w.block_off, w.diag_shift, w.cutoff, 1.0, "split_bf16",
                                  solver="mixed")
    r = _oracle_all(w)
    assert rel(dth.cpu().numpy(), r["dtheta"]) < 1e-2
    assert abs(em.cpu().numpy()[0] - r["e_mean"]) < 1e-12 * abs(r["e_mean"])
    assert np.array_equal(nk.cpu().numpy(), r["n_kept"])


def test_single_sample_step_is_zero():
    w = W.make_workload("chain10_rbm", 1)
    model, theta, x, ham = dev_inputs(w)
    dth, em, _, _ = nq().sr_step(model, theta, x, ham, w.block_off, 1e-4, 1e-10, 1.0, "fp64")
    assert torch.all(dth == 0)


@pytest.mark.parametrize("sizes", [[1, 2, 3], [17, 65, 130], [300, 64]])
@pytest.mark.parametrize("solver", ["mixed", "mixed_psd"])
def test_mixed_solver_matches_definition(sizes, solver):
    """FP32 reduction + FP64 refinement reaches the FP64 definition when the cutoff keeps all eigenvalues."""
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    rng = np.random.default_rng(9)
    blocks = []
    for b, n in enumerate(sizes):
        X = rng.normal(size=(2 * n + 3, n)) + 1j * rng.normal(size=(2 * n + 3, n))
        X[:, : n // 2] *= 1e-2  # spread the spectrum
        blocks.append(np.conj(X).T @ X / X.shape[0])
    F = rng.normal(size=off[-1]) + 1j * rng.normal(size=off[-1])
    S = torch.as_tensor(np.concatenate([B.ravel() for B in blocks]), device="cuda")
    dth, ev, nk = nq().qgt_block_solve(S, off, torch.as_tensor(F, device="cuda"), 1e-4, 1e-10, 0, 1.0,
                                       solver=solver)
    ref, sig, kept = oracle.qgt.block_solve(blocks, F, off, 1e-4, 1e-10, 1.0)
    assert np.array_equal(nk.cpu().numpy(), kept)
    assert rel(dth.cpu().numpy(), ref) < 1e-10
    evg = ev.cpu().numpy()
    for b in range(len(sizes)):
        np.testing.assert_allclose(evg[off[b]:off[b + 1]], sig[b], rtol=0, atol=1e-5 * sig[b].max())


@pytest.mark.parametrize("sizes", [[1, 2, 3], [17, 65, 130], [300, 64], [64, 129, 5], [700]])
@pytest.mark.parametrize("mode", [0, 1])
def test_cholesky_path_matches_definition(sizes, mode):
    """Gram-matrix blocks without eigenvalue output take the certified Cholesky path (FP32
    tiled factor, FP64 refinement): equal to the pseudo-inverse definition to 1e-10, in both
    cutoff modes, on ragged tiles (1 .. 700 parameters, 64-wide tiles)."""
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    rng = np.random.default_rng(19)
    blocks = []
    for n in sizes:
        X = rng.normal(size=(n + 7, n)) + 1j * rng.normal(size=(n + 7, n))
        X[:, : n // 3] *= 3e-2  # spread the spectrum
        blocks.append(np.conj(X).T @ X / X.shape[0])
    F = rng.normal(size=off[-1]) + 1j * rng.normal(size=off[-1])
    S = torch.as_tensor(np.concatenate([B.ravel() for B in blocks]), device="cuda")
    cut = 1e-10 if mode == 0 else 1e-6
    dth, ev, nk = nq().qgt_block_solve(S, off, torch.as_tensor(F, device="cuda"), 1e-3, cut, mode, 0.8,
                                       want_evals=False, solver="mixed_psd")
    assert ev is None
    ref, sig, kept = oracle.qgt.block_solve(blocks, F, off, 1e-3, cut, 0.8, absolute=mode == 1)
    assert np.array_equal(nk.cpu().numpy(), kept) and np.array_equal(kept, np.array(sizes))
    assert rel(dth.cpu().numpy(), ref) < 1e-10


def test_cholesky_path_hands_a_binding_cutoff_to_the_eigen_path():
    """When the certificate cannot show that the cutoff keeps everything, the solve must
    still equal the definition (eigen-decomposition path), with the dropped count exact."""
    sizes = [40, 9, 130]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    blocks = [_herm_psd(n, 3 + n, np.logspace(-6, 0, n)) for n in sizes]
    F = np.random.default_rng(1).normal(size=off[-1]) + 0j
    S = torch.as_tensor(np.concatenate([B.ravel() for B in blocks]), device="cuda")
    dth, _, nk = nq().qgt_block_solve(S, off, torch.as_tensor(F, device="cuda"), 1e-8, 3e-3, 0, 1.0,
                                      want_evals=False, solver="mixed_psd")
    ref, _, kept = oracle.qgt.block_solve(blocks, F, off, 1e-8, 3e-3, 1.0)
    assert np.array_equal(nk.cpu().numpy(), kept) and kept.min() < min(sizes)
    assert rel(dth.cpu().numpy(), ref) < 1e-9


def test_mixed_solver_falls_back_when_cutoff_binds():
    sizes = [40, 9]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    blocks = [_herm_psd(n, 3 + n, np.logspace(-6, 0, n)) for n in sizes]
    F = np.random.default_rng(1).normal(size=off[-1]) + 0j
    S = torch.as_tensor(np.concatenate([B.ravel() for B in blocks]), device="cuda")
    dth, _, nk = nq().qgt_block_solve(S, off, torch.as_tensor(F, device="cuda"), 1e-8, 3e-3, 0, 1.0,
                                      solver="mixed")
    ref, _, kept = oracle.qgt.block_solve(blocks, F, off, 1e-8, 3e-3, 1.0)
    assert np.array_equal(nk.cpu().numpy(), kept)
    assert rel(dth.cpu().numpy(), ref) < 1e-9


@pytest.mark.parametrize("name,ns,prec,tol", [
    ("chain10_rbm", 512, "fp64", 1e-10),
    ("j1j2_6x6_ffnn", 300, "fp64", 1e-10),
])
def test_sr_step_mixed_solver(name, ns, prec, tol):
    w = W.make_workload(name, ns)
    model, theta, x, ham = dev_inputs(w)
    dth, em, ev, nk = nq().sr_step(model, theta, x, ham, w.block_off, w.diag_shift, w.cutoff, 1.0, prec,
                                   solver="mixed", want_evals=False)
    r = _oracle_all(w)
    assert rel(dth.cpu().numpy(), r["dtheta"]) < tol
    assert np.array_equal(nk.cpu().numpy(), r["n_kept"])


@pytest.mark.parametrize("name,ns,prec,tol", [
    ("j1j2_6x6_ffnn", 300, "fp64", 1e-10),
    ("j1j2_6x6_ffnn", 300, "split_bf16_exact", 1e-6),
    ("chain10_rbm", 64, "fp64", 1e-10),
])
def test_sample_space_blocks_match_oracle(name, ns, prec, tol):
    """Blocks wider than the sample count (2368 and 4160 parameters at 300 samples; the RBM's
    100 weights at 64 samples) are solved in sample space by the push-through identity: the
    step equals the oracle's eigen-decomposition definition, and the parameter-space form of
    the same step."""
    w = W.make_workload(name, ns)
    assert max(np.diff(w.block_off)) > ns
    model, theta, x, ham = dev_inputs(w)
    dth, em, _, nk = nq().sr_step(model, theta, x, ham, w.block_off, w.diag_shift, w.cutoff, 1.0, prec,
                                  solver="mixed", want_evals=False)
    r = _oracle_all(w)
    assert rel(dth.cpu().numpy(), r["dtheta"]) < tol
    assert np.array_equal(nk.cpu().numpy(), r["n_kept"])
    assert abs(em.cpu().numpy()[0] - r["e_mean"]) < 1e-12 * abs(r["e_mean"])
    dp, _, _, nkp = nq().sr_step(model, theta, x, ham, w.block_off, w.diag_shift, w.cutoff, 1.0, prec,
                                 solver="mixed", want_evals=False, param_space=True)
    assert rel(dth.cpu().numpy(), dp.cpu().numpy()) < tol
    assert np.array_equal(nk.cpu().numpy(), nkp.cpu().numpy())


@pytest.mark.parametrize("cutoff,mode", [(1e-3, 0), (3e-6, 1)])
def test_sample_space_block_with_binding_cutoff(cutoff, mode):
    """A binding cutoff on a block wider than the sample count: the sample-space eigen
    solve with the same threshold still equals the definition, and n_kept counts the
    eigenvalues of S_b + lambda I (the lambda eigenvalues of the null space included)."""
    model = W.Model(W.FFNN, (16, 24, 8, 1))
    rng = np.random.default_rng(31)
    theta = W.init_params(model, rng)
    xs = W.zero_sz_configs(16, 100, rng)
    ij, jj = W.square_j1j2_bonds(4, 4, 1.0, 0.4)
    w = W.Workload("ffnn4x4_cut", model, theta, xs, ij, jj, model.block_offsets(), 1e-6, cutoff, "fp64")
    m, th, x, ham = dev_inputs(w)
    dth, _, _, nk = nq().sr_step(m, th, x, ham, w.block_off, w.diag_shift, cutoff, 1.0, "fp64", cutoff_mode=mode,
                                 solver="mixed", want_evals=False)
    r = oracle.qgt.sr_step(w.model, w.theta, w.configs, w.bond_ij, w.bond_j, w.block_off, w.diag_shift, cutoff,
                           absolute=mode == 1)
    assert r["n_kept"].min() < np.diff(w.block_off).max()  # the cutoff binds
    assert np.array_equal(nk.cpu().numpy(), r["n_kept"])
    assert rel(dth.cpu().numpy(), r["dtheta"]) < 1e-8


def _golden(name):
    import os
    p = os.path.join(os.path.dirname(__file__), "golden", f"oracle_{name}.npz")
    if not os.path.exists(p):
        pytest.skip(f"{p} not generated (tests/golden/make_fullsize.py)")
    return np.load(p)


@pytest.mark.parametrize("name,prec,solver,tol", [
    ("j1j2_6x6_ffnn", "fp64", "fp64", 1e-10),
    ("j1j2_6x6_ffnn", "fp64", "mixed", 1e-10),
    ("j1j2_6x6_ffnn", "split_bf16_exact", "mixed", 1e-6),
    ("j1j2_6x6_ffnn", "split_bf16x3", "mixed", 1e-4),
    ("j1j2_6x6_ffnn", "fp32", "mixed", 1e-4),
    ("j1j2_10x10_ffnn5", "split_bf16_exact", "mixed", 1e-6),
    ("j1j2_10x10_ffnn5", "split_bf16_exact", "fp64", 1e-6),
    ("j1j2_10x10_ffnn5", "split_bf16_exact/diff32", "mixed", 1e-6),
    ("j1j2_6x6_ffnn", "split_bf16_exact/diff32", "mixed", 1e-6),
])
def test_fullsize_against_oracle(name, prec, solver, tol):
    """Full-size workloads (6x6: FFNN 36-64-64-1, 4096 samples; 10x10: FFNN 100-64x4-1,
    16384 samples) against the FP64 oracle results stored by tests/golden/make_fullsize.py."""
    g = _golden(name)
    w = W.make_workload(name)
    model, theta, x, ham = dev_inputs(w)
    prec, _, opt = prec.partition("/")
    diff32 = opt == "diff32"
    dth, em, _, nk = nq().sr_step(model, theta, x, ham, w.block_off, w.diag_shift, w.cutoff, 1.0, prec,
                                  solver=solver, want_evals=False, eloc_diff32=diff32)
    assert rel(dth.cpu().numpy(), g["dtheta"]) < tol
    etol = 1e-7 if prec == "fp32" else emean_bar(w.configs.shape[0], diff32)
    assert abs(em.cpu().numpy()[0] - g["e_mean"]) < etol * abs(g["e_mean"])
    assert np.array_equal(nk.cpu().numpy(), g["n_kept"])
    if diff32:
        el = nq().nqs_local_energy(model, theta, x, ham, prec, diff32=True).cpu().numpy()
        ref = g["eloc"]
        assert np.max(np.abs(el[g["eloc_idx"]] - ref) / np.maximum(np.abs(ref), 1.0)) < ELOC_SPLIT_BAR
    # FP64 local energies at full size: the same 1e-12 bar (relative to max(|E_loc|, 1)) as
    # the small cases
    el = nq().nqs_local_energy(model, theta, x, ham, "fp64").cpu().numpy()
    ref = g["eloc"]
    assert np.max(np.abs(el[g["eloc_idx"]] - ref) / np.maximum(np.abs(ref), 1.0)) < 1e-12
