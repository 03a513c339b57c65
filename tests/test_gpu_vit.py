"""The transformer wavefunction on the device (NEXT #4: the module partition of Sec. 2 --
patching and embedding, encoder layers, output -- as the blocks of the block-layer QGT).

ln psi, the Jacobian and the local energies against the oracle; the whole SR step with the
module partition against the oracle's definition (wide encoder blocks through the
sample-space solve); the sampler's chains bit-identical to the oracle's; and the device VMC
loop training the transformer on the 16-site chain of Table 2, block-layer and full QGT.
"""
import ctypes as C

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


def _custom(widths, n_enc, ns, seed=0, scale=3.0):
    model = W.Model(W.VIT, widths, n_enc)
    theta = W.init_params(model, np.random.default_rng(seed)) * scale
    x = W.zero_sz_configs(widths[0], ns, np.random.default_rng(seed + 1))
    return model, theta, x


@pytest.mark.parametrize("case", ["chain16_vit", "j1j2_6x6_vit", "one_token_rbm_like", "no_encoder"])
def test_vit_log_psi_and_jacobian_match_oracle(case):
    if case == "chain16_vit":
        w = W.make_workload(case, 64)
        model_w, theta_np, x_np = w.model, w.theta * 10, w.configs   # away from the near-uniform start
    elif case == "j1j2_6x6_vit":
        w = W.make_workload(case, 16)
        model_w, theta_np, x_np = w.model, w.theta * 10, w.configs
    elif case == "one_token_rbm_like":
        model_w, theta_np, x_np = _custom((10, 10, 8, 4), 1, 40)
    else:
        model_w, theta_np, x_np = _custom((12, 3, 6, 5), 0, 40)
    model = nq().Model.from_workload(model_w)
    theta = torch.as_tensor(theta_np, device="cuda")
    x = torch.as_tensor(x_np, device="cuda")
    lp, O = nq().nqs_jacobian(model, theta, x, "fp64")
    lpo, Oo = oracle.nqs.jacobian(model_w, theta_np, x_np)
    assert rel(lp.cpu().numpy(), lpo) < 1e-12
    Og = O.cpu().numpy()[:, :x_np.shape[0]].T
    assert np.max(np.abs(Og - Oo)) <= 1e-12 * np.max(np.abs(Oo))
    assert np.all(O.cpu().numpy()[:, x_np.shape[0]:] == 0)  # padding columns


@pytest.mark.parametrize("name,ns", [("chain16_vit", 64), ("j1j2_6x6_vit", 8)])
def test_vit_local_energy_matches_oracle(name, ns):
    w = W.make_workload(name, ns)
    model, theta, x, ham = dev_inputs(w)
    theta = theta * 10
    el = nq().nqs_local_energy(model, theta, x, ham, "fp64").cpu().numpy()
    ref = oracle.hamiltonian.local_energy(w.model, w.theta * 10, w.configs, w.bond_ij, w.bond_j, w.c, w.sign_rule)
    assert np.max(np.abs(el - ref) / np.maximum(np.abs(ref), 1.0)) < 1e-12


@pytest.mark.parametrize("solver", ["fp64", "mixed"])
def test_vit_sr_step_with_module_blocks_matches_oracle(solver):
    w = W.make_workload("chain16_vit", 256)
    model, theta, x, ham = dev_inputs(w)
    th_np = w.theta * 10
    dth, em, _, nk = nq().sr_step(model, theta * 10, x, ham, w.block_off, w.diag_shift, w.cutoff, 1.0, "fp64",
                                  solver=solver, want_evals=False)
    r = oracle.qgt.sr_step(w.model, th_np, w.configs, w.bond_ij, w.bond_j, w.block_off, w.diag_shift, w.cutoff,
                           1.0, w.c, w.sign_rule)
    assert len(w.block_off) == 5  # embedding, two encoder layers, output
    assert rel(dth.cpu().numpy(), r["dtheta"]) < 1e-10
    assert abs(em.cpu().numpy()[0] - r["e_mean"]) < 1e-12 * abs(r["e_mean"])
    assert np.array_equal(nk.cpu().numpy(), r["n_kept"])


def test_vit_split_step_with_wide_encoder_blocks_matches_oracle():
    """6x6 J1-J2 transformer at 300 samples: both encoder blocks (5297 parameters) are wider
    than the sample count and go through the sample-space solve on the tensor-core Gram."""
    w = W.make_workload("j1j2_6x6_vit", 300)
    model, theta, x, ham = dev_inputs(w)
    dth, em, _, _ = nq().sr_step(model, theta * 10, x, ham, w.block_off, w.diag_shift, w.cutoff, 1.0,
                                 "split_bf16_exact", solver="mixed", want_evals=False)
    th_np = w.theta * 10
    _, O = oracle.nqs.jacobian(w.model, th_np, w.configs)
    el = oracle.hamiltonian.local_energy(w.model, th_np, w.configs, w.bond_ij, w.bond_j, w.c, w.sign_rule)
    e_mean, _, dO, e = oracle.qgt.center(O, el)
    ref = oracle.qgt.block_solve_sample_space(dO, e, w.block_off, w.diag_shift)
    assert max(np.diff(w.block_off)) > 300
    assert rel(dth.cpu().numpy(), ref) < 1e-6
    assert abs(em.cpu().numpy()[0] - e_mean) < 1e-12 * abs(e_mean)


def test_vit_metropolis_chains_match_oracle():
    w = W.make_workload("chain16_vit", 48)
    model, theta, x, _ = dev_inputs(w)
    u = W.metropolis_uniforms(12, 48, 41)
    acc = nq().metropolis(model, theta * 10, x, torch.as_tensor(u, device="cuda"))
    xo, acco = oracle.vmc.metropolis(w.model, w.theta * 10, w.configs, u)
    assert acc == acco and acc > 0
    assert np.array_equal(x.cpu().numpy(), xo)


def test_vit_fp32_is_unsupported():
    w = W.make_workload("chain16_vit", 8)
    model, theta, x, _ = dev_inputs(w)
    with pytest.raises(nq().NQSError):
        nq().nqs_jacobian(model, theta, x, "fp32")


@pytest.mark.parametrize("full_qgt", [False, True])
def test_vit_vmc_trains_chain16(full_qgt):
    """The device loop trains the two-encoder-layer transformer on the 16-site chain (1024
    chains, 16 Metropolis steps and one SR step per iteration, eta 0.02, shift 1e-2): the
    variational energy of the trained state (enumeration of the S^z = 0 sector) comes within
    5e-3 of the Lanczos ground energy in 40 iterations, with the module-partition block QGT
    and with the full QGT."""
    w = W.make_workload("chain16_vit")
    model, theta, x, ham = dev_inputs(w)
    off = np.array([0, w.model.n_params], dtype=np.int64) if full_qgt else w.block_off
    g = torch.Generator(device="cuda").manual_seed(9)
    out = nq().vmc_train(model, theta, x, ham, off, 40, 16, w.diag_shift, w.cutoff, 0.02, "fp64", "mixed",
                         generator=g)
    e0 = oracle.hamiltonian.ground_energy_sz0(16, w.bond_ij, w.bond_j, 1.0)
    xs = oracle.hamiltonian.all_configs(16)
    xs = xs[xs.sum(axis=1) == 0]
    th = theta.cpu().numpy()
    lp = oracle.nqs.log_psi(w.model, th, xs)
    p = np.exp(2 * (lp.real - lp.real.max()))
    el = oracle.hamiltonian.local_energy(w.model, th, xs, w.bond_ij, w.bond_j, w.c, w.sign_rule)
    e_var = float(np.real(np.sum(p * el) / p.sum()))
    assert np.all(np.isfinite(out["energies"]))
    assert e_var >= e0 - 1e-9
    assert (e_var - e0) / abs(e0) < 5e-3, (e_var, e0)


def test_vit_batched_with_rbm_equals_separate_steps():
    """A transformer and an RBM instance in one sr_step_batched call (FP64) give the steps of
    separate sr_step calls."""
    ws = [W.make_workload("chain16_vit", 128), W.make_workload("chain10_rbm", 96)]
    ins = [dev_inputs(w) for w in ws]
    thetas = [ins[0][1] * 10, ins[1][1]]
    dths, em, _, nk = nq().sr_step_batched([i[0] for i in ins], thetas, [i[2] for i in ins], [i[3] for i in ins],
                                           [w.block_off for w in ws], 1e-2, 1e-10, 1.0, "fp64", solver="fp64")
    for j, w in enumerate(ws):
        model, _, x, ham = ins[j]
        d1, e1, _, _ = nq().sr_step(model, thetas[j], x, ham, w.block_off, 1e-2, 1e-10, 1.0, "fp64", solver="fp64",
                                    want_evals=False, param_space=True)
        assert rel(dths[j].cpu().numpy(), d1.cpu().numpy()) < 1e-11, w.name
        assert abs(em[j].item() - e1.cpu().numpy()[0]) <= 1e-12 * abs(e1.cpu().numpy()[0])


def test_vit_sample_sharded_step_equals_unsharded():
    """The transformer through the sample-sharded step (three shards simulated on one GPU:
    shard sums, shard builds with the global means, owner solves) equals the one-call step."""
    from paper_2510_08430_gb300 import sharded
    w = W.make_workload("chain16_vit", 300)
    model, theta, x, ham = dev_inputs(w)
    theta = theta * 10
    shards = [x[idx] for idx in np.array_split(np.arange(300), 3)]
    be = sharded.LibraryShardBackend(model, ham, w.block_off, "fp64", "fp64")
    dth, em = sharded.step_simulated(be, theta, shards, w.block_off, w.diag_shift, w.cutoff)
    d1, e1, _, _ = nq().sr_step(model, theta, x, ham, w.block_off, w.diag_shift, w.cutoff, 1.0, "fp64", solver="fp64",
                                want_evals=False, param_space=True)
    assert rel(dth.cpu().numpy(), d1.cpu().numpy()) < 1e-11
    assert abs(em.cpu().numpy()[0] - e1.cpu().numpy()[0]) <= 1e-12 * abs(e1.cpu().numpy()[0])
