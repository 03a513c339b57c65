"""Host-side logic of the batched workload's memory plan and of the model descriptions (no GPU:
the library's workspace-size queries run on the host)."""
import ctypes as C

import numpy as np
import pytest

import workloads as W


@pytest.fixture(scope="module")
def nq():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2510_08430_gb300 as m
    return m


def _instances(nq, idx, ns):
    ws = [W.make_workload(f"batch8x8_{i}", 8) for i in idx]
    models = [nq.Model.from_workload(w.model) for w in ws]
    hams = [nq.Hamiltonian(64, w.bond_ij, w.bond_j, w.c, w.sign_rule, device="cpu") for w in ws]
    return models, [ns] * len(idx), hams, [w.block_off for w in ws]


def test_chunks_cover_instances_in_order_within_budget(nq):
    models, ns, hams, offs = _instances(nq, range(6), 2048)
    one = nq.sr_step_batched_workspace_size(models[:1], ns[:1], hams[:1], offs[:1])
    two = nq.sr_step_batched_workspace_size(models[:2], ns[:2], hams[:2], offs[:2])
    assert two > one
    budget = two + (two - one) // 2  # two instances fit, three do not
    groups, worst = nq.plan_batch_chunks(models, ns, hams, offs, budget)
    assert [i for g in groups for i in g] == list(range(6))
    assert all(len(g) == 2 for g in groups)
    for g in groups:
        need = nq.sr_step_batched_workspace_size([models[i] for i in g], [ns[i] for i in g], [hams[i] for i in g],
                                                 [offs[i] for i in g])
        assert need <= budget and need <= worst
    with pytest.raises(ValueError):
        nq.plan_batch_chunks(models, ns, hams, offs, one - 1)


def test_binding_block_offsets_match_the_workloads(nq):
    for name in ("chain16_vit", "j1j2_6x6_vit", "chain16_rbm", "j1j2_10x10_ffnn5"):
        w = W.make_workload(name, 4)
        assert np.array_equal(nq.Model.from_workload(w.model).block_offsets(), w.block_off), name
    # the library's descriptor agrees on n_p (Jacobian workspace grows with n_p x n_s)
    lib = nq._lib.load()
    out = C.c_size_t(0)
    vit = nq.Model.from_workload(W.make_workload("chain16_vit", 4).model)
    assert lib.nqs_jacobian_workspace_size(C.byref(vit.c), 64, 0, C.byref(out)) == 0 and out.value > 0
