"""sr_step captured into a CUDA graph (NQS_GRAPH) and replayed on new inputs equals the
direct call."""
import numpy as np
import pytest
import torch

import workloads as W
from gpu_util import dev_inputs, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("name,ns,prec,solver", [
    ("j1j2_6x6_ffnn", 300, "split_bf16_exact", "mixed"),
    ("chain10_rbm", 256, "fp64", "fp64"),
])
def test_graph_replay_equals_direct_step(name, ns, prec, solver):
    import paper_2510_08430_gb300 as nq
    w = W.make_workload(name, ns)
    model, theta, x, ham = dev_inputs(w)
    step = nq.SRStep(model, ns, ham, w.block_off, prec, w.diag_shift, w.cutoff, solver=solver)
    step.capture(theta, x)
    for k in range(2):  # two replays on different inputs
        th = theta * (1.0 + 0.01 * k)
        xk = torch.roll(x, shifts=k, dims=0)
        d_g, e_g = step.replay(th, xk)
        d_g, e_g = d_g.clone(), e_g.clone()
        step.ws.sync_status()
        direct = nq.SRStep(model, ns, ham, w.block_off, prec, w.diag_shift, w.cutoff, solver=solver)
        d_d, e_d = direct(th, xk, sync=True)
        assert rel(d_g.cpu().numpy(), d_d.cpu().numpy()) < 1e-12
        assert abs(e_g.item() - e_d.item()) <= 1e-13 * abs(e_d.item())
