"""The Gram tile-order autotuner on the device: every group edge G gives the same S bit for
bit (only the order of the tiles changes), and tune() times the candidates and installs the
fastest."""
import numpy as np
import pytest
import torch

import workloads as W
from gpu_util import dev_inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    yield
    from paper_2510_08430_gb300 import tune
    tune.install({})


@pytest.mark.parametrize("prec", ["split_bf16_exact", "split_bf16x3"])
def test_tile_order_leaves_S_unchanged(prec):
    import paper_2510_08430_gb300 as nq
    from paper_2510_08430_gb300 import tune
    w = W.make_workload("j1j2_6x6_ffnn", 640)
    model, theta, x, ham = dev_inputs(w)
    _, O = nq.nqs_jacobian(model, theta, x, prec)
    el = nq.nqs_local_energy(model, theta, x, ham, prec)
    ref = None
    for G in (1, 3, 8, 16, 64):
        tune.install({(1 << 30, 1 << 30): G})
        assert tune.group_edge(4160, 640) == G
        S, F, _, _ = nq.qgt_block_build(O, 640, w.block_off, el, prec)
        if ref is None:
            ref = S.clone()
        assert torch.equal(S, ref), G
    tune.install({})


def test_tune_on_device_installs_a_candidate(tmp_path):
    from paper_2510_08430_gb300 import tune
    shapes = [([2368, 4160, 65], 1024)]
    res = tune.tune(shapes, cache_path=str(tmp_path / "t.json"))
    rec = res[tune.bucket(4160, 1024)]
    assert rec["group"] in tune.CANDIDATES
    assert set(int(g) for g in rec["ms"]) == set(tune.CANDIDATES)
    assert tune.group_edge(4160, 1024) == rec["group"]
    tune.install({})
