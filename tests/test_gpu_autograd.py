"""NQSLogPsi: the library's per-sample backward exposed to torch.autograd, checked against
the oracle Jacobian and against central finite differences of the GPU forward."""
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


@pytest.mark.parametrize("name,ns", [("chain10_rbm", 64), ("j1j2_6x6_ffnn", 48)])
def test_log_psi_gradient(name, ns):
    import paper_2510_08430_gb300 as nq
    w = W.make_workload(name, ns)
    model, theta, x, _ = dev_inputs(w)
    rng = np.random.default_rng(3)
    c = rng.normal(size=ns) + 1j * rng.normal(size=ns)
    ct = torch.as_tensor(c, device="cuda")
    th = theta.clone().requires_grad_(True)
    lp = nq.log_psi(model, th, x)
    loss = torch.real(torch.sum(ct * lp))
    loss.backward()
    g = th.grad.cpu().numpy()
    # oracle: for L = Re(sum_s c_s ln psi_s), dL/dRe + i dL/dIm = conj(sum_s c_s O_sk)
    _, O = oracle.nqs.jacobian(w.model, w.theta, w.configs)
    ref = np.conj(c @ O)
    assert rel(g, ref) < 1e-12
    # central differences of the GPU forward on a few parameters
    h = 1e-6
    for k in rng.choice(theta.numel(), size=6, replace=False):
        d = []
        for step in (h, 1j * h):
            tp, tm = theta.clone(), theta.clone()
            tp[k] += step
            tm[k] -= step
            lp_p = nq.log_psi(model, tp, x)
            lp_m = nq.log_psi(model, tm, x)
            d.append(float(torch.real(torch.sum(ct * (lp_p - lp_m))).item()) / (2 * h))
        fd = d[0] + 1j * d[1]
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(g[k])), (k, fd, g[k])
