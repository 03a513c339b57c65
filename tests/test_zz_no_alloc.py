"""qgt_block_build_static (no workspace, static device scratch) against qgt_block_build.

The file name sorts last so that the static-scratch call also runs after every other
test in the session has used the library.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import workloads as W
from gpu_util import dev_inputs, rel, unpack_lower


def _lib():
    from paper_2510_08430_gb300 import _lib as L
    return L


def test_static_build_rejects_what_it_cannot_hold():
    """Host-side checks return before any CUDA call (the pointers are never touched)."""
    L = _lib()
    try:
        lib = L.load()
    except ImportError as e:  # library not built in this checkout
        pytest.skip(str(e))
    off = (C.c_int64 * 2)(0, 10)
    fake = C.c_void_p(256)
    too_many = L.NQS_STATIC_MAX_SAMPLES + 1
    rc = lib.qgt_block_build_static(fake, too_many, too_many, 10, None, off, 1, fake, L.NQS_FP64, fake, fake,
                                    None, None, None)
    assert rc == L.NQS_ERR_INVALID_ARG
    assert b"static scratch" in lib.nqs_last_error()
    for p in (L.NQS_SPLIT_BF16, L.NQS_SPLIT_BF16X3, L.NQS_SPLIT_BF16_EXACT, 9):
        rc = lib.qgt_block_build_static(fake, 64, 64, 10, None, off, 1, fake, p, fake, fake, None, None, None)
        assert rc == L.NQS_ERR_INVALID_ARG


def _inputs(name, n_s, prec, weighted):
    import paper_2510_08430_gb300 as nq
    w = W.make_workload(name, n_s)
    model, theta, x, ham = dev_inputs(w)
    _, O = nq.nqs_jacobian(model, theta, x, prec)
    el = nq.nqs_local_energy(model, theta, x, ham, prec)
    ws = None
    if weighted:
        r = np.random.default_rng(n_s).random(n_s) + 0.1
        ws = torch.as_tensor(r / r.sum(), device="cuda")
    return w, O, el, ws


def _compare(w, O, el, ws, prec, tol):
    import paper_2510_08430_gb300 as nq
    O_ref = O.clone()
    S_r, F_r, Om_r, Em_r = nq.qgt_block_build(O_ref, w.configs.shape[0], w.block_off, el, prec, w=ws)
    O_st = O.clone()
    S_s, F_s, Om_s, Em_s = nq.qgt_block_build_static(O_st, w.configs.shape[0], w.block_off, el, prec, w=ws)
    torch.cuda.synchronize()
    Sr = unpack_lower(S_r.cpu().numpy(), w.block_off)
    Ss = unpack_lower(S_s.cpu().numpy(), w.block_off)
    for b in range(len(Sr)):
        assert rel(Ss[b], Sr[b]) < tol, b
    assert rel(F_s.cpu().numpy(), F_r.cpu().numpy()) < tol
    assert rel(Om_s.cpu().numpy(), Om_r.cpu().numpy()) < tol
    assert rel(Em_s.cpu().numpy(), Em_r.cpu().numpy()) < tol
    assert rel(O_st.cpu().numpy(), O_ref.cpu().numpy()) < tol


@pytest.mark.gpu
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("fp32", 1e-6)])
def test_static_build_matches_workspace_build_on_consecutive_calls(prec, tol):
    # two different problems back to back, then the first again: the scratch holds
    # nothing a later call depends on
    a = _inputs("j1j2_6x6_ffnn", 1000, prec, False)
    b = _inputs("chain10_rbm", 333, prec, True)
    _compare(*a, prec, tol)
    _compare(*b, prec, tol)
    _compare(*a, prec, tol)


@pytest.mark.gpu
def test_static_build_at_its_sample_limit():
    """At the largest sample count the static scratch holds: against the workspace build and,
    on its own, against the FP64 oracle (weighted means, centring, force and block QGT)."""
    import oracle
    import paper_2510_08430_gb300 as nq
    from paper_2510_08430_gb300 import _lib as L
    ns = L.NQS_STATIC_MAX_SAMPLES
    w, O, el, ws = _inputs("chain10_rbm", ns, "fp64", True)
    _compare(w, O, el, ws, "fp64", 1e-13)
    S, F, Om, Em = nq.qgt_block_build_static(O.clone(), ns, w.block_off, el, "fp64", w=ws)
    wt = ws.cpu().numpy()
    _, Oo = oracle.nqs.jacobian(w.model, w.theta, w.configs)
    elo = oracle.hamiltonian.local_energy(w.model, w.theta, w.configs, w.bond_ij, w.bond_j, w.c, w.sign_rule)
    e_mean, o_mean, dO, e = oracle.qgt.center(Oo, elo, wt)
    assert rel(F.cpu().numpy(), oracle.qgt.force(dO, e, wt)) < 1e-11
    assert rel(Om.cpu().numpy(), o_mean) < 1e-12
    assert abs(Em.cpu().numpy()[0] - e_mean) < 1e-12 * abs(e_mean)
    Sg = unpack_lower(S.cpu().numpy(), w.block_off)
    for b, Sb in enumerate(oracle.qgt.block_qgt(dO, w.block_off, wt)):
        assert rel(Sg[b], np.tril(Sb)) < 1e-12, b
