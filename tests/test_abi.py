"""Host-side checks of the C ABI: the library loads, exports every symbol the
header declares, and validates arguments without touching a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"NQS_API\s+[\w\s\*]+?\b(\w+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2510_08430_gb300 import _lib
    if not os.path.exists(_lib.LIB_PATH):
        from paper_2510_08430_gb300 import build
        build.build()
    return _lib.load()


def test_every_declared_symbol_is_exported_and_bound(lib):
    from paper_2510_08430_gb300 import _lib
    names = _declared()
    assert len(names) >= 17
    for n in names:
        assert hasattr(lib, n), n
        assert n in _lib.SIGNATURES, n


def test_version_and_error_string(lib):
    assert b"sm_103a" in lib.nqs_version()
    assert lib.nqs_last_error() is not None


def _model(kind, widths):
    from paper_2510_08430_gb300 import Model
    return Model(kind, widths)


def test_workspace_size_queries(lib):
    from paper_2510_08430_gb300 import _lib
    m = _model(1, [36, 64, 64, 1])
    out = C.c_size_t(0)
    assert lib.nqs_jacobian_workspace_size(C.byref(m.c), 4096, 1, C.byref(out)) == 0
    # thR + W^T + Z + G (c64) + logpsi: grows with n_s
    small = out.value
    assert lib.nqs_jacobian_workspace_size(C.byref(m.c), 8192, 1, C.byref(out)) == 0
    assert out.value > small
    off = (C.c_int64 * 4)(0, 2368, 6528, 6593)
    assert lib.qgt_packed_size(off, 3) == 2368 ** 2 + 4160 ** 2 + 65 ** 2
    assert lib.qgt_block_solve_workspace_size(off, 3, C.byref(out)) == 0 and out.value > 0
    h = _lib.nqs_hamiltonian(36, 144, None, None, 1.0, 1)
    assert lib.sr_step_workspace_size(C.byref(m.c), 4096, C.byref(h), off, 3, 2, C.byref(out)) == 0
    assert out.value > 6593 * 4096 * 8


def test_invalid_arguments_are_rejected(lib):
    out = C.c_size_t(0)
    bad = (C.c_int64 * 4)(0, 10, 10, 20)  # not strictly increasing
    assert lib.qgt_block_solve_workspace_size(bad, 3, C.byref(out)) == -1
    assert b"strictly" in lib.nqs_last_error()
    bad0 = (C.c_int64 * 2)(1, 5)
    assert lib.qgt_block_solve_workspace_size(bad0, 1, C.byref(out)) == -1
    m = _model(1, [36, 64, 64, 2])  # FFNN must end in one output
    assert lib.nqs_jacobian_workspace_size(C.byref(m.c), 16, 0, C.byref(out)) == -1
    m = _model(1, [36, 64, 1])
    assert lib.nqs_jacobian_workspace_size(C.byref(m.c), 16, 7, C.byref(out)) == -1  # precision
    off = (C.c_int64 * 3)(0, 100, 2368)
    assert lib.qgt_block_build_workspace_size(16, 999, off, 2, 0, C.byref(out)) == -1  # n_p mismatch
    assert lib.nqs_workspace_create(None, 1024, C.byref(C.c_void_p())) == -1


def test_newer_entry_points_validate_on_the_host(lib):
    """Argument errors of the batched, sharded, NTK and VJP calls are caught before any
    device work (the fake pointers below are never dereferenced)."""
    from paper_2510_08430_gb300 import _lib
    out = C.c_size_t(0)
    fake = C.c_void_p(256)
    # batched: no instance
    assert lib.sr_step_batched_workspace_size(0, None, None, None, None, None, 0, C.byref(out)) == -1
    # NTK: split precisions are not an NTK Gram option
    assert lib.ntk_solve_workspace_size(64, 100, _lib.NQS_SPLIT_BF16_EXACT, C.byref(out)) == -1
    assert lib.ntk_solve_workspace_size(64, 100, _lib.NQS_FP32, C.byref(out)) == 0 and out.value > 64 * 64 * 16
    # shard build: the total sample count cannot be below the shard's
    off = (C.c_int64 * 2)(0, 10)
    assert lib.qgt_block_build_shard(fake, 64, 64, 10, 63, off, 1, fake, fake, fake, 0, fake, fake, None, None,
                                     None, None) == -1
    assert b"qgt_block_build_shard" in lib.nqs_last_error()
    # test hook: negative limits are rejected, zeros restore the defaults
    assert lib.nqs_set_limits(-1, 0) == -1 and lib.nqs_set_limits(0, -5) == -1
    assert lib.nqs_set_limits(0, 0) == 0
    assert lib.nqs_set_eloc_fallback_all(1) == 0 and lib.nqs_set_eloc_fallback_all(0) == 0
    # local energies: unknown flag bits, and the difference propagation without an FP64 forward
    from paper_2510_08430_gb300 import _lib
    m = _model(1, [36, 64, 64, 1])
    h = _lib.nqs_hamiltonian(36, 144, None, None, 1.0, 1)
    assert lib.nqs_local_energy_ex(C.byref(m.c), fake, fake, 8, C.byref(h), 4, 16, fake, None, None) == -1
    assert lib.nqs_local_energy_ex(C.byref(m.c), fake, fake, 8, C.byref(h), 1, _lib.NQS_ELOC_DIFF32, fake, None,
                                   None) == -1
    assert b"NQS_ELOC_DIFF32" in lib.nqs_last_error()
    # sampler: no chains, negative steps, missing uniforms
    assert lib.nqs_metropolis(C.byref(m.c), fake, fake, 0, 1, fake, None, None, None) == -1
    assert lib.nqs_metropolis(C.byref(m.c), fake, fake, 4, -1, fake, None, None, None) == -1
    assert lib.nqs_metropolis(C.byref(m.c), fake, fake, 4, 3, None, None, None, None) == -1
    assert lib.nqs_theta_update(None, fake, 4, None) == -1
    out = C.c_size_t(0)
    assert lib.nqs_metropolis_workspace_size(C.byref(m.c), 64, C.byref(out)) == 0 and out.value > 0
    # transformer: FP64 only; the patch must divide N
    import paper_2510_08430_gb300 as nq
    vit = nq.Model(2, [16, 4, 16, 32], 2)
    assert lib.nqs_jacobian_workspace_size(C.byref(vit.c), 64, 0, C.byref(out)) == 0
    assert lib.nqs_jacobian_workspace_size(C.byref(vit.c), 64, 1, C.byref(out)) == -7
    bad = nq.Model(2, [16, 5, 16, 32], 2)
    assert lib.nqs_jacobian_workspace_size(C.byref(bad.c), 64, 0, C.byref(out)) == -1
    # shard sums and VJP: leading dimension below n_s
    assert lib.nqs_shard_sums(fake, 10, 64, 10, 0, fake, fake, fake, None) == -1
    assert lib.nqs_vjp(fake, 10, 64, 10, 0, fake, fake, None) == -1
