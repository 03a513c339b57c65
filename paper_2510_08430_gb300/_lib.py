"""ctypes loader for libnqs_sr.so (built in-tree by ``build.py``).

There is no fallback: if the shared library is missing the import fails.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnqs_sr.so")

NQS_OK = 0
NQS_ERR_INVALID_ARG = -1
NQS_ERR_CUDA = -2
NQS_ERR_WORKSPACE = -3
NQS_ERR_NOT_CONVERGED = -4
NQS_ERR_TIMEOUT = -5
NQS_ERR_NONFINITE = -6
NQS_ERR_UNSUPPORTED = -7
NQS_ERR_RETRY = -8

NQS_FP64, NQS_FP32, NQS_SPLIT_BF16, NQS_SPLIT_BF16X3, NQS_SPLIT_BF16_EXACT = 0, 1, 2, 3, 4
NQS_RBM, NQS_FFNN, NQS_VIT = 0, 1, 2
NQS_SYNC = 1
NQS_GRAPH = 2
NQS_PARAM_SPACE = 4
NQS_ELOC_DIFF32 = 8
NQS_SOLVE_FP64, NQS_SOLVE_MIXED, NQS_SOLVE_MIXED_PSD = 0, 1, 2
NQS_STATIC_MAX_SAMPLES = 65536


class nqs_model(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_layers", C.c_int32), ("widths", C.POINTER(C.c_int32))]


class nqs_hamiltonian(C.Structure):
    _fields_ = [("n_sites", C.c_int32), ("n_bonds", C.c_int32), ("bond_ij", C.c_void_p),
                ("bond_J", C.c_void_p), ("c", C.c_double), ("sign_rule", C.c_int32)]


P = C.c_void_p
I32 = C.c_int32
I64 = C.c_int64
D = C.c_double
SZ = C.POINTER(C.c_size_t)
MP = C.POINTER(nqs_model)
HP = C.POINTER(nqs_hamiltonian)
OFF = C.POINTER(C.c_int64)

# name -> (restype, argtypes); every symbol declared in include/nqs_sr.h
SIGNATURES = {
    "nqs_workspace_create": (C.c_int, [P, C.c_size_t, C.POINTER(P)]),
    "nqs_workspace_destroy": (C.c_int, [P]),
    "nqs_sync_status": (C.c_int, [P, P]),
    "nqs_last_error": (C.c_char_p, []),
    "nqs_version": (C.c_char_p, []),
    "nqs_jacobian_workspace_size": (C.c_int, [MP, I64, I32, SZ]),
    "nqs_local_energy_workspace_size": (C.c_int, [MP, I64, HP, I32, SZ]),
    "qgt_block_build_workspace_size": (C.c_int, [I64, I64, OFF, I32, I32, SZ]),
    "qgt_block_solve_workspace_size": (C.c_int, [OFF, I32, SZ]),
    "sr_step_workspace_size": (C.c_int, [MP, I64, HP, OFF, I32, I32, SZ]),
    "sr_step_workspace_size2": (C.c_int, [MP, I64, HP, OFF, I32, D, I32, I32, I32, SZ]),
    "qgt_packed_size": (C.c_int64, [OFF, I32]),
    "nqs_jacobian": (C.c_int, [MP, P, P, I64, I32, P, P, I64, P, P]),
    "nqs_local_energy": (C.c_int, [MP, P, P, I64, HP, I32, P, P, P]),
    "nqs_local_energy_ex": (C.c_int, [MP, P, P, I64, HP, I32, I32, P, P, P]),
    "nqs_metropolis_workspace_size": (C.c_int, [MP, I64, SZ]),
    "nqs_metropolis": (C.c_int, [MP, P, P, I64, I32, P, P, P, P]),
    "nqs_theta_update": (C.c_int, [P, P, I64, P]),
    "nqs_connections": (C.c_int, [P, I64, HP, P, P, P, I64, C.POINTER(C.c_int64), P, P]),
    "nqs_vjp": (C.c_int, [P, I64, I64, I64, I32, P, P, P]),
    "ntk_solve_workspace_size": (C.c_int, [I64, I64, I32, SZ]),
    "ntk_solve": (C.c_int, [P, I64, I64, I64, P, D, D, D, I32, P, P, P, P]),
    "nqs_shard_sums": (C.c_int, [P, I64, I64, I64, I32, P, P, P, P]),
    "qgt_block_build_shard": (C.c_int, [P, I64, I64, I64, I64, OFF, I32, P, P, P, I32, P, P, P, P, P, P]),
    "qgt_block_build": (C.c_int, [P, I64, I64, I64, P, OFF, I32, P, I32, P, P, P, P, P, P]),
    "qgt_block_build_static": (C.c_int, [P, I64, I64, I64, P, OFF, I32, P, I32, P, P, P, P, P]),
    "qgt_block_solve": (C.c_int, [P, OFF, I32, P, D, D, I32, D, I32, P, P, P, P, P]),
    "sr_step": (C.c_int, [MP, P, P, I64, HP, OFF, I32, D, D, I32, D, I32, I32, P, P, P, P, I32, P, P]),
    "sr_step_batched_workspace_size": (C.c_int, [I32, P, OFF, P, OFF, P, I32, SZ]),
    "sr_step_batched": (C.c_int, [I32, P, P, P, OFF, P, OFF, P, D, D, I32, D, I32, I32, P, P, P, P, I32, P, P]),
    "nqs_stage_timing": (C.c_int, [P, I32]),
    "nqs_stage_times": (C.c_int, [P, C.POINTER(C.c_double), I32, C.POINTER(C.c_int32)]),
    "nqs_launch_count": (C.c_int64, []),
    "nqs_set_limits": (C.c_int, [I32, I64]),
    "nqs_set_eloc_fallback_all": (C.c_int, [I32]),
    "nqs_born_weights": (C.c_int, [P, I64, P, P]),
    "nqs_set_gram_tuning": (C.c_int, [I32, OFF, OFF, C.POINTER(C.c_int32)]),
    "nqs_gram_group_edge": (C.c_int32, [I64, I64]),
    "qgt_inverse_diagnostics_workspace_size": (C.c_int, [I64, SZ]),
    "qgt_inverse_diagnostics": (C.c_int, [P, OFF, I32, P, I64, D, D, I32, P, P, P]),
}

_lib = None


def load() -> C.CDLL:
    """Load libnqs_sr.so with argument types set; raises if it is not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run paper_2510_08430_gb300/build.py "
                          "(there is no CPU or Python fallback)")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class NQSError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"nqs_sr status {code}: {msg}")
        self.code = code


def check(rc: int) -> None:
    if rc != NQS_OK:
        raise NQSError(rc, load().nqs_last_error().decode())
