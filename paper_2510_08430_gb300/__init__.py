"""Block-layer stochastic reconfiguration for neural quantum states on GB300.

The compute path is libnqs_sr.so (hand-written CUDA for sm_103a, C ABI in
include/nqs_sr.h); this package is its thin Python binding.
"""
from .api import (Hamiltonian, Model, NQSLogPsi, SRStep, Workspace, born_weights, inverse_metric_study,  # noqa: F401
                  launch_count, log_psi, nqs_connections, nqs_jacobian, nqs_local_energy, ntk_solve, qgt_block_build,
                  qgt_block_build_static, qgt_block_solve, qgt_inverse_diagnostics, set_eloc_fallback_all, set_limits,
                  plan_batch_chunks, sr_step, sr_step_batched, sr_step_batched_workspace_size, theta_update,
                  metropolis, version, vmc_train)
from ._lib import NQS_FFNN, NQS_FP32, NQS_FP64, NQS_RBM, NQS_SPLIT_BF16, NQS_VIT, NQSError  # noqa: F401
