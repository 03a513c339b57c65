"""Helpers shared by the GPU parity tests (inputs come from `workloads`)."""
import numpy as np
import torch

import workloads as W


def dev_inputs(w: W.Workload):
    import paper_2510_08430_gb300 as nq
    model = nq.Model.from_workload(w.model)
    theta = torch.as_tensor(w.theta, device="cuda")
    x = torch.as_tensor(w.configs, device="cuda")
    ham = nq.Hamiltonian(w.model.n_sites, w.bond_ij, w.bond_j, w.c, w.sign_rule)
    return model, theta, x, ham


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def unpack_lower(S_packed: np.ndarray, block_off):
    """List of n_b x n_b lower triangles (upper set to 0) from the packed layout."""
    out, p = [], 0
    for b in range(len(block_off) - 1):
        n = int(block_off[b + 1] - block_off[b])
        m = S_packed[p:p + n * n].reshape(n, n)
        out.append(np.tril(m))
        p += n * n
    return out


# Per-sample local-energy bar of the FP32 difference propagation (NQS_ELOC_DIFF32), relative
# to max(|E_loc|, 1); FP64-class local energies are held to 1e-12.
ELOC_SPLIT_BAR = 2e-6


def emean_bar(n_s: int, diff32: bool) -> float:
    """Relative bar on <E>: 1e-12 with FP64-class local energies; with the FP32 difference
    propagation the per-sample rounding errors (round to nearest, independent between
    samples) average down, so the mean is held to ELOC_SPLIT_BAR / sqrt(n_s)."""
    return max(ELOC_SPLIT_BAR / np.sqrt(n_s), 1e-12) if diff32 else 1e-12
