"""Sample-sharded block-SR step: one SR instance whose samples are split over ranks.

The step has two exchanges:

1. After the Jacobian and local energies of each shard, the global means <O> and <E>.
   These come from an all-reduce of the per-shard sums (n_p + 1 complex numbers).
2. After each shard's part of the block Gram and the force (centred with the global
   means, weight 1/N per sample), the sum of those parts.

The blocks are then independent (Sec. 2, block-layer paragraph). Each rank solves the
blocks it owns; owners are chosen to balance sum n_b^3. dtheta is assembled by summing
the owners' disjoint slices.

The compute is the library's (`LibraryShardBackend`). This module only partitions the
work and reduces it, either over a process group (`step_distributed`) or with all shards
in one process (`step_simulated`).
"""
from __future__ import annotations

import ctypes as C
from typing import Callable, List, Sequence

import numpy as np
import torch

from . import _lib
from ._lib import check
from .api import Hamiltonian, Model, Workspace, _off, _prec, _ptr, _size, _solver, _stream, nqs_jacobian, \
    nqs_local_energy, qgt_block_solve


def block_owners(block_off: Sequence[int], world: int) -> List[List[int]]:
    """Greedy assignment of blocks to ranks by descending cost n_b^3."""
    sizes = np.diff(np.asarray(block_off, dtype=np.int64))
    load = [0.0] * world
    owners: List[List[int]] = [[] for _ in range(world)]
    for b in sorted(range(len(sizes)), key=lambda i: -float(sizes[i]) ** 3):
        r = int(np.argmin(load))
        owners[r].append(b)
        load[r] += float(sizes[b]) ** 3
    return [sorted(o) for o in owners]


def packed_ranges(block_off: Sequence[int]):
    """(start, end) of each block's n_b x n_b matrix in the packed S."""
    out, p = [], 0
    for b in range(len(block_off) - 1):
        n = int(block_off[b + 1] - block_off[b])
        out.append((p, p + n * n))
        p += n * n
    return out


class LibraryShardBackend:
    """One shard's compute through the C ABI (device tensors)."""

    def __init__(self, model: Model, ham: Hamiltonian, block_off, precision="fp64", solver="fp64"):
        self.model, self.ham = model, ham
        self.block_off = np.asarray(block_off, dtype=np.int64)
        self.precision, self.solver = precision, solver
        self.n_p = int(self.block_off[-1])

    def local(self, theta: torch.Tensor, configs: torch.Tensor):
        """Jacobian, local energies and the shard sums: (state, osum [n_p], esum [1])."""
        lib = _lib.load()
        _, O = nqs_jacobian(self.model, theta, configs, self.precision)
        eloc = nqs_local_energy(self.model, theta, configs, self.ham, self.precision)
        osum = torch.empty(self.n_p, dtype=torch.complex128, device=O.device)
        esum = torch.empty(1, dtype=torch.complex128, device=O.device)
        ns = int(configs.shape[0])
        check(lib.nqs_shard_sums(_ptr(O), int(O.shape[1]), ns, self.n_p, _prec(self.precision), _ptr(eloc),
                                 _ptr(osum), _ptr(esum), _stream()))
        return (O, eloc, ns), osum, esum

    def build(self, state, omean: torch.Tensor, emean: torch.Tensor, weight: float):
        """This shard's weighted S (packed) and F with the global means."""
        lib = _lib.load()
        O, eloc, ns = state
        off = _off(self.block_off)
        nb = len(self.block_off) - 1
        p = _prec(self.precision)
        ws = Workspace(_size(lib.qgt_block_build_workspace_size, ns, self.n_p, off, nb, p), device=O.device)
        S = torch.zeros(int(lib.qgt_packed_size(off, nb)), dtype=torch.complex128, device=O.device)
        F = torch.empty(self.n_p, dtype=torch.complex128, device=O.device)
        check(lib.qgt_block_build_shard(_ptr(O), int(O.shape[1]), ns, self.n_p, float(weight), off, nb, _ptr(eloc),
                                        _ptr(omean.contiguous()), _ptr(emean.contiguous()), p, _ptr(S), _ptr(F),
                                        ws.h, _stream()))
        ws.sync_status()
        return S, F

    def solve(self, S_sub: torch.Tensor, off_sub, F_sub: torch.Tensor, diag_shift: float, cutoff: float,
              cutoff_mode: int, eta: float) -> torch.Tensor:
        solver = "mixed_psd" if self.solver == "mixed" else self.solver
        dth, _, _ = qgt_block_solve(S_sub, off_sub, F_sub, diag_shift, cutoff, cutoff_mode, eta, want_evals=False,
                                    solver=solver)
        return dth


def _solve_owned(backend, S, F, block_off, owned, diag_shift, cutoff, cutoff_mode, eta):
    """dtheta with this rank's owned blocks filled in and zeros elsewhere."""
    block_off = np.asarray(block_off, dtype=np.int64)
    dth = torch.zeros(int(block_off[-1]), dtype=torch.complex128, device=F.device)
    if not owned:
        return dth
    pr = packed_ranges(block_off)
    S_sub = torch.cat([S[pr[b][0]:pr[b][1]] for b in owned])
    F_sub = torch.cat([F[block_off[b]:block_off[b + 1]] for b in owned])
    sizes = [int(block_off[b + 1] - block_off[b]) for b in owned]
    off_sub = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    d = backend.solve(S_sub, off_sub, F_sub, diag_shift, cutoff, cutoff_mode, eta)
    for k, b in enumerate(owned):
        dth[block_off[b]:block_off[b + 1]] = d[off_sub[k]:off_sub[k + 1]]
    return dth


def step_distributed(backend, theta: torch.Tensor, configs_local: torch.Tensor, n_total: int, block_off,
                     diag_shift: float, cutoff: float, cutoff_mode: int = 0, eta: float = 1.0,
                     all_reduce: Callable[[torch.Tensor], None] = None, rank: int = 0, world: int = 1):
    """One sharded step on this rank (its shard `configs_local` of n_total samples).
    `all_reduce(t)` sums t in place over the ranks (torch.distributed.all_reduce)."""
    if all_reduce is None:
        import torch.distributed as dist

        def all_reduce(t):
            dist.all_reduce(t)
    state, osum, esum = backend.local(theta, configs_local)
    sums = torch.cat([osum, esum])
    all_reduce(sums)
    means = sums / n_total
    S, F = backend.build(state, means[:-1], means[-1:], 1.0 / n_total)
    all_reduce(S)
    all_reduce(F)
    dth = _solve_owned(backend, S, F, block_off, block_owners(block_off, world)[rank], diag_shift, cutoff,
                       cutoff_mode, eta)
    all_reduce(dth)
    return dth, means[-1:]


def step_simulated(backend, theta: torch.Tensor, shards: Sequence[torch.Tensor], block_off, diag_shift: float,
                   cutoff: float, cutoff_mode: int = 0, eta: float = 1.0, world: int = None):
    """The same step with every shard processed in turn in this process and the reductions
    summed here (ranks simulated on one device). `world` ranks own the blocks (default:
    one per shard)."""
    world = len(shards) if world is None else world
    n_total = sum(int(x.shape[0]) for x in shards)
    parts = [backend.local(theta, x) for x in shards]
    sums = sum(torch.cat([o, e]) for _, o, e in parts)
    means = sums / n_total
    S, F = None, None
    for state, _, _ in parts:
        s, f = backend.build(state, means[:-1], means[-1:], 1.0 / n_total)
        S = s if S is None else S + s
        F = f if F is None else F + f
    dth = None
    for r, owned in enumerate(block_owners(block_off, world)):
        d = _solve_owned(backend, S.clone(), F, block_off, owned, diag_shift, cutoff, cutoff_mode, eta)
        dth = d if dth is None else dth + d
    return dth, means[-1:]
