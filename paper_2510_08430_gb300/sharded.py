"""Sample-sharded block-SR step: one SR instance whose samples are split over ranks.

The step has three exchanges:

1. After the Jacobian and local energies of each shard, an all-reduce of the per-shard
   sums (n_p + 1 complex numbers). The library turns the summed values into the global
   means <O> and <E> (qgt_block_build_shard).
2. After each shard's part of the block Gram and the force (centred with the global
   means, weight 1/N per sample), a reduce-scatter by block owner: rank r receives the
   sum over all shards of the S_b and F_b of the blocks it owns, and nothing else.
3. After each owner has solved its blocks (Sec. 2, block-layer paragraph: the blocks are
   independent), an all-gather of the owners' dtheta slices.

Owners are chosen to balance sum n_b^3, the cost of the per-block solve.

The compute is the library's (`LibraryShardBackend`). This module only partitions the
work and moves it between ranks, either over a process group (`step_distributed`) or
with all shards in one process (`step_simulated`).
"""
from __future__ import annotations

import ctypes as C
from typing import List, Sequence

import numpy as np
import torch

from . import _lib
from ._lib import check
from .api import Hamiltonian, Model, Workspace, _off, _on, _prec, _ptr, _size, _stream, nqs_jacobian, \
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


def owned_pack(S: torch.Tensor, F: torch.Tensor, block_off, owned: Sequence[int]) -> torch.Tensor:
    """One contiguous buffer of the owned blocks: their packed S_b in order, then their F_b."""
    block_off = np.asarray(block_off, dtype=np.int64)
    pr = packed_ranges(block_off)
    parts = [S[pr[b][0]:pr[b][1]] for b in owned] + [F[block_off[b]:block_off[b + 1]] for b in owned]
    if not parts:
        return torch.zeros(0, dtype=S.dtype, device=S.device)
    return torch.cat(parts)


def owned_unpack(buf: torch.Tensor, block_off, owned: Sequence[int]):
    """(S_sub packed, offsets of the owned blocks, F_sub) from an owned_pack buffer."""
    block_off = np.asarray(block_off, dtype=np.int64)
    sizes = [int(block_off[b + 1] - block_off[b]) for b in owned]
    nsq = sum(n * n for n in sizes)
    off_sub = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return buf[:nsq], off_sub, buf[nsq:nsq + int(off_sub[-1])]


class LibraryShardBackend:
    """One shard's compute through the C ABI (device tensors)."""

    def __init__(self, model: Model, ham: Hamiltonian, block_off, precision="fp64", solver="fp64",
                 eloc_diff32: bool = False):
        self.model, self.ham = model, ham
        self.block_off = np.asarray(block_off, dtype=np.int64)
        self.precision, self.solver = precision, solver
        self.eloc_diff32 = eloc_diff32
        self.n_p = int(self.block_off[-1])

    def local(self, theta: torch.Tensor, configs: torch.Tensor):
        """Jacobian, local energies and the shard sums: (state, osum [n_p], esum [1])."""
        lib = _lib.load()
        _, O = nqs_jacobian(self.model, theta, configs, self.precision)
        eloc = nqs_local_energy(self.model, theta, configs, self.ham, self.precision, diff32=self.eloc_diff32)
        osum = torch.empty(self.n_p, dtype=torch.complex128, device=O.device)
        esum = torch.empty(1, dtype=torch.complex128, device=O.device)
        ns = int(configs.shape[0])
        with _on(O, eloc):
            check(lib.nqs_shard_sums(_ptr(O), int(O.shape[1]), ns, self.n_p, _prec(self.precision), _ptr(eloc),
                                     _ptr(osum), _ptr(esum), _stream()))
        return (O, eloc, ns), osum, esum

    def build(self, state, osum: torch.Tensor, esum: torch.Tensor, n_total: int):
        """This shard's weighted S (packed) and F, centred with the global means that the
        library forms from the all-reduced sums; also returns <E> (c128 [1])."""
        lib = _lib.load()
        O, eloc, ns = state
        off = _off(self.block_off)
        nb = len(self.block_off) - 1
        p = _prec(self.precision)
        ws = Workspace(_size(lib.qgt_block_build_workspace_size, ns, self.n_p, off, nb, p), device=O.device)
        S = torch.zeros(int(lib.qgt_packed_size(off, nb)), dtype=torch.complex128, device=O.device)
        F = torch.empty(self.n_p, dtype=torch.complex128, device=O.device)
        em = torch.empty(1, dtype=torch.complex128, device=O.device)
        osum, esum = osum.contiguous(), esum.contiguous()
        with _on(O, eloc, osum, esum):
            check(lib.qgt_block_build_shard(_ptr(O), int(O.shape[1]), ns, self.n_p, int(n_total), off, nb,
                                            _ptr(eloc), _ptr(osum), _ptr(esum), p, _ptr(S), _ptr(F), None,
                                            _ptr(em), ws.h, _stream()))
        ws.sync_status()
        return S, F, em

    def solve(self, S_sub: torch.Tensor, off_sub, F_sub: torch.Tensor, diag_shift: float, cutoff: float,
              cutoff_mode: int, eta: float) -> torch.Tensor:
        solver = "mixed_psd" if self.solver == "mixed" else self.solver
        dth, _, _ = qgt_block_solve(S_sub, off_sub, F_sub, diag_shift, cutoff, cutoff_mode, eta, want_evals=False,
                                    solver=solver)
        return dth


class TorchComm:
    """The three collectives of the step over the default torch.distributed process group."""

    def all_reduce(self, t: torch.Tensor) -> None:
        import torch.distributed as dist
        dist.all_reduce(t)

    def reduce(self, t: torch.Tensor, dst: int) -> None:
        import torch.distributed as dist
        dist.reduce(t, dst=dst)

    def all_gather(self, out: List[torch.Tensor], t: torch.Tensor) -> None:
        import torch.distributed as dist
        dist.all_gather(out, t)


def _solve_owned_buf(backend, buf, block_off, owned, diag_shift, cutoff, cutoff_mode, eta):
    """dtheta of the owned blocks, concatenated in owned order."""
    if not owned:
        return torch.zeros(0, dtype=torch.complex128, device=buf.device)
    S_sub, off_sub, F_sub = owned_unpack(buf, block_off, owned)
    return backend.solve(S_sub.clone(), off_sub, F_sub.contiguous(), diag_shift, cutoff, cutoff_mode, eta)


def _assemble(slices: Sequence[torch.Tensor], owners, block_off, n_p: int, device) -> torch.Tensor:
    """dtheta from every rank's owned slice (owned blocks in owned order)."""
    block_off = np.asarray(block_off, dtype=np.int64)
    dth = torch.empty(n_p, dtype=torch.complex128, device=device)
    for r, owned in enumerate(owners):
        p = 0
        for b in owned:
            n = int(block_off[b + 1] - block_off[b])
            dth[block_off[b]:block_off[b + 1]] = slices[r][p:p + n]
            p += n
    return dth


def step_distributed(backend, theta: torch.Tensor, configs_local: torch.Tensor, n_total: int, block_off,
                     diag_shift: float, cutoff: float, cutoff_mode: int = 0, eta: float = 1.0, comm=None,
                     rank: int = 0, world: int = 1):
    """One sharded step on this rank (its shard `configs_local` of n_total samples).
    `comm` provides all_reduce(t), reduce(t, dst) and all_gather(list, t) (default: the
    torch.distributed process group). Returns (dtheta [n_p], <E> [1]) on every rank."""
    comm = TorchComm() if comm is None else comm
    block_off = np.asarray(block_off, dtype=np.int64)
    n_p = int(block_off[-1])
    # exchange 1: the shard sums -> global means (formed in the library)
    state, osum, esum = backend.local(theta, configs_local)
    sums = torch.cat([osum, esum])
    comm.all_reduce(sums)
    S, F, emean = backend.build(state, sums[:-1], sums[-1:], n_total)
    # exchange 2: reduce-scatter of S and F by block owner
    owners = block_owners(block_off, world)
    mine = None
    for r in range(world):
        buf = owned_pack(S, F, block_off, owners[r])
        if buf.numel():
            comm.reduce(buf, dst=r)
        if r == rank:
            mine = buf
    del S, F
    d_own = _solve_owned_buf(backend, mine, block_off, owners[rank], diag_shift, cutoff, cutoff_mode, eta)
    # exchange 3: all-gather of the owners' dtheta slices (padded to the largest)
    width = max(int(sum(block_off[b + 1] - block_off[b] for b in o)) for o in owners)
    pad = torch.zeros(width, dtype=torch.complex128, device=d_own.device)
    pad[:d_own.numel()] = d_own
    gathered = [torch.empty_like(pad) for _ in range(world)]
    comm.all_gather(gathered, pad)
    return _assemble(gathered, owners, block_off, n_p, d_own.device), emean


def step_simulated(backend, theta: torch.Tensor, shards: Sequence[torch.Tensor], block_off, diag_shift: float,
                   cutoff: float, cutoff_mode: int = 0, eta: float = 1.0, world: int = None):
    """The same step with every shard processed in turn in this process and the exchanges
    done here (ranks simulated on one device). `world` ranks own the blocks (default:
    one per shard)."""
    world = len(shards) if world is None else world
    block_off = np.asarray(block_off, dtype=np.int64)
    n_total = sum(int(x.shape[0]) for x in shards)
    parts = [backend.local(theta, x) for x in shards]
    sums = sum(torch.cat([o, e]) for _, o, e in parts)
    owners = block_owners(block_off, world)
    bufs = [None] * world
    emean = None
    for state, _, _ in parts:
        s, f, em = backend.build(state, sums[:-1], sums[-1:], n_total)
        emean = em
        for r in range(world):
            b = owned_pack(s, f, block_off, owners[r])
            bufs[r] = b if bufs[r] is None else bufs[r] + b
    slices = [_solve_owned_buf(backend, bufs[r], block_off, owners[r], diag_shift, cutoff, cutoff_mode, eta)
              for r in range(world)]
    return _assemble(slices, owners, block_off, int(block_off[-1]), theta.device), emean
