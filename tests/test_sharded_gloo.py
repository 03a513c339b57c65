"""Host logic of the sample-sharded step on two gloo ranks (CPU). The per-shard compute is
the FP64 oracle's, so the test checks the partition and the two exchanges: the sharded
step must equal the unsharded oracle step."""
import os
import socket
import tempfile

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle
import workloads as W


class OracleShardBackend:
    """One shard's compute with the oracle (CPU tensors)."""

    def __init__(self, w):
        self.w = w

    def local(self, theta, configs):
        w = self.w
        x = configs.numpy()
        _, O = oracle.nqs.jacobian(w.model, w.theta, x)
        el = oracle.hamiltonian.local_energy(w.model, w.theta, x, w.bond_ij, w.bond_j, w.c, w.sign_rule)
        return (O, el), torch.as_tensor(O.sum(axis=0)), torch.as_tensor(np.array([el.sum()]))

    def build(self, state, osum, esum, n_total):
        O, el = state
        weight = 1.0 / n_total
        omean, emean = osum.numpy() * weight, esum.numpy() * weight
        dO = O - omean[None, :]
        e = el - emean[0]
        F = weight * (np.conj(dO).T @ e)
        S = []
        off = self.w.block_off
        for b in range(len(off) - 1):
            X = dO[:, off[b]:off[b + 1]]
            S.append((weight * (np.conj(X).T @ X)).ravel())
        return torch.as_tensor(np.concatenate(S)), torch.as_tensor(F), torch.as_tensor(emean)

    def solve(self, S_sub, off_sub, F_sub, diag_shift, cutoff, cutoff_mode, eta):
        S = S_sub.numpy()
        blocks, p = [], 0
        for b in range(len(off_sub) - 1):
            n = int(off_sub[b + 1] - off_sub[b])
            blocks.append(S[p:p + n * n].reshape(n, n))
            p += n * n
        d, _, _ = oracle.qgt.block_solve(blocks, F_sub.numpy(), off_sub, diag_shift, cutoff, eta,
                                         absolute=cutoff_mode == 1)
        return torch.as_tensor(d)


def _workload(name, ns):
    if name == "ffnn4x4":  # three blocks of unequal size, small enough for the oracle's eigh
        model = W.Model(W.FFNN, (16, 24, 8, 1))
        rng = np.random.default_rng(7)
        theta = W.init_params(model, rng)
        x = W.zero_sz_configs(16, ns, rng)
        ij, jj = W.square_j1j2_bonds(4, 4, 1.0, 0.3)
        return W.Workload(name, model, theta, x, ij, jj, model.block_offsets(), 1e-3, 1e-10, "fp64")
    return W.make_workload(name, ns)


def _rank(rank, world, port, name, ns, out_dir):
    import torch.distributed as dist
    from paper_2510_08430_gb300 import sharded
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", world_size=world, rank=rank)
    w = _workload(name, ns)
    shard = np.array_split(np.arange(ns), world)[rank]
    x = torch.as_tensor(w.configs[shard])
    dth, em = sharded.step_distributed(OracleShardBackend(w), torch.as_tensor(w.theta), x, ns, w.block_off,
                                       w.diag_shift, w.cutoff, rank=rank, world=world)
    np.save(os.path.join(out_dir, f"dth{rank}.npy"), dth.numpy())
    np.save(os.path.join(out_dir, f"em{rank}.npy"), em.numpy())
    dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


@pytest.mark.parametrize("name,ns", [("chain10_rbm", 120), ("ffnn4x4", 90)])
def test_two_rank_sharded_step_equals_unsharded(name, ns):
    world = 2
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_rank, args=(world, _free_port(), name, ns, d), nprocs=world, join=True,
                           start_method="spawn")
        w = _workload(name, ns)
        r = oracle.qgt.sr_step(w.model, w.theta, w.configs, w.bond_ij, w.bond_j, w.block_off, w.diag_shift,
                               w.cutoff, 1.0, w.c, w.sign_rule)
        for rank in range(world):
            dth = np.load(os.path.join(d, f"dth{rank}.npy"))
            em = np.load(os.path.join(d, f"em{rank}.npy"))
            assert np.linalg.norm(dth - r["dtheta"]) <= 1e-10 * np.linalg.norm(r["dtheta"])
            assert abs(em[0] - r["e_mean"]) <= 1e-12 * abs(r["e_mean"])


class CountingComm:
    """torch.distributed collectives that record the element counts each rank sends."""

    def __init__(self):
        from paper_2510_08430_gb300.sharded import TorchComm
        self.inner = TorchComm()
        self.log = []

    def all_reduce(self, t):
        self.log.append(("all_reduce", t.numel()))
        self.inner.all_reduce(t)

    def reduce(self, t, dst):
        self.log.append(("reduce", t.numel(), dst))
        self.inner.reduce(t, dst)

    def all_gather(self, out, t):
        self.log.append(("all_gather", t.numel()))
        self.inner.all_gather(out, t)


def _rank_counted(rank, world, port, name, ns, out_dir):
    import json
    import torch.distributed as dist
    from paper_2510_08430_gb300 import sharded
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", world_size=world, rank=rank)
    w = _workload(name, ns)
    shard = np.array_split(np.arange(ns), world)[rank]
    comm = CountingComm()
    dth, _ = sharded.step_distributed(OracleShardBackend(w), torch.as_tensor(w.theta),
                                      torch.as_tensor(w.configs[shard]), ns, w.block_off, w.diag_shift, w.cutoff,
                                      comm=comm, rank=rank, world=world)
    np.save(os.path.join(out_dir, f"dth{rank}.npy"), dth.numpy())
    json.dump(comm.log, open(os.path.join(out_dir, f"log{rank}.json"), "w"))
    dist.destroy_process_group()


def test_exchanges_are_reduce_scatter_and_all_gather():
    """Exchange 2 sends each owner only its blocks (sum over owners = the packed S and F once);
    exchange 3 gathers dtheta slices no longer than the largest owner's share."""
    import json
    from paper_2510_08430_gb300.sharded import block_owners
    world, name, ns = 2, "ffnn4x4", 60
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_rank_counted, args=(world, _free_port(), name, ns, d), nprocs=world, join=True,
                           start_method="spawn")
        w = _workload(name, ns)
        off = w.block_off
        sizes = np.diff(off)
        owners = block_owners(off, world)
        r = oracle.qgt.sr_step(w.model, w.theta, w.configs, w.bond_ij, w.bond_j, off, w.diag_shift, w.cutoff)
        for rank in range(world):
            dth = np.load(os.path.join(d, f"dth{rank}.npy"))
            assert np.linalg.norm(dth - r["dtheta"]) <= 1e-10 * np.linalg.norm(r["dtheta"])
            log = json.load(open(os.path.join(d, f"log{rank}.json")))
            assert log[0] == ["all_reduce", int(off[-1]) + 1]
            reduces = [e for e in log if e[0] == "reduce"]
            assert [e[2] for e in reduces] == [q for q in range(world) if owners[q]]
            for e in reduces:
                own = owners[e[2]]
                assert e[1] == int(sum(sizes[b] ** 2 + sizes[b] for b in own))
            assert sum(e[1] for e in reduces) == int(np.sum(sizes ** 2) + off[-1])
            gathers = [e for e in log if e[0] == "all_gather"]
            assert gathers == [["all_gather", max(int(sum(sizes[b] for b in o)) for o in owners)]]
            assert not any(e[0] == "all_reduce" for e in log[1:])


def _rank_leaves(rank, world, port, name, ns, out_dir):
    """Both ranks take one step; rank 1 then leaves between steps (its process ends with
    nothing in flight). Rank 0's next step must fail with an error, within the process
    group's short timeout, instead of waiting for ever."""
    import datetime
    import torch.distributed as dist
    from paper_2510_08430_gb300 import sharded
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", world_size=world, rank=rank,
                            timeout=datetime.timedelta(seconds=20))
    w = _workload(name, ns)
    shard = np.array_split(np.arange(ns), world)[rank]
    x = torch.as_tensor(w.configs[shard])
    args = (torch.as_tensor(w.theta), x, ns, w.block_off, w.diag_shift, w.cutoff)
    dth, _ = sharded.step_distributed(OracleShardBackend(w), *args, rank=rank, world=world)
    np.save(os.path.join(out_dir, f"dth{rank}.npy"), dth.numpy())
    if rank == 1:
        return  # leaves without taking the next step
    import time
    t0 = time.monotonic()
    try:
        sharded.step_distributed(OracleShardBackend(w), *args, rank=rank, world=world)
        outcome = "completed"
    except Exception as exc:  # the collective of the missing rank fails
        outcome = "error: " + type(exc).__name__
    with open(os.path.join(out_dir, "rank0.txt"), "w") as f:
        f.write(f"{outcome}\n{time.monotonic() - t0:.3f}\n")


def test_rank_leaving_between_steps_is_detected():
    world, name, ns = 2, "chain10_rbm", 40
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_rank_leaves, args=(world, _free_port(), name, ns, d), nprocs=world, join=True,
                           start_method="spawn")
        w = _workload(name, ns)
        r = oracle.qgt.sr_step(w.model, w.theta, w.configs, w.bond_ij, w.bond_j, w.block_off, w.diag_shift,
                               w.cutoff)
        for rank in range(world):
            dth = np.load(os.path.join(d, f"dth{rank}.npy"))
            assert np.linalg.norm(dth - r["dtheta"]) <= 1e-10 * np.linalg.norm(r["dtheta"])
        outcome, secs = open(os.path.join(d, "rank0.txt")).read().splitlines()
        assert outcome.startswith("error"), outcome
        assert float(secs) < 60.0


def test_block_owners_balance_and_cover():
    from paper_2510_08430_gb300.sharded import block_owners
    off = np.concatenate([[0], np.cumsum([6464, 4160, 4160, 4160, 65])])
    own = block_owners(off, 2)
    assert sorted(sum(own, [])) == list(range(5))
    assert own[0] == [0] or own[1] == [0]
    own4 = block_owners(off, 8)
    assert sorted(sum(own4, [])) == list(range(5)) and sum(1 for o in own4 if o) == 5
