#!/usr/bin/env python
"""Benchmark of one block-layer stochastic-reconfiguration step on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

A step is the whole hot path: Jacobian of ln psi, local energies, centring and
force, the per-layer QGT blocks (tcgen05 BF16 hi+lo Gram) and the per-block
FP64 shifted pseudo-inverse solve, from (theta, configs) to (dtheta, <E>).
Default workload: FFNN 100-64-64-64-64-1 on the periodic 10x10 J1-J2 lattice
(J2/J1 = 0.5), 16384 zero-magnetisation samples, blocks 6464/4160/4160/4160/65,
seeded synthetic inputs. Prints one JSON line (rank 0).

Timing: W untimed warm-up steps; K timed steps bracketed by a barrier and
device synchronisation, each step timed with CUDA events on the launching
stream, L2 flushed (256 MB write) between steps; the maximum over ranks is
reported. With N > 1 every rank runs its own independent replica of the
workload (no data-path collective; weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "block-SR steps/sec and Gram TFLOP/s (% of peak) at δθ rel err ≤1e-6 vs FP64"
WORKLOAD = "j1j2_10x10_ffnn5"
W_DEFAULT_NS = {"j1j2_6x6_ffnn": 4096, "j1j2_10x10_ffnn5": 16384}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--samples", type=int, default=None, help="override N_s (profiling of small cases)")
    ap.add_argument("--solver", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


SOLVER_DESC = {"fp64": "FP64 Householder eigensolver",
               "mixed": "FP32 Householder reduction + FP64-residual refinement (PSD certificate, FP64 fallback)"}


def workload_desc(w, solver="mixed") -> dict:
    import numpy as np
    return {
        "workload": f"{w.name}: widths {[int(v) for v in w.model.widths]}, {int(w.bond_ij.shape[0])} bonds, "
                    f"N_s={int(w.n_samples)}, blocks {[int(v) for v in np.diff(w.block_off)]}, {w.precision} Gram, "
                    f"{SOLVER_DESC[solver]}",
        "solver": solver,
        "n_s": int(w.n_samples),
        "n_p": int(w.model.n_params),
        "blocks": [int(v) for v in np.diff(w.block_off)],
        "precision": w.precision,
        "diag_shift": w.diag_shift,
        "cutoff": w.cutoff,
        "l2": "flushed between timed steps (256 MB write); each step also streams > 2 GB",
    }


def dtype_of(prec: str) -> str:
    return {"fp64": "f64", "fp32": "f32+f64", "split_bf16": "bf16 hi+lo (3 products, f32 acc)+f32+f64",
            "split_bf16x3": "bf16 hi+mid+lo (6 products, f32 acc)+f32+f64",
            "split_bf16_exact": "bf16 x5 grouped error-free split (15 products, f32 TMEM acc, double-float sums)"
                                "+f32+f64"}[prec]


# ------------------------------------------------------------------ counts
def gram_flops(w) -> tuple:
    import numpy as np
    nb = np.diff(w.block_off).astype(np.float64)
    ns = float(w.n_samples)
    alg = float(np.sum(4.0 * nb * (nb + 1.0) * ns))  # unique lower triangle, 8 flops per complex MAC
    full = float(np.sum(8.0 * nb * nb * ns))
    tiles = np.ceil(2 * nb / 128.0)
    kpad = np.ceil(ns / 64.0) * 64.0
    nprod = {"split_bf16": 3, "split_bf16x3": 6, "split_bf16_exact": 15}.get(w.precision, 1)
    issued = float(np.sum(tiles * (tiles + 1) / 2 * nprod * 2 * 128 * 128 * kpad))
    return alg, full, issued


def trd_bytes(w, solver: str) -> float:
    """Algorithmic DRAM bytes of one launch of the (unblocked, fused) Householder reduction
    of all blocks: for every column, the lower triangle (diagonal included) of the trailing
    m x m matrix is read once (Hermitian matvec) and written once (rank-2 update),
    m = n_b - 1 .. 1, i.e. 2 * esize * (n_b - 1) n_b (n_b + 1) / 6 bytes per block; esize is
    8 (complex64, mixed solver) or 16 (complex128, FP64 solver)."""
    import numpy as np
    nb = np.diff(w.block_off).astype(np.float64)
    es = 8.0 if solver == "mixed" else 16.0
    return float(np.sum(2.0 * es * (nb - 1.0) * nb * (nb + 1.0) / 6.0))


def trd_traffic(w, solver: str):
    """DRAM bytes per launch of the reduction kernel from the committed ncu summary, or None
    when the summary is missing, is for another workload/solver, or the kernel source has
    changed since it was taken (sha256 of eigh_persist.cu recorded in the summary)."""
    import hashlib
    import numpy as np
    path = os.path.join(ROOT, "profiles", f"trd_persist_{w.name}.md")
    src = os.path.join(ROOT, "paper_2510_08430_gb300", "csrc", "eigh_persist.cu")
    if not os.path.exists(path) or not os.path.exists(src):
        return None
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    rec = {}
    for line in open(path):
        if line.startswith("- ") and ": " in line:
            k, v = line[2:].split(": ", 1)
            rec[k.strip()] = v.strip().strip("`")
    blocks = ",".join(str(int(v)) for v in np.diff(w.block_off))
    if rec.get("source_sha256") != sha or rec.get("solver") != solver or rec.get("blocks") != blocks:
        return None  # the reduction's traffic depends on the blocks only, not on N_s
    try:
        return float(rec["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


# ------------------------------------------------------------------ clocks
class Clocks:
    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(gpu_index)], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ CPU oracle (bounded sample)
def oracle_sample(w, n_sample: int = 1024, eig_n: int = 2048) -> dict:
    """Time the FP64 oracle on a bounded sample of the workload and extrapolate one step.

    Stages linear in N_s (Jacobian, E_loc, centring, force, block Gram) run on
    the first n_sample samples and scale by N_s / n_sample; the per-block eigh +
    pseudo-inverse runs on one eig_n x eig_n Hermitian block and scales by
    sum_b n_b^3 / eig_n^3.
    """
    import numpy as np
    import oracle
    import workloads as W
    ws = W.make_workload(w.name, n_sample)
    t0 = time.perf_counter()
    lp, O = oracle.nqs.jacobian(ws.model, ws.theta, ws.configs)
    el = oracle.hamiltonian.local_energy(ws.model, ws.theta, ws.configs, ws.bond_ij, ws.bond_j, ws.c, ws.sign_rule)
    _, _, dO, e = oracle.qgt.center(O, el)
    F = oracle.qgt.force(dO, e)
    S = oracle.qgt.block_qgt(dO, ws.block_off)
    t_lin = time.perf_counter() - t0
    rng = np.random.default_rng(0)
    X = rng.normal(size=(eig_n, eig_n)) + 1j * rng.normal(size=(eig_n, eig_n))
    Sb = X @ np.conj(X).T / eig_n
    t1 = time.perf_counter()
    oracle.qgt.pinv_solve(Sb, F[:eig_n] if F.shape[0] >= eig_n else np.ones(eig_n, complex), w.diag_shift,
                          w.cutoff)
    t_eig = time.perf_counter() - t1
    nb = np.diff(w.block_off).astype(np.float64)
    est = t_lin * w.n_samples / n_sample + t_eig * float(np.sum(nb ** 3)) / eig_n ** 3
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count()
    return {"seconds_per_step": est, "measured_seconds": t_lin + t_eig, "cores": cores,
            "sample": (f"oracle on {n_sample} of {w.n_samples} samples (Jacobian, E_loc, centring, force, "
                       f"block Gram; scaled x{w.n_samples / n_sample:g}) plus one {eig_n}x{eig_n} eigh+pinv "
                       f"(scaled by sum n_b^3/{eig_n}^3); NumPy/LAPACK threads = all cores")}


# ------------------------------------------------------------------ measured peaks
def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return {"hbm_gbs": d.get("hbm_gbs"), "bf16_tflops": d.get("bf16_tflops"),
                "bf16_tflops_sustained": d.get("bf16_tflops_sustained"), "source": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "source": "fallback"}


# ------------------------------------------------------------------ same-GPU comparisons
def _timed_step(torch, step, theta, x):
    step(theta, x)  # warm
    torch.cuda.synchronize()
    s = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    s.record()
    d, _ = step(theta, x)
    e.record()
    e.synchronize()
    return s.elapsed_time(e) / 1e3, d.cpu().numpy()


def compare_steps(nq, torch, np, w, model, ham, theta, x, dth, solver) -> dict:
    """The plain FP64 and FP32 GPU steps and the cheaper split variants on the same GPU and
    inputs, each with its dtheta error against the FP64 GPU step and against the stored FP64
    oracle result of this workload (tests/golden, written from the oracle alone)."""
    out = {}
    gold = os.path.join(ROOT, "tests", "golden", f"oracle_{w.name}.npz")
    ref = np.load(gold)["dtheta"] if os.path.exists(gold) and w.n_samples == W_DEFAULT_NS.get(w.name) else None

    def err(a, b):
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))

    st = nq.SRStep(model, w.n_samples, ham, w.block_off, "fp64", w.diag_shift, w.cutoff, solver="fp64")
    t64, d64 = _timed_step(torch, st, theta, x)
    del st
    out["fp64_fp64solve"] = {"seconds": t64, "dtheta_rel_err_vs_oracle": err(d64, ref) if ref is not None else None}
    out[f"{w.precision}_{solver}solve (timed line)"] = {
        "dtheta_rel_err_vs_fp64_gpu": err(dth, d64),
        "dtheta_rel_err_vs_oracle": err(dth, ref) if ref is not None else None}
    # the full QGT (one block of all n_p parameters; the paper's comparison) on the same inputs
    full_off = np.array([0, int(w.block_off[-1])], dtype=np.int64)
    stf = nq.SRStep(model, w.n_samples, ham, full_off, w.precision, w.diag_shift, w.cutoff, solver=solver)
    tf, dfull = _timed_step(torch, stf, theta, x)
    del stf
    out[f"full_qgt_{w.precision}_{solver}solve"] = {
        "seconds": tf, "blocks": [int(w.block_off[-1])],
        "dtheta_rel_diff_vs_block": err(dfull, dth),
        "note": "full-QGT update: a different method; it is not expected to equal the block-layer update"}
    # the sample-space (NTK) form of the full-QGT update (FP32 N_s x N_s Gram, mixed solver),
    # timed from the FP64 Jacobian and local energies
    try:
        _, O64 = nq.nqs_jacobian(model, theta, x, "fp64")
        el64 = nq.nqs_local_energy(model, theta, x, ham, "fp64")
        torch.cuda.synchronize()
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record()
        dntk, _ = nq.ntk_solve(O64, w.n_samples, el64, w.diag_shift, w.cutoff, 1.0, "fp32")
        e.record()
        e.synchronize()
        dntk = dntk.cpu().numpy()
        del O64, el64
        out["ntk_fp32gram_mixedsolve"] = {
            "seconds": s.elapsed_time(e) / 1e3, "what": "centring, N_s x N_s Gram, solve, back-projection",
            "dtheta_rel_diff_vs_full_qgt": err(dntk, dfull)}
    except Exception as exc:
        out["ntk_fp32gram_mixedsolve"] = {"unavailable": str(exc)[:200]}
    for prec in ("fp32", "split_bf16", "split_bf16x3"):
        if prec == w.precision:
            continue
        st = nq.SRStep(model, w.n_samples, ham, w.block_off, prec, w.diag_shift, w.cutoff, solver=solver)
        t, d = _timed_step(torch, st, theta, x)
        del st
        out[f"{prec}_{solver}solve"] = {"seconds": t, "dtheta_rel_err_vs_fp64_gpu": err(d, d64),
                                         "dtheta_rel_err_vs_oracle": err(d, ref) if ref is not None else None}
    return out


# ------------------------------------------------------------------ reference arm
def run_reference(args, rank: int, world: int) -> None:
    import workloads as W
    if rank != 0:
        return
    w = W.make_workload(args.workload, args.samples)
    for _ in range(args.warmup):
        oracle_sample(w)
    secs = []
    info = None
    for _ in range(args.steps):
        info = oracle_sample(w)
        secs.append(info["seconds_per_step"])
    t = sum(secs)
    value = args.steps / t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_desc(w, "mixed"),
        "reference_impl": "FP64 NumPy oracle (same workload and metric; FP64 Jacobian, E_loc, Gram and LAPACK eigh)",
        "cpu_baseline": {"value": value, "unit": "steps/s", "cores": info["cores"], "kind": "oracle",
                         "sample": info["sample"]},
        "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm
def run_ours(args, rank: int, world: int, local_rank: int) -> None:
    import numpy as np
    import torch
    import torch.distributed as dist

    import __graft_entry__
    __graft_entry__.build()
    import paper_2510_08430_gb300 as nq
    import workloads as W

    torch.cuda.set_device(local_rank)
    w = W.make_workload(args.workload, args.samples)
    model = nq.Model.from_workload(w.model)
    theta = torch.as_tensor(w.theta, device="cuda")
    x = torch.as_tensor(w.configs, device="cuda")
    ham = nq.Hamiltonian(w.model.n_sites, w.bond_ij, w.bond_j, w.c, w.sign_rule)
    step = nq.SRStep(model, w.n_samples, ham, w.block_off, w.precision, w.diag_shift, w.cutoff, solver=args.solver)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step(theta, x)
    step.ws.sync_status()
    step.enable_stage_timing(True)
    barrier()
    clocks = Clocks(local_rank)
    l0 = nq.launch_count()
    per_step, stages = [], []
    for _ in range(args.steps):
        flush.fill_(1.0)
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record()
        step(theta, x)
        e.record()
        e.synchronize()
        per_step.append(s.elapsed_time(e) / 1e3)
        stages.append(step.stage_times())
    barrier()
    launches = nq.launch_count() - l0
    clk = clocks.stop()
    step.ws.sync_status()
    step.enable_stage_timing(False)
    total = torch.tensor([sum(per_step)], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(total, op=dist.ReduceOp.MAX)
    t_max = float(total.item())
    value = world * args.steps / t_max

    # end to end through the public API with host buffers (pinned), copies timed
    th_h = torch.as_tensor(w.theta).pin_memory()
    x_h = torch.as_tensor(w.configs).pin_memory()
    out_h = torch.empty(w.model.n_params, dtype=torch.complex128).pin_memory()
    em_h = torch.empty(1, dtype=torch.complex128).pin_memory()
    th_d = torch.empty_like(theta)
    x_d = torch.empty_like(x)
    e2e_t = []
    barrier()
    for _ in range(args.steps):
        flush.fill_(1.0)
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record()
        th_d.copy_(th_h, non_blocking=True)
        x_d.copy_(x_h, non_blocking=True)
        dth, em = step(th_d, x_d)
        out_h.copy_(dth, non_blocking=True)
        em_h.copy_(em, non_blocking=True)
        e.record()
        e.synchronize()
        e2e_t.append(s.elapsed_time(e) / 1e3)
    barrier()
    e2e_total = torch.tensor([sum(e2e_t)], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(e2e_total, op=dist.ReduceOp.MAX)
    e2e_value = world * args.steps / float(e2e_total.item())
    h2d = int(th_h.numel() * th_h.element_size() + x_h.numel() * x_h.element_size())
    d2h = int(out_h.numel() * out_h.element_size() + em_h.numel() * em_h.element_size())
    dth_split = out_h.numpy().copy()

    if rank != 0:
        return
    peaks = measured_peaks()
    st_mean = {k: statistics.mean(d[k] for d in stages) for k in stages[0]}
    alg, full, issued = gram_flops(w)
    gram_s = st_mean["gram"] / 1e3
    trd_s = st_mean["tridiagonal_reduction"] / 1e3
    hbm = peaks["hbm_gbs"]
    trd_alg = trd_bytes(w, args.solver)
    trd_gbs = trd_alg / trd_s / 1e9
    traffic = trd_traffic(w, args.solver)
    bf16_peak = peaks["bf16_tflops"]
    gram_tf = alg / gram_s / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": dtype_of(w.precision), "data": "synthetic",
        "config": dict(workload_desc(w, args.solver), parallelism=("replicas" if world > 1 else "single")),
        "stage_ms": st_mean,
        "roofline": {"kernel": ("trd_persist_kernel<float>" if args.solver == "mixed" else
                                "trd_persist_kernel<double>") + " (Householder reduction of all blocks, one launch)",
                     "bound": "hbm", "achieved": trd_gbs, "peak": hbm, "unit": "GB/s", "frac": trd_gbs / hbm,
                     "traffic": traffic,
                     "peak_source": f"hbm_gbs, {peaks['source']}",
                     "algorithmic": "per block 2 * esize * (n_b-1) n_b (n_b+1) / 6 bytes (trailing lower triangle "
                                    "read + written once per column)",
                     "algorithmic_bytes": trd_alg, "ms_per_launch": st_mean["tridiagonal_reduction"]},
        "roofline_gram": {"kernel": f"gram_tc_kernel (tcgen05, {w.precision})", "bound": "tensor",
                          "achieved": gram_tf, "peak": bf16_peak, "unit": "TFLOP/s", "frac": gram_tf / bf16_peak,
                          "peak_source": f"bf16_tflops burst, {peaks['source']}",
                          "issued_tflops": issued / gram_s / 1e12,
                          "algorithmic": "sum_b 4 n_b (n_b+1) N_s flops (unique lower triangle)",
                          "full_count_tflops": full / gram_s / 1e12},
        "clocks": clk,
        "e2e": {"value": e2e_value, "unit": "steps/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
    }
    # the same step captured as one CUDA graph and replayed (launch overhead removed)
    try:
        step.capture(theta, x)
        for _ in range(2):
            step.replay()
        torch.cuda.synchronize()
        gt = []
        for _ in range(args.steps):
            flush.fill_(1.0)
            s = torch.cuda.Event(enable_timing=True)
            e = torch.cuda.Event(enable_timing=True)
            s.record()
            step.replay()
            e.record()
            e.synchronize()
            gt.append(s.elapsed_time(e) / 1e3)
        step.ws.sync_status()
        line["graph_replay"] = {"value": args.steps / sum(gt), "unit": "steps/s",
                                "ms_per_step": 1e3 * sum(gt) / args.steps}
    except Exception as exc:  # capture not possible here: report why, keep the direct timing
        line["graph_replay"] = {"unavailable": str(exc)[:200]}
    if world == 1 and not args.no_fp64_compare:
        line["comparisons"] = compare_steps(nq, torch, np, w, model, ham, theta, x, dth_split, args.solver)
    if world == 1 and not args.no_cpu_baseline:
        info = oracle_sample(w)
        line["cpu_baseline"] = {"value": 1.0 / info["seconds_per_step"], "unit": "steps/s", "cores": info["cores"],
                                "kind": "oracle", "sample": info["sample"]}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
