"""Python binding of the nqs_sr C ABI: argument marshalling only.

Each function has the name of the C entry point it calls. Tensors are torch
CUDA tensors (PyTorch supplies device memory and the current stream); every
stage of the computation runs in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
from typing import Optional, Sequence

import numpy as np
import torch

from . import _lib
from ._lib import (NQS_FFNN, NQS_FP32, NQS_FP64, NQS_RBM, NQS_VIT, NQS_SPLIT_BF16, NQS_SPLIT_BF16_EXACT, NQS_SPLIT_BF16X3,
                   NQS_ELOC_DIFF32, NQS_GRAPH, NQS_PARAM_SPACE, NQS_SYNC, check, nqs_hamiltonian, nqs_model)

PRECISIONS = {"fp64": NQS_FP64, "fp32": NQS_FP32, "split_bf16": NQS_SPLIT_BF16, "split_bf16x3": NQS_SPLIT_BF16X3,
              "split_bf16_exact": NQS_SPLIT_BF16_EXACT}
SOLVERS = {"fp64": 0, "mixed": 1, "mixed_psd": 2}


def _solver(s) -> int:
    return SOLVERS[s] if isinstance(s, str) else int(s)


def _prec(p) -> int:
    return PRECISIONS[p] if isinstance(p, str) else int(p)


def _stream() -> C.c_void_p:
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t: Optional[torch.Tensor]) -> C.c_void_p:
    return C.c_void_p(0 if t is None else t.data_ptr())


def _on(*tensors):
    """Make the tensors' (common) device current for the library call, so that the
    stream, the static scratch and every pointer belong to one device."""
    devs = {t.device for t in tensors if t is not None}
    if len(devs) != 1:
        raise ValueError(f"arguments on several devices: {sorted(map(str, devs))}")
    d = devs.pop()
    if d.type != "cuda":
        raise ValueError(f"arguments must be CUDA tensors, got {d}")
    return torch.cuda.device(d)


class Model:
    """Network description: kind (0 RBM, 1 FFNN, 2 VIT), widths, and for the transformer the
    number of encoder layers (widths = (N, patch, d_model, d_mlp))."""

    def __init__(self, kind: int, widths: Sequence[int], n_enc: int = 0):
        self.kind = int(kind)
        self.widths = [int(w) for w in widths]
        self.n_enc = int(n_enc)
        self._w = (C.c_int32 * len(self.widths))(*self.widths)
        n_layers = self.n_enc if self.kind == NQS_VIT else len(self.widths) - 1
        self.c = nqs_model(self.kind, n_layers, self._w)

    @classmethod
    def from_workload(cls, m) -> "Model":
        return cls(m.kind, m.widths, getattr(m, "n_enc", 0))

    def block_offsets(self) -> np.ndarray:
        if self.kind == NQS_RBM:
            n, m = self.widths
            sz = [n, m, m * n]
        elif self.kind == NQS_VIT:
            n, p, d, h = self.widths
            t = n // p
            sz = [d * p + d] + [t * t + d * d + 2 * h * d + h + d] * self.n_enc + [d + 1]
        else:
            sz = [self.widths[i + 1] * self.widths[i] + self.widths[i + 1] for i in range(len(self.widths) - 1)]
        return np.concatenate([[0], np.cumsum(sz)]).astype(np.int64)


class Hamiltonian:
    """Bond Hamiltonian; bond arrays are copied to the device."""

    def __init__(self, n_sites: int, bond_ij, bond_j, c: float = 1.0, sign_rule: int = 1, device="cuda"):
        self.bond_ij = torch.as_tensor(np.ascontiguousarray(bond_ij, dtype=np.int32), device=device)
        self.bond_j = torch.as_tensor(np.ascontiguousarray(bond_j, dtype=np.float64), device=device)
        self.c = nqs_hamiltonian(int(n_sites), int(self.bond_ij.shape[0]), self.bond_ij.data_ptr(),
                                 self.bond_j.data_ptr(), float(c), int(sign_rule))


class Workspace:
    """Caller-owned device scratch (a torch uint8 tensor) wrapped in a library handle."""

    def __init__(self, nbytes: int = 0, device="cuda"):
        self.device = device
        self.buf = None
        self.h = C.c_void_p(0)
        self.nbytes = 0
        if nbytes:
            self.ensure(nbytes)

    def ensure(self, nbytes: int) -> "Workspace":
        if nbytes <= self.nbytes:
            return self
        lib = _lib.load()
        if self.h.value:
            lib.nqs_workspace_destroy(self.h)
        self.buf = torch.empty(int(nbytes) + 256, dtype=torch.uint8, device=self.device)
        base = (self.buf.data_ptr() + 255) // 256 * 256
        self.h = C.c_void_p(0)
        check(lib.nqs_workspace_create(C.c_void_p(base), C.c_size_t(int(nbytes)), C.byref(self.h)))
        self.nbytes = int(nbytes)
        return self

    def sync_status(self) -> None:
        check(_lib.load().nqs_sync_status(self.h, _stream()))

    def __del__(self):
        try:
            if self.h.value:
                _lib.load().nqs_workspace_destroy(self.h)
        except Exception:
            pass


def _size(fn, *args) -> int:
    out = C.c_size_t(0)
    check(fn(*args, C.byref(out)))
    return out.value


def _off(block_off) -> C.Array:
    arr = np.ascontiguousarray(block_off, dtype=np.int64)
    return (C.c_int64 * len(arr))(*arr.tolist())


def _cdt(precision: int):
    """dtype of the Jacobian O: complex64 only in fp32 mode (split modes use an FP64 Jacobian)."""
    return torch.complex64 if precision == NQS_FP32 else torch.complex128


def nqs_jacobian(model: Model, theta: torch.Tensor, configs: torch.Tensor, precision="fp64",
                 ldo: Optional[int] = None, ws: Optional[Workspace] = None, sync: bool = True):
    """(logpsi c128 [n_s], O parameter-major [n_p, ldo] c128/c64)."""
    lib = _lib.load()
    p = _prec(precision)
    ns = int(configs.shape[0])
    ldo = ns if ldo is None else int(ldo)
    n_p = int(model.block_offsets()[-1])
    ws = ws or Workspace()
    ws.ensure(_size(lib.nqs_jacobian_workspace_size, C.byref(model.c), ns, p))
    logpsi = torch.empty(ns, dtype=torch.complex128, device=configs.device)
    O = torch.empty((n_p, ldo), dtype=_cdt(p), device=configs.device)
    with _on(theta, configs):
        check(lib.nqs_jacobian(C.byref(model.c), _ptr(theta), _ptr(configs), ns, p, _ptr(logpsi), _ptr(O), ldo,
                               ws.h, _stream()))
    if sync:
        ws.sync_status()
    return logpsi, O


class NQSLogPsi(torch.autograd.Function):
    """ln psi(configs; theta) with the hand-written per-sample backward of the library:
    forward runs nqs_jacobian (ln psi and the Jacobian O in one pass); backward returns
    sum_s conj(O_sk) g_s (nqs_vjp), the gradient of a holomorphic function in PyTorch's
    conjugate-Wirtinger convention."""

    @staticmethod
    def forward(ctx, theta: torch.Tensor, model: "Model", configs: torch.Tensor, precision: str = "fp64"):
        logpsi, O = nqs_jacobian(model, theta.detach(), configs, precision)
        ctx.save_for_backward(O)
        ctx.precision = precision
        ctx.n_s = int(configs.shape[0])
        return logpsi

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        (O,) = ctx.saved_tensors
        lib = _lib.load()
        g = grad_out.to(torch.complex128).contiguous()
        out = torch.empty(O.shape[0], dtype=torch.complex128, device=O.device)
        with _on(O, g):
            check(lib.nqs_vjp(_ptr(O), int(O.shape[1]), ctx.n_s, int(O.shape[0]), _prec(ctx.precision), _ptr(g),
                              _ptr(out), _stream()))
        return out, None, None, None


def log_psi(model: "Model", theta: torch.Tensor, configs: torch.Tensor, precision: str = "fp64") -> torch.Tensor:
    """Differentiable ln psi (see NQSLogPsi)."""
    return NQSLogPsi.apply(theta, model, configs, precision)


def nqs_local_energy(model: Model, theta: torch.Tensor, configs: torch.Tensor, ham: Hamiltonian,
                     precision="fp64", ws: Optional[Workspace] = None, sync: bool = True,
                     diff32: bool = False) -> torch.Tensor:
    """E_loc c128 [n_s]; diff32: FP32 difference propagation (nqs_local_energy_ex, NQS_ELOC_DIFF32)."""
    lib = _lib.load()
    p = _prec(precision)
    ns = int(configs.shape[0])
    ws = ws or Workspace()
    ws.ensure(_size(lib.nqs_local_energy_workspace_size, C.byref(model.c), ns, C.byref(ham.c), p))
    eloc = torch.empty(ns, dtype=torch.complex128, device=configs.device)
    with _on(theta, configs, ham.bond_ij):
        check(lib.nqs_local_energy_ex(C.byref(model.c), _ptr(theta), _ptr(configs), ns, C.byref(ham.c), p,
                                      NQS_ELOC_DIFF32 if diff32 else 0, _ptr(eloc), ws.h, _stream()))
    if sync:
        ws.sync_status()
    return eloc


def nqs_connections(configs: torch.Tensor, ham: Hamiltonian, ws: Optional[Workspace] = None):
    """(count int32 [n_s], offset int64 [n_s+1], bond int32 [n_conn])."""
    lib = _lib.load()
    ns = int(configs.shape[0])
    maxc = ns * int(ham.c.n_bonds)
    ws = ws or Workspace()
    ws.ensure(4 * maxc + 1024)
    cnt = torch.empty(ns, dtype=torch.int32, device=configs.device)
    off = torch.empty(ns + 1, dtype=torch.int64, device=configs.device)
    bond = torch.empty(max(maxc, 1), dtype=torch.int32, device=configs.device)
    n = C.c_int64(0)
    with _on(configs, ham.bond_ij):
        check(lib.nqs_connections(_ptr(configs), ns, C.byref(ham.c), _ptr(cnt), _ptr(off), _ptr(bond), maxc,
                                  C.byref(n), ws.h, _stream()))
    ws.sync_status()
    return cnt, off, bond[: n.value]


def qgt_block_build(O: torch.Tensor, n_s: int, block_off, eloc: torch.Tensor, precision="fp64",
                    w: Optional[torch.Tensor] = None, ws: Optional[Workspace] = None, sync: bool = True):
    """(S_packed c128, F c128 [n_p], Omean c128 [n_p], Emean c128 [1]). O is overwritten
    with the centred dO in fp64/fp32 modes."""
    lib = _lib.load()
    p = _prec(precision)
    off = _off(block_off)
    nb = len(off) - 1
    n_p = int(block_off[-1])
    ldo = int(O.shape[1])
    ws = ws or Workspace()
    ws.ensure(_size(lib.qgt_block_build_workspace_size, n_s, n_p, off, nb, p))
    dev = O.device
    S = torch.zeros(int(lib.qgt_packed_size(off, nb)), dtype=torch.complex128, device=dev)
    F = torch.empty(n_p, dtype=torch.complex128, device=dev)
    Om = torch.empty(n_p, dtype=torch.complex128, device=dev)
    Em = torch.empty(1, dtype=torch.complex128, device=dev)
    with _on(O, eloc, w):
        check(lib.qgt_block_build(_ptr(O), ldo, n_s, n_p, _ptr(w), off, nb, _ptr(eloc), p, _ptr(S), _ptr(F),
                                  _ptr(Om), _ptr(Em), ws.h, _stream()))
    if sync:
        ws.sync_status()
    return S, F, Om, Em


def qgt_block_build_static(O: torch.Tensor, n_s: int, block_off, eloc: torch.Tensor, precision="fp64",
                           w: Optional[torch.Tensor] = None):
    """qgt_block_build without a workspace (fp64/fp32, n_s <= NQS_STATIC_MAX_SAMPLES);
    same results. The outputs are allocated here by torch; the library call allocates nothing."""
    lib = _lib.load()
    p = _prec(precision)
    off = _off(block_off)
    nb = len(off) - 1
    n_p = int(block_off[-1])
    dev = O.device
    S = torch.zeros(int(lib.qgt_packed_size(off, nb)), dtype=torch.complex128, device=dev)
    F = torch.empty(n_p, dtype=torch.complex128, device=dev)
    Om = torch.empty(n_p, dtype=torch.complex128, device=dev)
    Em = torch.empty(1, dtype=torch.complex128, device=dev)
    with _on(O, eloc, w):
        check(lib.qgt_block_build_static(_ptr(O), int(O.shape[1]), n_s, n_p, _ptr(w), off, nb, _ptr(eloc), p,
                                         _ptr(S), _ptr(F), _ptr(Om), _ptr(Em), _stream()))
    return S, F, Om, Em


def qgt_block_solve(S: torch.Tensor, block_off, F: torch.Tensor, diag_shift: float, cutoff: float,
                    cutoff_mode: int = 0, eta: float = 1.0, want_evals: bool = True, solver="fp64",
                    ws: Optional[Workspace] = None, sync: bool = True):
    """(dtheta c128 [n_p], evals f64 [n_p] or None, n_kept int32 [n_blocks]). S is overwritten."""
    lib = _lib.load()
    off = _off(block_off)
    nb = len(off) - 1
    n_p = int(block_off[-1])
    ws = ws or Workspace()
    ws.ensure(_size(lib.qgt_block_solve_workspace_size, off, nb))
    dev = S.device
    dth = torch.empty(n_p, dtype=torch.complex128, device=dev)
    ev = torch.empty(n_p, dtype=torch.float64, device=dev) if want_evals else None
    nk = torch.empty(nb, dtype=torch.int32, device=dev)
    with _on(S, F):
        check(lib.qgt_block_solve(_ptr(S), off, nb, _ptr(F), float(diag_shift), float(cutoff), int(cutoff_mode),
                                  float(eta), _solver(solver), _ptr(dth), _ptr(ev), _ptr(nk), ws.h, _stream()))
    if sync:
        ws.sync_status()
    return dth, ev, nk


class SRStep:
    """A prepared block-layer SR step: sizes the workspace once, then runs
    ``sr_step`` on new (theta, configs) of the same shape."""

    def __init__(self, model: Model, n_s: int, ham: Hamiltonian, block_off, precision="split_bf16x3",
                 diag_shift: float = 1e-3, cutoff: float = 1e-10, cutoff_mode: int = 0, eta: float = 1.0,
                 want_evals: bool = False, solver="fp64", device="cuda", param_space: bool = False,
                 eloc_diff32: bool = False):
        lib = _lib.load()
        self.model, self.ham = model, ham
        self.n_s = int(n_s)
        self.p = _prec(precision)
        self.solver = _solver(solver)
        self.off = _off(block_off)
        self.nb = len(self.off) - 1
        self.n_p = int(block_off[-1])
        self.shift, self.cutoff, self.mode, self.eta = float(diag_shift), float(cutoff), int(cutoff_mode), float(eta)
        # blocks wider than n_s are solved in sample space unless param_space is set
        self.flags = (NQS_PARAM_SPACE if param_space else 0) | (NQS_ELOC_DIFF32 if eloc_diff32 else 0)
        self.ws = Workspace(_size(lib.sr_step_workspace_size2, C.byref(model.c), self.n_s, C.byref(ham.c), self.off,
                                  self.nb, self.shift, self.p, self.solver, self.flags), device=device)
        self.dtheta = torch.empty(self.n_p, dtype=torch.complex128, device=device)
        self.emean = torch.empty(1, dtype=torch.complex128, device=device)
        self.evals = torch.empty(self.n_p, dtype=torch.float64, device=device) if want_evals else None
        self.n_kept = torch.empty(self.nb, dtype=torch.int32, device=device)

    STAGES = ("jacobian", "local_energy", "centring_force", "gram", "factorization", "solve")

    def enable_stage_timing(self, on: bool = True) -> None:
        check(_lib.load().nqs_stage_timing(self.ws.h, 1 if on else 0))

    def stage_times(self) -> dict:
        """Milliseconds per stage of the last sr_step with timing enabled."""
        ms = (C.c_double * 8)()
        n = C.c_int32(0)
        check(_lib.load().nqs_stage_times(self.ws.h, ms, 8, C.byref(n)))
        return {self.STAGES[i]: ms[i] for i in range(n.value)}

    def __call__(self, theta: torch.Tensor, configs: torch.Tensor, sync: bool = False, _flags: int = 0):
        lib = _lib.load()
        with _on(theta, configs, self.dtheta):
            check(lib.sr_step(C.byref(self.model.c), _ptr(theta), _ptr(configs), self.n_s, C.byref(self.ham.c),
                              self.off, self.nb, self.shift, self.cutoff, self.mode, self.eta, self.p, self.solver,
                              _ptr(self.dtheta), _ptr(self.emean), _ptr(self.evals), _ptr(self.n_kept),
                              (NQS_SYNC if sync else 0) | self.flags | _flags, self.ws.h, _stream()))
        return self.dtheta, self.emean

    def capture(self, theta: torch.Tensor, configs: torch.Tensor) -> "torch.cuda.CUDAGraph":
        """Capture one step into a CUDA graph over static copies of (theta, configs); replay()
        then runs it for new inputs of the same shape. One uncaptured step runs first."""
        self._g_theta = theta.detach().clone()
        self._g_configs = configs.detach().clone()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            self(self._g_theta, self._g_configs)
        torch.cuda.current_stream().wait_stream(side)
        self.ws.sync_status()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, capture_error_mode="thread_local"):
            self(self._g_theta, self._g_configs, _flags=NQS_GRAPH)
        self._graph = g
        return g

    def replay(self, theta: Optional[torch.Tensor] = None, configs: Optional[torch.Tensor] = None):
        """Run the captured step (copying new inputs into its static buffers first)."""
        if theta is not None:
            self._g_theta.copy_(theta, non_blocking=True)
        if configs is not None:
            self._g_configs.copy_(configs, non_blocking=True)
        self._graph.replay()
        return self.dtheta, self.emean


def sr_step(model: Model, theta: torch.Tensor, configs: torch.Tensor, ham: Hamiltonian, block_off,
            diag_shift: float, cutoff: float, eta: float = 1.0, precision="fp64", cutoff_mode: int = 0,
            want_evals: bool = True, solver="fp64", param_space: bool = False, eloc_diff32: bool = False):
    """One whole block-layer SR step: (dtheta, Emean, evals, n_kept). eloc_diff32: FFNN local
    energies by FP32 difference propagation (NQS_ELOC_DIFF32) instead of FP64-class arithmetic."""
    st = SRStep(model, int(configs.shape[0]), ham, block_off, precision, diag_shift, cutoff, cutoff_mode, eta,
                want_evals, solver, device=configs.device, param_space=param_space, eloc_diff32=eloc_diff32)
    st(theta, configs, sync=True)
    return st.dtheta, st.emean, st.evals, st.n_kept


def _batch_args(models, n_s, hams, block_offs):
    n = len(models)
    mods = (nqs_model * n)(*[m.c for m in models])
    hs = (nqs_hamiltonian * n)(*[h.c for h in hams])
    ns = (C.c_int64 * n)(*[int(v) for v in n_s])
    nbs = (C.c_int32 * n)(*[len(o) - 1 for o in block_offs])
    offs = np.concatenate([np.asarray(o, dtype=np.int64) for o in block_offs])
    off_c = (C.c_int64 * len(offs))(*offs.tolist())
    return n, mods, hs, ns, nbs, off_c


def sr_step_batched_workspace_size(models, n_s, hams, block_offs, precision="split_bf16_exact") -> int:
    """Bytes of workspace one sr_step_batched call over these instances needs."""
    n, mods, hs, ns, nbs, off_c = _batch_args(models, n_s, hams, block_offs)
    sz = C.c_size_t(0)
    check(_lib.load().sr_step_batched_workspace_size(n, mods, ns, hs, off_c, nbs, _prec(precision), C.byref(sz)))
    return int(sz.value)


def plan_batch_chunks(models, n_s, hams, block_offs, max_bytes: int, precision="split_bf16_exact"):
    """Memory plan of a batch that does not fit at once: consecutive groups of instances, each
    as large as possible with its sr_step_batched workspace within max_bytes. Returns (list of
    index lists, the largest group's workspace bytes); a single instance above max_bytes is an
    error."""
    groups, cur, worst = [], [], 0
    for i in range(len(models)):
        trial = cur + [i]
        need = sr_step_batched_workspace_size([models[k] for k in trial], [n_s[k] for k in trial],
                                              [hams[k] for k in trial], [block_offs[k] for k in trial], precision)
        if need <= max_bytes:
            cur, last = trial, need
            continue
        if not cur:
            raise ValueError(f"instance {i} alone needs {need} bytes > {max_bytes}")
        groups.append(cur)
        worst = max(worst, last)
        cur = [i]
        last = sr_step_batched_workspace_size([models[i]], [n_s[i]], [hams[i]], [block_offs[i]], precision)
        if last > max_bytes:
            raise ValueError(f"instance {i} alone needs {last} bytes > {max_bytes}")
    if cur:
        groups.append(cur)
        worst = max(worst, last)
    return groups, worst


def sr_step_batched(models, thetas, configs, hams, block_offs, diag_shift: float, cutoff: float, eta: float = 1.0,
                    precision="split_bf16", cutoff_mode: int = 0, solver="mixed", want_evals: bool = False,
                    eloc_diff32: bool = False, ws: Optional[Workspace] = None):
    """Several independent SR steps in one call (one grouped Gram and one eigensolver launch).
    Lists of per-instance Model, theta (c128 device), configs (int8 device), Hamiltonian and block
    offsets. Returns (list of dtheta, Emean c128 [n_inst], evals or None, n_kept int32 [sum blocks]).
    ws: a workspace to (grow and) reuse across calls."""
    lib = _lib.load()
    n, mods, hs, ns, nbs, off_c = _batch_args(models, [int(x.shape[0]) for x in configs], hams, block_offs)
    p = _prec(precision)
    sz = C.c_size_t(0)
    check(lib.sr_step_batched_workspace_size(n, mods, ns, hs, off_c, nbs, p, C.byref(sz)))
    dev = thetas[0].device
    if ws is None:
        ws = Workspace(int(sz.value), device=dev)
    else:
        ws.ensure(int(sz.value))
    th = torch.cat([t.reshape(-1) for t in thetas]).contiguous()
    xc = torch.cat([x.reshape(-1) for x in configs]).contiguous()
    np_tot = int(th.numel())
    dth = torch.empty(np_tot, dtype=torch.complex128, device=dev)
    em = torch.empty(n, dtype=torch.complex128, device=dev)
    ev = torch.empty(np_tot, dtype=torch.float64, device=dev) if want_evals else None
    nk = torch.empty(int(sum(len(o) - 1 for o in block_offs)), dtype=torch.int32, device=dev)
    with _on(th, xc):
        check(lib.sr_step_batched(n, mods, _ptr(th), _ptr(xc), ns, hs, off_c, nbs, float(diag_shift), float(cutoff),
                                  int(cutoff_mode), float(eta), p, _solver(solver), _ptr(dth), _ptr(em), _ptr(ev),
                                  _ptr(nk), NQS_SYNC | (NQS_ELOC_DIFF32 if eloc_diff32 else 0), ws.h, _stream()))
    sizes = [int(o[-1]) for o in block_offs]
    return list(torch.split(dth, sizes)), em, ev, nk


def ntk_solve(O: torch.Tensor, n_s: int, eloc: torch.Tensor, diag_shift: float, cutoff: float = 1e-10,
              eta: float = 1.0, precision="fp64"):
    """Sample-space (NTK) form of the full-QGT update from a c128 Jacobian O [n_p, ldo]
    (overwritten with dO). Returns (dtheta c128 [n_p], Emean c128 [1])."""
    lib = _lib.load()
    p = _prec(precision)
    n_p = int(O.shape[0])
    ws = Workspace(_size(lib.ntk_solve_workspace_size, n_s, n_p, p), device=O.device)
    dth = torch.empty(n_p, dtype=torch.complex128, device=O.device)
    em = torch.empty(1, dtype=torch.complex128, device=O.device)
    with _on(O, eloc):
        check(lib.ntk_solve(_ptr(O), int(O.shape[1]), n_s, n_p, _ptr(eloc), float(diag_shift), float(cutoff),
                            float(eta), p, _ptr(dth), _ptr(em), ws.h, _stream()))
    ws.sync_status()
    return dth, em


def born_weights(logpsi: torch.Tensor) -> torch.Tensor:
    """|psi|^2 / Z over the given configurations (nqs_born_weights), float64 [n]."""
    w = torch.empty(int(logpsi.shape[0]), dtype=torch.float64, device=logpsi.device)
    with _on(logpsi):
        check(_lib.load().nqs_born_weights(_ptr(logpsi), int(logpsi.shape[0]), _ptr(w), _stream()))
    return w


def qgt_inverse_diagnostics(S_a: torch.Tensor, block_off_a, S_b: torch.Tensor, diag_shift: float, cutoff: float,
                            cutoff_mode: int = 0) -> dict:
    """Eq. 4 diagnostics of A = pinv(blocks of S_a + shift I) against B = pinv(S_b + shift I)
    (S_a, S_b: n x n complex128, lower triangle used)."""
    lib = _lib.load()
    n = int(S_b.shape[-1])
    off = _off(block_off_a)
    ws = Workspace(_size(lib.qgt_inverse_diagnostics_workspace_size, n), device=S_b.device)
    out = torch.empty(5, dtype=torch.float64, device=S_b.device)
    Sa, Sb = S_a.contiguous(), S_b.contiguous()
    with _on(Sa, Sb):
        check(lib.qgt_inverse_diagnostics(_ptr(Sa), off, len(off) - 1, _ptr(Sb), n, float(diag_shift), float(cutoff),
                                          int(cutoff_mode), _ptr(out), ws.h, _stream()))
    ws.sync_status()
    v = out.cpu().tolist()
    return {"F": v[0], "eps_F": v[1], "kappa_A": v[2], "kappa_B": v[3], "r_lambda": v[4]}


def inverse_metric_study(model: Model, theta: torch.Tensor, configs: torch.Tensor, block_off, diag_shift: float,
                         cutoff: float) -> dict:
    """Eq. 4 diagnostics on a system small enough to enumerate (N <= 12 sites): B is the
    pseudo-inverse of the exact QGT (all 2^N configurations, Born weights); A that of
    (i) the block-layer QGT of the sampled QGT, (ii) the full sampled QGT, (iii) the
    block-layer QGT of the exact QGT. Every number is computed by the library."""
    n_sites = model.widths[0]
    if n_sites > 12:
        raise ValueError("enumeration limited to 12 sites")
    dev = configs.device
    idx = torch.arange(2 ** n_sites, device=dev)
    bits = (idx[:, None] >> torch.arange(n_sites - 1, -1, -1, device=dev)[None, :]) & 1
    x_all = (2 * bits - 1).to(torch.int8).contiguous()
    n_p = int(np.asarray(block_off)[-1])
    full = np.array([0, n_p], dtype=np.int64)

    def full_qgt(x, w):
        lp, O = nqs_jacobian(model, theta, x, "fp64")
        zero = torch.zeros(int(x.shape[0]), dtype=torch.complex128, device=dev)
        S, _, _, _ = qgt_block_build(O, int(x.shape[0]), full, zero, "fp64", w=w)
        return S.view(n_p, n_p), lp

    lp_all, _ = nqs_jacobian(model, theta, x_all, "fp64")
    S_exact, _ = full_qgt(x_all, born_weights(lp_all))
    S_samp, _ = full_qgt(configs, None)
    return {
        "block_sampled_vs_exact": qgt_inverse_diagnostics(S_samp, block_off, S_exact, diag_shift, cutoff),
        "full_sampled_vs_exact": qgt_inverse_diagnostics(S_samp, full, S_exact, diag_shift, cutoff),
        "block_exact_vs_exact": qgt_inverse_diagnostics(S_exact, block_off, S_exact, diag_shift, cutoff),
    }


def set_limits(max_sweeps: int = 0, wait_ns: int = 0) -> None:
    """Test hook of the failure paths (nqs_set_limits): lower the eigen-solver and refinement
    sweep limits and the device wait budget of the persistent solver kernels; 0 restores
    the defaults."""
    check(_lib.load().nqs_set_limits(int(max_sweeps), int(wait_ns)))


def metropolis(model: Model, theta: torch.Tensor, configs: torch.Tensor, uniforms: torch.Tensor,
               ws: Optional[Workspace] = None, count: bool = True) -> Optional[int]:
    """nqs_metropolis: uniforms.shape[0] exchange-move Metropolis steps on every chain (rows of
    configs, int8, updated in place). uniforms: float64 [n_steps, n_chains, 3] on the device.
    Returns the number of accepted moves (count=True; this synchronises) or None."""
    lib = _lib.load()
    n = int(configs.shape[0])
    steps = int(uniforms.shape[0])
    if tuple(uniforms.shape) != (steps, n, 3) or uniforms.dtype != torch.float64:
        raise ValueError("uniforms must be float64 [n_steps, n_chains, 3]")
    ws = ws or Workspace()
    ws.ensure(_size(lib.nqs_metropolis_workspace_size, C.byref(model.c), n))
    acc = torch.zeros(1, dtype=torch.int64, device=configs.device) if count else None
    u = uniforms.contiguous()
    with _on(theta, configs, u):
        check(lib.nqs_metropolis(C.byref(model.c), _ptr(theta), _ptr(configs), n, steps, _ptr(u), _ptr(acc), ws.h,
                                 _stream()))
    return int(acc.item()) if count else None


def theta_update(theta: torch.Tensor, dtheta: torch.Tensor) -> None:
    """theta += dtheta in place (nqs_theta_update; c128 device vectors)."""
    with _on(theta, dtheta):
        check(_lib.load().nqs_theta_update(_ptr(theta), _ptr(dtheta), int(theta.numel()), _stream()))


def vmc_train(model: Model, theta: torch.Tensor, configs: torch.Tensor, ham: Hamiltonian, block_off,
              n_iter: int, n_steps: int, diag_shift: float, cutoff: float, eta: float, precision="fp64",
              solver="fp64", uniforms=None, generator: Optional[torch.Generator] = None) -> dict:
    """The VMC loop on the device: per iteration n_steps Metropolis steps of every chain
    (nqs_metropolis), one block-layer SR step on the chains' configurations (sr_step with the
    given blocks; one block [0, n_p] is the full QGT) and theta += dtheta (nqs_theta_update).
    theta (c128) and configs (int8) are updated in place. uniforms: optional list of n_iter
    float64 [n_steps, n_chains, 3] device tensors (default: drawn from `generator`). Returns
    {"energies": <E> per iteration (c128, CPU), "accepted": accepted moves per iteration}."""
    n = int(configs.shape[0])
    step = SRStep(model, n, ham, block_off, precision, diag_shift, cutoff, 0, eta, solver=solver,
                  device=configs.device)
    ws = Workspace()
    emeans = torch.empty(n_iter, dtype=torch.complex128, device=configs.device)
    accepted = torch.zeros(n_iter, dtype=torch.int64, device=configs.device)
    lib = _lib.load()
    ws.ensure(_size(lib.nqs_metropolis_workspace_size, C.byref(model.c), n))
    for it in range(n_iter):
        u = uniforms[it] if uniforms is not None else torch.rand(
            (n_steps, n, 3), dtype=torch.float64, device=configs.device, generator=generator)
        u = u.contiguous()
        acc = accepted[it:it + 1]
        with _on(theta, configs, u):
            check(lib.nqs_metropolis(C.byref(model.c), _ptr(theta), _ptr(configs), n, int(u.shape[0]), _ptr(u),
                                     _ptr(acc), ws.h, _stream()))
        dth, em = step(theta, configs)
        emeans[it:it + 1].copy_(em)
        theta_update(theta, dth)
    step.ws.sync_status()
    ws.sync_status()
    return {"energies": emeans.cpu().numpy(), "accepted": accepted.cpu().numpy()}


def set_eloc_fallback_all(on: bool) -> None:
    """Test hook (nqs_set_eloc_fallback_all): every connection of the FP32 difference-propagation
    local energies goes to the FP64-class kernel that otherwise takes only the connections FP32
    cannot follow."""
    check(_lib.load().nqs_set_eloc_fallback_all(1 if on else 0))


def launch_count() -> int:
    """Kernels launched by libnqs_sr in this process."""
    return int(_lib.load().nqs_launch_count())


def version() -> str:
    return _lib.load().nqs_version().decode()
