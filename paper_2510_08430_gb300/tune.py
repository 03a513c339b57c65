"""Autotuner of the tensor-core Gram's tile order.

The persistent tcgen05 Gram takes the 128 x 128 tiles of a block in square groups of G x G
tiles so that the CTAs running at the same time share row and column panels in L2 while
they stream the samples (see nqs_set_gram_tuning in include/nqs_sr.h). The best G depends on
the block sizes and the sample count. For every shape bucket (largest block, sample count,
each rounded up to a power of two) this module times the library's block Gram for each
candidate G on the current GPU with CUDA events, keeps the fastest and installs the table in
the library. Results are cached as JSON keyed by the GPU name, so a later process installs
them without timing. The choice changes only the order of the tiles, never S.
"""
from __future__ import annotations

import ctypes as C
import json
import os
from typing import Callable, Dict, Iterable, List, Optional, Sequence, Tuple

import numpy as np

from . import _lib
from ._lib import check

CANDIDATES = (1, 2, 4, 8, 12, 16)
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "nqs_sr", "gram_tuning.json")


def bucket(max_nb: int, n_s: int) -> Tuple[int, int]:
    """(largest block, sample count), each rounded up to a power of two."""
    return 1 << max(0, int(max_nb - 1).bit_length()), 1 << max(0, int(n_s - 1).bit_length())


def install(table: Dict[Tuple[int, int], int]) -> None:
    """Install {(max_nb, max_ns): G} in the library, smallest buckets first (first match wins)."""
    keys = sorted(table, key=lambda k: (k[0], k[1]))
    n = len(keys)
    nb = (C.c_int64 * max(n, 1))(*[k[0] for k in keys])
    ns = (C.c_int64 * max(n, 1))(*[k[1] for k in keys])
    g = (C.c_int32 * max(n, 1))(*[int(table[k]) for k in keys])
    check(_lib.load().nqs_set_gram_tuning(n, nb, ns, g))


def group_edge(max_nb: int, n_s: int) -> int:
    """G the library uses for a Gram of this shape."""
    return int(_lib.load().nqs_gram_group_edge(int(max_nb), int(n_s)))


def _gpu_name() -> str:
    import torch
    return torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"


def _load_cache(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save_cache(path: str, data: dict) -> None:
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def gram_timer(block_sizes: Sequence[int], n_s: int, precision: str = "split_bf16_exact",
               reps: int = 2) -> Callable[[int], float]:
    """A timer of the library's block Gram (qgt_block_build) on synthetic centred data of this
    shape: returns f(G) -> milliseconds (median of reps, after one warm-up)."""
    import torch

    from .api import qgt_block_build
    off = np.concatenate([[0], np.cumsum(block_sizes)]).astype(np.int64)
    n_p = int(off[-1])
    gen = torch.Generator(device="cuda").manual_seed(0)
    O = torch.randn((n_p, n_s), dtype=torch.complex128, device="cuda", generator=gen)
    el = torch.randn(n_s, dtype=torch.complex128, device="cuda", generator=gen)

    def run(G: int) -> float:
        install({bucket(max(block_sizes), n_s): G})
        qgt_block_build(O, n_s, off, el, precision)  # warm-up (and O is left unchanged in split modes)
        ts = []
        for _ in range(reps):
            s = torch.cuda.Event(enable_timing=True)
            e = torch.cuda.Event(enable_timing=True)
            s.record()
            qgt_block_build(O, n_s, off, el, precision, sync=False)
            e.record()
            e.synchronize()
            ts.append(s.elapsed_time(e))
        return float(np.median(ts))

    return run


def tune(shapes: Iterable[Tuple[Sequence[int], int]], candidates: Sequence[int] = CANDIDATES,
         precision: str = "split_bf16_exact", cache_path: Optional[str] = DEFAULT_CACHE,
         timer_factory: Optional[Callable] = None, gpu: Optional[str] = None) -> Dict[Tuple[int, int], dict]:
    """Pick G for every shape (block sizes, sample count) and install the table.

    A bucket already in the cache for this GPU is not timed again. `timer_factory(blocks,
    n_s, precision)` returns f(G) -> ms (default: gram_timer on the device). Returns
    {bucket: {"group": G, "ms": {G: ms}}} for every bucket of the table."""
    gpu = gpu or _gpu_name()
    cache = _load_cache(cache_path) if cache_path else {}
    known = cache.get(gpu, {})
    timer_factory = timer_factory or gram_timer
    for blocks, n_s in shapes:
        key = bucket(max(blocks), n_s)
        skey = f"{key[0]}x{key[1]}"
        if skey in known:
            continue
        f = timer_factory(list(blocks), int(n_s), precision)
        ms = {int(G): f(int(G)) for G in candidates}
        best = min(ms, key=lambda G: (ms[G], G))
        known[skey] = {"group": best, "ms": {str(G): v for G, v in ms.items()},
                       "shape": {"blocks": [int(b) for b in blocks], "n_s": int(n_s)}}
    cache[gpu] = known
    if cache_path:
        _save_cache(cache_path, cache)
    table = {}
    for skey, rec in known.items():
        a, b = skey.split("x")
        table[(int(a), int(b))] = int(rec["group"])
    install(table)
    return {(int(k.split("x")[0]), int(k.split("x")[1])): v for k, v in known.items()}


def load(cache_path: str = DEFAULT_CACHE, gpu: Optional[str] = None) -> int:
    """Install the cached table of this GPU (no timing); returns the number of entries."""
    gpu = gpu or _gpu_name()
    known = _load_cache(cache_path).get(gpu, {})
    install({(int(k.split("x")[0]), int(k.split("x")[1])): int(v["group"]) for k, v in known.items()})
    return len(known)
