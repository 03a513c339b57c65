"""Write full-size oracle results used by the GPU parity tests.

Runs the FP64 oracle (and nothing else) on the full-size seeded workloads and
stores dtheta, <E>, n_kept and a sample of E_loc as .npz files next to this
script. Usage: python tests/golden/make_fullsize.py [workload ...]
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import workloads as W  # noqa: E402


def main(names):
    for name in names:
        t0 = time.time()
        w = W.make_workload(name)
        r = oracle.qgt.sr_step(w.model, w.theta, w.configs, w.bond_ij, w.bond_j, w.block_off, w.diag_shift,
                               w.cutoff, 1.0, w.c, w.sign_rule)
        idx = np.linspace(0, w.n_samples - 1, 64).astype(np.int64)
        np.savez_compressed(os.path.join(HERE, f"oracle_{name}.npz"), dtheta=r["dtheta"], e_mean=r["e_mean"],
                            n_kept=r["n_kept"], eloc_idx=idx, eloc=r["eloc"][idx],
                            sigma_max=np.array([s.max() for s in r["sigma"]]),
                            sigma_min=np.array([s.min() for s in r["sigma"]]))
        print(name, "done in", round(time.time() - t0, 1), "s", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["j1j2_6x6_ffnn", "j1j2_10x10_ffnn5"])
