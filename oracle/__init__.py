"""FP64 CPU oracle of the block-layer stochastic-reconfiguration step.

TEST INFRASTRUCTURE ONLY. Nothing on the product path may import, call, link
or execute anything in this package; only the tests, the smoke check of
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` use it. It shares
no code with the CUDA path (it imports only NumPy/SciPy and the seeded input
generators of ``workloads``).

Every function follows the paper's definitions directly, in float64/complex128:

* ``nqs``          ln psi and the log-derivative Jacobian O = d ln psi / d theta
                   (Sec. 2, definition below Eq. 2), for the RBM and the ln cosh FFNN.
* ``hamiltonian``  local energies E_loc (Eq. 1) of the periodic Heisenberg
                   chain and the J1-J2 square lattice (Sec. 3), dense H and
                   Lanczos ground energies for pins.
* ``qgt``          means, centring, force F, the block-layer QGT S_b (Eq. 3 /
                   Eq. 2), the shifted per-block pseudo-inverse solve (Sec. 2,
                   block-layer paragraph), the full-QGT and NTK comparators.
* ``exact``        exact expectations by enumeration of all 2^N states.
* ``diagnostics``  the inverse-metric diagnostics of Eq. 4 and the infidelity.
* ``vit``          the transformer wavefunction (embedding, encoder layers, output) whose
                   modules give the block partition of Sec. 2.
* ``vmc``          exchange-move Metropolis sampling of |psi|^2 and the VMC loop
                   (sample, block-layer SR step, theta += dtheta).

Parity status of each function is listed in its docstring; all are pinned by
tests in ``tests/test_oracle_*.py`` except the Table 1 diagnostics values,
which need the paper's trained network (parity unpinned for those numbers;
the diagnostic formulas themselves are pinned by identities).
"""
from . import nqs, hamiltonian, qgt, exact, diagnostics, vmc, vit  # noqa: F401
