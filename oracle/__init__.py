"""CPU oracle for the parallel multicanonical lattice gas.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously-correct
reference that the CUDA path is checked against.  Only ``tests/``, the smoke
check in ``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may
import it.  It shares no code with the CUDA library and imports nothing from
it; the library never imports this package.

Contents (paper section / equation each function follows):

* ``mucal_oracle.c`` (compiled with gcc, loaded with ctypes): Philox4x32-10,
  lattice geometry, the energy of Eq. 5, initial placement, acceptance
  thresholds for min(1, W(E_n)/W(E_o)) (Sec. 2), the walker chain (Sec. 2),
  exact enumeration of Omega(E), and the fixed-magnetisation Ising Metropolis
  run of Sec. 4.
* ``recursion.py`` (numpy, float64): the simple weight iteration
  W^{i+1} = W^i / H^i (Sec. 2), the accumulated-statistics recursion named in
  Sec. 2, normalisation, flatness and the ln Omega estimate.
* ``muca.py``: the iteration loop of Sec. 2 (run p walkers with fixed weights,
  sum their histograms by Eq. 2, update the weights), the exact transition
  matrix for detailed-balance checks, reweighting and the Ising map of Eq. 5.
* ``mlp.py`` (numpy, float64): the 4-128-128-1 GELU network that maps
  (d, L, rho, E/V) to ln Omega(E)/V, forward and backward.

Parity pins for each function are in ``tests/test_oracle_*.py``.
"""
from .build import build_oracle, load_oracle  # noqa: F401
