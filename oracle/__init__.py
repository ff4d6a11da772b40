"""FP64 CPU oracle of the multislice ptychography loss-and-gradient path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product imports, calls or executes
this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it.  It
shares no code with the CUDA path (no kernels, headers, tables or helpers);
the only thing both sides have in common is the seeded input generator
module, which holds none of the method's arithmetic.

Contents
  dft.py    naive DFT by explicit FP64 DFT matrices (no FFT library)
  model.py  forward model (Algorithm 1, Eqs. ri_modulation, fresnel_prop,
            paraxial_kernel, fraunhofer, fourier_shift, multimode,
            rotation_transform), losses (Eqs. lsq_loss, poisson_loss) and the
            hand-derived adjoint; the near-field multi-distance variant.

Every function is pinned by ``tests/test_oracle_*.py`` against closed forms,
invariants, library routines on special cases, or brute-force finite
differences; no function is left with unpinned parity.
"""
from .dft import dft2, dft_minus, dft_plus, freq, idft_minus  # noqa: F401
from .model import (Problem, forward, loss, loss_grad, rotate, rotate_T,  # noqa: F401
                    split_positions)
