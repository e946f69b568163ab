"""CPU oracle for the symbol-based tau-preconditioned Krylov solve of fractional
diffusion equations (Barakitis, Ekstrom, Vassalos, "Preconditioners for
Fractional Diffusion Equations Based on the Spectral Symbol").

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or links
anything in this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it.

Everything here is plain FP64 numpy written from the paper's definitions:
dense Toeplitz matrices built entry by entry from the Grunwald weights, an
explicit dense sine matrix, textbook PCG and GMRES(m).  It shares no code,
constant or table generator with the CUDA path.
"""

from .fde_oracle import *  # noqa: F401,F403
