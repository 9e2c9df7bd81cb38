"""CPU oracle for the Zeitlin-Euler IsoMP step (complex128, NumPy/SciPy).

TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the
benchmark's CPU-baseline leg may import this package. The product path (the
CUDA library and its Python binding) never imports, calls or links it, and
it shares no code with that path.

Contents (each function cites the passage of Cifani, Viviani & Modin,
"An efficient geometric method for incompressible hydrodynamics on the
sphere", that it follows):
  laplacian_block   -- tridiagonal block of diagonal m, Sec. 3.2 Eq. 13
  laplacian_apply   -- W = Delta_N P, block by block, Sec. 3.2-3.3
  stream_solve      -- P = Delta_N^{-1} W, Sec. 3.3 Eq. 14
  isomp_step        -- one IsoMP step by fixed-point sweeps, Sec. 2 Eqs.
                       8 and 9, Sec. 3.1
  isomp_run         -- repeated steps
  casimirs          -- C_k = tr(W^k), Sec. 2 Eq. 7
  basis (module)    -- quantised spherical-harmonic basis T^_lm by Wigner 3j
                       symbols and by eigenvectors of the blocks, W from
                       omega_lm and back, Sec. 3.2 Eqs. 10-12
  spectrum (module) -- kinetic-energy spectrum E_l over the basis, Sec. 4

Every function is pinned by tests/test_oracle_*.py against facts that do not
come from this package (closed-form spectrum, the textbook spin-Casimir
operator, dense pseudo-inverses, exact algebraic identities of the scheme,
an independent high-order ODE integration, hand-computed blocks).
"""
from .zeitlin import (  # noqa: F401
    laplacian_block,
    laplacian_apply,
    stream_solve,
    isomp_step,
    isomp_run,
    casimirs,
    StepInfo,
)
