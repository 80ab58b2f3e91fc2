"""CPU oracle for the trigonometric-collocation Lippmann-Schwinger solver.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only the test suite, the smoke check and the CPU
baseline leg of the benchmark use it.  It shares no code with the CUDA
library (no kernels, headers, tables or helpers); the only common input is
the seeded microstructure generator, which holds none of the method's
arithmetic.

Everything here is plain, slow and in float64:

``operator``   the collocation operator ``A = I + B`` of Eq. (linear_system)
               and Eq. (mtrx_B), with a library FFT (scipy.fft) as the DFT step.
``dense``      Tier 1, tiny grids only: the DFT matrices of Eq. (DFT_def)
               written out, ``I + B`` assembled densely and solved by LU; and
               an independent potential (equilibrium) formulation of the same
               discrete problem, solved by Cholesky.
``solvers``    CG (Saad Alg. 6.18), BiCG (Saad Alg. 7.3) and the FFTH
               Neumann iteration Eq. (orig_fft), in the paper's order, plus the
               stopping norms Eq. (errE_def), Eq. (errR_def) and the effective
               tensor.

Every function is pinned by ``tests/test_oracle_*.py`` against closed forms,
invariants and brute force (see each docstring for what pins it).
"""
from . import dense, operator, solvers  # noqa: F401
from .operator import (  # noqa: F401
    apply_A,
    apply_AT,
    apply_B,
    gamma_hat,
    polarisation,
    reference_medium,
    signed_frequencies,
)
from .solvers import (  # noqa: F401
    bicg,
    cg,
    effective_tensor,
    eta_e,
    fixed_point,
    solve,
)
