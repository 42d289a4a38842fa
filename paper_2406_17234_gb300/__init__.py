"""GB300-native JFNK solver for multilevel NLTE radiative transfer.

The hot path -- residual F(n) of the statistical-equilibrium equations, its
Jacobian-vector products, the block-Jacobi preconditioner and the on-device
Newton-Krylov driver -- lives in ``libjfnk.so`` (CUDA, sm_103a), behind the C
ABI of ``include/jfnk.h``. ``binding`` marshals arguments to it with ctypes;
there is no CPU fallback: loading fails loudly when the library is missing.
"""
from . import binding  # noqa: F401
from .binding import (Atmosphere, Atom, Context, JFNKError, batch_solve, block_jacobi,  # noqa: F401
                      default_options, jvp, load, residual, rh92_update, solve)
