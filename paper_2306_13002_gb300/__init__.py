"""GB300-native (sm_103a) library for the as-written and saturated forms of two FP64 3D
stencil loop bodies: a compressible-flow RHS and a 25-point star stencil.

The compute path is `libacs.so` (CUDA, built in-tree by `build.build()`); `binding`
exposes its C-ABI entry points under the same names. `inputs` holds the seeded input
generators. Importing the package does not load the CUDA library; the first call does,
and fails loudly if it is missing.
"""
from .binding import (AcsError, acs_abi_version, acs_rhs_form, acs_rhs_plain, acs_rhs_saturated,  # noqa: F401
                      acs_stencil_plain, acs_stencil_saturated, acs_status_string)
