"""nlpot: NUFFT evaluation of nonlocal potentials phi = U * rho on one GB300 (sm_103a).

Method of Bao, Jiang, Tang & Zhang (arXiv:1410.3584): spherical/polar Fourier quadrature
with the Jacobian cancelling the kernel singularity, type-2 / type-1 NUFFTs, the Gaussian
subtraction for the 2D Laplace kernel (Algorithm 1), the normalized gradient flow
(Sec. 3) and time splitting (Sec. 4).  The compute lives in libnlpot.so (C-ABI in
include/nlpot.h); this package is its thin binding.
"""
from ._binding import *  # noqa: F401,F403
from ._binding import Plan, Surrogate, NlpError, LIB_PATH  # noqa: F401
