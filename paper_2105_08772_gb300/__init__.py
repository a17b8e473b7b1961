"""GB300-native Shan-Chen droplet/bubble lattice Boltzmann library.

The hot path -- the D3Q19 BGK + Guo-forcing Shan-Chen step and the FP64
reductions that give R_e, Delta P, sigma[R], R_s (arXiv:2105.08772,
Secs. II-IV) -- lives in liblbm.so (hand-written CUDA for sm_103a behind the
C ABI of include/lbm.h).  This package is its Python binding.
"""
from .lbm import *  # noqa: F401,F403
from .lbm import Batch, Group, Lattice, make_box, make_eos  # noqa: F401
from ._lib import (EXPORTS, LBM_ECOLLAPSE, LBM_EINVAL, LBM_ENOTCONV, LBM_ENUMERIC,  # noqa: F401
                   LBM_ETIMEOUT, LBM_OK, LBMError, lbm_obs)
