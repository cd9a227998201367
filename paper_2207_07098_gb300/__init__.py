"""GB300 (sm_103a) spectral-element Poisson solver: Python binding of libsem.

The compute path lives in csrc/*.cu (built into libsem.so, C ABI in
include/sem.h); this package only marshals arguments.  Functions keep the C
names: sem_setup, sem_setup_batch, sem_ax, sem_gs, sem_mass, sem_dot,
sem_get_geometry, sem_get_jacobi, sem_cg_solve, sem_cg_solve_batch,
sem_destroy, sem_get_info, sem_get_offsets, sem_gll, sem_set_helmholtz,
sem_projection_reset, sem_projection_size, sem_dot_noalloc, sem_grad, sem_div,
sem_curl, sem_pressure_rhs.
"""
from ._lib import *  # noqa: F401,F403
from ._lib import (SEM_EBREAKDOWN, SEM_ECUDA, SEM_EINVAL, SEM_ENOMEM, SEM_ENOTCONV, SEM_ESTAGNATE,
                   SEM_ETIMEOUT, SEM_FP32, SEM_FP64, SEM_FP64_NATIVE, SEM_FP64_PAIR, SEM_TC_SPLIT, SEM_MODE_FP64, SEM_MODE_MIXED_IR, SEM_MODE_GMRES,
                   SEM_OK, LIB_PATH, SemError, load, exported_symbols, SEM_FLAG_VARIANT, SEM_FLAG_TEST_STALL,
                   SEM_FLAG_METRICS, SEM_FLAG_SCHWARZ)
from .build import build  # noqa: F401
