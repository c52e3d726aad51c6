"""GB300-native matrix-free DG solver for compressible Euler on 2:1 non-conforming meshes.

The computation lives in the CUDA library ``_lib/libdgatmo.so`` (C ABI in
``include/dg_atmo.h``); this package only marshals arguments.  Importing it
without the built library raises ImportError: there is no CPU fallback.
"""

from .api import (  # noqa: F401
    DG_FP32,
    DG_FP64,
    DG_KRYLOV_AUTO,
    DG_KRYLOV_CG,
    DG_KRYLOV_CHEBYSHEV,
    DG_KRYLOV_GMRES,
    DG_KRYLOV_GMRES_CGS2,
    DG_TERMS_FULL,
    DG_TERMS_IMEX_EXPLICIT,
    BatchPlan,
    Context,
    DGError,
    Mesh,
    Server,
    State,
    dg_apply_div,
    dg_batch_barrier_test,
    dg_batch_step,
    dg_apply_explicit,
    dg_apply_grad,
    dg_apply_implicit,
    dg_apply_implicit_noalloc,
    dg_background,
    dg_conservation,
    dg_init_state,
    dg_launch_count,
    dg_math_selftest,
    dg_peak_fma,
    dg_profile_enable,
    dg_profile_read,
    dg_profile_read_cta_passes,
    dg_profile_read_gmres_phases,
    dg_profile_reset,
    imex_rk2_step,
    solver_opts,
)
