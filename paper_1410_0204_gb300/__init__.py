"""GB300-native (sm_103a, FP64) Transport Matrix Method year map of Metos3D (arXiv:1410.0204).

The compute path is the CUDA library ``libmetos3d.so`` (C ABI in ``include/metos3d.h``);
this package holds its sources (``csrc/``), its build (``build.py``) and a thin ctypes
binding (``binding.py``) that passes torch CUDA tensors and streams to it.
"""
from .binding import (Context, Metos3dError, bgc, declared_symbols, load, library_path,  # noqa: F401
                      MODEL_NONE, MODEL_NDOP, M3D_OK, M3D_ERR_ARG, M3D_ERR_CUDA, M3D_ERR_NONFINITE,
                      M3D_ERR_TIMEOUT, M3D_ERR_UNSUPPORTED, M3D_NOT_CONVERGED, OPT_YEAR_PLAN,
                      OPT_WAIT_TIMEOUT_NS, OPT_TEST_WITHHOLD_TILE, OPT_NTILES, PLAN_PERSISTENT, PLAN_GRAPH,
                      PLAN_RESIDENT, OPT_IMPLICIT_FORM, OPT_ADJOINT_PLAN, OPT_STEP_OPERATORS,
                      OPT_STEP_OPERATOR_BYTES, OPT_KERNEL_TIMING, OPT_LAST_KERNEL_NS,
                      OPT_TANGENT_FORM, TANGENT_DUAL, TANGENT_LINEARISED, IMPLICIT_DENSE, IMPLICIT_TRIDIAGONAL,
                      JV_FD, JV_TANGENT, NewtonOptions, NewtonReport, GradientOptions, GradientReport,
                      year_map_autograd, Ensemble, MODEL_N, MODEL_PHY, MODEL_NPZD, MODEL_NTRACER)
