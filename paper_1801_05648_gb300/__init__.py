"""GB300-native block-preconditioned FGMRES for monolithic ALE fluid-structure
Jacobians (Jodlbauer, Langer & Wick, arXiv:1801.05648, Sec. 4).

The solver lives in ``libfsi.so`` (CUDA, sm_103a) behind the C ABI of
``include/fsi.h``; ``fsi.py`` is its ctypes binding and ``learned.py`` the
training / evaluation driver of the learned correction stage.
"""
from .fsi import (FSISolver, FSIAssembler, FSIError, Params, SolveStats, Trainer, TrainParams, default_params,
                  default_train_params, load_library, BLOCKS, EXPORTED, FSI_FP64, FSI_FP32_AMG, FSI_X0_GIVEN,
                  FSI_USE_GRAPHS, FSI_NO_RIGID_MODES, FSI_CLUSTER_COARSE, FSI_LEARNED, FSI_NO_PDL, FSI_GRID_COARSE,
                  FSI_FLUID_GMRES, FSI_MLP_CUDA_CORES, FSI_PRECOND_LDU, FSI_PRECOND_LOWER, FSI_PRECOND_UPPER,
                  FSI_PRECOND_DIAG, FSI_MLP_PARAMS, FSI_MLP_PARAMS_3D, mlp_params, mlp_inputs, LIB_PATH,
                  probe_fma_rate, FSI_OK, FSI_EINVAL, FSI_ENOMEM,
                  FSI_ECUDA, FSI_ENOTCONV, FSI_EBREAKDOWN, FSI_ENONFINITE, FSI_INJECT_COARSE_BARRIER,
                  FSI_INJECT_MLP_COMMIT)

__all__ = ["FSISolver", "FSIAssembler", "FSIError", "Params", "SolveStats", "Trainer", "TrainParams", "default_params",
           "default_train_params", "load_library", "BLOCKS", "EXPORTED", "FSI_FP64", "FSI_FP32_AMG", "FSI_X0_GIVEN",
           "FSI_USE_GRAPHS", "FSI_NO_RIGID_MODES", "FSI_CLUSTER_COARSE", "FSI_LEARNED", "FSI_NO_PDL",
           "FSI_GRID_COARSE", "FSI_FLUID_GMRES", "FSI_MLP_CUDA_CORES", "FSI_PRECOND_LDU", "FSI_PRECOND_LOWER",
           "FSI_PRECOND_UPPER", "FSI_PRECOND_DIAG", "FSI_MLP_PARAMS", "FSI_MLP_PARAMS_3D", "mlp_params",
           "mlp_inputs", "LIB_PATH", "probe_fma_rate", "FSI_OK",
           "FSI_EINVAL", "FSI_ENOMEM", "FSI_ECUDA", "FSI_ENOTCONV", "FSI_EBREAKDOWN", "FSI_ENONFINITE",
           "FSI_INJECT_COARSE_BARRIER", "FSI_INJECT_MLP_COMMIT"]
