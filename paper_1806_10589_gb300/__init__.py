"""GB300 (sm_103a) D3Q19 lattice Boltzmann solver with the adaptive volumetric-flux
boundary condition of arXiv:1806.10589.

The compute path is the CUDA library libgb300lbm.so (C ABI in include/lbm.h);
this package only builds it (build.py) and binds it (lbm.py).
"""
from .lbm import (  # noqa: F401
    Lattice, Batch, ColorLattice, WarmStartNet, LBMError, conv3d_bf16, load_library, LIB_PATH, SIGNATURES,
    LBM_FACE_ZMIN, LBM_FACE_ZMAX, LBM_PREC_FP64, LBM_PREC_FP32, LBM_PREC_FP16DEV, LBM_PREC_BF16DEV,
    LBM_MODEL_BGK, LBM_MODEL_MRT, PRECISIONS, MODELS, BATCH_CONFIGS, LBM_BATCH_GRAPH, LBM_BATCH_GRAPH_CAPPED,
    LBM_BATCH_PERSISTENT, LBM_BATCH_PERSISTENT_CAPPED, LBM_BATCH_AA, LBM_BATCH_AA_CAPPED,
)
