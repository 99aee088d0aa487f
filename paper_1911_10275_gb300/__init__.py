"""GB300-native hot path of the fully-coupled DG/CZM + lubrication method of
arXiv 1911.10275: per-Newton assembly and ILU(0) block-Jacobi GMRES solve,
hand-written CUDA for sm_103a behind the C ABI of include/hf.h."""
from ._lib import (HFMesh, HFError, load, hf_mesh_desc, hf_solver_opts, hf_newton_report,
                   HF_PREC_FP64, HF_PREC_MIXED, SIGNATURES)
