"""GB300-native hot path of the fully-coupled DG/CZM + lubrication method of
arXiv 1911.10275: per-Newton assembly and ILU(0) block-Jacobi GMRES solve,
hand-written CUDA for sm_103a behind the C ABI of include/hf.h."""
from ._lib import (HFMesh, HFRuntime, HFError, load, hf_mesh_desc, hf_solver_opts, hf_newton_report,
                   hf_step_opts, hf_step_report, hf_request, hf_result, hf_runtime_opts, hf_mesh_sizes,
                   hf_estimate_device_bytes, solver_opts, step_opts, HF_PREC_FP64, HF_PREC_MIXED, SIGNATURES)
