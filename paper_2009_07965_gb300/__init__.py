"""GB300-native Recursive MRCM (arXiv 2009.07965) for 2D Darcy flow.

The compute path is libmrcm.so (hand-written sm_103a CUDA behind the C ABI
of include/mrcm.h); this package only builds it and marshals arguments.
"""
from .binding import (mrcm_setup, mrcm_setup_batch, mrcm_plan_query, mrcm_set_permeability, mrcm_build_basis, mrcm_solve,
                      mrcm_query, mrcm_node_info, mrcm_node_segments, mrcm_segment_info,
                      mrcm_node_operator, mrcm_destroy, mrcm_error_string, mrcm_enable_timing, mrcm_use_graphs,
                      mrcm_last_cuda_error,
                      mrcm_phase_times, mrcm_merge_pair_noalloc, mrcm_set_refinement, mrcm_set_residual,
                      mrcm_residual_history, mrcm_phase_flops, mrcm_group_times, mrcm_check_reciprocal, mrcm_set_wait_limit, mrcm_probe_peak, mrcm_set_mixed_split, mrcm_set_mixed_leaves, mrcm_set_root_form, mrcm_autotune, mrcm_tune_info,
                      mrcm_interior_leaves, mrcm_leaf_fields, mrcm_leaf_patches, mrcm_leaf_gate, mrcm_leaf_apply,
                      mrcm_cnn_conv_forward, mrcm_cnn_conv_wgrad, mrcm_cnn_flip_weights, mrcm_cnn_relu_grad,
                      mrcm_cnn_mse_grad, mrcm_cnn_adam, PROBES, MrcmError, PHASES, PHASE_KERNELS,
                      EXPORTS, LIB_PATH)
from .solver import Solver, Solver3D, BatchSolver

__all__ = ["mrcm_setup", "mrcm_setup_batch", "mrcm_plan_query", "mrcm_set_permeability", "mrcm_build_basis", "mrcm_solve", "mrcm_query",
           "mrcm_node_info", "mrcm_node_segments", "mrcm_segment_info", "mrcm_node_operator",
           "mrcm_destroy", "mrcm_error_string", "mrcm_enable_timing", "mrcm_phase_times", "mrcm_use_graphs",
           "mrcm_last_cuda_error",
           "mrcm_merge_pair_noalloc", "mrcm_set_refinement", "mrcm_set_residual", "mrcm_residual_history", "mrcm_phase_flops",
           "mrcm_group_times", "mrcm_check_reciprocal", "mrcm_set_wait_limit", "mrcm_probe_peak", "mrcm_set_mixed_split", "mrcm_set_mixed_leaves", "mrcm_set_root_form", "mrcm_autotune", "mrcm_tune_info",
           "mrcm_interior_leaves", "mrcm_leaf_fields", "mrcm_leaf_patches", "mrcm_leaf_gate", "mrcm_leaf_apply",
           "mrcm_cnn_conv_forward", "mrcm_cnn_conv_wgrad", "mrcm_cnn_flip_weights", "mrcm_cnn_relu_grad",
           "mrcm_cnn_mse_grad", "mrcm_cnn_adam", "PROBES", "MrcmError", "PHASE_KERNELS", "PHASES", "EXPORTS", "LIB_PATH", "Solver", "Solver3D", "BatchSolver"]
