"""Importance-sampling Gaussian shape overlap on B300 (sm_103a).

Python face of the C ABI in ``include/shape.h`` (library ``libshape.so``):
molecule sets live in device memory, the estimators of Eq. expectation /
Eq. union-is run in hand-written CUDA kernels, and results come back as
torch CUDA tensors. ``synth`` builds the seeded synthetic molecule sets.
"""
from ._binding import (ANTITHETIC, EXPORTS, ID_STREAMS, LIB_PATH, MAX_ATOMS, OBJ_FO, OBJ_FO_CLOSED, OBJ_UNION, SYMMETRIC,
                       TAG_AB, TAG_BA,
                       TAG_SELF, PoseOverlap, align_crn_points, align_rigid, overlap_pose_grad, pose_overlap,
                       ShapeError, ShapeSet, fo_overlap, load_library, overlap_estimate, screen_config,
                       fail_next_allocations, eval_probe, fo_tanimoto_screen, fo_prefilter_select, prefilter_db_ids, screen_variant_info, screen_variants, self_overlaps, shape_set_load, tanimoto_screen, tanimoto_screen_tune,
                       union_volume_estimate, union_attributions, union_volume_cv, union_self_estimate, cv_features, cv_fit_weights, mlp_forward,
                       mlp_loss_grad, mlp_adam, mlp_train_epoch, MLP_PARAMS)
from .graph import StepGraph
from . import pipeline

__all__ = ["ANTITHETIC", "EXPORTS", "ID_STREAMS", "LIB_PATH", "MAX_ATOMS", "OBJ_FO", "OBJ_FO_CLOSED", "OBJ_UNION", "SYMMETRIC",
           "TAG_AB", "TAG_BA",
           "TAG_SELF", "PoseOverlap", "align_crn_points", "align_rigid", "overlap_pose_grad", "pose_overlap",
           "ShapeError", "ShapeSet", "fo_overlap", "load_library", "overlap_estimate", "screen_config",
           "fail_next_allocations", "eval_probe", "fo_tanimoto_screen", "fo_prefilter_select", "prefilter_db_ids", "screen_variant_info", "screen_variants", "self_overlaps", "shape_set_load", "tanimoto_screen", "tanimoto_screen_tune",
           "union_volume_estimate", "union_attributions", "union_volume_cv", "union_self_estimate", "cv_features", "cv_fit_weights", "mlp_forward",
           "mlp_loss_grad", "mlp_adam", "mlp_train_epoch", "MLP_PARAMS", "StepGraph", "pipeline"]
