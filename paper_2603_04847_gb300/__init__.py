"""GB300-native joint pose-appearance training step of GloSplat
(arXiv 2603.04847): differentiable 3D Gaussian splatting with camera poses
as parameters, fused with the feature-track reprojection term.

The compute path is libgs (hand-written CUDA for sm_103a behind the C ABI
in include/gs.h).  This package only marshals arguments; it raises if the
library is missing and has no CPU fallback."""
from ._lib import GsError, load  # noqa: F401
from .core import (Batch, Cameras, Gaussians, Projected, TileLists, gs_adam_update, gs_photo_loss,  # noqa: F401
                   gs_project, gs_render_bwd, gs_render_fwd, gs_sort_tiles, gs_step_advance, gs_zero, pose_se3_update,
                   track_reproj_fwd_bwd)
from .step import Hyper, JointStep, Renderer  # noqa: F401
