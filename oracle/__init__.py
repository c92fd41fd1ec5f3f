"""FP64 CPU oracle of the object-centric 2DGS rasterizer (test infrastructure only).

Only tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
import this package; the CUDA product path never does.
"""
from .ocgs_oracle import *  # noqa: F401,F403
from .ocgs_oracle import (ALPHA_MAX, ALPHA_MIN, RHO_CUT, SIGMA_F2, T_EPS, background_loss,  # noqa: F401
                          background_loss_grad, composite, contribution_score, keep_set, project,
                          prune, quat_to_rotmat, render, render_views, sh_basis, adam_step,
                          masked_psnr, masked_ssim, ssim_blur, ssim_map, ssim_window,
                          depth_distortion, normal_consistency, project_ewa, render_3d,
                          contribution_score_3d)
