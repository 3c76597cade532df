"""FP64 CPU oracle for non-rectified variational fisheye stereo (Roxas & Oishi).

TEST INFRASTRUCTURE ONLY.  This package is the slow, plain reference that the
CUDA path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The product path (``paper_1909_07545_gb300``) never imports it and shares no
code with it: camera models, interpolation, pyramid, tensor, primal-dual and
triangulation are all written again here, in float64 numpy, one step per
paper equation, with no blocking, fusion or reordering.

Modules
-------
camera       projection pi / unprojection pi^-1 (Sec. III-A, III-B, III-D)
interp       bilinear and Keys-bicubic sampling (Sec. III-B, Eq. 9)
geometry     trajectory field (Sec. III-B, Eq. 6-7), calibration field and
             pre-rotation (Sec. IV-A), ray triangulation (Sec. III-D end)
pyramid      levels, circular FOV mask, down/up-sampling (Sec. IV-B)
variational  tensor (Eq. 12), masked gradient/divergence, preconditioning,
             primal-dual step (Eq. 11, 13), linearisation (Eq. 3, 5), energy
tgv          the TGV-L1 energy of Eq. 10 and its primal-dual step (Eq. 11)
solve        Algorithm 1 driven coarse-to-fine (Algorithm 1, Sec. IV)

Pinning status (what fixes each function independently of itself) is listed
in ``tests/test_oracle_*.py``; the one function whose result is not pinned
beyond self-consistency is the full multi-warp solve on textured scenes
("parity unpinned" for exact iteration-count behaviour: the paper prints no
worked example); the end-to-end fronto-parallel plane test bounds it.
"""

from .camera import Calib, calib_from_dict, project, unproject, radial, fov_radius
from .interp import bilinear, bicubic
from .geometry import (trajectory_field, trajectory_vector, calibration_field,
                       prerotate, triangulate_range, virtual_translation)
from .pyramid import level_sizes, scaled_calib, fov_mask, downsample, upsample
from .variational import (Params, grad_masks, grad, div, tensor_sqrt, precondition,
                          dual_step, shrink, primal_step, pd_iteration,
                          warp_linearize, clip_update, energy, accel_schedule,
                          check_accel)
from .solve import solve, solve_level_warps, warm_start_w
from .tgv import div_q, grad_v, tgv_energy, tgv_iteration, tgv_steps

__all__ = [
    "Calib", "calib_from_dict", "project", "unproject", "radial", "fov_radius",
    "bilinear", "bicubic",
    "trajectory_field", "trajectory_vector", "calibration_field", "prerotate",
    "triangulate_range", "virtual_translation",
    "level_sizes", "scaled_calib", "fov_mask", "downsample", "upsample",
    "Params", "grad_masks", "grad", "div", "tensor_sqrt", "precondition",
    "dual_step", "shrink", "primal_step", "pd_iteration", "warp_linearize",
    "clip_update", "energy", "accel_schedule", "check_accel", "solve",
    "solve_level_warps", "warm_start_w",
    "grad_v", "div_q", "tgv_steps", "tgv_iteration", "tgv_energy",
]
