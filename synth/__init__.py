"""Seeded synthetic fisheye stereo inputs (scene simulator, no stereo method)."""
from .workloads import (auto_levels, disparity_errors, draw_kb, fronto_plane,
                        gt_disparity, mixed_2048, plain_kb, plain_small, rig_sequence)

__all__ = ["plain_small", "plain_kb", "mixed_2048", "fronto_plane", "draw_kb",
           "auto_levels", "rig_sequence", "gt_disparity", "disparity_errors"]
