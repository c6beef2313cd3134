"""Seeded synthetic inputs: tetrahedral voxel meshes, rigs and rig poses.

This module produces the *inputs* of a pose solve (rest vertices, tets, joint
positions, parent links, per-handle rigid transforms, material constants).  It
holds none of the skinning method's arithmetic (no deformation gradients,
energies, clustering, pin selection or solves), so both the FP64 oracle and the
CUDA library can be fed from it without sharing any of the method's code.
"""
from .meshes import (kuhn_voxel_mesh, bar_mesh, figure_rig, character_rig, figure_mesh,
                     figure_mesh_for_tets)
from .poses import rodrigues, figure_pose, figure_animation, bar_twist_pose, identity_pose, rigid_pose
from .configs import (bar_twist_config, bar_pull_config, character_config, face_traction_loads, figure_config,
                      lame_from_young, SNH_E, SNH_NU)

__all__ = [
    "kuhn_voxel_mesh", "bar_mesh", "figure_rig", "character_rig", "character_config", "figure_mesh", "figure_mesh_for_tets",
    "rodrigues", "figure_pose", "figure_animation", "bar_twist_pose", "identity_pose", "rigid_pose",
    "bar_twist_config", "bar_pull_config", "face_traction_loads", "figure_config", "lame_from_young", "SNH_E", "SNH_NU",
]
