"""Writes the stored regression fixtures in this folder.  Calls only the
oracle and the seeded input generators; run from the repository root:
    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth   # noqa: E402


def forward_tiny():
    rng = np.random.default_rng(2024)
    views = synth.circular_views(2, 150.0, 250.0, 1.7, 1.9, angles=[0.2, 2.1])
    g = synth.Geometry(7, 6, 5, 1.0, 1.2, 0.9, 6, 5, views, 0.45, (0.3, -0.2, 0.1))
    mu = rng.uniform(0, 1, g.vol_shape)
    poses = np.array([[0.5, -0.3, 0.2, 0.05, -0.1, 0.2], [-0.4, 0.1, 0.0, 0.0, 0.15, -0.05]])
    inst_view = np.array([0, 1, 1], dtype=np.int32)
    inst_pose = np.array([0, 0, 1], dtype=np.int32)
    proj = oracle.forward(g, mu, poses, inst_view=inst_view, inst_pose=inst_pose)
    np.savez(os.path.join(HERE, "forward_tiny.npz"), dims=[g.nx, g.ny, g.nz],
             vox=[g.vx, g.vy, g.vz], det=[g.nu, g.nv], views=views, step=g.step,
             off=np.array(g.off), mu=mu, poses=poses, inst_view=inst_view,
             inst_pose=inst_pose, proj=proj)


if __name__ == "__main__":
    forward_tiny()
