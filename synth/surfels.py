"""Seeded synthetic surfel maps and keyframe trajectories for the dense model
correction (inputs only: no correction arithmetic here).

A room-sized map: surfel positions on the floor, walls and boxes of the room
scene generator's extent, random unit normals, and for each surfel an
initialisation and last-update time stamp a few dozen keyframes apart. The
keyframes walk a loop around the room at eye height looking toward its middle
(camera-to-world poses, z forward); the corrected poses apply a drift
correction that grows along the loop to about 1.5 deg and 6 cm at its end, as
a loop closure does.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
from scipy.spatial.transform import Rotation

CAM = (525.0, 525.0, 319.5, 239.5, 640.0, 480.0, 4.0)  # fx, fy, cx, cy, width, height, max depth (m)


@dataclass
class SurfelMap:
    pos: np.ndarray    # n x 3 float32
    nrm: np.ndarray    # n x 3 float32, unit
    t0: np.ndarray     # n float32
    tu: np.ndarray     # n float32
    T_old: np.ndarray  # m x 4 x 4 float64 camera-to-world
    T_new: np.ndarray  # m x 4 x 4 float64
    t_kf: np.ndarray   # m float32, ascending
    cam: tuple


def _look_at(eye, target):
    z = target - eye
    z /= np.linalg.norm(z)
    x = np.cross(z, [0.0, 0.0, 1.0])
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    T = np.eye(4)
    T[:3, 0], T[:3, 1], T[:3, 2], T[:3, 3] = x, y, z, eye
    return T


def make_surfels(n: int = 1_000_000, m: int = 200, seed: int = 7, window: tuple = (2, 40)) -> SurfelMap:
    rng = np.random.default_rng(seed)
    W, D, H = 4.0, 3.5, 2.5
    # surfels on the floor (40%), the four walls (50%) and the ceiling (10%) of a W x D x H room
    u = rng.random(n)
    pos = np.empty((n, 3))
    a, b = rng.random(n), rng.random(n)
    floor, walls = u < 0.4, (u >= 0.4) & (u < 0.9)
    pos[floor] = np.stack([a[floor] * W, b[floor] * D, np.zeros(floor.sum())], 1)
    ceil = ~floor & ~walls
    pos[ceil] = np.stack([a[ceil] * W, b[ceil] * D, np.full(ceil.sum(), H)], 1)
    side = rng.integers(0, 4, n)
    for s in range(4):
        sel = walls & (side == s)
        k = sel.sum()
        t, h = a[sel], b[sel] * H
        if s == 0:
            pos[sel] = np.stack([t * W, np.zeros(k), h], 1)
        elif s == 1:
            pos[sel] = np.stack([t * W, np.full(k, D), h], 1)
        elif s == 2:
            pos[sel] = np.stack([np.zeros(k), t * D, h], 1)
        else:
            pos[sel] = np.stack([np.full(k, W), t * D, h], 1)
    pos += rng.normal(0, 0.003, pos.shape)
    nrm = rng.normal(size=(n, 3))
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    # keyframes on a loop at eye height
    centre = np.array([W / 2, D / 2, 1.4])
    T_old = np.empty((m, 4, 4))
    T_new = np.empty((m, 4, 4))
    for f in range(m):
        ang = 2 * np.pi * f / m
        eye = centre + np.array([1.2 * np.cos(ang), 1.0 * np.sin(ang), 0.1 * np.sin(3 * ang)])
        target = centre + np.array([-0.8 * np.cos(ang + 0.3), -0.7 * np.sin(ang + 0.3), -0.3])
        T_old[f] = _look_at(eye, target)
        s = f / max(m - 1, 1)
        C = np.eye(4)
        C[:3, :3] = Rotation.from_rotvec(np.array([0.2, -0.4, 1.0]) / np.linalg.norm([0.2, -0.4, 1.0]) *
                                         np.deg2rad(1.5) * s).as_matrix()
        C[:3, 3] = np.array([0.04, -0.03, 0.02]) * s
        T_new[f] = C @ T_old[f]
    t_kf = np.arange(m, dtype=np.float32)
    t0 = rng.integers(0, m, n).astype(np.float32) - 0.5
    tu = t0 + rng.integers(window[0], window[1] + 1, n).astype(np.float32)
    return SurfelMap(pos.astype(np.float32), nrm.astype(np.float32), t0, tu, T_old, T_new, t_kf, CAM)
