"""Start/goal acceptance through the device collision checker, for building
problem sets (workload.problem_set's `accept` predicate) without the CPU oracle.

The predicate returns, for candidate configurations Q [n x dof], whether each is
collision-free and the world position of each end-effector frame origin (from
the two outermost spheres on the frame's link axis)."""
from __future__ import annotations

import numpy as np

from . import prrtc as P


def device_accept():
    cache = {}

    def accept(robot, scene, Q):
        key = (robot.name, id(scene))
        if key not in cache:
            cache.clear()
            cache[key] = (P.make_robot(robot), P.make_env(scene))
        rb, ev = cache[key]
        valid, sph = P.prrtc_check_states(rb, ev, Q, want_spheres=True)
        ee = np.zeros((len(Q), len(robot.ee_frames), 3))
        for k, f in enumerate(robot.ee_frames):
            idx = np.nonzero(robot.sphere_frame == f)[0]
            z = robot.sphere_offset[idx, 2]
            order = idx[np.argsort(z)]
            a, b = order[-2], order[-1]          # two outermost spheres on the link axis
            za, zb = robot.sphere_offset[a, 2], robot.sphere_offset[b, 2]
            ca, cb = sph[:, a, :3].astype(np.float64), sph[:, b, :3].astype(np.float64)
            ee[:, k] = cb + (cb - ca) * ((0.0 - zb) / (zb - za))   # frame origin at offset 0
        return valid, ee

    return accept
