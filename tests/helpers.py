"""Small hand-built robots and scenes used by the pins and parity tests."""
import numpy as np

from paper_2503_06757_gb300 import workload as W


def robot(types, lengths, parents=None, bases=None, lower=None, upper=None, spheres=(), pairs=(), name="custom"):
    d = len(types)
    parents = list(range(-1, d - 1)) if parents is None else parents
    bases = [[0.0, 0.0, 0.0]] * d if bases is None else bases
    lower = [-np.pi] * d if lower is None else lower
    upper = [np.pi] * d if upper is None else upper
    fr = [s[0] for s in spheres]
    off = [s[1] for s in spheres]
    rad = [s[2] for s in spheres]
    return W.Robot(
        name=name, dof=d,
        joint_type=np.asarray(types, np.int32), joint_parent=np.asarray(parents, np.int32),
        joint_base=np.asarray(bases, np.float64).reshape(d, 3), link_length=np.asarray(lengths, np.float64),
        lower=np.asarray(lower, np.float64), upper=np.asarray(upper, np.float64),
        sphere_frame=np.asarray(fr, np.int32).reshape(-1),
        sphere_offset=np.asarray(off, np.float64).reshape(-1, 3),
        sphere_radius=np.asarray(rad, np.float64).reshape(-1),
        sphere_link=np.asarray(fr, np.int32).reshape(-1),
        self_pairs=np.asarray(pairs, np.int32).reshape(-1, 2),
        ee_frames=[d - 1],
    )


def empty_scene():
    return W.Scene(boxes=np.zeros((0, 15)), cylinders=np.zeros((0, 8)), spheres=np.zeros((0, 4)))


def scene(boxes=(), cylinders=(), spheres=()):
    b = np.asarray(boxes, np.float64).reshape(-1, 15)
    c = np.asarray(cylinders, np.float64).reshape(-1, 8)
    s = np.asarray(spheres, np.float64).reshape(-1, 4)
    return W.Scene(boxes=b, cylinders=c, spheres=s)


def aabb(c, h):
    return np.concatenate([np.asarray(c, float), np.asarray(h, float), np.eye(3).reshape(9)])


def no_self(rb):
    """Copy of a robot with self-collision checking switched off."""
    import dataclasses
    return dataclasses.replace(rb, self_pairs=np.zeros((0, 2), np.int32))


def point_robot(z0=0.5, radius=0.02, lo=0.0, hi=1.2):
    """2-DoF point robot: prismatic x then prismatic y, one sphere."""
    return robot([W.JOINT_PRISM_X, W.JOINT_PRISM_Y], [0.0, 0.0], bases=[[0.0, 0.0, z0], [0.0, 0.0, 0.0]],
                 lower=[lo, lo], upper=[hi, hi], spheres=[(1, (0.0, 0.0, 0.0), radius)], name="point2")


def maze(seed, n=6, cell=0.2, wall=0.02, z0=0.5, open_frac=0.55, enclose=None):
    """Grid maze of n x n cells in the plane z = z0.

    Returns (scene, open_edges) where open_edges[(a, b)] is True when the wall
    between adjacent cells a and b is absent.  Reachability between cells is a
    plain graph question on this adjacency, independent of any geometry code.
    """
    st = W.Stream(seed, 7)
    boxes = []
    open_edges = {}
    t = 0.5 * wall
    for i in range(n):
        for j in range(n):
            for (di, dj) in ((1, 0), (0, 1)):
                a, b = (i, j), (i + di, j + dj)
                inside = b[0] < n and b[1] < n
                is_open = inside and st.uniform(1)[0] < open_frac
                if enclose is not None and (a == enclose or b == enclose):
                    is_open = False
                if inside:
                    open_edges[(a, b)] = open_edges[(b, a)] = is_open
                if is_open:
                    continue
                if di == 1:   # wall on the x = (i+1)*cell line, spanning cell j in y
                    c = [(i + 1) * cell, (j + 0.5) * cell, z0]
                    h = [t, 0.5 * cell + t, 0.5]
                else:         # wall on the y = (j+1)*cell line
                    c = [(i + 0.5) * cell, (j + 1) * cell, z0]
                    h = [0.5 * cell + t, t, 0.5]
                boxes.append(aabb(c, h))
    # outer walls on x = 0 and y = 0
    for k in range(n):
        boxes.append(aabb([0.0, (k + 0.5) * cell, z0], [t, 0.5 * cell + t, 0.5]))
        boxes.append(aabb([(k + 0.5) * cell, 0.0, z0], [0.5 * cell + t, t, 0.5]))
    return scene(boxes=boxes), open_edges


def maze_reachable(open_edges, n, a, b):
    seen = {a}
    todo = [a]
    while todo:
        x = todo.pop()
        if x == b:
            return True
        for (di, dj) in ((1, 0), (-1, 0), (0, 1), (0, -1)):
            y = (x[0] + di, x[1] + dj)
            if 0 <= y[0] < n and 0 <= y[1] < n and open_edges.get((x, y), False) and y not in seen:
                seen.add(y)
                todo.append(y)
    return False


def bf16_round(x):
    """Round binary32 values to bfloat16 (nearest, ties to even), returned as float32."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    bits = a.view(np.uint32).astype(np.uint64)
    lsb = (bits >> 16) & 1
    bits = (bits + 0x7FFF + lsb) & 0xFFFF0000
    return bits.astype(np.uint32).view(np.float32).reshape(a.shape)


def revalidation_counts(items, res):
    """Re-check paths with the oracle at resolution `res` (4x finer than planning).

    items: (robot, scene, path [k x dof], esdf or None) per path.  Returns
    (segments, bad segments, lowest clearance seen)."""
    from oracle import oracle as O
    segs = bad = 0
    worst = float("inf")
    for robot, scene, path, esdf in items:
        path = np.asarray(path, np.float64)
        b, mc = O.revalidate(robot, scene, path, res, esdf=esdf)
        segs += max(0, len(path) - 1)
        bad += b
        worst = min(worst, mc)
    return segs, bad, worst


def assert_same_revalidation_rate(gpu, oracle, what=""):
    """Discrete edge checking can pass a segment that a finer re-check flags, for
    the oracle's own paths as much as for the GPU's; the hot-path contract is
    that both flag segments at the same rate.  gpu / oracle: revalidation_counts
    results on the same problems.  The rates must agree within three standard
    errors of the pooled rate (floored at one flagged segment in the pool)."""
    (ng, bg, wg), (no, bo, wo) = gpu, oracle
    assert ng > 0 and no > 0, (gpu, oracle)
    pool = (bg + bo) / (ng + no)
    p = max(pool, 1.0 / (ng + no))
    tol = 3.0 * np.sqrt(p * (1.0 - p) * (1.0 / ng + 1.0 / no))
    print(f"revalidation {what}: GPU {bg}/{ng} segments flagged (lowest clearance {wg:.2e}), "
          f"oracle {bo}/{no} ({wo:.2e})")
    assert abs(bg / ng - bo / no) <= tol, (what, gpu, oracle, tol)
