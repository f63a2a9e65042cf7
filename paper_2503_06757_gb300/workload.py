"""Seeded synthetic robots, scenes and candidate configurations.

This module only *draws inputs*: joint tables, sphere placements, obstacle
sets and streams of candidate configurations.  It holds none of the planner's
arithmetic (no kinematics, no distances, no collision tests, no sampling of
the planner itself), so that both the CUDA path and the FP64 oracle can consume
exactly the same inputs without sharing any of the method's code.

Every floating-point value it emits is exactly representable in IEEE binary32,
so the FP32 device path and the FP64 oracle see bit-identical geometry.

Randomness comes from a counter-based splitmix64 hash evaluated with numpy
uint64 arithmetic, which gives the same stream on every platform and numpy
version.

Robots (synthetic stand-ins for the paper's 7-, 8- and 14-DoF Panda / Fetch /
Baxter, Sec. IV-A):
  * ``arm7``   serial arm, revolute axes z,y,z,y,z,y,z, link lengths
               0.33/0/0.32/0/0.38/0/0.1 m, limits +-2.8 rad, 4 spheres of
               radius 0.06 m per link.
  * ``arm8``   the same arm on a prismatic torso (0..0.4 m) carrying 4 more
               spheres.
  * ``dual14`` two arms with bases 0.6 m apart and cross-arm self-collision.

Kinematic convention shared by both sides (an input convention, not code):
frame i is ``T_parent * J_i(q_i) * Trans(0, 0, L_i)`` where ``J_i`` rotates
about, or translates along, the local x, y or z axis; a joint whose parent
is -1 hangs off the world at ``joint_base[i]``.  Sphere k sits at
``T_frame * [offset, 1]``.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np

JOINT_REV_Z = 0
JOINT_REV_Y = 1
JOINT_PRISM_Z = 2
JOINT_PRISM_X = 3
JOINT_PRISM_Y = 4
JOINT_REV_X = 5
PRISMATIC = (JOINT_PRISM_Z, JOINT_PRISM_X, JOINT_PRISM_Y)

OBS_BOX = 0
OBS_CYLINDER = 1
OBS_SPHERE = 2

# Planner workspace used by every scene generator (metres).
WORKSPACE_LO = np.array([-0.8, -0.8, 0.0])
WORKSPACE_HI = np.array([0.8, 0.8, 1.2])

_M64 = (1 << 64) - 1
_GOLD = np.uint64(0x9E3779B97F4A7C15)


def _f32(x):
    """Round to the nearest binary32 value and return it as float64."""
    return np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)


def _mix64(x: np.ndarray) -> np.ndarray:
    x = np.asarray(x, dtype=np.uint64)
    x = (x ^ (x >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    x = (x ^ (x >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return x ^ (x >> np.uint64(31))


class Stream:
    """Counter-based uniform stream keyed by (seed, stream id)."""

    def __init__(self, seed: int, stream: int = 0):
        base = (int(seed) * 0x9E3779B97F4A7C15 + int(stream) * 0xD1B54A32D192ED03 + 0x632BE59BD9B4E019) & _M64
        self._base = _mix64(np.array([base], dtype=np.uint64))[0]
        self._pos = 0

    def uniform(self, n: int) -> np.ndarray:
        ctr = self._base + _GOLD * (np.arange(n, dtype=np.uint64) + np.uint64(self._pos))
        self._pos += n
        return (_mix64(ctr) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def range(self, lo, hi, n: int | None = None):
        lo = np.asarray(lo, dtype=np.float64)
        hi = np.asarray(hi, dtype=np.float64)
        shape = np.broadcast(lo, hi).shape if n is None else (n,) + np.broadcast(lo, hi).shape
        u = self.uniform(int(np.prod(shape)) if shape else 1).reshape(shape)
        return lo + u * (hi - lo)

    def integers(self, lo: int, hi: int, n: int | None = None):
        """Uniform integers in [lo, hi] inclusive."""
        m = 1 if n is None else n
        v = lo + np.floor(self.uniform(m) * (hi - lo + 1)).astype(np.int64)
        v = np.minimum(v, hi)
        return int(v[0]) if n is None else v

    def normal(self, n: int) -> np.ndarray:
        u1 = np.maximum(self.uniform(n), 1e-300)
        u2 = self.uniform(n)
        return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


# --------------------------------------------------------------------------- robots

@dataclass
class Robot:
    name: str
    dof: int
    joint_type: np.ndarray      # int32 [d]
    joint_parent: np.ndarray    # int32 [d]   (-1: world)
    joint_base: np.ndarray      # f64 [d,3]   world offset of world-parented joints
    link_length: np.ndarray     # f64 [d]
    lower: np.ndarray           # f64 [d]
    upper: np.ndarray           # f64 [d]
    sphere_frame: np.ndarray    # int32 [S]
    sphere_offset: np.ndarray   # f64 [S,3]   in the frame's coordinates
    sphere_radius: np.ndarray   # f64 [S]
    sphere_link: np.ndarray     # int32 [S]   link id (for the self-pair rule)
    self_pairs: np.ndarray      # int32 [P,2] sphere index pairs checked for self-collision
    ee_frames: list = field(default_factory=list)  # frames whose origin is an end effector

    @property
    def n_spheres(self) -> int:
        return int(self.sphere_frame.shape[0])


_ARM_TYPES = [JOINT_REV_Z, JOINT_REV_Y] * 3 + [JOINT_REV_Z]
_ARM_LENGTHS = [0.33, 0.0, 0.32, 0.0, 0.38, 0.0, 0.1]
_ARM_LIMIT = 2.8
_SPHERE_R = 0.06
_SPHERES_PER_LINK = 4


def _link_pairs_chain(lengths, first_link):
    """Link pairs of one serial chain that are checked for self-collision.

    Links i < j are checked when j - i >= 2, except when the only link between
    them has zero length (a joint housing): such neighbours are adjacent in
    effect and always touch.
    """
    n = len(lengths)
    pairs = []
    for i in range(n):
        for j in range(i + 2, n):
            if j - i == 2 and lengths[i + 1] == 0.0:
                continue
            pairs.append((first_link + i, first_link + j))
    return pairs


def _build_robot(name, types, parents, bases, lengths, lower, upper, extra_spheres, link_pairs, ee_frames):
    d = len(types)
    frames, offs, radii, links = [], [], [], []
    for f, (extra) in enumerate(extra_spheres):
        for (off, r) in extra:
            frames.append(f)
            offs.append(off)
            radii.append(r)
            links.append(f)
    for f in range(d):
        if types[f] in PRISMATIC:
            continue
        L = lengths[f]
        for k in range(_SPHERES_PER_LINK):
            t = (k + 0.5) / _SPHERES_PER_LINK
            frames.append(f)
            offs.append((0.0, 0.0, (t - 1.0) * L))
            radii.append(_SPHERE_R)
            links.append(f)
    frames = np.asarray(frames, dtype=np.int32)
    links = np.asarray(links, dtype=np.int32)
    sp = []
    for (a, b) in link_pairs:
        ia = np.nonzero(links == a)[0]
        ib = np.nonzero(links == b)[0]
        for x in ia:
            for y in ib:
                sp.append((int(x), int(y)))
    return Robot(
        name=name,
        dof=d,
        joint_type=np.asarray(types, dtype=np.int32),
        joint_parent=np.asarray(parents, dtype=np.int32),
        joint_base=_f32(np.asarray(bases, dtype=np.float64).reshape(d, 3)),
        link_length=_f32(lengths),
        lower=_f32(lower),
        upper=_f32(upper),
        sphere_frame=frames,
        sphere_offset=_f32(np.asarray(offs, dtype=np.float64).reshape(-1, 3)),
        sphere_radius=_f32(radii),
        sphere_link=links,
        self_pairs=np.asarray(sp, dtype=np.int32).reshape(-1, 2),
        ee_frames=list(ee_frames),
    )


def arm7(base=(0.0, 0.0, 0.0)) -> Robot:
    """Synthetic 7-DoF serial arm (28 spheres, 12 checked link pairs)."""
    d = 7
    parents = [-1] + list(range(d - 1))
    bases = [list(base)] + [[0.0, 0.0, 0.0]] * (d - 1)
    extra = [[] for _ in range(d)]
    return _build_robot("arm7", _ARM_TYPES, parents, bases, _ARM_LENGTHS,
                        [-_ARM_LIMIT] * d, [_ARM_LIMIT] * d, extra,
                        _link_pairs_chain(_ARM_LENGTHS, 0), [d - 1])


def arm8() -> Robot:
    """The 7-DoF arm on a prismatic torso (0..0.4 m), 32 spheres."""
    types = [JOINT_PRISM_Z] + _ARM_TYPES
    lengths = [0.0] + _ARM_LENGTHS
    d = 8
    parents = [-1] + list(range(d - 1))
    bases = [[0.0, 0.0, 0.0]] * d
    torso = [((0.0, 0.0, z), _SPHERE_R) for z in (-0.05, -0.15, -0.25, -0.35)]
    extra = [torso] + [[] for _ in range(d - 1)]
    lower = [0.0] + [-_ARM_LIMIT] * 7
    upper = [0.4] + [_ARM_LIMIT] * 7
    # The torso link is adjacent to arm link 0 only; the generic rule gives
    # exactly that because the link between them has non-zero length.
    pairs = _link_pairs_chain(lengths, 0)
    return _build_robot("arm8", types, parents, bases, lengths, lower, upper, extra, pairs, [d - 1])


def dual14() -> Robot:
    """Two 7-DoF arms with bases at x = -0.3 and +0.3 m (56 spheres)."""
    types = _ARM_TYPES + _ARM_TYPES
    lengths = _ARM_LENGTHS + _ARM_LENGTHS
    parents = [-1] + list(range(6)) + [-1] + list(range(7, 13))
    bases = [[-0.3, 0.0, 0.0]] + [[0.0, 0.0, 0.0]] * 6 + [[0.3, 0.0, 0.0]] + [[0.0, 0.0, 0.0]] * 6
    extra = [[] for _ in range(14)]
    pairs = _link_pairs_chain(_ARM_LENGTHS, 0) + _link_pairs_chain(_ARM_LENGTHS, 7)
    pairs += [(a, b) for a in range(7) for b in range(7, 14)]
    return _build_robot("dual14", types, parents, bases, lengths,
                        [-_ARM_LIMIT] * 14, [_ARM_LIMIT] * 14, extra, pairs, [6, 13])


ROBOTS = {"arm7": arm7, "arm8": arm8, "dual14": dual14}


def point2(lo=0.0, hi=1.2, z0=0.5, radius=0.02) -> Robot:
    """2-DoF point robot: prismatic x then prismatic y at height z0, one sphere."""
    return Robot(name="point2", dof=2, joint_type=np.asarray([JOINT_PRISM_X, JOINT_PRISM_Y], np.int32),
                 joint_parent=np.asarray([-1, 0], np.int32),
                 joint_base=_f32(np.asarray([[0.0, 0.0, z0], [0.0, 0.0, 0.0]])), link_length=_f32([0.0, 0.0]),
                 lower=_f32([lo, lo]), upper=_f32([hi, hi]), sphere_frame=np.asarray([1], np.int32),
                 sphere_offset=_f32(np.zeros((1, 3))), sphere_radius=_f32([radius]),
                 sphere_link=np.asarray([1], np.int32), self_pairs=np.zeros((0, 2), np.int32), ee_frames=[1])


def scene_two_rooms(z0=0.5, door=(0.85, 0.93)) -> "Scene":
    """Two rooms of the point robot's plane joined by a narrow door: a wall at
    x in [0.58, 0.62] with an opening for y in door (8 cm by default; the
    point robot's 2 cm sphere leaves its centre 4 cm)."""
    eye = np.eye(3).reshape(9)
    y0, y1 = door
    below = np.concatenate([[0.60, y0 / 2, z0], [0.02, y0 / 2, 0.3], eye])
    above = np.concatenate([[0.60, (y1 + 1.2) / 2, z0], [0.02, (1.2 - y1) / 2, 0.3], eye])
    return Scene(boxes=_f32(np.stack([below, above])), cylinders=np.zeros((0, 8)), spheres=np.zeros((0, 4)))


def two_rooms_pairs(n: int, seed: int):
    """Start in the left room, goal in the right room."""
    st = Stream(seed, 1)
    u = st.uniform(4 * n).reshape(n, 4)
    s = np.stack([0.05 + 0.45 * u[:, 0], 0.05 + 1.1 * u[:, 1]], 1)
    g = np.stack([0.70 + 0.45 * u[:, 2], 0.05 + 1.1 * u[:, 3]], 1)
    return _f32(s), _f32(g)


def robot_bases(robot: Robot) -> np.ndarray:
    """World positions of the chain roots (used for the base keep-out rule)."""
    return robot.joint_base[robot.joint_parent < 0]


# --------------------------------------------------------------------------- scenes

@dataclass
class Scene:
    boxes: np.ndarray      # f64 [nb,15]: centre(3), half extents(3), rotation(9, row-major, world = R*local + c)
    cylinders: np.ndarray  # f64 [nc,8]:  centre(3), unit axis(3), radius, half length
    spheres: np.ndarray    # f64 [ns,4]:  centre(3), radius
    cells: np.ndarray = field(default_factory=lambda: np.zeros((0, 6)))  # goal regions [lo(3), hi(3)]

    @property
    def n_obstacles(self) -> int:
        return int(self.boxes.shape[0] + self.cylinders.shape[0] + self.spheres.shape[0])


_EYE9 = np.eye(3).reshape(9)


def _box_row(c, h, R=None):
    R = _EYE9 if R is None else np.asarray(R).reshape(9)
    return np.concatenate([c, h, R])


def _quat_to_axis(qw, qx, qy, qz):
    """Third column of the rotation matrix of a unit quaternion (local z in world)."""
    return np.array([
        2.0 * (qx * qz + qw * qy),
        2.0 * (qy * qz - qw * qx),
        1.0 - 2.0 * (qx * qx + qy * qy),
    ])


def _bound_radius_box(h):
    return float(np.sqrt(np.sum(np.asarray(h) ** 2)))


def _clear_of_bases(c, rb, bases, margin=0.15, height=0.45):
    """Generator rule: keep obstacles off the fixed base column of each arm.

    The first link of every arm rotates about the vertical axis only, so an
    obstacle touching it would make every configuration invalid.
    """
    for b in bases:
        horiz = np.hypot(c[0] - b[0], c[1] - b[1])
        if horiz < rb + margin and c[2] - rb < height:
            return False
    return True


def _draw_box(st: Stream, side_lo=0.05, side_hi=0.3):
    c = st.range(WORKSPACE_LO, WORKSPACE_HI)
    h = 0.5 * st.range([side_lo] * 3, [side_hi] * 3)
    return c, h


def _draw_cylinder(st: Stream, centre=None):
    c = st.range(WORKSPACE_LO, WORKSPACE_HI) if centre is None else centre
    r = st.range(0.03, 0.1)
    length = st.range(0.1, 0.5)
    q = st.normal(4)
    q = q / np.linalg.norm(q)
    axis = _quat_to_axis(*q)
    axis = axis / np.linalg.norm(axis)
    return c, axis, float(r), float(0.5 * length)


def _draw_sphere(st: Stream, centre=None):
    c = st.range(WORKSPACE_LO, WORKSPACE_HI) if centre is None else centre
    r = float(st.range(0.03, 0.15))
    return c, r


def _finish(boxes, cyls, sphs, cells=None):
    b = _f32(np.asarray(boxes, dtype=np.float64).reshape(-1, 15))
    cy = np.asarray(cyls, dtype=np.float64).reshape(-1, 8)
    if cy.shape[0]:
        # unit axis rounded to binary32 (re-normalised first in float64)
        ax = cy[:, 3:6] / np.linalg.norm(cy[:, 3:6], axis=1, keepdims=True)
        cy = cy.copy()
        cy[:, 3:6] = ax
    cy = _f32(cy)
    s = _f32(np.asarray(sphs, dtype=np.float64).reshape(-1, 4))
    cl = np.zeros((0, 6)) if cells is None else _f32(np.asarray(cells, dtype=np.float64).reshape(-1, 6))
    return Scene(boxes=b, cylinders=cy, spheres=s, cells=cl)


def scene_random_boxes(seed: int, n: int = 8, bases=((0.0, 0.0, 0.0),)) -> Scene:
    """Axis-aligned cuboids with sides U[0.05,0.3] m, centres uniform in the workspace."""
    st = Stream(seed, 11)
    boxes = []
    while len(boxes) < n:
        c, h = _draw_box(st)
        if _clear_of_bases(c, _bound_radius_box(h), bases):
            boxes.append(_box_row(c, h))
    return _finish(boxes, [], [])


SHELF_FRONT_X = 0.45
SHELF_CELL = 0.3
SHELF_WALL = 0.02
SHELF_BOTTOM_Z = 0.2


def shelf_cells() -> np.ndarray:
    """Interior boxes [lo, hi] of the 3x3 cubby grid (goal regions)."""
    cells = []
    t = 0.5 * SHELF_WALL
    for iy in range(3):
        for iz in range(3):
            y0 = -1.5 * SHELF_CELL + iy * SHELF_CELL
            z0 = SHELF_BOTTOM_Z + iz * SHELF_CELL
            cells.append([SHELF_FRONT_X, y0 + t, z0 + t, SHELF_FRONT_X + SHELF_CELL - t, y0 + SHELF_CELL - t, z0 + SHELF_CELL - t])
    return np.asarray(cells)


def _shelf_structure():
    t = 0.5 * SHELF_WALL
    x0, x1 = SHELF_FRONT_X, SHELF_FRONT_X + SHELF_CELL
    y0, y1 = -1.5 * SHELF_CELL, 1.5 * SHELF_CELL
    z0, z1 = SHELF_BOTTOM_Z, SHELF_BOTTOM_Z + 3 * SHELF_CELL
    xm, zm = 0.5 * (x0 + x1), 0.5 * (z0 + z1)
    boxes = [_box_row([x1 + t, 0.0, zm], [t, 0.5 * (y1 - y0) + t, 0.5 * (z1 - z0) + t])]  # back wall
    for k in range(4):                                                                       # verticals
        y = y0 + k * SHELF_CELL
        boxes.append(_box_row([xm, y, zm], [0.5 * SHELF_CELL, t, 0.5 * (z1 - z0) + t]))
    for k in range(4):                                                                       # horizontals
        z = z0 + k * SHELF_CELL
        boxes.append(_box_row([xm, 0.0, z], [0.5 * SHELF_CELL, 0.5 * (y1 - y0) + t, t]))
    return boxes


def scene_shelf(seed: int, facing: str = "x") -> Scene:
    """3x3 cubby shelf (9 cuboids) plus clutter inside the cubbies.

    Clutter: 21 more cuboids (sides U[0.05,0.3] m), 10 capped cylinders
    (radius U[0.03,0.1] m, length U[0.1,0.5] m, uniform random unit
    quaternion) and 10 spheres (radius U[0.03,0.15] m), each centred at a
    uniform point inside a uniformly chosen cell; objects may protrude.
    facing "x": the shelf's front is the plane x = 0.45 (the single arm at the
    origin faces it).  facing "y": the same scene turned 90 degrees about the
    vertical axis, front plane y = 0.45 -- in front of both arms of the dual
    arm (bases at x = -0.3 and +0.3), each 0.45 m from it as the single arm is.
    """
    sc = _scene_shelf_x(seed)
    return sc if facing == "x" else rotate_scene_z90(sc)


def shelf_facing(robot: Robot) -> str:
    """Shelf placement for a robot: in front of the single arm ("x") or of both
    arms of the dual arm ("y")."""
    return "y" if len(robot_bases(robot)) > 1 else "x"


def rotate_scene_z90(sc: Scene) -> Scene:
    """The scene turned +90 degrees about the z axis: (x, y, z) -> (-y, x, z).
    Axis-aligned boxes stay axis-aligned with their x and y half extents
    swapped; cylinder axes and sphere centres turn; goal cells are re-sorted."""
    def rot(p):
        p = np.asarray(p, np.float64)
        return np.stack([-p[..., 1], p[..., 0], p[..., 2]], axis=-1)
    boxes = []
    for b in sc.boxes:
        R = b[6:15].reshape(3, 3)
        Rz = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
        boxes.append(np.concatenate([rot(b[0:3]), b[3:6], (Rz @ R).reshape(9)]))
        if np.allclose(R, np.eye(3)):   # keep axis-aligned boxes in the identity form
            boxes[-1] = np.concatenate([rot(b[0:3]), [b[4], b[3], b[5]], np.eye(3).reshape(9)])
    cyls = [np.concatenate([rot(c[0:3]), rot(c[3:6]), c[6:8]]) for c in sc.cylinders]
    sphs = [np.concatenate([rot(q[0:3]), q[3:4]]) for q in sc.spheres]
    cells = []
    for c in sc.cells:
        a, b = rot(c[0:3]), rot(c[3:6])
        cells.append(np.concatenate([np.minimum(a, b), np.maximum(a, b)]))
    return _finish(boxes, cyls, sphs, cells)


def _scene_shelf_x(seed: int) -> Scene:
    st = Stream(seed, 12)
    cells = shelf_cells()
    boxes = _shelf_structure()

    def in_cell():
        k = st.integers(0, 8)
        lo, hi = cells[k, :3], cells[k, 3:]
        return st.range(lo, hi)

    cyls, sphs = [], []
    for _ in range(21):
        c = in_cell()
        h = 0.5 * st.range([0.05] * 3, [0.3] * 3)
        boxes.append(_box_row(c, h))
    for _ in range(10):
        c, a, r, hl = _draw_cylinder(st, in_cell())
        cyls.append(np.concatenate([c, a, [r, hl]]))
    for _ in range(10):
        c, r = _draw_sphere(st, in_cell())
        sphs.append(np.concatenate([c, [r]]))
    return _finish(boxes, cyls, sphs, cells)


def scene_mixed(seed: int, n_obstacles: int, bases=((0.0, 0.0, 0.0),), n_moving: int = 0) -> Scene:
    """Random cuboids / cylinders / spheres in ratio 3:1:1 over the workspace."""
    st = Stream(seed, 13)
    n_cyl = int(round(n_obstacles * 0.2))
    n_sph = int(round(n_obstacles * 0.2))
    n_box = n_obstacles - n_cyl - n_sph
    boxes, cyls, sphs = [], [], []
    while len(boxes) < n_box:
        c, h = _draw_box(st)
        if _clear_of_bases(c, _bound_radius_box(h), bases):
            boxes.append(_box_row(c, h))
    while len(cyls) < n_cyl:
        c, a, r, hl = _draw_cylinder(st)
        if _clear_of_bases(c, float(np.hypot(r, hl)), bases):
            cyls.append(np.concatenate([c, a, [r, hl]]))
    while len(sphs) < n_sph:
        c, r = _draw_sphere(st)
        if _clear_of_bases(c, r, bases):
            sphs.append(np.concatenate([c, [r]]))
    return _finish(boxes, cyls, sphs)


# --------------------------------------------------------------------------- moving spheres

@dataclass
class MovingSpheres:
    """Spherical obstacles that move at a fixed speed with a random-walk heading.

    ``positions(k)`` gives the centres after k update ticks; they reflect at
    the workspace walls.
    """
    centres0: np.ndarray
    radii: np.ndarray
    seed: int
    speed: float = 0.5
    rate_hz: float = 30.0

    def positions(self, k: int) -> np.ndarray:
        return self.positions_track(k)[k]

    def positions_track(self, n: int) -> np.ndarray:
        """Centres after 0..n ticks, shape [n + 1, spheres, 3]."""
        st = Stream(self.seed, 99)
        p = self.centres0.copy()
        dt = 1.0 / self.rate_hz
        m = p.shape[0]
        head = st.normal(3 * m).reshape(m, 3)
        out = [_f32(p)]
        for _ in range(n):
            head = head + 0.3 * st.normal(3 * m).reshape(m, 3)
            v = head / np.linalg.norm(head, axis=1, keepdims=True) * self.speed
            p = p + v * dt
            lo = WORKSPACE_LO + self.radii[:, None]
            hi = WORKSPACE_HI - self.radii[:, None]
            over = p > hi
            under = p < lo
            p = np.where(over, 2 * hi - p, p)
            p = np.where(under, 2 * lo - p, p)
            head = np.where(over | under, -head, head)
            out.append(_f32(p))
        return np.stack(out)


def moving_spheres(seed: int, n: int = 5, bases=((0.0, 0.0, 0.0),)) -> MovingSpheres:
    st = Stream(seed, 14)
    cs, rs = [], []
    while len(cs) < n:
        c, r = st.range(WORKSPACE_LO, WORKSPACE_HI), float(st.range(0.05, 0.15))
        if _clear_of_bases(c, r, bases):
            cs.append(c)
            rs.append(r)
    return MovingSpheres(_f32(np.asarray(cs)), _f32(np.asarray(rs)), seed)


# --------------------------------------------------------------------------- configurations

def candidates(robot: Robot, seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """Candidate configurations, uniform within the joint limits (float32-exact)."""
    st = Stream(seed, 1000 + stream)
    if offset:
        st._pos = offset * robot.dof
    u = st.uniform(n * robot.dof).reshape(n, robot.dof)
    q = robot.lower + u * (robot.upper - robot.lower)
    return _f32(q)


@dataclass
class Problem:
    robot: Robot
    scene: Scene
    q_start: np.ndarray
    q_goal: np.ndarray
    seed: int
    name: str = ""


def choose_problem(robot: Robot, scene: Scene, seed: int, accept, goal_in_cells: bool = False,
                   chunk: int = 4096, max_chunks: int = 64):
    """Pick start and goal as the first acceptable candidates of a seeded stream.

    ``accept(robot, scene, Q)`` is supplied by the caller (the oracle in tests,
    the device collision checker in the benchmark); it returns a boolean
    free-mask for the rows of Q and the world positions of the end-effector
    frames, shape [n, len(robot.ee_frames), 3].  Returns None if no pair was
    found within the candidate budget.
    """
    start = goal = None
    for ci in range(max_chunks):
        Q = candidates(robot, seed, 0, chunk, offset=ci * chunk)
        free, ee = accept(robot, scene, Q)
        for i in np.nonzero(free)[0]:
            if start is None:
                start = Q[i]
                continue
            if goal_in_cells and scene.cells.shape[0]:
                p = ee[i, 0]
                inside = np.any(np.all((p >= scene.cells[:, :3]) & (p <= scene.cells[:, 3:]), axis=1))
                if not inside:
                    continue
            goal = Q[i]
            break
        if goal is not None:
            break
    if start is None or goal is None:
        return None
    return start, goal


def problem_set(kind: str, count: int, seed0: int, accept, n_obstacles=None):
    """Seeded problem sets shaped like the paper's workloads.

    kind: "boxes8" 8 random cuboids + arm7; "shelf" cubby shelf + arm7 (goals in
    cubbies); "mixed" 7/8/14-DoF in equal thirds with 10..120 mixed obstacles.
    Scenes for which no start/goal pair is found are replaced by the next seed.
    """
    out = []
    seed = seed0
    while len(out) < count:
        if kind == "boxes8":
            robot = arm7()
            scene = scene_random_boxes(seed)
            pair = choose_problem(robot, scene, seed, accept)
        elif kind == "shelf":
            robot = arm7()
            scene = scene_shelf(seed)
            pair = choose_problem(robot, scene, seed, accept, goal_in_cells=True)
        elif kind == "mixed":
            which = ["arm7", "arm8", "dual14"][len(out) % 3]
            robot = ROBOTS[which]()
            st = Stream(seed, 15)
            n_obs = st.integers(10, 120) if n_obstacles is None else int(n_obstacles)
            scene = scene_mixed(seed, n_obs, bases=robot_bases(robot))
            pair = choose_problem(robot, scene, seed, accept)
        else:
            raise ValueError(kind)
        if pair is not None:
            out.append(Problem(robot, scene, pair[0], pair[1], seed, f"{kind}-{seed}"))
        seed += 1
    return out


# --------------------------------------------------------------------------- learned proposal inputs

PROPOSAL_IN = 16 ** 3 + 2 * 32      # occupancy voxels + padded start + padded goal
PROPOSAL_HIDDEN = (1024, 512, 512)
PROPOSAL_COMPONENTS = 8


def proposal_head_pad(dof: int) -> int:
    """Head width (8 logits + 8*dof means + 8*dof log-sigmas) rounded up to 128."""
    return ((PROPOSAL_COMPONENTS * (1 + 2 * dof) + 127) // 128) * 128


def proposal_init(dof: int, seed: int):
    """Seeded He-normal initial weights (W [out, in], b [out]) of the proposal MLP,
    binary32-exact; biases start at zero."""
    dims = (PROPOSAL_IN,) + PROPOSAL_HIDDEN + (proposal_head_pad(dof),)
    st = Stream(seed, 77)
    params = []
    for i in range(4):
        fan_in, fan_out = dims[i], dims[i + 1]
        scale = np.sqrt(2.0 / fan_in) if i < 3 else 0.1 * np.sqrt(1.0 / fan_in)
        W = _f32(st.normal(fan_out * fan_in).reshape(fan_out, fan_in) * scale)
        params.append((W, np.zeros(fan_out)))
    return params


def random_mixture(dof: int, seed: int, spread: float = 0.6):
    """Seeded mixture parameters [logits(8) | means(8*dof) | log-sigmas(8*dof)]
    over normalised joint values (inputs for sampler parity tests)."""
    st = Stream(seed, 78)
    logits = st.normal(PROPOSAL_COMPONENTS)
    means = st.range(-spread, spread, PROPOSAL_COMPONENTS * dof)
    logsig = st.range(-3.0, -1.0, PROPOSAL_COMPONENTS * dof)
    return _f32(np.concatenate([logits, means, logsig]))
