"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each pin is chosen so that a plausible slip in the oracle (a constant, a sign,
an axis, an operand order, a transposed rotation, a dropped term, a wrong
index) fails at least one of them:
  * Philox4x32-10: the published known-answer vectors (tests/golden).
  * Forward kinematics: closed forms of 1-, 2- and 3-link chains, prismatic
    joints, sphere placement along a link, the straight arm, orthonormality.
  * Signed distances: brute-force minimum over dense surface samples of tiny
    cuboids / capped cylinders / spheres, plus inside/on-surface special cases.
  * Clearance composition: one sphere vs one obstacle, two-sphere self pair.
  * Planner (Alg. 1 / Alg. 2): obstacle-free special cases, balanced first
    extension, maze reachability against a graph BFS, walled-off goal, start /
    goal in collision, tree invariants, determinism.
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_06757_gb300 import workload as W
from tests import helpers as H

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- Philox

def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert O.philox(v[0:4], v[4:6]) == v[6:10]


def test_sample_inside_limits_and_goal_fraction():
    rb = W.arm8()
    n, goals = 20000, 0
    lo, hi = rb.lower, rb.upper
    for it in range(n):
        g, q = O.sample(rb, 7, 3, it, 0.05)
        if g:
            goals += 1
        else:
            assert np.all(q >= lo) and np.all(q < hi)
    # binomial(20000, 0.05): sd = 30.8
    assert abs(goals - 0.05 * n) < 5 * 30.8


def test_sample_uniform_per_dimension():
    rb = W.arm7()
    qs = np.array([O.sample(rb, 11, 0, it, 0.0)[1] for it in range(4000)])
    u = (qs - rb.lower) / (rb.upper - rb.lower)
    # mean 1/2, variance 1/12 per dimension; loose 5-sigma bounds
    assert np.all(np.abs(u.mean(0) - 0.5) < 5 * np.sqrt(1 / 12 / 4000))
    assert np.all(np.abs(u.var(0) - 1 / 12) < 0.01)
    # dimensions are not copies of one another
    assert np.all(np.abs(np.corrcoef(u.T)[np.triu_indices(7, 1)]) < 0.1)


# ----------------------------------------------------------------- FK

def _tip(rb, q):
    _, fr = O.fk(rb, np.asarray(q, float))
    return fr[-1][:3, 3]


def _rz(a):
    c, s = np.cos(a), np.sin(a)
    return np.array([[c, -s, 0], [s, c, 0], [0, 0, 1.0]])


@pytest.mark.parametrize("q", [0.0, 0.3, -1.2, 2.5])
def test_fk_one_link_revolute_y(q):
    L = 0.7
    rb = H.robot([W.JOINT_REV_Y], [L], bases=[[0.1, -0.2, 0.3]])
    np.testing.assert_allclose(_tip(rb, [q]), [0.1 + L * np.sin(q), -0.2, 0.3 + L * np.cos(q)], atol=1e-14)


def test_fk_one_link_revolute_x():
    L, q = 0.5, 0.9
    rb = H.robot([W.JOINT_REV_X], [L])
    np.testing.assert_allclose(_tip(rb, [q]), [0.0, -L * np.sin(q), L * np.cos(q)], atol=1e-14)


@pytest.mark.parametrize("q1,q2", [(0.0, 0.0), (0.4, -0.7), (-2.0, 1.3), (3.0, 2.9)])
def test_fk_two_link_zy(q1, q2):
    L1, L2 = 0.33, 0.45
    rb = H.robot([W.JOINT_REV_Z, W.JOINT_REV_Y], [L1, L2])
    want = _rz(q1) @ np.array([L2 * np.sin(q2), 0.0, L1 + L2 * np.cos(q2)])
    np.testing.assert_allclose(_tip(rb, [q1, q2]), want, atol=1e-14)


@pytest.mark.parametrize("q", [(0.2, 0.5, -0.4), (-1.0, 2.0, 1.0), (2.7, -1.1, -2.2)])
def test_fk_three_link_zyy(q):
    L1, L2, L3 = 0.3, 0.4, 0.25
    q1, q2, q3 = q
    rb = H.robot([W.JOINT_REV_Z, W.JOINT_REV_Y, W.JOINT_REV_Y], [L1, L2, L3])
    planar = np.array([L2 * np.sin(q2) + L3 * np.sin(q2 + q3), 0.0, L1 + L2 * np.cos(q2) + L3 * np.cos(q2 + q3)])
    np.testing.assert_allclose(_tip(rb, q), _rz(q1) @ planar, atol=1e-14)


def test_fk_prismatic_xyz():
    rb = H.robot([W.JOINT_PRISM_X, W.JOINT_PRISM_Y, W.JOINT_PRISM_Z], [0.0, 0.0, 0.2], bases=[[1.0, 2.0, 3.0], [0, 0, 0], [0, 0, 0]])
    np.testing.assert_allclose(_tip(rb, [0.1, -0.3, 0.4]), [1.1, 1.7, 3.6], atol=1e-14)


def test_fk_sphere_placement_along_link():
    L, q = 0.6, 0.8
    spheres = [(0, (0.0, 0.0, (t - 1.0) * L), 0.05) for t in (0.125, 0.375, 0.625, 0.875)]
    rb = H.robot([W.JOINT_REV_Y], [L], spheres=spheres)
    cen, _ = O.fk(rb, np.array([q]))
    for k, t in enumerate((0.125, 0.375, 0.625, 0.875)):
        np.testing.assert_allclose(cen[k], [t * L * np.sin(q), 0.0, t * L * np.cos(q)], atol=1e-14)


def test_fk_arm7_straight_and_bent():
    rb = W.arm7()
    np.testing.assert_allclose(_tip(rb, np.zeros(7)), [0, 0, 1.13], atol=1e-7)
    q = np.zeros(7)
    q[1] = np.pi / 2
    np.testing.assert_allclose(_tip(rb, q), [0.8, 0, 0.33], atol=1e-7)
    q[0] = np.pi / 2     # rotate the bent arm about the vertical axis
    np.testing.assert_allclose(_tip(rb, q), [0, 0.8, 0.33], atol=1e-7)


def test_fk_dual_arm_bases():
    rb = W.dual14()
    _, fr = O.fk(rb, np.zeros(14))
    np.testing.assert_allclose(fr[6][:3, 3], [-0.3, 0, 1.13], atol=1e-7)
    np.testing.assert_allclose(fr[13][:3, 3], [0.3, 0, 1.13], atol=1e-7)


@pytest.mark.parametrize("name", ["arm7", "arm8", "dual14"])
def test_fk_rotations_orthonormal_and_link_lengths(name):
    rb = W.ROBOTS[name]()
    rng = np.random.default_rng(0)
    for _ in range(20):
        q = rb.lower + rng.random(rb.dof) * (rb.upper - rb.lower)
        _, fr = O.fk(rb, q)
        for i in range(rb.dof):
            R = fr[i][:3, :3]
            np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-12)
            assert abs(np.linalg.det(R) - 1) < 1e-12
            par = rb.joint_parent[i]
            p0 = rb.joint_base[i] if par < 0 else fr[par][:3, 3]
            if rb.joint_type[i] in W.PRISMATIC:
                continue
            # a revolute joint does not move its own origin: link i has length L_i
            assert abs(np.linalg.norm(fr[i][:3, 3] - p0) - rb.link_length[i]) < 1e-12


# ----------------------------------------------------------------- signed distances

def _box_surface(c, h, R, step=1e-3):
    pts = []
    for axis in range(3):
        o = [a for a in range(3) if a != axis]
        u = np.arange(-h[o[0]], h[o[0]] + step / 2, step)
        v = np.arange(-h[o[1]], h[o[1]] + step / 2, step)
        U, V = np.meshgrid(u, v)
        for sgn in (-1, 1):
            P = np.zeros((U.size, 3))
            P[:, o[0]] = U.ravel()
            P[:, o[1]] = V.ravel()
            P[:, axis] = sgn * h[axis]
            pts.append(P)
    P = np.concatenate(pts)
    return P @ R.T + c


def _rot(seed):
    rng = np.random.default_rng(seed)
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


@pytest.mark.parametrize("rotated", [False, True])
def test_box_distance_brute_force(rotated):
    c = np.array([0.1, -0.05, 0.2])
    h = np.array([0.03, 0.05, 0.02])
    R = _rot(3) if rotated else np.eye(3)
    box = np.concatenate([c, h, R.reshape(9)])
    S = _box_surface(c, h, R)
    rng = np.random.default_rng(1)
    step = 1e-3
    for _ in range(60):
        p = c + rng.uniform(-0.1, 0.1, 3)
        local = R.T @ (p - c)
        inside = np.all(np.abs(local) < h)
        brute = np.min(np.linalg.norm(S - p, axis=1)) * (-1 if inside else 1)
        assert abs(O.sd_box(box, p) - brute) <= step * np.sqrt(2) / 2 + 1e-12


def test_box_distance_special_cases():
    c, h = np.array([0.0, 0.0, 0.0]), np.array([0.1, 0.2, 0.3])
    box = H.aabb(c, h)
    assert abs(O.sd_box(box, c) + 0.1) < 1e-15                      # centre: -min(h)
    assert abs(O.sd_box(box, [0.1, 0.05, -0.1])) < 1e-15             # on a face
    assert abs(O.sd_box(box, [0.5, 0.0, 0.0]) - 0.4) < 1e-15         # off a face
    assert abs(O.sd_box(box, [0.4, 0.6, 0.0]) - 0.5) < 1e-15         # off an edge (3-4-5)


def _cyl_surface(c, a, r, hl, step=1e-3):
    # orthonormal frame with third axis a
    t = np.array([1.0, 0, 0]) if abs(a[0]) < 0.9 else np.array([0, 1.0, 0])
    e1 = np.cross(a, t)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(a, e1)
    nth = int(np.ceil(2 * np.pi * r / step))
    th = np.linspace(0, 2 * np.pi, nth, endpoint=False)
    z = np.arange(-hl, hl + step / 2, step)
    TH, Z = np.meshgrid(th, z)
    side = (r * np.cos(TH.ravel()))[:, None] * e1 + (r * np.sin(TH.ravel()))[:, None] * e2 + Z.ravel()[:, None] * a
    rr = np.arange(0, r + step / 2, step)
    caps = []
    for zz in (-hl, hl):
        for rad in rr:
            n = max(1, int(np.ceil(2 * np.pi * rad / step)))
            th2 = np.linspace(0, 2 * np.pi, n, endpoint=False)
            caps.append((rad * np.cos(th2))[:, None] * e1 + (rad * np.sin(th2))[:, None] * e2 + zz * a)
    return np.concatenate([side] + caps) + c


def test_cylinder_distance_brute_force():
    c = np.array([0.05, 0.0, 0.1])
    a = np.array([1.0, 2.0, 2.0]) / 3.0
    r, hl = 0.03, 0.04
    cyl = np.concatenate([c, a, [r, hl]])
    S = _cyl_surface(c, a, r, hl)
    rng = np.random.default_rng(2)
    step = 1e-3
    for _ in range(60):
        p = c + rng.uniform(-0.09, 0.09, 3)
        v = p - c
        z = v @ a
        rho = np.linalg.norm(v - z * a)
        inside = rho < r and abs(z) < hl
        brute = np.min(np.linalg.norm(S - p, axis=1)) * (-1 if inside else 1)
        assert abs(O.sd_cyl(cyl, p) - brute) <= step * 1.5 + 1e-12


def test_cylinder_distance_special_cases():
    cyl = np.array([0, 0, 0, 0, 0, 1.0, 0.1, 0.3])
    assert abs(O.sd_cyl(cyl, [0, 0, 0]) + 0.1) < 1e-15         # centre: -min(r, hl)
    assert abs(O.sd_cyl(cyl, [0, 0, 0.25]) + 0.05) < 1e-15      # near a cap, inside
    assert abs(O.sd_cyl(cyl, [0, 0, 0.5]) - 0.2) < 1e-15        # beyond a cap on the axis (flat cap)
    assert abs(O.sd_cyl(cyl, [0.4, 0, 0]) - 0.3) < 1e-15        # radial
    assert abs(O.sd_cyl(cyl, [0.4, 0, 0.7]) - 0.5) < 1e-15      # off the rim (3-4-5)
    # a capsule would give 0.2 - ... at this point; the flat cap gives the axial distance
    assert abs(O.sd_cyl(cyl, [0.05, 0, 0.4]) - 0.1) < 1e-15


def test_sphere_distance_brute_force():
    s = np.array([0.0, 0.1, 0.2, 0.04])
    n = 40000
    i = np.arange(n) + 0.5
    phi = np.arccos(1 - 2 * i / n)
    th = np.pi * (1 + 5 ** 0.5) * i
    S = s[:3] + s[3] * np.stack([np.cos(th) * np.sin(phi), np.sin(th) * np.sin(phi), np.cos(phi)], 1)
    rng = np.random.default_rng(3)
    for _ in range(40):
        p = s[:3] + rng.uniform(-0.08, 0.08, 3)
        inside = np.linalg.norm(p - s[:3]) < s[3]
        brute = np.min(np.linalg.norm(S - p, axis=1)) * (-1 if inside else 1)
        assert abs(O.sd_sph(s, p) - brute) <= 1e-3


# ----------------------------------------------------------------- clearance

def test_clearance_one_sphere_one_obstacle():
    rb = H.robot([W.JOINT_PRISM_X, W.JOINT_PRISM_Y, W.JOINT_PRISM_Z], [0, 0, 0], spheres=[(2, (0, 0, 0), 0.05)])
    sc = H.scene(spheres=[[1.0, 0.0, 0.0, 0.2]])
    q = np.array([0.3, 0.4, 0.0])  # centre (0.3, 0.4, 0): distance to (1,0,0) is sqrt(0.49+0.16)
    tot, env, slf = O.clearance(rb, sc, q)
    assert abs(env - (np.sqrt(0.65) - 0.25)) < 1e-15
    assert slf > 1e300 and tot == env
    free, cl = O.check_states(rb, sc, np.array([[0.8, 0.0, 0.0], [0.3, 0.4, 0.0]]))
    assert list(free) == [False, True]


def test_clearance_self_pair():
    # sphere A rides a prismatic-x joint, sphere B a world-parented prismatic-y joint
    rb = H.robot([W.JOINT_PRISM_X, W.JOINT_PRISM_Y], [0, 0], parents=[-1, -1],
                 spheres=[(0, (0, 0, 0), 0.1), (1, (0, 0, 0), 0.15)], pairs=[(0, 1)])
    q = np.array([0.3, 0.4])
    tot, env, slf = O.clearance(rb, H.empty_scene(), q)
    assert abs(slf - (0.5 - 0.25)) < 1e-15 and env > 1e300
    free, _ = O.check_states(rb, H.empty_scene(), np.array([[0.1, 0.1], [0.3, 0.4]]))
    assert list(free) == [False, True]


def test_arm_home_is_self_collision_free():
    for name in ("arm7", "arm8", "dual14"):
        rb = W.ROBOTS[name]()
        q = np.zeros(rb.dof)
        if name == "arm8":
            q[0] = 0.2
        _, _, slf = O.clearance(rb, H.empty_scene(), q)
        assert slf > 0.0, name


def test_arm_folded_back_self_collides():
    rb = W.arm7()
    q = np.zeros(7)
    q[3] = 2.8   # fold the forearm back onto the upper arm
    _, _, slf = O.clearance(rb, H.empty_scene(), q)
    assert slf < 0.0


# ----------------------------------------------------------------- planner

def _free_problem(seed):
    rb = H.no_self(W.arm7())
    rng = np.random.default_rng(seed)
    s = rb.lower + rng.random(7) * (rb.upper - rb.lower)
    g = rb.lower + rng.random(7) * (rb.upper - rb.lower)
    return rb, H.empty_scene(), s, g


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_plan_free_space_first_iteration(seed):
    rb, sc, s, g = _free_problem(seed)
    r = O.plan(rb, sc, s, g, seed=seed + 10, goal_bias=0.0)
    assert r["status"] == 0 and r["iterations"] == 1
    P = r["path"]
    np.testing.assert_array_equal(P[0], s)
    np.testing.assert_array_equal(P[-1], g)
    seg = np.linalg.norm(np.diff(P, axis=0), axis=1)
    assert np.all(seg <= 1.0 + 1e-12)
    D = np.linalg.norm(g - s)
    assert D - 1e-12 <= r["cost"] <= D + 2.0 + 1e-12
    # iteration 0 extends T_a (tie of the sizes): the first step is the steered sample
    is_goal, c_rand = O.sample(rb, seed + 10, 0, 0, 0.0)
    v = c_rand - s
    dist = np.linalg.norm(v)
    want = s + v * min(1.0, 1.0 / dist)
    np.testing.assert_allclose(P[1], want, atol=1e-12)


def test_plan_free_space_goal_bias_straight_line():
    rb, sc, s, g = _free_problem(5)
    r = O.plan(rb, sc, s, g, seed=3, goal_bias=1.0)
    assert r["status"] == 0
    D = np.linalg.norm(g - s)
    assert abs(r["cost"] - D) < 1e-9 * D
    P = r["path"]
    # collinear, evenly spaced by delta except the last step
    u = (g - s) / D
    for k, p in enumerate(P):
        off = p - s
        assert np.linalg.norm(off - (off @ u) * u) < 1e-9
    assert len(P) == int(np.ceil(D / 1.0)) + 1


def test_plan_start_or_goal_in_collision():
    rb = W.arm7()
    sc = H.scene(boxes=[H.aabb([0, 0, 1.13], [0.1, 0.1, 0.1])])
    q0 = np.zeros(7)
    q1 = np.zeros(7)
    q1[1] = 1.5
    assert O.plan(rb, sc, q0, q1)["status"] == 1
    assert O.plan(rb, sc, q1, q0)["status"] == 2


@pytest.mark.parametrize("seed", [1, 2, 3, 4, 5, 6])
def test_plan_maze_matches_graph_reachability(seed):
    n, cell = 6, 0.2
    sc, edges = H.maze(seed, n=n, cell=cell)
    rb = H.point_robot()
    a, b = (0, 0), (n - 1, n - 1)
    s = np.array([(a[0] + 0.5) * cell, (a[1] + 0.5) * cell])
    g = np.array([(b[0] + 0.5) * cell, (b[1] + 0.5) * cell])
    reach = H.maze_reachable(edges, n, a, b)
    r = O.plan(rb, sc, s, g, seed=seed, range=0.2, resolution=0.01, max_iters=4000)
    assert (r["status"] == 0) == reach, (seed, reach, r["status_name"])
    if reach:
        bad, mc = O.revalidate(rb, sc, r["path"], 0.0025)
        assert bad == 0


def test_plan_walled_off_goal_fails():
    n, cell = 6, 0.2
    sc, edges = H.maze(9, n=n, cell=cell, open_frac=1.0, enclose=(n - 1, n - 1))
    assert not H.maze_reachable(edges, n, (0, 0), (n - 1, n - 1))
    rb = H.point_robot()
    s = np.array([0.1, 0.1])
    g = np.array([(n - 0.5) * cell, (n - 0.5) * cell])
    r = O.plan(rb, sc, s, g, seed=1, range=0.2, resolution=0.01, max_iters=1500)
    assert r["status"] == 3 and r["iterations"] == 1500


def _boxes8_problems(k):
    return W.problem_set("boxes8", k, 1, O.accept)


def test_plan_tree_invariants_boxes8():
    for pb in _boxes8_problems(3):
        for seed in (1, 2):
            r = O.plan(pb.robot, pb.scene, pb.q_start, pb.q_goal, seed=seed, want_trees=True, tree_capacity=1 << 14)
            assert r["status"] == 0
            for nodes, par, root in ((r["nodes_a"], r["parent_a"], pb.q_start), (r["nodes_b"], r["parent_b"], pb.q_goal)):
                np.testing.assert_array_equal(nodes[0], root)
                assert par[0] == -1
                idx = np.arange(len(par))
                assert np.all(par[1:] >= 0) and np.all(par[1:] < idx[1:])
                for i in range(1, len(par)):
                    a, b = nodes[par[i]], nodes[i]
                    L = np.linalg.norm(b - a)
                    assert L <= 1.0 + 1e-12
                    m = int(np.ceil(L * 32 - 1e-9))
                    Q = np.array([a + (k / m) * (b - a) for k in range(1, m + 1)])
                    free, _ = O.check_states(pb.robot, pb.scene, Q)
                    assert free.all()
            P = r["path"]
            np.testing.assert_array_equal(P[0], pb.q_start)
            np.testing.assert_array_equal(P[-1], pb.q_goal)
            allnodes = np.concatenate([r["nodes_a"], r["nodes_b"]])
            for p in P:
                assert np.min(np.linalg.norm(allnodes - p, axis=1)) == 0.0
            assert r["cost"] >= np.linalg.norm(pb.q_goal - pb.q_start) - 1e-12
            assert abs(r["cost"] - np.sum(np.linalg.norm(np.diff(P, axis=0), axis=1))) < 1e-9


def test_plan_deterministic_and_seed_dependent():
    pb = _boxes8_problems(1)[0]
    r1 = O.plan(pb.robot, pb.scene, pb.q_start, pb.q_goal, seed=4)
    r2 = O.plan(pb.robot, pb.scene, pb.q_start, pb.q_goal, seed=4)
    r3 = O.plan(pb.robot, pb.scene, pb.q_start, pb.q_goal, seed=5)
    assert r1["cost"] == r2["cost"] and np.array_equal(r1["path"], r2["path"])
    assert r1["cost"] != r3["cost"]


def test_plan_batch_matches_single():
    pbs = _boxes8_problems(3)
    rs = O.plan_batch(pbs, threads=3, seed=2)
    for pb, r in zip(pbs, rs):
        one = O.plan(pb.robot, pb.scene, pb.q_start, pb.q_goal, seed=2)
        assert one["cost"] == r["cost"] and one["iterations"] == r["iterations"]


@pytest.mark.parametrize("D", [0.7, 2.3, 3.61, 5.05])
def test_plan_straight_line_state_counts(D):
    """Free space with goal bias 1: the first extension moves delta toward the goal,
    then the connect covers D - delta in ceil((D - delta)/delta) steps.  Every edge of
    length l is checked at ceil(l / res) states, endpoint included, so the counts
    are fixed in closed form."""
    rb = H.no_self(W.arm7())
    s = np.zeros(7)
    u = np.array([1.0, -2.0, 0.5, 0.0, 1.5, -1.0, 0.25])
    u /= np.linalg.norm(u)
    g = s + D * u
    delta, res = 1.0, 1.0 / 32
    r = O.plan(rb, H.empty_scene(), s, g, seed=1, goal_bias=1.0, range=delta, resolution=res)
    assert r["status"] == 0 and r["iterations"] == 1
    if D <= delta:
        edges, states = 1, int(np.ceil(D / res))
    else:
        rest = D - delta
        n_ext = int(np.ceil(rest / delta))
        last = rest - (n_ext - 1) * delta
        edges = 1 + n_ext
        states = int(round(delta / res)) * n_ext + int(np.ceil(last / res))
    assert r["edges_checked"] == edges
    assert r["edge_states"] == states
    assert r["states_checked"] == states


# ----------------------------------------------------------------- revalidation

def _point_scene_path(obstacle_spheres=(), boxes=(), z0=0.5):
    return H.point_robot(z0=z0, radius=0.001), H.scene(boxes=boxes, spheres=obstacle_spheres)


def test_revalidate_through_a_box_reports_the_analytic_penetration():
    """A straight two-waypoint path through the centre of a box: one bad segment,
    and the deepest state (the box centre, reached at t = 1/2) has clearance
    -(smallest half extent) - r."""
    rb, sc = _point_scene_path(boxes=[H.aabb([0.6, 0.6, 0.5], [0.1, 0.15, 0.5])])
    path = np.array([[0.2, 0.6], [1.0, 0.6]])
    bad, mc = O.revalidate(rb, sc, path, 0.01)       # 80 states, state 40 at the centre
    assert bad == 1
    assert abs(mc - (-0.1 - 0.001)) < 1e-12
    # two segments, only the second crosses the box
    path3 = np.array([[0.2, 0.2], [0.2, 0.6], [1.0, 0.6]])
    bad3, mc3 = O.revalidate(rb, sc, path3, 0.01)
    assert bad3 == 1 and abs(mc3 - (-0.101)) < 1e-12


def test_revalidate_catches_what_the_coarse_resolution_misses():
    """An obstacle sphere of radius 3 mm centred half way between two states of a
    1/32 check: free at 1/32 (the nearest states are 1/64 away), caught at 1/128,
    where a state lands on its centre with clearance -(3 mm + 1 mm)."""
    x0 = 0.1 + 10.5 / 32
    rb, sc = _point_scene_path(obstacle_spheres=[[x0, 0.5, 0.5, 0.003]])
    path = np.array([[0.1, 0.5], [1.1, 0.5]])
    bad_c, mc_c = O.revalidate(rb, sc, path, 1 / 32)
    assert bad_c == 0 and abs(mc_c - (1 / 64 - 0.004)) < 1e-9
    bad_f, mc_f = O.revalidate(rb, sc, path, 1 / 128)
    assert bad_f == 1 and abs(mc_f - (-0.004)) < 1e-9


def test_revalidate_free_path_reports_exact_clearance():
    """A path parallel to a wall at 5 cm: no bad segment, minimum clearance
    5 cm - r at every state."""
    rb, sc = _point_scene_path(boxes=[H.aabb([0.5, 0.8, 0.5], [0.5, 0.05, 0.5])])
    path = np.array([[0.1, 0.7], [0.5, 0.7], [0.9, 0.7]])
    bad, mc = O.revalidate(rb, sc, path, 0.01)
    assert bad == 0
    assert abs(mc - (0.05 - 0.001)) < 1e-12


def test_revalidate_counts_the_first_waypoint_in_the_clearance_only():
    """The first waypoint enters the minimum clearance but not the segment count
    (segments test the states after their first waypoint)."""
    rb, sc = _point_scene_path(obstacle_spheres=[[0.2, 0.5, 0.5, 0.004]])
    path = np.array([[0.2, 0.5], [0.6, 0.5]])
    bad, mc = O.revalidate(rb, sc, path, 0.01)   # the next state is 1 cm on: free
    assert bad == 0
    assert abs(mc - (-0.005)) < 1e-12


def test_philox_batch_equals_single_blocks():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and not l.startswith("#")]
    for r in rows:
        v = [int(x, 16) for x in r]
        out = O.philox_blocks(np.array([v[0:4]] * 3, np.uint32), v[4] | (v[5] << 32))
        assert all([int(x) for x in o] == v[6:10] for o in out)
