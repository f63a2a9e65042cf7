"""Parity of the CUDA collision checker (prrtc_check_states) with the FP64 oracle.

The oracle evaluates the GPU's exact FP32 configurations upcast to FP64.
Verdicts must agree bit for bit wherever the oracle clearance is outside the
1e-5 m band; every disagreement is listed with its clearance.  Sphere centres
must agree within 1e-5 m.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_06757_gb300 import prrtc as P
from paper_2503_06757_gb300 import workload as W
from tests import helpers as H

pytestmark = pytest.mark.gpu

BAND = 1e-5
CENTRE_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2503_06757_gb300 import build
    build.build()


def _states(robot, n, seed):
    st = W.Stream(seed, 5)
    u = st.uniform(n * robot.dof).reshape(n, robot.dof)
    return (robot.lower + u * (robot.upper - robot.lower)).astype(np.float32)


def compare(robot, scene, Q, check_centres=True, max_centre_rows=3000):
    rb, ev = P.make_robot(robot), P.make_env(scene)
    valid, sph = P.prrtc_check_states(rb, ev, Q, want_spheres=True)
    Qd = Q.astype(np.float64)
    free, cl = O.check_states(robot, scene, Qd)
    dis = np.nonzero(valid != free)[0]
    report = [(int(i), float(cl[i]), bool(valid[i]), bool(free[i])) for i in dis]
    assert all(abs(c) <= BAND for _, c, _, _ in report), f"disagreements outside the band: {report[:20]}"
    if check_centres and len(Q):
        rows = np.arange(len(Q)) if len(Q) <= max_centre_rows else np.linspace(0, len(Q) - 1, max_centre_rows).astype(int)
        worst = 0.0
        for i in rows:
            cen, _ = O.fk(robot, Qd[i])
            worst = max(worst, float(np.max(np.abs(sph[i, :, :3] - cen))))
            np.testing.assert_array_equal(sph[i, :, 3], robot.sphere_radius.astype(np.float32))
        assert worst <= CENTRE_TOL, worst
    return dict(n=len(Q), free=int(free.sum()), disagreements=report)


SCENES = {
    "boxes8": lambda: (W.arm7(), W.scene_random_boxes(1)),
    "shelf": lambda: (W.arm7(), W.scene_shelf(1000)),
    "mixed_arm8": lambda: (W.arm8(), W.scene_mixed(2001, 60)),
    "mixed_dual14": lambda: (W.dual14(), W.scene_mixed(2002, 120, bases=W.robot_bases(W.dual14()))),
}


@pytest.mark.parametrize("name", sorted(SCENES))
def test_verdicts_and_centres_match_oracle(name):
    robot, scene = SCENES[name]()
    Q = _states(robot, 4099, 17)  # several blocks and a ragged last warp
    r = compare(robot, scene, Q)
    assert 0 < r["free"] < r["n"], r["free"]  # both verdicts occur


def test_oriented_boxes_and_cylinders():
    rng = np.random.default_rng(4)
    boxes, cyls = [], []
    for _ in range(12):
        q = rng.normal(size=4)
        q /= np.linalg.norm(q)
        w, x, y, z = q
        R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                      [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                      [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
        c = rng.uniform([-0.6, -0.6, 0.3], [0.6, 0.6, 1.1])
        h = rng.uniform(0.03, 0.15, 3)
        boxes.append(np.concatenate([c, h, R.reshape(9)]))
    for _ in range(8):
        a = rng.normal(size=3)
        a /= np.linalg.norm(a)
        cyls.append(np.concatenate([rng.uniform([-0.6, -0.6, 0.3], [0.6, 0.6, 1.1]), a, [0.05, 0.15]]))
    scene = H.scene(boxes=np.asarray(boxes).astype(np.float32), cylinders=np.asarray(cyls).astype(np.float32))
    robot = W.arm7()
    env = P.make_env(scene)
    assert env.info() == (0, 12, 8, 0)
    compare(robot, scene, _states(robot, 2048, 3))


def test_empty_scene_and_no_self_pairs():
    robot = H.no_self(W.arm7())
    Q = _states(robot, 300, 9)
    valid = P.prrtc_check_states(P.make_robot(robot), P.make_env(H.empty_scene()), Q)
    assert valid.all()
    # with self-collision on, folded configurations are rejected exactly as the oracle says
    compare(W.arm7(), H.empty_scene(), Q)


@pytest.mark.parametrize("n", [0, 1, 31, 32, 33])
def test_small_and_ragged_sizes(n):
    robot, scene = SCENES["boxes8"]()
    Q = _states(robot, max(n, 1), 5)[:n]
    if n == 0:
        valid = P.prrtc_check_states(P.make_robot(robot), P.make_env(scene), np.zeros((0, 7), np.float32))
        assert valid.shape == (0,)
    else:
        compare(robot, scene, Q)


def test_point_robot_prismatic_joints():
    sc, _ = H.maze(3)
    robot = H.point_robot()
    Q = _states(robot, 5000, 2)
    compare(robot, sc, Q)


def test_merged_sphere_counts():
    r7 = P.make_robot(W.arm7()).info()
    assert r7 == dict(dof=7, n_spheres=19, n_pairs=75, dpad=8)
    r14 = P.make_robot(W.dual14()).info()
    assert r14["n_spheres"] == 38 and r14["n_pairs"] == 2 * 75 + 19 * 19 and r14["dpad"] == 16


def test_full_size_sampled():
    """10^6 states on the cubby shelf (the benchmark's launch shape): a sample of
    rows against the oracle, and the all-free property of the free-state set."""
    robot, scene = SCENES["shelf"]()
    rb, ev = P.make_robot(robot), P.make_env(scene)
    Q = _states(robot, 1_000_000, 23)
    valid = P.prrtc_check_states(rb, ev, Q)
    idx = np.random.default_rng(0).choice(len(Q), 3000, replace=False)
    free, cl = O.check_states(robot, scene, Q[idx].astype(np.float64))
    bad = [(int(i), float(c)) for i, f, c, v in zip(idx, free, cl, valid[idx]) if f != v and abs(c) > BAND]
    assert not bad, bad
    # the collision-free subset re-checked is all free (no state depends on its neighbours)
    F = Q[valid]
    assert P.prrtc_check_states(rb, ev, F).all()


def test_device_pointer_variant_matches_host():
    torch = pytest.importorskip("torch")
    robot, scene = SCENES["mixed_arm8"]()
    rb, ev = P.make_robot(robot), P.make_env(scene)
    Q = _states(robot, 10000, 8)
    host = P.prrtc_check_states(rb, ev, Q)
    q = torch.from_numpy(Q).cuda()
    v = torch.zeros(len(Q), dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream()
    P.prrtc_check_states_device(rb, ev, q.data_ptr(), len(Q), v.data_ptr(), 0, s.cuda_stream)
    s.synchronize()
    np.testing.assert_array_equal(v.cpu().numpy().astype(bool), host)


def test_env_update_moves_obstacle():
    robot = W.arm7()
    scene = H.scene(spheres=[[2.0, 2.0, 2.0, 0.1]])
    env = P.make_env(scene)
    rb = P.make_robot(robot)
    q = np.zeros((1, 7), np.float32)
    assert P.prrtc_check_states(rb, env, q)[0]
    moved = H.scene(spheres=[[0.0, 0.0, 1.1, 0.1]])
    env.update([0], P.obstacles_from_scene(moved))
    assert not P.prrtc_check_states(rb, env, q)[0]
    with pytest.raises(P.PrrtcError):
        env.update([0], P.obstacles_from_scene(H.scene(boxes=[H.aabb([0, 0, 0], [0.1, 0.1, 0.1])])))


def test_invalid_inputs_rejected():
    with pytest.raises(P.PrrtcError) as e:
        P.make_env(H.scene(spheres=[[0, 0, 0, -1.0]]))
    assert e.value.code == P.ERR_INVALID_ARG
    bad = H.robot([W.JOINT_REV_Z, W.JOINT_REV_Z], [0.1, 0.1], parents=[-1, -1 + 0])
    bad.joint_parent[1] = 5
    with pytest.raises(P.PrrtcError):
        P.make_robot(bad)
