"""Edge cases of the planning and checking entry points on the GPU: non-finite
inputs, degenerate problems, the wall-clock budget, size limits and empty calls.
Each expectation is the oracle's where the oracle defines one, else the error
contract of include/prrtc.h."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_06757_gb300 import prrtc as P
from paper_2503_06757_gb300 import workload as W
from tests import helpers as H

pytestmark = pytest.mark.gpu

F32 = lambda x: float(np.float32(x))


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2503_06757_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def boxes8():
    return W.problem_set("boxes8", 1, 1, O.accept)[0]


@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf])
def test_non_finite_endpoints_rejected(boxes8, bad):
    rb, ev = P.make_robot(boxes8.robot), P.make_env(boxes8.scene)
    q = boxes8.q_start.astype(np.float32).copy()
    q[3] = bad
    for s, g in ((q, boxes8.q_goal), (boxes8.q_start, q)):
        with pytest.raises(P.PrrtcError) as e:
            P.prrtc_plan(rb, ev, s, g, P.params())
        assert e.value.code == P.ERR_INVALID_ARG


def test_start_equals_goal_matches_oracle(boxes8):
    rb, ev = P.make_robot(boxes8.robot), P.make_env(boxes8.scene)
    q = boxes8.q_start.astype(np.float32)
    g = P.prrtc_plan(rb, ev, q, q, P.params(seed=1, mode=P.MODE_SERIAL, tree_capacity=1024))
    o = O.plan(boxes8.robot, boxes8.scene, q.astype(np.float64), q.astype(np.float64), seed=1, tree_capacity=1024,
               range=1.0, resolution=F32(1 / 32), goal_bias=F32(0.05))
    assert g["status"] == o["status"] == P.SOLVED
    assert g["iterations"] == o["iterations"]
    assert g["n"] == o["path_n"]
    np.testing.assert_allclose(g["path"], o["path"], atol=1e-4)
    np.testing.assert_array_equal(g["path"][0], q)
    np.testing.assert_array_equal(g["path"][-1], q)


def test_time_limit_on_unsolvable_problem():
    """A goal sealed in a box: the device budget ends the search with PRRTC_TIME_LIMIT."""
    n, cell = 6, 0.2
    sc, _ = H.maze(9, n=n, cell=cell, open_frac=1.0, enclose=(n - 1, n - 1))
    rb = H.point_robot()
    s = np.array([0.1, 0.1], np.float32)
    g = np.array([(n - 0.5) * cell, (n - 0.5) * cell], np.float32)
    r = P.prrtc_plan(P.make_robot(rb), P.make_env(sc), s, g,
                     P.params(range=0.2, resolution=0.01, max_iters=10_000_000, time_limit_s=0.002))
    assert r["status"] == P.TIME_LIMIT
    assert r["iterations"] > 0


def test_obstacle_count_limit():
    sph = [[0.0, 0.0, 5.0 + 0.01 * k, 0.001] for k in range(1024)]
    env = P.make_env(H.scene(spheres=sph))
    assert env.info() == (0, 0, 0, 1024)
    rb = W.arm7()
    h = P.make_robot(rb)
    Q = W.candidates(rb, 5, 1, 64).astype(np.float32)
    got = P.prrtc_check_states(h, env, Q)
    free, cl = O.check_states(rb, H.scene(spheres=sph), Q.astype(np.float64))
    clear = np.abs(cl) > 1e-5
    np.testing.assert_array_equal(got[clear], free[clear])
    with pytest.raises(P.PrrtcError) as e:
        P.make_env(H.scene(spheres=sph + [[0.0, 0.0, 20.0, 0.001]]))
    assert e.value.code == P.ERR_INVALID_ARG


def test_dof_limit():
    d = 17
    types = [W.JOINT_REV_Z] * d
    with pytest.raises(P.PrrtcError) as e:
        P.make_robot(H.robot(types, [0.1] * d, spheres=[(0, (0.0, 0.0, 0.0), 0.05)]))
    assert e.value.code == P.ERR_INVALID_ARG


def test_sixteen_dof_chain_checks_against_oracle():
    d = 16
    types = [W.JOINT_REV_Z if j % 2 == 0 else W.JOINT_REV_Y for j in range(d)]
    spheres = [(j, (0.0, 0.0, -0.03), 0.02) for j in range(d)]
    pairs = [(i, j) for i in range(d) for j in range(i + 3, d)]
    rb = H.robot(types, [0.06] * d, lower=[-1.5] * d, upper=[1.5] * d, spheres=spheres, pairs=pairs)
    h = P.make_robot(rb)
    assert h.info()["dpad"] == 16
    sc = W.scene_random_boxes(7)
    ev = P.make_env(sc)
    Q = W.candidates(rb, 11, 2, 500).astype(np.float32)
    got = P.prrtc_check_states(h, ev, Q)
    free, cl = O.check_states(rb, sc, Q.astype(np.float64))
    clear = np.abs(cl) > 1e-5
    np.testing.assert_array_equal(got[clear], free[clear])
    assert 0.02 < free.mean() < 0.98


def test_empty_calls(boxes8):
    rb, ev = P.make_robot(boxes8.robot), P.make_env(boxes8.scene)
    assert P.prrtc_check_states(rb, ev, np.zeros((0, 7), np.float32)).shape == (0,)
    with pytest.raises(P.PrrtcError) as e:
        P.prrtc_plan_batch([], P.params())
    assert e.value.code == P.ERR_INVALID_ARG


@pytest.mark.parametrize("mode", [P.MODE_SERIAL, P.MODE_ASYNC, P.MODE_LOCKSTEP])
def test_bounded_device_wait_gives_up_and_the_next_call_works(boxes8, mode):
    """Failure detection without a GPU fault: the test hook makes the path
    extraction's bounded wait spin on a flag that nothing sets.  The wait must
    give up after its poll limit, the problem and the call must report
    PRRTC_ERR_TIMEOUT, and the next call on the same handles must plan as if
    nothing had happened (serial mode: the same path as a clean call)."""
    rb, ev = P.make_robot(boxes8.robot), P.make_env(boxes8.scene)
    kw = dict(seed=4, mode=mode, workers=4, tree_capacity=1 << 14)
    clean = P.prrtc_plan(rb, ev, boxes8.q_start, boxes8.q_goal, P.params(**kw))
    assert clean["status"] == P.SOLVED
    with pytest.raises(P.PrrtcError) as e:
        P.prrtc_plan(rb, ev, boxes8.q_start, boxes8.q_goal, P.params(debug_wait_polls=2000, **kw))
    assert e.value.code == P.ERR_TIMEOUT
    again = P.prrtc_plan(rb, ev, boxes8.q_start, boxes8.q_goal, P.params(**kw))
    assert again["status"] == P.SOLVED
    if mode != P.MODE_ASYNC:
        np.testing.assert_array_equal(again["path"], clean["path"])
        assert again["iterations"] == clean["iterations"]
    # a batch: every solved problem reports the timeout, the call fails, the next batch works
    items = [(rb, ev, boxes8.q_start, boxes8.q_goal, s, 0) for s in (1, 2, 3)]
    with pytest.raises(P.PrrtcError) as e:
        P.prrtc_plan_batch(items, P.params(debug_wait_polls=100, **kw))
    assert e.value.code == P.ERR_TIMEOUT
    assert all(r["status"] == P.SOLVED for r in P.prrtc_plan_batch(items, P.params(**kw)))
