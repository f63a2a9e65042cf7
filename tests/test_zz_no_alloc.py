"""prrtc_plan_noalloc: planning for callers that cannot allocate device memory
(real-time threads, frameworks that own all device memory, code running under
someone else's stream capture).  Its results must equal those of prrtc_plan,
the allocating entry point, on consecutive calls that share its fixed scratch.

Kept in its own file so that it is collected after every other test; it must
pass both alone in a fresh process and after the rest of the suite.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_06757_gb300 import prrtc as P
from paper_2503_06757_gb300 import workload as W
from tests import helpers as H

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def problems():
    from paper_2503_06757_gb300 import build
    build.build()
    return W.problem_set("boxes8", 2, 1, O.accept)


def _same(a, b):
    assert a["status"] == b["status"] == P.SOLVED
    assert a["iterations"] == b["iterations"]
    assert (a["nodes_a"], a["nodes_b"]) == (b["nodes_a"], b["nodes_b"])
    np.testing.assert_allclose(a["path"], b["path"], atol=TOL)
    assert abs(a["cost"] - b["cost"]) <= TOL * max(1.0, b["cost"])


def test_noalloc_matches_plan_on_consecutive_calls(problems):
    # serial mode is deterministic, so both entry points must give the same tree and path
    calls = [(problems[0], 1), (problems[1], 2), (problems[0], 3)]
    for pb, seed in calls:
        rb, ev = P.make_robot(pb.robot), P.make_env(pb.scene)
        prm = P.params(seed=seed, mode=P.MODE_SERIAL, tree_capacity=4096, path_capacity=4096)
        ref = P.prrtc_plan(rb, ev, pb.q_start, pb.q_goal, prm)
        got = P.prrtc_plan_noalloc(rb, ev, pb.q_start, pb.q_goal, prm)
        _same(got, ref)


def test_noalloc_async_paths_valid_twice(problems):
    pb = problems[0]
    rb, ev = P.make_robot(pb.robot), P.make_env(pb.scene)
    prm = P.params(seed=5, tree_capacity=4096, path_capacity=4096)
    res = float(np.float32(1 / 32)) / 4
    o = O.plan(pb.robot, pb.scene, pb.q_start.astype(np.float32).astype(np.float64),
               pb.q_goal.astype(np.float32).astype(np.float64), seed=5, range=1.0,
               resolution=float(np.float32(1 / 32)), goal_bias=float(np.float32(0.05)))
    assert o["status"] == 0
    for _ in range(2):
        r = P.prrtc_plan_noalloc(rb, ev, pb.q_start, pb.q_goal, prm)
        assert r["status"] == P.SOLVED
        np.testing.assert_array_equal(r["path"][0], pb.q_start.astype(np.float32))
        np.testing.assert_array_equal(r["path"][-1], pb.q_goal.astype(np.float32))
        # re-checked at 4x resolution, flagged at the rate of the oracle's own path
        H.assert_same_revalidation_rate(H.revalidation_counts([(pb.robot, pb.scene, r["path"], None)], res),
                                        H.revalidation_counts([(pb.robot, pb.scene, o["path"], None)], res),
                                        "allocation-free call")


def test_noalloc_rejects_sizes_beyond_scratch(problems):
    pb = problems[0]
    rb, ev = P.make_robot(pb.robot), P.make_env(pb.scene)
    for kw in (dict(tree_capacity=4097), dict(path_capacity=1 << 14)):
        with pytest.raises(P.PrrtcError) as e:
            P.prrtc_plan_noalloc(rb, ev, pb.q_start, pb.q_goal, P.params(**dict(dict(tree_capacity=4096,
                                                                                    path_capacity=4096), **kw)))
        assert e.value.code == P.ERR_INVALID_ARG


def test_noalloc_path_overflow_reported(problems):
    pb = problems[1]
    rb, ev = P.make_robot(pb.robot), P.make_env(pb.scene)
    prm = P.params(seed=2, mode=P.MODE_SERIAL, tree_capacity=4096, path_capacity=4096)
    ref = P.prrtc_plan(rb, ev, pb.q_start, pb.q_goal, prm)
    if ref["n"] > 2:
        r = P.prrtc_plan_noalloc(rb, ev, pb.q_start, pb.q_goal, prm, path_rows=2)
        assert r["status"] == P.PATH_OVERFLOW and r["n"] == ref["n"]
