"""prrtc_plan_noalloc: planning for callers that cannot allocate device memory
(real-time threads that must not block in an allocator, frameworks that own all
device memory).  Its results must equal those of prrtc_plan, the allocating
entry point, on consecutive calls that share its fixed scratch -- also when the
arm's DoF (row width) and the tree capacity change from one call to the next --
and the calls must leave the device's free memory unchanged.

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


def _same_outcome(a, b):
    assert a["status"] == b["status"]
    assert a["iterations"] == b["iterations"]
    assert (a["nodes_a"], a["nodes_b"]) == (b["nodes_a"], b["nodes_b"])
    if b["status"] == P.SOLVED:
        np.testing.assert_allclose(a["path"], b["path"], atol=TOL)


def test_noalloc_row_width_and_capacity_change_between_calls():
    """14-DoF rows (stride 16) after 7-DoF rows (stride 8) and back, with the tree
    capacity shrinking and growing: each call's setup must clear exactly the rows
    the previous call wrote, whatever their stride."""
    probs = W.problem_set("mixed", 3, 2000, O.accept)   # 7-, 8- and 14-DoF arms in turn
    by_dof = {pb.robot.dof: pb for pb in probs}
    seq = [(14, 4096), (7, 512), (14, 2048), (8, 256), (7, 4096), (14, 1024)]
    for k, (dof, cap) in enumerate(seq):
        pb = by_dof[dof]
        rb, ev = P.make_robot(pb.robot), P.make_env(pb.scene)
        prm = P.params(seed=11 + k, mode=P.MODE_SERIAL, tree_capacity=cap, path_capacity=4096, max_iters=3000)
        ref = P.prrtc_plan(rb, ev, pb.q_start, pb.q_goal, prm)
        got = P.prrtc_plan_noalloc(rb, ev, pb.q_start, pb.q_goal, prm)
        _same_outcome(got, ref)


def test_noalloc_calls_leave_device_memory_unchanged(problems):
    torch = pytest.importorskip("torch")
    pb = problems[0]
    rb, ev = P.make_robot(pb.robot), P.make_env(pb.scene)
    prm = P.params(seed=3, mode=P.MODE_SERIAL, tree_capacity=4096, path_capacity=4096)
    P.prrtc_plan_noalloc(rb, ev, pb.q_start, pb.q_goal, prm)   # the first call does the set-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for seed in range(4, 9):
        prm.seed = seed
        P.prrtc_plan_noalloc(rb, ev, pb.q_start, pb.q_goal, prm)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
