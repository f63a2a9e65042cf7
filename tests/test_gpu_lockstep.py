"""The concurrent planner (Sec. III) against the oracle: lockstep rounds exactly,
the async mode statistically.

* Lockstep mode (PRRTC_MODE_LOCKSTEP, B workers per round): the GPU must build
  the oracle's lockstep trees and return its path wherever the oracle met no
  ambiguous decision, for B = 4 and B = 32, whatever the warps per block.
* Async mode has no fixed schedule.  Its statistics are compared with the
  oracle's lockstep form at the same number of concurrent workers: one block
  of 8 warps per problem (8 workers, no other problem's blocks joining) against
  B = 8 rounds, over 200 cubby-shelf problems and 5 Philox keys.  Success rate
  must agree within 1 percentage point and mean initial-path cost within 2%,
  and the oracle's re-check at 4x resolution must flag the GPU's path segments
  at the rate it flags its own.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_06757_gb300 import prrtc as P
from paper_2503_06757_gb300 import workload as W

pytestmark = pytest.mark.gpu

F32 = lambda x: float(np.float32(x))
RANGE, RES, BIAS = 1.0, F32(1 / 32), F32(0.05)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2503_06757_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def boxes8_problems():
    return W.problem_set("boxes8", 6, 1, O.accept)


def gpu_plan(pb, seed, **kw):
    rb, ev = P.make_robot(pb.robot), P.make_env(pb.scene)
    return P.prrtc_plan(rb, ev, pb.q_start, pb.q_goal, P.params(seed=seed, **kw))


def oracle_plan(pb, seed, **kw):
    return O.plan(pb.robot, pb.scene, pb.q_start.astype(np.float32).astype(np.float64),
                  pb.q_goal.astype(np.float32).astype(np.float64), seed=seed, want_trees=True,
                  range=RANGE, resolution=RES, goal_bias=BIAS, **kw)


def ambiguous(o):
    return o["first_amb_iter"] != -1 and o["first_amb_iter"] < o["iterations"]


@pytest.mark.parametrize("B", [4, 32])
@pytest.mark.parametrize("k", range(6))
@pytest.mark.parametrize("seed", [1, 2])
def test_lockstep_mode_matches_oracle(boxes8_problems, B, k, seed):
    pb = boxes8_problems[k]
    o = oracle_plan(pb, seed, workers=B, tree_capacity=1 << 14)
    if ambiguous(o):
        pytest.skip(f"oracle met an ambiguous decision at iteration {o['first_amb_iter']} (kind {o['first_amb_kind']})")
    g = gpu_plan(pb, seed, mode=P.MODE_LOCKSTEP, workers=B, tree_capacity=1 << 14)
    assert g["status"] == o["status"] == 0
    assert g["iterations"] == o["iterations"]
    assert (g["nodes_a"], g["nodes_b"]) == (o["n_a"], o["n_b"])
    for t, (nodes, par) in enumerate(((o["nodes_a"], o["parent_a"]), (o["nodes_b"], o["parent_b"]))):
        gn, gp = P.prrtc_debug_tree(0, t, pb.robot.dof)
        np.testing.assert_array_equal(gp, par)
        np.testing.assert_allclose(gn, nodes, atol=1e-4)
    np.testing.assert_allclose(g["path"], o["path"], atol=1e-4)
    assert abs(g["cost"] - o["cost"]) <= 1e-4 * o["cost"]
    assert g["edges_checked"] == o["edges_checked"]
    assert g["edge_states"] == o["edge_states"]


@pytest.mark.parametrize("B", [4, 32])
def test_lockstep_unambiguous_cases_exist(boxes8_problems, B):
    """The exact comparison above must not be vacuous."""
    clean = sum(not ambiguous(oracle_plan(pb, seed, workers=B, tree_capacity=1 << 14))
                for pb in boxes8_problems for seed in (1, 2))
    assert clean >= 5


def test_lockstep_one_worker_is_serial_mode(boxes8_problems):
    for k, pb in enumerate(boxes8_problems):
        s = gpu_plan(pb, 3, mode=P.MODE_SERIAL, tree_capacity=1 << 14)
        l1 = gpu_plan(pb, 3, mode=P.MODE_LOCKSTEP, workers=1, tree_capacity=1 << 14)
        for name in ("status", "iterations", "nodes_a", "nodes_b", "edges_checked", "edge_states", "cost"):
            assert s[name] == l1[name], (k, name)
        np.testing.assert_array_equal(s["path"], l1["path"])


def test_lockstep_result_does_not_depend_on_the_launch_shape(boxes8_problems):
    """Virtual worker b runs on warp b % warps: 12 workers on 3, 5 or 12 warps, alone
    or in a batch of six problems, give bitwise the same plans."""
    probs = [(P.make_robot(pb.robot), P.make_env(pb.scene), pb.q_start, pb.q_goal, 7, k)
             for k, pb in enumerate(boxes8_problems)]
    ref = P.prrtc_plan_batch(probs, P.params(mode=P.MODE_LOCKSTEP, workers=12, warps_per_block=3,
                                             tree_capacity=1 << 14))
    for warps in (5, 12):
        out = P.prrtc_plan_batch(probs, P.params(mode=P.MODE_LOCKSTEP, workers=12, warps_per_block=warps,
                                                 tree_capacity=1 << 14))
        for k in range(len(probs)):
            assert out[k]["iterations"] == ref[k]["iterations"]
            np.testing.assert_array_equal(out[k]["path"], ref[k]["path"])
    for k, pr in enumerate(probs):
        alone = P.prrtc_plan_batch([pr], P.params(mode=P.MODE_LOCKSTEP, workers=12, tree_capacity=1 << 14))[0]
        assert alone["iterations"] == ref[k]["iterations"]
        np.testing.assert_array_equal(alone["path"], ref[k]["path"])


def test_lockstep_rejects_bad_worker_counts(boxes8_problems):
    pb = boxes8_problems[0]
    for bad in (0, 1025):
        with pytest.raises(RuntimeError):
            gpu_plan(pb, 1, mode=P.MODE_LOCKSTEP, workers=bad)


@pytest.fixture(scope="module")
def shelf200():
    from paper_2503_06757_gb300.accept import device_accept
    return W.problem_set("shelf", 200, 1000, device_accept())


def test_async_statistics_match_the_lockstep_oracle(shelf200):
    """Async mode with 8 workers per problem against the oracle's B = 8 rounds on
    the same 200 shelf problems and keys: success within 1 pp, mean cost within 2%."""
    keys = (1, 2, 3, 4, 5)
    rb = P.make_robot(shelf200[0].robot)
    envs = [P.make_env(pb.scene) for pb in shelf200]
    prm = P.params(mode=P.MODE_ASYNC, blocks=1, warps_per_block=8)
    g_cost, g_ok, o_cost, o_ok, n = [], 0, [], 0, 0
    g_items, o_items = [], []
    for key in keys:
        for k, pb in enumerate(shelf200):
            r = P.prrtc_plan_batch([(rb, envs[k], pb.q_start.astype(np.float32), pb.q_goal.astype(np.float32),
                                     key, k)], prm)[0]
            n += 1
            if r["status"] == P.SOLVED:
                g_ok += 1
                g_cost.append(r["cost"])
                g_items.append((pb.robot, pb.scene, r["path"], None))
        rs = O.plan_batch(shelf200, seed=key, problem_ids=list(range(len(shelf200))), range=RANGE,
                          resolution=RES, goal_bias=BIAS, workers=8)
        for pb, r in zip(shelf200, rs):
            if r["status"] == 0:
                o_ok += 1
                o_cost.append(r["cost"])
                o_items.append((pb.robot, pb.scene, r["path"], None))
    # every returned path re-checked by the oracle at 4x resolution: the GPU's
    # segments are flagged at the rate of the oracle's own paths
    from tests import helpers as H
    H.assert_same_revalidation_rate(H.revalidation_counts(g_items, RES / 4), H.revalidation_counts(o_items, RES / 4),
                                    "shelf-200 x 5 keys")
    g_mean, o_mean = float(np.mean(g_cost)), float(np.mean(o_cost))
    print(f"async W=8: success {g_ok / n:.4f} cost {g_mean:.4f}; oracle B=8: success {o_ok / n:.4f} "
          f"cost {o_mean:.4f} ({100 * (g_mean / o_mean - 1):+.2f}%)")
    assert abs(g_ok - o_ok) / n <= 0.01
    assert abs(g_mean / o_mean - 1.0) <= 0.02
