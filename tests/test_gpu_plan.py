"""Parity of the CUDA planner (prrtc_plan / prrtc_plan_batch) with the FP64 oracle.

* Serial mode runs Alg. 1 in iteration order on one warp; it must build the
  same trees and return the same path as the serial oracle wherever the
  oracle met no ambiguous decision (a clearance inside 1e-5 m, a near tie in
  the nearest-neighbour scan, a ceil() argument next to an integer).
* Async mode (many warps over shared trees, Sec. III) is nondeterministic:
  every returned path must start at q_start, end at q_goal and take steps of
  at most delta; re-checked by the oracle at 4x finer resolution, its segments
  must be flagged at the rate of the oracle's own paths on the same problems
  (discrete edge checking lets both miss thin contacts); every tree edge must
  be collision-free at the planning resolution.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_06757_gb300 import prrtc as P
from paper_2503_06757_gb300 import workload as W
from tests import helpers as H

pytestmark = pytest.mark.gpu

F32 = lambda x: float(np.float32(x))
RANGE, RES, BIAS = 1.0, F32(1 / 32), F32(0.05)
BAND = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2503_06757_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def boxes8_problems():
    return W.problem_set("boxes8", 6, 1, O.accept)


def gpu_plan(pb, seed, **kw):
    rb, ev = P.make_robot(pb.robot), P.make_env(pb.scene)
    prm = P.params(seed=seed, **kw)
    return P.prrtc_plan(rb, ev, pb.q_start, pb.q_goal, prm)


def oracle_plan(pb, seed, **kw):
    kw.setdefault("range", RANGE)
    kw.setdefault("resolution", RES)
    kw.setdefault("goal_bias", BIAS)
    return O.plan(pb.robot, pb.scene, pb.q_start.astype(np.float32).astype(np.float64),
                  pb.q_goal.astype(np.float32).astype(np.float64), seed=seed, want_trees=True, **kw)


def assert_path_valid(pb, r, delta=RANGE):
    P_ = r["path"].astype(np.float64)
    assert r["status"] == P.SOLVED
    np.testing.assert_array_equal(r["path"][0], pb.q_start.astype(np.float32))
    np.testing.assert_array_equal(r["path"][-1], pb.q_goal.astype(np.float32))
    seg = np.linalg.norm(np.diff(P_, axis=0), axis=1)
    assert np.all(seg <= delta * (1 + 1e-5)), seg.max()
    assert abs(r["cost"] - seg.sum()) <= 1e-4 * max(1.0, seg.sum())


# ------------------------------------------------------------------ serial lockstep parity

@pytest.mark.parametrize("k", range(6))
@pytest.mark.parametrize("seed", [1, 2])
def test_serial_mode_matches_oracle(boxes8_problems, k, seed):
    pb = boxes8_problems[k]
    g = gpu_plan(pb, seed, mode=P.MODE_SERIAL, tree_capacity=1 << 14)
    o = oracle_plan(pb, seed, tree_capacity=1 << 14)
    amb = o["first_amb_iter"]
    if amb != -1 and amb < o["iterations"]:
        pytest.skip(f"oracle met an ambiguous decision at iteration {amb} (kind {o['first_amb_kind']})")
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


def test_serial_mode_unambiguous_cases_exist(boxes8_problems):
    """The lockstep comparison above must not be vacuous."""
    clean = 0
    for pb in boxes8_problems:
        for seed in (1, 2):
            o = oracle_plan(pb, seed, tree_capacity=1 << 14)
            clean += o["first_amb_iter"] == -1 or o["first_amb_iter"] >= o["iterations"]
    assert clean >= 6


def test_serial_batch_equals_serial_alone(boxes8_problems):
    """Each problem's result is the same alone and in a batch (serial mode: bitwise)."""
    probs = [(P.make_robot(pb.robot), P.make_env(pb.scene), pb.q_start, pb.q_goal, 3, k)
             for k, pb in enumerate(boxes8_problems)]
    prm = P.params(mode=P.MODE_SERIAL, tree_capacity=1 << 14)
    batch = P.prrtc_plan_batch(probs, prm)
    for k, pr in enumerate(probs):
        alone = P.prrtc_plan_batch([pr], prm)[0]
        assert alone["status"] == batch[k]["status"]
        np.testing.assert_array_equal(alone["path"], batch[k]["path"])
        assert alone["iterations"] == batch[k]["iterations"]


def test_batch_paths_come_back_with_the_results():
    """A batch copies the first 32 rows of every path back with its results; a
    longer path takes the gather after the results are read.  Either way each
    problem's path equals the one it gets alone (serial mode: bitwise)."""
    robot = H.point_robot()
    rb, ev = P.make_robot(robot), P.make_env(H.empty_scene())
    s = np.array([0.1, 0.1], np.float32)
    prm = P.params(mode=P.MODE_SERIAL, range=F32(0.02), resolution=F32(0.01), goal_bias=1.0, max_iters=200)
    short = [(rb, ev, s, np.array([0.15, 0.12], np.float32), 1, k) for k in range(3)]
    long_ = short + [(rb, ev, s, np.array([1.1, 1.1], np.float32), 1, 3)]
    for items, want_gather in ((short, False), (long_, True)):
        batch = P.prrtc_plan_batch(items, prm)
        st = P.prrtc_last_launch_stats()
        assert st["kernels"] == (5 if want_gather else 4), st["kernels"]
        rows = [len(r["path"]) for r in batch]
        assert (max(rows) > 32) == want_gather, rows
        for k, it in enumerate(items):
            alone = P.prrtc_plan_batch([it], prm)[0]
            assert alone["status"] == batch[k]["status"] == P.SOLVED
            np.testing.assert_array_equal(alone["path"], batch[k]["path"])


def test_lean_planner_instance_serves_only_plain_batches(boxes8_problems):
    """The lean planner instance (no learned draw, Halton, dynamic domain, distance
    fields, oriented boxes or one-stage links in its code) is launched only for batches that need none of
    them, and plans exactly as the full instance: a zero-ratio mixture puts the
    same problems on the full instance without changing a sample (serial mode,
    bitwise)."""
    pbs = boxes8_problems[:3]
    rbs = [P.make_robot(pb.robot) for pb in pbs]
    evs = [P.make_env(pb.scene) for pb in pbs]
    items = [(rbs[k], evs[k], pb.q_start, pb.q_goal, 3, k) for k, pb in enumerate(pbs)]
    prm = P.params(mode=P.MODE_SERIAL, tree_capacity=1 << 14)
    lean = P.prrtc_plan_batch(items, prm)
    assert P.prrtc_last_launch_stats()["lean_kernel"] == 1
    dof = pbs[0].robot.dof
    zero_mix = np.zeros(8 + 16 * dof, np.float32)
    full = P.prrtc_plan_batch([it + (zero_mix,) for it in items], prm)
    assert P.prrtc_last_launch_stats()["lean_kernel"] == 0
    for a, b in zip(lean, full):
        assert a["status"] == b["status"] and a["iterations"] == b["iterations"]
        np.testing.assert_array_equal(a["path"], b["path"])
    # each feature the lean instance leaves out puts the batch on the full one
    P.prrtc_plan_batch(items, P.params(mode=P.MODE_SERIAL, tree_capacity=1 << 14, sampler=P.SAMPLER_HALTON))
    assert P.prrtc_last_launch_stats()["lean_kernel"] == 0
    P.prrtc_plan_batch(items, P.params(mode=P.MODE_SERIAL, tree_capacity=1 << 14, dd_radius=5.0))
    assert P.prrtc_last_launch_stats()["lean_kernel"] == 0
    rbs[0].set_two_stage(False)
    P.prrtc_plan_batch(items, prm)
    assert P.prrtc_last_launch_stats()["lean_kernel"] == 0
    rbs[0].set_two_stage(True)
    c, sn = np.cos(0.5), np.sin(0.5)
    turned = H.scene(boxes=[np.concatenate([[0.5, 0.5, 1.5], [0.05, 0.05, 0.05], [c, -sn, 0, sn, c, 0, 0, 0, 1]])])
    P.prrtc_plan_batch([(rbs[0], P.make_env(turned), pbs[0].q_start, pbs[0].q_goal, 3, 0)] + items[1:], prm)
    assert P.prrtc_last_launch_stats()["lean_kernel"] == 0
    empty = P.make_env(H.empty_scene())
    P.prrtc_plan_batch([(rbs[0], empty, pbs[0].q_start, pbs[0].q_goal, 3, 0)] + items[1:], prm)
    assert P.prrtc_last_launch_stats()["lean_kernel"] == 0
    P.prrtc_plan_batch(items, prm)
    assert P.prrtc_last_launch_stats()["lean_kernel"] == 1


def test_plan_batch_object_equals_list_call(boxes8_problems):
    """PlanBatch (marshalled once, run many times, results as columns) returns what
    prrtc_plan_batch returns, run after run (serial mode: bitwise)."""
    probs = [(P.make_robot(pb.robot), P.make_env(pb.scene), pb.q_start, pb.q_goal, 5, k)
             for k, pb in enumerate(boxes8_problems)]
    prm = P.params(mode=P.MODE_SERIAL, tree_capacity=1 << 14)
    ref = P.prrtc_plan_batch(probs, prm)
    batch = P.PlanBatch(probs)
    for _ in range(2):
        out = batch.run(prm)
        for k, r in enumerate(ref):
            for name in ("status", "iterations", "cost", "nodes_a", "nodes_b", "edge_states", "verdict_states"):
                assert out[name][k] == r[name], (k, name)
            np.testing.assert_array_equal(out.path(k), r["path"])
    batch.set_seeds([6] * len(probs))
    other = batch.run(prm)
    assert any(other["iterations"][k] != ref[k]["iterations"] for k in range(len(probs)))


# ------------------------------------------------------------------ async mode

@pytest.mark.parametrize("seed", [1, 2, 3])
def test_async_paths_revalidate(boxes8_problems, seed):
    g_items, o_items = [], []
    for pb in boxes8_problems:
        r = gpu_plan(pb, seed)
        assert_path_valid(pb, r)
        g_items.append((pb.robot, pb.scene, r["path"], None))
        o = oracle_plan(pb, seed)
        assert o["status"] == 0
        o_items.append((pb.robot, pb.scene, o["path"], None))
    H.assert_same_revalidation_rate(H.revalidation_counts(g_items, RES / 4), H.revalidation_counts(o_items, RES / 4),
                                    f"boxes8, key {seed}")


def test_async_tree_invariants(boxes8_problems):
    pb = boxes8_problems[0]
    r = gpu_plan(pb, 7, goal_bias=0.0, max_iters=400)  # no goal bias: trees grow before they meet
    rng = np.random.default_rng(0)
    for t, root in ((0, pb.q_start), (1, pb.q_goal)):
        nodes, par = P.prrtc_debug_tree(0, t, pb.robot.dof)
        assert np.all(np.isfinite(nodes))
        np.testing.assert_array_equal(nodes[0], root.astype(np.float32))
        assert par[0] == -1
        assert np.all(par[1:] >= 0) and np.all(par[1:] < np.arange(1, len(par)))
        L = np.linalg.norm(nodes[1:] - nodes[par[1:]], axis=1)
        assert np.all(L <= RANGE * (1 + 1e-5))
        for i in rng.choice(np.arange(1, len(par)), min(60, len(par) - 1), replace=False):
            a, b = nodes[par[i]].astype(np.float64), nodes[i].astype(np.float64)
            m = max(1, int(np.ceil(np.float32(np.linalg.norm(b - a)) / np.float32(RES))))
            Q = np.array([a + (k / m) * (b - a) for k in range(1, m + 1)])
            _, cl = O.check_states(pb.robot, pb.scene, Q)
            assert np.all(cl >= -BAND), (t, i, cl.min())
    assert r["status"] in (P.SOLVED, P.NO_SOLUTION)


def test_async_success_matches_oracle_on_boxes8_keys(boxes8_problems):
    pb = boxes8_problems[1]
    g_ok = o_ok = 0
    for seed in range(1, 21):
        g_ok += gpu_plan(pb, seed)["status"] == P.SOLVED
        o_ok += oracle_plan(pb, seed)["status"] == 0
    assert g_ok == o_ok == 20


# ------------------------------------------------------------------ special cases

def test_free_space_solves_immediately():
    robot = H.no_self(W.arm7())
    rb, ev = P.make_robot(robot), P.make_env(H.empty_scene())
    s = np.zeros(7, np.float32)
    g = np.full(7, 0.5, np.float32)
    r = P.prrtc_plan(rb, ev, s, g, P.params(goal_bias=1.0, mode=P.MODE_SERIAL))
    assert r["status"] == P.SOLVED and r["iterations"] == 1
    assert abs(r["cost"] - np.linalg.norm(g - s)) < 1e-5


def test_start_goal_in_collision():
    robot = W.arm7()
    sc = H.scene(boxes=[H.aabb([0, 0, 1.13], [0.1, 0.1, 0.1])])
    rb, ev = P.make_robot(robot), P.make_env(sc)
    q0 = np.zeros(7, np.float32)
    q1 = np.zeros(7, np.float32)
    q1[1] = 1.5
    assert P.prrtc_plan(rb, ev, q0, q1)["status"] == P.START_IN_COLLISION
    assert P.prrtc_plan(rb, ev, q1, q0)["status"] == P.GOAL_IN_COLLISION


@pytest.mark.parametrize("mode", [P.MODE_SERIAL, P.MODE_ASYNC])
@pytest.mark.parametrize("seed", [1, 2, 3, 4, 5, 6])
def test_maze_reachability(mode, seed):
    n, cell = 6, 0.2
    sc, edges = H.maze(seed, n=n, cell=cell)
    robot = H.point_robot()
    s = np.array([0.1, 0.1], np.float32)
    g = np.array([(n - 0.5) * cell, (n - 0.5) * cell], np.float32)
    reach = H.maze_reachable(edges, n, (0, 0), (n - 1, n - 1))
    rb, ev = P.make_robot(robot), P.make_env(sc)
    r = P.prrtc_plan(rb, ev, s, g, P.params(seed=seed, range=F32(0.2), resolution=F32(0.01), max_iters=4000,
                                            mode=mode))
    assert (r["status"] == P.SOLVED) == reach, (seed, reach, r["status"])
    if reach:
        pb = W.Problem(robot, sc, s.astype(np.float64), g.astype(np.float64), seed)
        assert_path_valid(pb, r, delta=F32(0.2))
        # checked at 1 cm, a segment may graze a wall corner between two states,
        # which the re-check at 2.5 mm reports; the oracle's own path of the same
        # maze is held to the same re-check
        o = O.plan(robot, sc, s.astype(np.float64), g.astype(np.float64), seed=seed, range=F32(0.2),
                   resolution=F32(0.01), max_iters=4000)
        assert o["status"] == 0
        H.assert_same_revalidation_rate(H.revalidation_counts([(robot, sc, r["path"], None)], F32(0.01) / 4),
                                        H.revalidation_counts([(robot, sc, o["path"], None)], F32(0.01) / 4),
                                        f"maze {seed}")


def test_walled_off_goal_no_solution():
    n, cell = 6, 0.2
    sc, _ = H.maze(9, n=n, cell=cell, open_frac=1.0, enclose=(n - 1, n - 1))
    rb, ev = P.make_robot(H.point_robot()), P.make_env(sc)
    r = P.prrtc_plan(rb, ev, np.array([0.1, 0.1], np.float32), np.array([1.1, 1.1], np.float32),
                     P.params(range=F32(0.2), resolution=F32(0.01), max_iters=1500))
    assert r["status"] == P.NO_SOLUTION and r["iterations"] == 1500


def test_budget_and_capacity_edges(boxes8_problems):
    pb = boxes8_problems[2]
    r = gpu_plan(pb, 1, max_iters=1, goal_bias=0.0)
    assert r["iterations"] == 1 and r["status"] in (P.SOLVED, P.NO_SOLUTION)
    r = gpu_plan(pb, 1, tree_capacity=2)
    assert r["nodes_a"] <= 2 and r["nodes_b"] <= 2
    r = gpu_plan(pb, 1, path_capacity=2)
    assert r["status"] in (P.PATH_OVERFLOW, P.SOLVED)
    if r["status"] == P.PATH_OVERFLOW:
        assert r["n"] > 2


def test_invalid_params_rejected(boxes8_problems):
    pb = boxes8_problems[0]
    for bad in (dict(range=0.0), dict(resolution=-1.0), dict(goal_bias=2.0), dict(max_iters=0), dict(mode=7)):
        with pytest.raises(P.PrrtcError) as e:
            gpu_plan(pb, 1, **bad)
        assert e.value.code == P.ERR_INVALID_ARG


# ------------------------------------------------------------------ batches

def test_mixed_dof_batch_one_launch():
    probs = W.problem_set("mixed", 9, 2000, O.accept)
    items = [(P.make_robot(p.robot), P.make_env(p.scene), p.q_start, p.q_goal, 5, k) for k, p in enumerate(probs)]
    res = P.prrtc_plan_batch(items, P.params())
    st = P.prrtc_last_launch_stats()
    assert st["problems"] == 9
    orc = O.plan_batch(probs, seed=5, problem_ids=list(range(len(probs))), range=RANGE, resolution=RES,
                       goal_bias=BIAS)
    g_items, o_items = [], []
    for p, r, o in zip(probs, res, orc):
        assert r["status"] in (P.SOLVED, P.NO_SOLUTION)
        if r["status"] == P.SOLVED:
            assert_path_valid(p, r)
            g_items.append((p.robot, p.scene, r["path"], None))
        if o["status"] == 0:
            o_items.append((p.robot, p.scene, o["path"], None))
    H.assert_same_revalidation_rate(H.revalidation_counts(g_items, RES / 4), H.revalidation_counts(o_items, RES / 4),
                                    "mixed 9")
    # some dense 8/14-DoF scenes are not solved within the budget (the oracle does
    # not solve them either); the 7-DoF ones and most others are
    assert sum(r["status"] == P.SOLVED for r in res) >= 5


# ------------------------------------------------------------------ graph replay and autotuning

def test_graph_replay_is_exact_and_recaptures_on_shape_change(boxes8_problems):
    pb = boxes8_problems[3]
    rb, ev = P.make_robot(pb.robot), P.make_env(pb.scene)
    prm = P.params(seed=4, mode=P.MODE_SERIAL, tree_capacity=1 << 14)
    first = P.prrtc_plan(rb, ev, pb.q_start, pb.q_goal, prm)          # captures
    again = P.prrtc_plan(rb, ev, pb.q_start, pb.q_goal, prm)          # replays
    items = [(P.make_robot(q.robot), P.make_env(q.scene), q.q_start, q.q_goal, 4, k) for k, q in enumerate(boxes8_problems)]
    P.prrtc_plan_batch(items, prm)                                     # another shape
    third = P.prrtc_plan(rb, ev, pb.q_start, pb.q_goal, prm)           # re-captures
    for r in (again, third):
        assert r["status"] == first["status"] == P.SOLVED
        np.testing.assert_array_equal(r["path"], first["path"])
        assert r["iterations"] == first["iterations"]
    # a single-problem path comes back without the gather kernel
    assert P.prrtc_last_launch_stats()["kernels"] == 3


def test_autotune_picks_a_candidate_and_later_calls_use_it(boxes8_problems):
    items = [(P.make_robot(q.robot), P.make_env(q.scene), q.q_start, q.q_goal, 1, k) for k, q in enumerate(boxes8_problems)]
    best, ms = P.prrtc_autotune(items, P.params(), trials=2)
    assert best.warps_per_block in (2, 3, 4, 6, 8) and best.blocks >= 1 and ms > 0
    assert best.obstacle_tile in (32, 64) and best.expansions in (1, 2, 4, 8)
    res = P.prrtc_plan_batch(items, P.params())
    st = P.prrtc_last_launch_stats()
    assert st["grid"] == best.blocks and st["block_threads"] == 32 * best.warps_per_block
    assert all(r["status"] == P.SOLVED for r in res)


@pytest.mark.parametrize("seed", [1, 2])
def test_obstacle_tile_does_not_change_serial_plans(seed):
    """Two primitives per lane in the first stage test the same spheres against
    the same primitives: serial plans are bitwise those of one per lane, also on
    scenes with more than 64 primitives of a type."""
    probs = W.problem_set("mixed", 6, 2000, O.accept, n_obstacles=120)
    items = [(P.make_robot(q.robot), P.make_env(q.scene), q.q_start, q.q_goal, seed, k) for k, q in enumerate(probs)]
    kw = dict(mode=P.MODE_SERIAL, tree_capacity=1 << 14, max_iters=3000)
    a = P.prrtc_plan_batch(items, P.params(obstacle_tile=32, **kw))
    b = P.prrtc_plan_batch(items, P.params(obstacle_tile=64, **kw))
    for x, y in zip(a, b):
        for name in ("status", "iterations", "nodes_a", "nodes_b", "edge_states", "verdict_states"):
            assert x[name] == y[name], name
        np.testing.assert_array_equal(x["path"], y["path"])


def test_expansions_per_claim(boxes8_problems):
    """Claims of several iteration ids at once: async plans stay valid, the count
    of iterations run stays within the budget, and serial mode ignores it."""
    items = [(P.make_robot(q.robot), P.make_env(q.scene), q.q_start, q.q_goal, 3, k) for k, q in enumerate(boxes8_problems)]
    for e in (1, 4, 16):
        for r, pb in zip(P.prrtc_plan_batch(items, P.params(expansions=e)), boxes8_problems):
            assert_path_valid(pb, r)
    small = P.prrtc_plan_batch(items, P.params(expansions=8, max_iters=5, goal_bias=0.0))
    assert all(r["iterations"] <= 5 for r in small)
    s1 = P.prrtc_plan_batch(items, P.params(mode=P.MODE_SERIAL, expansions=1))
    s8 = P.prrtc_plan_batch(items, P.params(mode=P.MODE_SERIAL, expansions=8))
    for x, y in zip(s1, s8):
        assert x["iterations"] == y["iterations"]
        np.testing.assert_array_equal(x["path"], y["path"])
    for bad in (dict(expansions=65), dict(expansions=-1), dict(obstacle_tile=48)):
        with pytest.raises(P.PrrtcError) as e:
            P.prrtc_plan_batch(items, P.params(**bad))
        assert e.value.code == P.ERR_INVALID_ARG


def test_serial_batch_success_and_mean_cost_match_oracle():
    """Over 64 cubby-shelf problems (one launch, one worker per problem), success rate
    within 1 percentage point and mean path cost within 2% of the serial oracle's.
    Problems whose runs part at an ambiguous decision still count: the bound is on
    the set, not on each problem."""
    probs = W.problem_set("shelf", 64, 1000, O.accept)
    robots = {}
    items = []
    for k, pb in enumerate(probs):
        rb = robots.setdefault(pb.robot.name, P.make_robot(pb.robot))
        items.append((rb, P.make_env(pb.scene), pb.q_start, pb.q_goal, 1, k))
    g = P.prrtc_plan_batch(items, P.params(mode=P.MODE_SERIAL, tree_capacity=1 << 15, max_iters=20000))
    o = O.plan_batch(probs, seeds=[1] * len(probs), problem_ids=list(range(len(probs))), range=1.0,
                     resolution=RES, goal_bias=BIAS, tree_capacity=1 << 15, max_iters=20000)
    g_ok = np.array([r["status"] == P.SOLVED for r in g])
    o_ok = np.array([r["status"] == 0 for r in o])
    assert abs(g_ok.mean() - o_ok.mean()) <= 0.01 + 1e-9
    both = g_ok & o_ok
    g_cost = np.mean([r["cost"] for r, b in zip(g, both) if b])
    o_cost = np.mean([r["cost"] for r, b in zip(o, both) if b])
    assert abs(g_cost - o_cost) <= 0.02 * o_cost, (g_cost, o_cost)
    # and most problems are decided identically end to end
    same = sum(abs(a["cost"] - b["cost"]) <= 1e-4 * b["cost"] for a, b, ok in zip(g, o, both) if ok)
    assert same >= 0.5 * both.sum()


def test_mixed_600_one_launch_at_full_size():
    """The mixed-DoF configuration at full size: 600 problems (7/8/14-DoF in turn,
    10-120 obstacles) in one persistent launch.  Inputs are accepted by the device
    checker (the oracle's acceptance would take minutes); outputs are checked
    against the oracle on a sample: every solved path's endpoints, its cost against
    the straight line, and 60 paths revalidated at 4x the resolution."""
    from paper_2503_06757_gb300.accept import device_accept
    probs = W.problem_set("mixed", 600, 2000, device_accept())
    assert len(probs) == 600
    robots, items = {}, []
    for k, p in enumerate(probs):
        if p.robot.name not in robots:
            robots[p.robot.name] = P.make_robot(p.robot)
        items.append((robots[p.robot.name], P.make_env(p.scene), p.q_start, p.q_goal, 1, k))
    res = P.prrtc_plan_batch(items, P.params())
    st = P.prrtc_last_launch_stats()
    assert st["problems"] == 600
    solved = [k for k, r in enumerate(res) if r["status"] == P.SOLVED]
    assert all(r["status"] in (P.SOLVED, P.NO_SOLUTION) for r in res)
    by_dof = {d: [k for k, p in enumerate(probs) if p.robot.dof == d] for d in (7, 8, 14)}
    for d, ks in by_dof.items():
        assert len(ks) == 200
        # measured 178 / 166 / 144 of 200 (7 / 8 / 14-DoF); dense scenes leave the rest
        # unsolved within the budget
        assert sum(res[k]["status"] == P.SOLVED for k in ks) >= 110, d
    for k in solved:
        path, p = res[k]["path"], probs[k]
        np.testing.assert_array_equal(path[0], p.q_start.astype(np.float32))
        np.testing.assert_array_equal(path[-1], p.q_goal.astype(np.float32))
        assert res[k]["cost"] >= np.linalg.norm(p.q_goal - p.q_start) - 1e-4
    rng = np.random.default_rng(600)
    pick = sorted(int(k) for k in rng.choice(solved, 60, replace=False))
    for k in pick:
        assert_path_valid(probs[k], res[k])
    orc = O.plan_batch([probs[k] for k in pick], seed=1, problem_ids=pick, range=RANGE, resolution=RES,
                       goal_bias=BIAS)
    g_items = [(probs[k].robot, probs[k].scene, res[k]["path"], None) for k in pick]
    o_items = [(probs[k].robot, probs[k].scene, o["path"], None) for k, o in zip(pick, orc) if o["status"] == 0]
    H.assert_same_revalidation_rate(H.revalidation_counts(g_items, RES / 4), H.revalidation_counts(o_items, RES / 4),
                                    "mixed 600, 60 sampled")
