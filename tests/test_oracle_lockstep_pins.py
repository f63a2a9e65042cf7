"""Pins of the oracle's lockstep form of the concurrent planner (Sec. III).

In a lockstep round of B workers, worker b runs iteration r B + b of Alg. 1
(sampling, nearest neighbour, pEXTEND, greedy connect) against the trees as
they stood when the round began and holds its new rows back; the rows are
appended in worker order at the end of the round, and the connected worker
that checked the fewest edges (ties: lowest b) wins.  The pins below come from
outside that code:
  * one worker per round is the serial Alg. 1, computed by the oracle's
    separate serial loop: identical trees, path, iterations and edge counts;
  * in a scene without obstacles every worker of round 0 extends the start
    root and connects straight to the goal root, so the trees, the winner, the
    path and its cost follow in closed form from the sampler's draws;
  * a walled-off goal spends exactly max_iters iterations, also when the
    budget is not a multiple of B;
  * tree capacity: rows past the capacity are dropped in worker order and a
    worker whose rows did not all fit cannot win (closed form again);
  * every tree built with B > 1 keeps the invariants of a valid RRT forest.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_06757_gb300 import workload as W
from tests import helpers as H

RANGE, RES, BIAS = 1.0, float(np.float32(1 / 32)), float(np.float32(0.05))


def plan(rb, sc, qs, qg, **kw):
    kw.setdefault("range", RANGE)
    kw.setdefault("resolution", RES)
    kw.setdefault("goal_bias", BIAS)
    return O.plan(rb, sc, np.asarray(qs, np.float64), np.asarray(qg, np.float64), want_trees=True, **kw)


@pytest.fixture(scope="module")
def boxes8():
    return W.problem_set("boxes8", 3, 1, O.accept)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_one_worker_rounds_are_the_serial_planner(boxes8, seed):
    for pb in boxes8:
        s = plan(pb.robot, pb.scene, pb.q_start, pb.q_goal, seed=seed, workers=0)
        l1 = plan(pb.robot, pb.scene, pb.q_start, pb.q_goal, seed=seed, workers=1)
        for k in ("status", "iterations", "n_a", "n_b", "join_a", "join_b", "path_n", "edges_checked",
                  "states_checked", "edge_states", "first_amb_iter"):
            assert s[k] == l1[k], k
        for k in ("nodes_a", "parent_a", "nodes_b", "parent_b", "path"):
            np.testing.assert_array_equal(s[k], l1[k])
        assert s["cost"] == l1["cost"]


def test_one_worker_rounds_are_the_serial_planner_in_a_maze():
    sc, _ = H.maze(5, n=6)
    rb = H.point_robot()
    qs, qg = [0.1, 0.1], [1.1, 1.1]
    for seed in (1, 2):
        s = plan(rb, sc, qs, qg, seed=seed, workers=0, range=0.3, resolution=0.01)
        l1 = plan(rb, sc, qs, qg, seed=seed, workers=1, range=0.3, resolution=0.01)
        assert (s["status"], s["iterations"], s["n_a"], s["n_b"]) == (l1["status"], l1["iterations"], l1["n_a"], l1["n_b"])
        np.testing.assert_array_equal(s["parent_a"], l1["parent_a"])
        np.testing.assert_array_equal(s["path"], l1["path"])


def free_round(rb, qs, qg, seed, B, cap=1 << 16):
    """Round 0 of B workers without obstacles, written out from the sampler's
    draws: every worker extends T_a (both trees hold one node, ties go to T_a)
    from its root toward its sample and connects straight to the goal root."""
    qs, qg = np.asarray(qs, float), np.asarray(qg, float)
    rows, conn, edges = [], [], []
    for b in range(B):
        goal, q = O.sample(rb, seed, 0, b, BIAS)
        c_rand = qg if goal else q
        d = np.linalg.norm(c_rand - qs)
        if d == 0.0:
            rows.append([]), conn.append(False), edges.append(0)
            continue
        c_new = qs + (c_rand - qs) * (RANGE / d) if d > RANGE else c_rand.copy()
        D = np.linalg.norm(qg - c_new)
        n_ext = math.ceil(D / RANGE) if D > 0 else 0
        steps = [c_new + (i * RANGE / D) * (qg - c_new) for i in range(1, n_ext)] + ([qg.copy()] if n_ext else [])
        want = [c_new] + steps
        held = want[: max(0, cap - 1)]            # a worker stops once its own rows fill the tree
        rows.append(held)
        conn.append(len(held) == len(want))
        edges.append(1 + n_ext if len(held) == len(want) else None)
    nodes, parents, winner, join = [qs], [-1], -1, -1
    for b in range(B):
        prev = 0
        all_in = True
        for r in rows[b]:
            if len(nodes) >= cap:
                all_in = False
                break
            nodes.append(r)
            parents.append(prev)
            prev = len(nodes) - 1
        if conn[b] and all_in and (winner < 0 or edges[b] < edges[winner]):
            winner, join = b, prev
    return np.array(nodes), np.array(parents), winner, join


@pytest.mark.parametrize("B", [4, 7])
@pytest.mark.parametrize("seed", range(1, 13))
def test_obstacle_free_round_in_closed_form(B, seed):
    rb = H.no_self(W.arm7())
    qs = np.array([0.3, -0.5, 0.2, 1.0, -0.7, 0.4, 0.0])
    qg = np.array([-2.2, 1.4, -1.9, -1.2, 2.1, -1.5, 2.0])
    nodes, parents, w, join = free_round(rb, qs, qg, seed, B)
    o = plan(rb, H.empty_scene(), qs, qg, seed=seed, workers=B)
    assert o["status"] == 0
    assert o["iterations"] == B
    assert (o["n_a"], o["n_b"]) == (len(nodes), 1)
    np.testing.assert_array_equal(o["parent_a"], parents)
    np.testing.assert_allclose(o["nodes_a"], nodes, rtol=0, atol=1e-12)
    assert o["join_a"] == join and o["join_b"] == 0
    chain = [join]
    while parents[chain[-1]] >= 0:
        chain.append(parents[chain[-1]])
    path = nodes[chain[::-1]]  # T_a's chain ends on the goal root's configuration
    np.testing.assert_allclose(o["path"], path, atol=1e-12)
    cost = float(np.linalg.norm(np.diff(path, axis=0), axis=1).sum())
    assert abs(o["cost"] - cost) <= 1e-12 * cost
    # the winner checked the fewest edges: its connect is the shortest of the round
    assert w >= 0


@pytest.mark.parametrize("cap", [3, 4, 6, 9])
def test_capacity_drops_rows_in_worker_order(cap):
    rb = H.no_self(W.arm7())
    qs = np.array([0.3, -0.5, 0.2, 1.0, -0.7, 0.4, 0.0])
    qg = np.array([-2.2, 1.4, -1.9, -1.2, 2.1, -1.5, 2.0])
    B = 5
    nodes, parents, w, join = free_round(rb, qs, qg, 3, B, cap=cap)
    o = plan(rb, H.empty_scene(), qs, qg, seed=3, workers=B, tree_capacity=cap, max_iters=B)
    assert o["n_a"] == len(nodes)
    np.testing.assert_array_equal(o["parent_a"], parents)
    if w >= 0:
        assert o["status"] == 0 and o["join_a"] == join
    else:
        assert o["status"] == 3  # no worker fitted its whole connect: budget spent


@pytest.mark.parametrize("B,max_iters", [(4, 30), (3, 31), (8, 8), (16, 5)])
def test_walled_off_goal_spends_the_budget(B, max_iters):
    sc, _ = H.maze(3, n=4, enclose=(3, 3))
    rb = H.point_robot()
    o = plan(rb, sc, [0.1, 0.1], [0.7, 0.7], seed=1, workers=B, range=0.3, resolution=0.01,
             max_iters=max_iters)
    assert o["status"] == 3
    assert o["iterations"] == max_iters


@pytest.mark.parametrize("B", [2, 8, 32])
def test_lockstep_trees_are_valid_forests(boxes8, B):
    for k, pb in enumerate(boxes8):
        o = plan(pb.robot, pb.scene, pb.q_start, pb.q_goal, seed=4, workers=B, tree_capacity=1 << 14)
        assert o["status"] == 0
        assert o["iterations"] % B == 0 or o["iterations"] == 50000
        for nodes, par, root in ((o["nodes_a"], o["parent_a"], pb.q_start), (o["nodes_b"], o["parent_b"], pb.q_goal)):
            np.testing.assert_array_equal(nodes[0], root)
            assert par[0] == -1
            assert np.all((par[1:] >= 0) & (par[1:] < np.arange(1, len(par))))
            # every tree edge is collision-free at the planning resolution and at most delta long
            seg = np.linalg.norm(nodes[1:] - nodes[par[1:]], axis=1)
            assert np.all(seg <= RANGE * (1 + 1e-12))
            for i in np.random.default_rng(k).choice(np.arange(1, len(par)), size=min(40, len(par) - 1), replace=False):
                a, b = nodes[par[i]], nodes[i]
                n = max(1, math.ceil(np.linalg.norm(b - a) / RES))
                Q = a + (np.arange(1, n + 1)[:, None] / n) * (b - a)
                free, _ = O.check_states(pb.robot, pb.scene, Q)
                assert free.all()
        path = o["path"]
        np.testing.assert_array_equal(path[0], pb.q_start)
        np.testing.assert_array_equal(path[-1], pb.q_goal)
        assert o["cost"] >= np.linalg.norm(pb.q_goal - pb.q_start) - 1e-12
