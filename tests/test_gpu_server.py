"""The continuous-batching request loop (prrtc_server_*).

* Serial mode: a query's result is bitwise the same alone, in a mix of
  uneven queries, and from the one-shot prrtc_plan.
* Queries that arrive while another is in flight are admitted and finish
  without waiting for it (continuous batching, not a queue).
* Environment updates apply to queries admitted after them only.
* Async mode: every returned path passes the oracle's 4x-finer re-check.
"""
import time

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
def problems():
    return W.problem_set("boxes8", 3, 1, O.accept) + W.problem_set("mixed", 6, 2000, O.accept)


def handles(pb):
    return P.make_robot(pb.robot), P.make_env(pb.scene)


def by_ticket(results):
    return {r["ticket"]: r for r in results}


def collect(srv, completed_total, new, timeout=60.0):
    """Wait until `completed_total` queries have finished, then poll `new` results."""
    srv.wait(completed_total, timeout)
    out = []
    t0 = time.time()
    while len(out) < new and time.time() - t0 < timeout:
        out += srv.poll()
    return out


def test_serial_result_same_alone_in_mix_and_one_shot(problems):
    prm = P.params(mode=P.MODE_SERIAL, tree_capacity=1 << 13, path_capacity=1 << 12, max_iters=20000)
    srv = P.Server(prm, slice_us=100)
    hs = [handles(pb) for pb in problems]
    tgt = problems[0]
    rb, ev = hs[0]
    t_alone = srv.submit(rb, ev, tgt.q_start, tgt.q_goal, seed=5, problem_id=0)
    alone = by_ticket(collect(srv, 1, 1))[t_alone]
    tickets = []
    for k, pb in enumerate(problems[1:], start=1):
        tickets.append(srv.submit(*hs[k], pb.q_start, pb.q_goal, seed=5, problem_id=k))
    t_mix = srv.submit(rb, ev, tgt.q_start, tgt.q_goal, seed=5, problem_id=0)
    res = by_ticket(collect(srv, 2 + len(tickets), 1 + len(tickets)))
    mixed = res[t_mix]
    one_shot = P.prrtc_plan(rb, ev, tgt.q_start, tgt.q_goal, P.params(mode=P.MODE_SERIAL, tree_capacity=1 << 13,
                                                                        path_capacity=1 << 12, max_iters=20000, seed=5))
    for other in (mixed, one_shot):
        assert other["status"] == alone["status"] == P.SOLVED
        np.testing.assert_array_equal(other["path"], alone["path"])
        assert other["iterations"] == alone["iterations"] and other["cost"] == alone["cost"]
    st = srv.stats()
    assert st["completed"] == 2 + len(tickets) and st["slices"] >= 2
    srv.close()


def test_late_query_overlaps_a_long_one():
    n, cell = 6, 0.2
    sc, _ = H.maze(9, n=n, cell=cell, open_frac=1.0, enclose=(n - 1, n - 1))
    prm = P.params(range=F32(0.2), resolution=F32(0.01), max_iters=400000, tree_capacity=1 << 13,
                   path_capacity=1 << 12)
    srv = P.Server(prm, slice_us=200)
    rb, ev = P.make_robot(H.point_robot()), P.make_env(sc)
    t_long = srv.submit(rb, ev, np.array([0.1, 0.1], np.float32), np.array([1.1, 1.1], np.float32), seed=1)
    time.sleep(0.02)
    t_short = srv.submit(rb, ev, np.array([0.1, 0.1], np.float32), np.array([0.1, 0.3], np.float32), seed=2)
    res = by_ticket(collect(srv, 2, 2, timeout=120))
    short, long_ = res[t_short], res[t_long]
    assert short["status"] == P.SOLVED and long_["status"] == P.NO_SOLUTION
    assert short["latency_ms"] < long_["latency_ms"]
    # the short query was admitted while the long one was running and did not wait for it
    assert short["queue_ms"] < 50.0
    srv.close()


def test_env_update_applies_to_later_admissions():
    robot = H.no_self(W.arm7())
    env = P.make_env(H.scene(spheres=[[2.0, 2.0, 2.0, 0.1]]))
    rb = P.make_robot(robot)
    srv = P.Server(P.params(mode=P.MODE_SERIAL, tree_capacity=1 << 12, path_capacity=1 << 10, max_iters=2000),
                   slice_us=100)
    q0 = np.zeros(7, np.float32)
    q1 = np.full(7, 0.4, np.float32)
    a = srv.submit(rb, env, q0, q1, seed=1)
    ra = by_ticket(collect(srv, 1, 1))[a]
    assert ra["status"] == P.SOLVED
    # move the sphere onto the straight arm: the start is now in collision
    env.update([0], P.obstacles_from_scene(H.scene(spheres=[[0.0, 0.0, 0.8, 0.1]])))
    b = srv.submit(rb, env, q0, q1, seed=1)
    rb_ = by_ticket(collect(srv, 2, 1))[b]
    assert rb_["status"] == P.START_IN_COLLISION
    srv.close()


def test_async_burst_paths_revalidate(problems):
    srv = P.Server(P.params(max_iters=20000, tree_capacity=1 << 13, path_capacity=1 << 12), slice_us=300)
    hs = [handles(pb) for pb in problems]
    tickets = {}
    for rep in range(3):
        for k, pb in enumerate(problems):
            tickets[srv.submit(*hs[k], pb.q_start, pb.q_goal, seed=10 + rep, problem_id=k)] = pb
    res = collect(srv, len(tickets), len(tickets), timeout=120)
    assert len(res) == len(tickets)
    g_items = []
    for r in res:
        pb = tickets[r["ticket"]]
        assert r["status"] in (P.SOLVED, P.NO_SOLUTION)
        if r["status"] == P.SOLVED:
            g_items.append((pb.robot, pb.scene, r["path"], None))
            np.testing.assert_array_equal(r["path"][0], pb.q_start.astype(np.float32))
            np.testing.assert_array_equal(r["path"][-1], pb.q_goal.astype(np.float32))
    # re-checked at 4x resolution, flagged at the rate of the oracle's paths for the same queries
    o_items = []
    for rep in range(3):
        orc = O.plan_batch(problems, seed=10 + rep, problem_ids=list(range(len(problems))), range=1.0,
                           resolution=F32(1 / 32), goal_bias=F32(0.05), max_iters=20000, tree_capacity=1 << 13,
                           path_capacity=1 << 12)
        o_items += [(pb.robot, pb.scene, o["path"], None) for pb, o in zip(problems, orc) if o["status"] == 0]
    H.assert_same_revalidation_rate(H.revalidation_counts(g_items, F32(1 / 32) / 4),
                                    H.revalidation_counts(o_items, F32(1 / 32) / 4), "server burst")
    assert sum(r["status"] == P.SOLVED for r in res) >= len(res) // 2
    srv.close()


def test_server_rejects_bad_config():
    with pytest.raises(P.PrrtcError):
        P.Server(P.params(), slice_us=1)
    with pytest.raises(P.PrrtcError):
        P.Server(P.params(), memory_budget_bytes=1000)
