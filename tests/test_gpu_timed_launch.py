"""Parity at full size in the launch configuration the benchmark times: the 200
cubby-shelf problems (7-DoF arm, 50 obstacles each) in one batched async launch
of 304 blocks x 4 worker warps, the shape the autotuner picks for this batch.

Async mode is nondeterministic (Sec. III: concurrent workers on shared trees),
so the checks are on outputs the oracle can verify one by one:

* every tree: the roots are the start and goal, parents precede their
  children, and every edge is at most delta long;
* sampled tree edges: every state at the planning resolution is collision-free
  for the FP64 oracle (outside the 1e-5 m band);
* every returned path starts at q_start, ends at q_goal and takes steps of at
  most delta; re-checked by the oracle at 4x finer resolution, its segments
  are flagged at the rate of the oracle's own paths on the same problems;
* success against the serial oracle on the same problems and keys (1 pp).
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
KEYS = (1, 2, 3)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2503_06757_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def shelf200():
    from paper_2503_06757_gb300.accept import device_accept
    return W.problem_set("shelf", 200, 1000, device_accept())


def _edge_states(a, b):
    """The states k = 1..N of edge a -> b at the planning resolution (Alg. 2)."""
    a, b = a.astype(np.float64), b.astype(np.float64)
    m = max(1, int(np.ceil(np.float32(np.linalg.norm(b - a)) / np.float32(RES))))
    return np.array([a + (k / m) * (b - a) for k in range(1, m + 1)])


def test_timed_launch_matches_the_oracle_on_sampled_outputs(shelf200):
    rb = P.make_robot(shelf200[0].robot)
    envs = [P.make_env(pb.scene) for pb in shelf200]
    items = [(rb, envs[k], pb.q_start.astype(np.float32), pb.q_goal.astype(np.float32), 1, k)
             for k, pb in enumerate(shelf200)]
    batch = P.PlanBatch(items)
    prm = P.params(blocks=304, warps_per_block=4)
    rng = np.random.default_rng(7)
    g_paths, g_ok, o_ok, n = [], 0, 0, 0
    o_items = []
    edges_checked = 0
    for key in KEYS:
        batch.set_seeds([key] * len(items))
        out = batch.run(prm)
        st = P.prrtc_last_launch_stats()
        assert st["grid"] == 304 and st["block_threads"] == 128
        for k, pb in enumerate(shelf200):
            n += 1
            if out["status"][k] == P.SOLVED:
                g_ok += 1
                path = out.path(k)
                assert np.array_equal(path[0], pb.q_start.astype(np.float32))
                assert np.array_equal(path[-1], pb.q_goal.astype(np.float32))
                steps = np.linalg.norm(np.diff(path.astype(np.float64), axis=0), axis=1)
                assert np.all(steps <= RANGE * (1 + 1e-5)), (key, k, steps.max())
                g_paths.append((pb.robot, pb.scene, path, None))
        # trees of 20 problems of this launch, 8 sampled edges per tree
        for k in rng.choice(len(shelf200), 20, replace=False):
            pb = shelf200[k]
            for t, root in ((0, pb.q_start), (1, pb.q_goal)):
                nodes, par = P.prrtc_debug_tree(int(k), t, pb.robot.dof)
                assert np.all(np.isfinite(nodes))
                np.testing.assert_array_equal(nodes[0], root.astype(np.float32))
                assert par[0] == -1
                assert np.all(par[1:] >= 0) and np.all(par[1:] < np.arange(1, len(par)))
                L = np.linalg.norm(nodes[1:].astype(np.float64) - nodes[par[1:]], axis=1)
                assert np.all(L <= RANGE * (1 + 1e-5))
                if len(par) < 2:
                    continue
                for i in rng.choice(np.arange(1, len(par)), min(8, len(par) - 1), replace=False):
                    _, cl = O.check_states(pb.robot, pb.scene, _edge_states(nodes[par[i]], nodes[i]))
                    assert np.all(cl >= -BAND), (key, int(k), t, int(i), cl.min())
                    edges_checked += 1
        rs = O.plan_batch(shelf200, seed=key, problem_ids=list(range(len(shelf200))), range=RANGE,
                          resolution=RES, goal_bias=BIAS)
        for pb, r in zip(shelf200, rs):
            if r["status"] == 0:
                o_ok += 1
                o_items.append((pb.robot, pb.scene, r["path"], None))
    assert edges_checked >= 300
    H.assert_same_revalidation_rate(H.revalidation_counts(g_paths, RES / 4), H.revalidation_counts(o_items, RES / 4),
                                    "shelf-200 timed launch x 3 keys")
    print(f"timed launch: success {g_ok}/{n}; serial oracle {o_ok}/{n}; {edges_checked} tree edges re-checked")
    assert abs(g_ok - o_ok) / n <= 0.01
