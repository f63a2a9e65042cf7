"""GPU parity of the Halton sampler, dynamic-domain sampling and the two-stage
collision check with the FP64 oracle.

* Two-stage check (Sec. III-A): the bounding spheres contain the fine spheres,
  and the verdicts, sphere centres and serial-mode plans are identical with
  and without the first stage; the oracle (one stage, FP64) agrees outside
  the 1e-5 m band.
* Halton sampler (Sec. IV-A) and dynamic-domain sampling (Sec. III,
  Yershova et al. 2005): serial mode builds the same trees as the serial
  oracle, takes the same iterations and rejects the same samples, wherever
  the oracle met no ambiguous decision.
* Async mode with both on: every path passes the oracle's 4x finer re-check.
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


def oracle_plan(pb, seed, **kw):
    kw.setdefault("range", RANGE)
    kw.setdefault("resolution", RES)
    kw.setdefault("goal_bias", BIAS)
    return O.plan(pb.robot, pb.scene, pb.q_start.astype(np.float32).astype(np.float64),
                  pb.q_goal.astype(np.float32).astype(np.float64), seed=seed, want_trees=True, **kw)


def compare_serial(pb, g, o):
    amb = o["first_amb_iter"]
    if amb != -1 and amb < o["iterations"]:
        pytest.skip(f"oracle met an ambiguous decision at iteration {amb} (kind {o['first_amb_kind']})")
    assert g["status"] == o["status"]
    assert g["iterations"] == o["iterations"]
    assert (g["nodes_a"], g["nodes_b"]) == (o["n_a"], o["n_b"])
    for t, (nodes, par) in enumerate(((o["nodes_a"], o["parent_a"]), (o["nodes_b"], o["parent_b"]))):
        gn, gp = P.prrtc_debug_tree(0, t, pb.robot.dof)
        np.testing.assert_array_equal(gp, par)
        np.testing.assert_allclose(gn, nodes, atol=1e-4)
    if o["status"] == 0:
        np.testing.assert_allclose(g["path"], o["path"], atol=1e-4)
    assert g["edges_checked"] == o["edges_checked"]
    assert g["edge_states"] == o["edge_states"]
    assert g["dd_rejected"] == o["dd_rejected"]


# ------------------------------------------------------------------ two-stage check

@pytest.mark.parametrize("name", ["arm7", "arm8", "dual14"])
def test_bounding_spheres_contain_fine_spheres(name):
    rb = W.ROBOTS[name]()
    b = P.make_robot(rb).bounds().astype(np.float64)
    for f in range(rb.dof):
        idx = np.nonzero(rb.sphere_frame == f)[0]
        rows = np.unique(np.concatenate([rb.sphere_offset[idx], rb.sphere_radius[idx, None]], 1).astype(np.float32),
                         axis=0).astype(np.float64)
        if len(rows) < 2:
            assert b[f, 3] == 0.0
            continue
        reach = np.linalg.norm(rows[:, :3] - b[f, :3], axis=1) + rows[:, 3]
        assert np.all(reach <= b[f, 3] - 0.9e-5), (f, reach.max(), b[f, 3])
        # and not loose: within 2 cm of the tightest enclosing reach
        assert b[f, 3] <= reach.max() + 0.02


def _scene(kind, seed):
    if kind == "shelf":
        return W.scene_shelf(seed)
    return W.scene_mixed(seed, 60)


@pytest.mark.parametrize("name,kind", [("arm7", "shelf"), ("arm8", "mixed"), ("dual14", "mixed"),
                                       ("arm7", "mixed")])
def test_two_stage_verdicts_equal_one_stage_and_oracle(name, kind):
    rb = W.ROBOTS[name]()
    sc = _scene(kind, 4000 + len(name))
    h, ev = P.make_robot(rb), P.make_env(sc)
    Q = W.candidates(rb, 17, 2, 3000).astype(np.float32)
    v2, s2 = P.prrtc_check_states(h, ev, Q, want_spheres=True)
    st2 = P.prrtc_last_launch_stats()
    h.set_two_stage(False)
    v1, s1 = P.prrtc_check_states(h, ev, Q, want_spheres=True)
    st1 = P.prrtc_last_launch_stats()
    h.set_two_stage(True)
    np.testing.assert_array_equal(v2, v1)
    np.testing.assert_array_equal(s2, s1)
    assert 0.02 < v1.mean() < 0.98  # both verdicts occur
    # the first stage replaces most sphere-environment passes
    assert st1["env_tests"] == 0 and sum(st1["prim_tests"]) == 0
    assert st2["sphere_tests"] < st1["sphere_tests"] and st2["env_tests"] > 0
    # the oracle (one stage, FP64) agrees outside the clearance band
    free, cl = O.check_states(rb, sc, Q.astype(np.float64))
    clear = np.abs(cl) > BAND
    np.testing.assert_array_equal(v2[clear], free[clear])


def test_two_stage_on_off_serial_plans_identical(boxes8_problems):
    shelf = W.problem_set("shelf", 2, 1, O.accept)
    second_stage = 0
    for pb in list(boxes8_problems[:3]) + shelf:
        h, ev = P.make_robot(pb.robot), P.make_env(pb.scene)
        prm = P.params(seed=5, mode=P.MODE_SERIAL, tree_capacity=1 << 14, max_iters=4000)
        a = P.prrtc_plan(h, ev, pb.q_start, pb.q_goal, prm)
        h.set_two_stage(False)
        b = P.prrtc_plan(h, ev, pb.q_start, pb.q_goal, prm)
        h.set_two_stage(True)
        assert a["status"] == b["status"] and a["iterations"] == b["iterations"]
        assert (a["nodes_a"], a["nodes_b"]) == (b["nodes_a"], b["nodes_b"])
        np.testing.assert_array_equal(a["path"], b["path"])
        assert a["edge_states"] == b["edge_states"]
        assert sum(b["prim_tests"]) == 0
        second_stage += sum(a["prim_tests"])
    assert second_stage > 0


# ------------------------------------------------------------------ Halton

def test_halton_first_step_free_space():
    rb = H.no_self(W.arm7())
    s = np.zeros(7, np.float32)
    g = np.full(7, 0.4, np.float32)
    h, ev = P.make_robot(rb), P.make_env(H.empty_scene())
    for offset in (0, 17, 1000):
        prm = P.params(seed=3, mode=P.MODE_SERIAL, goal_bias=0.0, sampler=P.SAMPLER_HALTON, halton_offset=offset,
                       tree_capacity=256)
        r = P.prrtc_plan(h, ev, s, g, prm)
        assert r["status"] == P.SOLVED and r["iterations"] == 1
        nodes, _ = P.prrtc_debug_tree(0, 0, 7)
        c_rand = rb.lower + O.halton(1 + offset, 7) * (rb.upper - rb.lower)
        want = c_rand * min(1.0, 1.0 / np.linalg.norm(c_rand))
        np.testing.assert_allclose(nodes[1], want, atol=2e-6)


@pytest.mark.parametrize("k", range(6))
def test_serial_halton_matches_oracle(boxes8_problems, k):
    pb = boxes8_problems[k]
    h, ev = P.make_robot(pb.robot), P.make_env(pb.scene)
    prm = P.params(seed=2, mode=P.MODE_SERIAL, tree_capacity=1 << 14, sampler=P.SAMPLER_HALTON,
                   halton_offset=37 * k)
    g = P.prrtc_plan(h, ev, pb.q_start, pb.q_goal, prm)
    o = oracle_plan(pb, 2, tree_capacity=1 << 14, sampler=O.SAMPLER_HALTON, halton_offset=37 * k)
    compare_serial(pb, g, o)


# ------------------------------------------------------------------ dynamic domain

DD = dict(dd_radius=F32(0.6), dd_alpha=F32(0.05), dd_min_radius=F32(0.3))


@pytest.mark.parametrize("k", range(6))
@pytest.mark.parametrize("seed", [1, 2])
def test_serial_dynamic_domain_matches_oracle(boxes8_problems, k, seed):
    pb = boxes8_problems[k]
    h, ev = P.make_robot(pb.robot), P.make_env(pb.scene)
    prm = P.params(seed=seed, mode=P.MODE_SERIAL, tree_capacity=1 << 14, **DD)
    g = P.prrtc_plan(h, ev, pb.q_start, pb.q_goal, prm)
    o = oracle_plan(pb, seed, tree_capacity=1 << 14, **DD)
    compare_serial(pb, g, o)


def test_serial_dynamic_domain_unambiguous_cases_exist(boxes8_problems):
    clean, rejected = 0, 0
    for pb in boxes8_problems:
        for seed in (1, 2):
            o = oracle_plan(pb, seed, tree_capacity=1 << 14, **DD)
            ok = o["first_amb_iter"] == -1 or o["first_amb_iter"] >= o["iterations"]
            clean += ok
            rejected += o["dd_rejected"] * ok
    assert clean >= 6 and rejected > 0


def _slider():
    rb = H.robot([W.JOINT_PRISM_X], [0.0], bases=[[0.0, 0.0, 0.5]], lower=[0.0], upper=[2.0],
                 spheres=[(0, (0.0, 0.0, 0.0), 0.02)], name="slider")
    wall = H.scene(boxes=[H.aabb([1.1, 0.0, 0.5], [0.1, 0.5, 0.5])])
    return rb, wall, np.array([0.1], np.float32), np.array([1.6], np.float32)


@pytest.mark.parametrize("seed", [4, 5, 6])
def test_serial_dynamic_domain_slider_matches_oracle(seed):
    rb, wall, s, g = _slider()
    kw = dict(range=F32(0.3), resolution=F32(0.01), max_iters=400, tree_capacity=1024, dd_radius=F32(0.05),
              dd_alpha=F32(0.25), dd_min_radius=F32(0.02), goal_bias=BIAS)
    h, ev = P.make_robot(rb), P.make_env(wall)
    r = P.prrtc_plan(h, ev, s, g, P.params(seed=seed, mode=P.MODE_SERIAL, **kw))
    o = O.plan(rb, wall, s.astype(np.float64), g.astype(np.float64), seed=seed, want_trees=True, **kw)
    pb = type("Pb", (), dict(robot=rb))
    assert o["status"] == 3 and o["dd_rejected"] > 0
    compare_serial(pb, r, o)


@pytest.mark.parametrize("seed", [1, 2])
def test_async_halton_dynamic_domain_paths_revalidate(boxes8_problems, seed):
    items = [(P.make_robot(pb.robot), P.make_env(pb.scene), pb.q_start, pb.q_goal, seed, k)
             for k, pb in enumerate(boxes8_problems)]
    prm = P.params(sampler=P.SAMPLER_HALTON, **DD)
    res = P.prrtc_plan_batch(items, prm)
    for pb, r in zip(boxes8_problems, res):
        assert r["status"] == P.SOLVED
        path = r["path"].astype(np.float64)
        np.testing.assert_array_equal(r["path"][0], pb.q_start.astype(np.float32))
        np.testing.assert_array_equal(r["path"][-1], pb.q_goal.astype(np.float32))
        seg = np.linalg.norm(np.diff(path, axis=0), axis=1)
        assert np.all(seg <= RANGE * (1 + 1e-5))
    # the oracle's own paths with the same sampler and dynamic domain set the re-check's rate
    orc = O.plan_batch(boxes8_problems, seed=seed, problem_ids=list(range(len(boxes8_problems))), range=RANGE,
                       resolution=RES, goal_bias=BIAS, sampler=O.SAMPLER_HALTON, **DD)
    H.assert_same_revalidation_rate(
        H.revalidation_counts([(pb.robot, pb.scene, r["path"], None) for pb, r in zip(boxes8_problems, res)], RES / 4),
        H.revalidation_counts([(pb.robot, pb.scene, o["path"], None) for pb, o in zip(boxes8_problems, orc)
                               if o["status"] == 0], RES / 4), f"Halton + dynamic domain, key {seed}")


def test_sampling_params_validated(boxes8_problems):
    pb = boxes8_problems[0]
    h, ev = P.make_robot(pb.robot), P.make_env(pb.scene)
    for bad in (dict(sampler=7), dict(dd_radius=-1.0), dict(dd_radius=0.5, dd_alpha=1.0),
                dict(dd_radius=0.5, dd_min_radius=float("nan"))):
        with pytest.raises(P.PrrtcError) as e:
            P.prrtc_plan(h, ev, pb.q_start, pb.q_goal, P.params(**bad))
        assert e.value.code == P.ERR_INVALID_ARG
