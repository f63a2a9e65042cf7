"""Pins of the oracle's Halton sampler and dynamic-domain sampling.

Halton (the sampler of the paper's experiments, Sec. IV-A): the van der Corput
fractions printed in every textbook treatment for bases 2, 3 and 5, and the
exact stratification of the first b^m points of each prime base.

Dynamic-domain sampling (Yershova et al. 2005, added to Alg. 1 in Sec. III,
radius adaptation of Jaillet et al. 2005): two settings reduce it to the plain
planner (an unbounded radius; a scene without obstacles, where no extension
fails), and a 1-DoF slider pushed against a wall shows the effects that the
method exists for: far samples are rejected, the number of wasted collision
checks drops, and every bounded radius takes one of the values the adaptation
rule allows.
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_06757_gb300 import workload as W
from tests import helpers as H

PRIMES = [2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37, 41, 43, 47, 53]


# ----------------------------------------------------------------- Halton

@pytest.mark.parametrize("dim,expected", [
    (0, ["1/2", "1/4", "3/4", "1/8", "5/8", "3/8", "7/8", "1/16"]),
    (1, ["1/3", "2/3", "1/9", "4/9", "7/9", "2/9", "5/9", "8/9", "1/27"]),
    (2, ["1/5", "2/5", "3/5", "4/5", "1/25", "6/25", "11/25"]),
])
def test_halton_van_der_corput_fractions(dim, expected):
    for i, frac in enumerate(expected, start=1):
        u = O.halton(i, dim + 1)[dim]
        assert u == float(Fraction(frac)), (dim, i, u, frac)


def test_halton_origin_and_dimensions():
    np.testing.assert_array_equal(O.halton(0, 16), np.zeros(16))
    # index 1 has the single digit 1 in every base: 1/p
    np.testing.assert_array_equal(O.halton(1, 16), [1.0 / p for p in PRIMES])


@pytest.mark.parametrize("j", range(16))
def test_halton_stratifies_first_power_of_base(j):
    b = PRIMES[j]
    m = 1
    while b ** (m + 1) <= 3000:
        m += 1
    n = b ** m
    u = np.array([O.halton(i, j + 1)[j] for i in range(n)])
    k = np.round(u * n).astype(int)
    # every point is the correctly rounded grid value k / b^m, one per cell
    assert all(float(ui) == kk / n for ui, kk in zip(u, k))
    assert sorted(k.tolist()) == list(range(n))


def test_plan_halton_first_sample_free_space():
    """With goal bias 0 in free space, iteration 0 steers toward Halton point 1 + offset."""
    rb = H.no_self(W.arm7())
    s = np.zeros(7)
    g = np.full(7, 0.4)
    for offset in (0, 17):
        r = O.plan(rb, H.empty_scene(), s, g, seed=3, goal_bias=0.0, sampler=O.SAMPLER_HALTON,
                   halton_offset=offset, want_trees=True, tree_capacity=256)
        assert r["status"] == 0 and r["iterations"] == 1
        c_rand = rb.lower + O.halton(1 + offset, 7) * (rb.upper - rb.lower)
        v = c_rand - s
        want = s + v * min(1.0, 1.0 / np.linalg.norm(v))
        np.testing.assert_allclose(r["nodes_a"][1], want, atol=1e-12)


def test_plan_halton_does_not_depend_on_seed_without_goal_bias():
    pb = W.problem_set("boxes8", 1, 1, O.accept)[0]
    kw = dict(goal_bias=0.0, sampler=O.SAMPLER_HALTON, max_iters=3000)
    r1 = O.plan(pb.robot, pb.scene, pb.q_start, pb.q_goal, seed=1, **kw)
    r2 = O.plan(pb.robot, pb.scene, pb.q_start, pb.q_goal, seed=99, **kw)
    assert r1["iterations"] == r2["iterations"] and r1["cost"] == r2["cost"]


# ----------------------------------------------------------------- dynamic domain

def _boxes8(k):
    return W.problem_set("boxes8", k, 1, O.accept)


def _same_plan(a, b):
    assert a["status"] == b["status"] and a["iterations"] == b["iterations"]
    assert (a["n_a"], a["n_b"]) == (b["n_a"], b["n_b"])
    np.testing.assert_array_equal(a["nodes_a"], b["nodes_a"])
    np.testing.assert_array_equal(a["parent_b"], b["parent_b"])
    assert a["edges_checked"] == b["edges_checked"]


def test_dynamic_domain_unbounded_radius_is_plain():
    for pb in _boxes8(2):
        plain = O.plan(pb.robot, pb.scene, pb.q_start, pb.q_goal, seed=2, want_trees=True, tree_capacity=1 << 14)
        dd = O.plan(pb.robot, pb.scene, pb.q_start, pb.q_goal, seed=2, want_trees=True, tree_capacity=1 << 14,
                    dd_radius=np.inf, dd_alpha=0.1, dd_min_radius=0.5)
        _same_plan(plain, dd)
        assert dd["dd_rejected"] == 0
        assert np.all(np.isinf(dd["radius_a"])) and np.all(np.isinf(dd["radius_b"]))


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_dynamic_domain_free_space_is_plain(seed):
    rb = H.no_self(W.arm7())
    rng = np.random.default_rng(seed)
    s = rb.lower + rng.random(7) * (rb.upper - rb.lower)
    g = rb.lower + rng.random(7) * (rb.upper - rb.lower)
    kw = dict(seed=seed, goal_bias=0.0, want_trees=True, tree_capacity=4096)
    plain = O.plan(rb, H.empty_scene(), s, g, **kw)
    dd = O.plan(rb, H.empty_scene(), s, g, dd_radius=0.3, dd_alpha=0.2, dd_min_radius=0.1, **kw)
    _same_plan(plain, dd)
    assert dd["dd_rejected"] == 0 and np.all(np.isinf(dd["radius_a"]))


def _slider():
    rb = H.robot([W.JOINT_PRISM_X], [0.0], bases=[[0.0, 0.0, 0.5]], lower=[0.0], upper=[2.0],
                 spheres=[(0, (0.0, 0.0, 0.0), 0.02)], name="slider")
    wall = H.scene(boxes=[H.aabb([1.1, 0.0, 0.5], [0.1, 0.5, 0.5])])
    return rb, wall, np.array([0.1]), np.array([1.6])


def test_dynamic_domain_slider_against_wall():
    rb, wall, s, g = _slider()
    kw = dict(seed=4, range=0.3, resolution=0.01, max_iters=400, want_trees=True, tree_capacity=1024)
    plain = O.plan(rb, wall, s, g, **kw)
    R = 0.05
    dd = O.plan(rb, wall, s, g, dd_radius=R, dd_alpha=0.0, dd_min_radius=R, **kw)
    assert plain["status"] == dd["status"] == 3  # the wall separates start and goal
    # far samples are rejected and fewer edges run into the wall
    assert dd["dd_rejected"] > 0
    assert dd["edges_checked"] < plain["edges_checked"]
    # with alpha = 0 a bounded radius is exactly R, and only nodes next to the wall carry one
    for nodes, rad in ((dd["nodes_a"], dd["radius_a"]), (dd["nodes_b"], dd["radius_b"])):
        bounded = np.isfinite(rad)
        assert bounded.any()
        np.testing.assert_array_equal(rad[bounded], R)
        # the wall occupies [1.0, 1.2]; with the sphere radius the slider is blocked
        # in (0.98, 1.22): a bounded node failed an extension, so it is within one
        # extension range (0.3) of the wall
        x = nodes[bounded, 0]
        assert np.all((x > 0.98 - 0.3) & (x < 1.22 + 0.3)), x
    # every node stays on its side of the wall
    assert np.all(dd["nodes_a"][:, 0] <= 0.98) and np.all(dd["nodes_b"][:, 0] >= 1.22)


def test_dynamic_domain_radius_adaptation_bounds():
    rb, wall, s, g = _slider()
    R, alpha, rmin = 0.2, 0.5, 0.15
    dd = O.plan(rb, wall, s, g, seed=5, range=0.3, resolution=0.01, max_iters=600, want_trees=True,
                tree_capacity=1024, dd_radius=R, dd_alpha=alpha, dd_min_radius=rmin)
    rad = np.concatenate([dd["radius_a"], dd["radius_b"]])
    fin = rad[np.isfinite(rad)]
    assert len(fin) > 0
    # shrinking stops at the floor: nothing below it, and repeated failures reach it
    assert np.all(fin >= rmin)
    assert np.any(fin == rmin)
    # every bounded radius is R (1 + alpha)^a (1 - alpha)^b, or the floor grown by (1 + alpha)^a
    ok = []
    for r in fin:
        hit = False
        for base in (R, rmin):
            for a in range(0, 60):
                for b in range(0, 60):
                    if abs(r - base * (1 + alpha) ** a * (1 - alpha) ** b) <= 1e-12 * r:
                        hit = True
                        break
                if hit:
                    break
            if hit:
                break
        ok.append(hit)
    assert all(ok)


def test_dynamic_domain_leaves_goal_bias_samples_alone():
    """The goal-bias branch targets the opposite root on purpose: it is never rejected,
    even once the wall has bounded the radius of the nodes facing it."""
    rb, wall, s, g = _slider()
    dd = O.plan(rb, wall, s, g, seed=6, range=0.3, resolution=0.01, max_iters=200, goal_bias=1.0,
                want_trees=True, tree_capacity=1024, dd_radius=0.05, dd_alpha=0.0, dd_min_radius=0.05)
    assert dd["status"] == 3
    assert np.isfinite(np.concatenate([dd["radius_a"], dd["radius_b"]])).any()
    assert dd["dd_rejected"] == 0
