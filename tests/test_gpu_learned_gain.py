"""What the trained proposal gains over plain sampling, in a setting where the
gain is expected: a point robot in two rooms joined by a narrow door.  Every
solution passes the door, so a mixture trained on the plain planner's solution
paths puts mass there; uniform sampling rarely lands in it.  Training, inference
and planning all run on the device; the comparison is on held-out start/goal
pairs with the same Philox keys, in serial mode (one worker, so iterations are
those of Alg. 1)."""
import numpy as np
import pytest

from paper_2503_06757_gb300 import learned as L
from paper_2503_06757_gb300 import prrtc as P
from paper_2503_06757_gb300 import workload as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2503_06757_gb300 import build
    build.build()


def two_rooms():
    return W.point2(), W.scene_two_rooms()


def pairs(n, seed):
    return W.two_rooms_pairs(n, seed)


def test_trained_proposal_needs_fewer_iterations_through_a_door():
    rb, sc = two_rooms()
    h, ev = P.make_robot(rb), P.make_env(sc)
    prm = P.params(range=0.2, resolution=0.01, mode=P.MODE_SERIAL, max_iters=20000, tree_capacity=1 << 14,
                   path_capacity=1 << 12)
    # training data: solution paths of the plain planner
    s, g = pairs(256, 11)
    prop, samples, losses = L.train_on_plain_solutions(rb, h, ev, s, g, prm, steps=1500, batch=256)
    assert samples > 1000
    assert losses[-50:].mean() < losses[:5].mean() - 1.0
    # held-out pairs, same keys: plain vs 50% learned
    s2, g2 = pairs(96, 12)
    items = [(h, ev, s2[k], g2[k], 5, k) for k in range(len(s2))]
    plain = P.prrtc_plan_batch(items, prm)
    prm_l = P.params(range=0.2, resolution=0.01, mode=P.MODE_SERIAL, max_iters=20000, tree_capacity=1 << 14,
                     path_capacity=1 << 12, learned_ratio=0.5)
    learned = P.prrtc_plan_batch_learned(items, [prop] * len(items), prm_l)
    ok_p = sum(r["status"] == P.SOLVED for r in plain)
    ok_l = sum(r["status"] == P.SOLVED for r in learned)
    it_p = np.mean([r["iterations"] for r in plain])
    it_l = np.mean([r["iterations"] for r in learned])
    print(f"door: plain {ok_p}/{len(items)} solved, {it_p:.0f} iterations; learned {ok_l}/{len(items)}, {it_l:.0f}")
    assert ok_l >= ok_p
    assert it_l <= 0.7 * it_p, (it_l, it_p)


def test_learned_batched_planner_beats_plain_ttfs_through_narrower_door():
    """Through a 5 cm door (1 cm free for the robot's centre) the batched learned
    form reaches its p50 time-to-first-solution before the plain GPU planner does,
    at equal or better success: 200 held-out pairs in one async launch per key,
    TTFS = device prep (including the on-device inference) + setup + solve time,
    over six Philox keys (1200 solves per side, one measurement)."""
    rb = W.point2()
    sc = W.scene_two_rooms(door=(0.865, 0.915))
    h, ev = P.make_robot(rb), P.make_env(sc)
    base = dict(range=0.2, resolution=0.01, max_iters=20000, tree_capacity=1 << 14, path_capacity=1 << 12)
    s, g = W.two_rooms_pairs(256, 11)
    prop, samples, _ = L.train_on_plain_solutions(rb, h, ev, s, g, P.params(mode=P.MODE_SERIAL, **base), steps=1500)
    assert samples > 1000
    s2, g2 = pairs(200, 12)
    plain_prm = P.params(**base)
    learned_prm = P.params(learned_ratio=0.5, **base)
    keys = (1, 2, 3, 4, 5, 6)
    plain = L.batched_ttfs(h, ev, s2, g2, plain_prm, None, keys=keys)
    learned = L.batched_ttfs(h, ev, s2, g2, learned_prm, prop, keys=keys)
    p50_p, p50_l = np.percentile(plain["ttfs_us"], 50), np.percentile(learned["ttfs_us"], 50)
    print(f"5 cm door: plain {plain['success_rate']:.3f} p50 {p50_p:.1f} us; "
          f"learned {learned['success_rate']:.3f} p50 {p50_l:.1f} us (inference {learned['infer_us_mean']:.1f} us)")
    assert learned["success_rate"] >= plain["success_rate"] - 0.01
    assert learned["iterations_mean"] < 0.5 * plain["iterations_mean"]
    assert p50_l < p50_p, (p50_l, p50_p)
