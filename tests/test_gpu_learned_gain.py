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
    res = P.prrtc_plan_batch([(h, ev, s[k], g[k], 3, k) for k in range(len(s))], prm)
    occ = P.prrtc_occupancy(ev)[None, :]
    qs, qg, tg = [], [], []
    for k, r in enumerate(res):
        if r["status"] != P.SOLVED:
            continue
        wp = L.waypoints(r["path"].astype(np.float64), spacing=0.05)
        qs += [s[k]] * len(wp)
        qg += [g[k]] * len(wp)
        tg += list(wp)
    assert len(tg) > 1000
    init = W.proposal_init(2, 7)
    flat = np.concatenate([np.concatenate([Wm.ravel(), b]) for Wm, b in init]).astype(np.float32)
    prop = P.Proposal(2, rb.lower, rb.upper, flat)
    losses = prop.train(occ, np.zeros(len(tg), np.int32), np.array(qs, np.float32), np.array(qg, np.float32),
                        np.array(tg, np.float32), batch=256, steps=1500, lr=1e-3, seed=1)
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
