"""Parity of the learned proposal's CUDA path with the FP64 oracle.

The device keeps BF16 weights and activations and accumulates in FP32, so its
forward output and gradients differ from the FP64 oracle (which uses the FP32
master weights exactly) by BF16 rounding: about 2^-9 per element, compounding
over four layers.  The bounds below are relative L2 errors of 2^-5 (forward)
and 2^-4 (gradients, which pass through the forward activations twice).
"""
import numpy as np
import pytest

from oracle import mlp_oracle as M
from oracle import oracle as O
from paper_2503_06757_gb300 import prrtc as P
from paper_2503_06757_gb300 import workload as W
from tests import helpers as H

pytestmark = pytest.mark.gpu

FWD_TOL = 2.0 ** -5
GRAD_TOL = 2.0 ** -4
F32 = lambda x: float(np.float32(x))


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2503_06757_gb300 import build
    build.build()


def flat(params):
    return np.concatenate([np.concatenate([Wm.ravel(), b]) for Wm, b in params]).astype(np.float32)


def unflat(v, d):
    out, k = [], 0
    for (o, i) in M.shapes(d):
        Wm = v[k:k + o * i].reshape(o, i).astype(np.float64)
        k += o * i
        b = v[k:k + o].astype(np.float64)
        k += o
        out.append((Wm, b))
    return out


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def make_batch(robot, B, seed):
    st = W.Stream(seed, 3)
    scenes = [W.scene_shelf(1000 + k) for k in range(3)]
    occ = np.stack([O.occupancy(scenes[k % 3]) for k in range(B)])
    u = st.uniform(3 * B * robot.dof).reshape(3, B, robot.dof)
    qs, qg, tg = (robot.lower + u[i] * (robot.upper - robot.lower) for i in range(3))
    return occ, qs.astype(np.float32), qg.astype(np.float32), tg.astype(np.float32)


def init(d, seed):
    params = W.proposal_init(d, seed)
    st = W.Stream(seed, 4)
    return [(Wm, (0.05 * st.normal(len(b))).astype(np.float32).astype(np.float64)) for Wm, b in params]


def oracle_x(robot, occ, qs, qg):
    us = M.normalise(qs.astype(np.float64), robot.lower, robot.upper)
    ug = M.normalise(qg.astype(np.float64), robot.lower, robot.upper)
    return M.features(occ, us, ug)


@pytest.mark.parametrize("name,B", [("arm7", 37), ("dual14", 256)])
def test_forward_matches_oracle(name, B):
    rb = W.ROBOTS[name]()
    params = init(rb.dof, 11)
    prop = P.Proposal(rb.dof, rb.lower, rb.upper, flat(params))
    occ, qs, qg, _ = make_batch(rb, B, 5)
    got = prop.forward(occ, qs, qg)
    ref, _ = M.forward(params, oracle_x(rb, occ, qs, qg))
    assert got.shape == ref.shape
    assert rel(got, ref) <= FWD_TOL, rel(got, ref)


@pytest.mark.parametrize("name,B", [("arm7", 40), ("dual14", 130)])
def test_gradients_match_oracle(name, B):
    rb = W.ROBOTS[name]()
    d = rb.dof
    params = init(d, 12)
    prop = P.Proposal(d, rb.lower, rb.upper, flat(params))
    occ, qs, qg, tg = make_batch(rb, B, 6)
    loss, g = prop.loss_and_grads(occ, qs, qg, tg)
    x = oracle_x(rb, occ, qs, qg)
    u = M.normalise(tg.astype(np.float64), rb.lower, rb.upper)
    ref_loss, ref_grads = M.loss_and_grads(params, x, u, d)
    assert abs(loss - ref_loss) <= 2 ** -6 * abs(ref_loss), (loss, ref_loss)
    got = unflat(g, d)
    for li in range(4):
        for which in (0, 1):
            a, b = got[li][which], ref_grads[li][which]
            r = rel(a, b)
            cos = float(np.sum(a * b) / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-30))
            assert r <= GRAD_TOL and cos >= 0.995, (li, which, r, cos)


def test_adam_step_direction_matches_oracle():
    rb = W.arm7()
    d = rb.dof
    params = init(d, 13)
    prop = P.Proposal(d, rb.lower, rb.upper, flat(params))
    occ, qs, qg, tg = make_batch(rb, 64, 7)
    before = prop.params().astype(np.float64)
    prop.train(occ, np.arange(64), qs, qg, tg, batch=64, steps=1, lr=1e-3, seed=1)
    delta = prop.params().astype(np.float64) - before
    x = oracle_x(rb, occ, qs, qg)
    u = M.normalise(tg.astype(np.float64), rb.lower, rb.upper)
    _, grads = M.loss_and_grads(params, x, u, d)
    new = M.adam(params, grads, M.adam_state(params), lr=1e-3)
    ref_delta = flat(new).astype(np.float64) - flat(params).astype(np.float64)
    g = flat(grads).astype(np.float64)
    strong = np.abs(g) > 1e-3 * np.max(np.abs(g))
    agree = np.mean(np.sign(delta[strong]) == np.sign(ref_delta[strong]))
    assert agree >= 0.99, agree
    # first Adam step moves every strong coordinate by ~lr
    assert np.median(np.abs(delta[strong])) == pytest.approx(1e-3, rel=0.05)


def test_training_lowers_the_loss_on_a_fixed_batch():
    rb = W.arm7()
    prop = P.Proposal(rb.dof, rb.lower, rb.upper, flat(init(rb.dof, 14)))
    occ, qs, qg, tg = make_batch(rb, 64, 8)
    losses = prop.train(occ, np.arange(64), qs, qg, tg, batch=64, steps=80, lr=1e-3, seed=2)
    assert np.all(np.isfinite(losses))
    assert losses[-10:].mean() < losses[:5].mean() - 1.0, (losses[:5], losses[-10:])
    assert prop.step == 80


def test_checkpoint_round_trip(tmp_path):
    rb = W.dual14()
    prop = P.Proposal(rb.dof, rb.lower, rb.upper, flat(init(rb.dof, 15)))
    occ, qs, qg, tg = make_batch(rb, 16, 9)
    prop.train(occ, np.arange(16), qs, qg, tg, batch=16, steps=3, lr=1e-3)
    path = tmp_path / "p.bin"
    prop.save(path)
    q = P.Proposal.load(path)
    assert q.step == 3 and q.dof == 14
    np.testing.assert_array_equal(q.params(), prop.params())
    np.testing.assert_array_equal(q.forward(occ, qs, qg), prop.forward(occ, qs, qg))


def test_occupancy_matches_oracle():
    for seed in (1000, 1001, 2005):
        sc = W.scene_shelf(seed) if seed < 2000 else W.scene_mixed(seed, 90)
        got = P.prrtc_occupancy(P.make_env(sc))
        want = O.occupancy(sc)
        bad = np.nonzero(got != want)[0]
        # any disagreement must sit on the 5 cm threshold (ambiguity band)
        for v in bad:
            i, j, k = v % 16, (v // 16) % 16, v // 256
            p = np.array([-0.8 + 0.1 * (i + 0.5), -0.8 + 0.1 * (j + 0.5), 0.1 * (k + 0.5)])
            sd = min([O.sd_box(b, p) for b in sc.boxes] + [O.sd_cyl(c, p) for c in sc.cylinders] +
                     [O.sd_sph(s, p) for s in sc.spheres])
            assert abs(sd - M.OCC_RADIUS) <= 1e-5, (v, sd)
        assert 0 < want.sum() < 4096


@pytest.fixture(scope="module")
def boxes8_problems():
    return W.problem_set("boxes8", 4, 1, O.accept)


@pytest.mark.parametrize("k", range(4))
def test_serial_planner_with_mixture_matches_oracle(boxes8_problems, k):
    pb = boxes8_problems[k]
    gmm = W.random_mixture(7, 100 + k)
    rb, ev = P.make_robot(pb.robot), P.make_env(pb.scene)
    prm = P.params(seed=3, mode=P.MODE_SERIAL, tree_capacity=1 << 14, learned_ratio=0.5)
    g = P.prrtc_plan_batch([(rb, ev, pb.q_start, pb.q_goal, 3, 0, gmm)], prm)[0]
    o = O.plan(pb.robot, pb.scene, pb.q_start, pb.q_goal, seed=3, want_trees=True, tree_capacity=1 << 14,
               range=1.0, resolution=F32(1 / 32), goal_bias=F32(0.05), gmm=gmm.astype(np.float64),
               learned_ratio=F32(0.5))
    if o["first_amb_iter"] != -1 and o["first_amb_iter"] < o["iterations"]:
        pytest.skip(f"ambiguous decision at iteration {o['first_amb_iter']}")
    assert g["status"] == o["status"] == 0
    assert g["iterations"] == o["iterations"]
    assert (g["nodes_a"], g["nodes_b"]) == (o["n_a"], o["n_b"])
    np.testing.assert_allclose(g["path"], o["path"], atol=1e-4)


def test_learned_batch_plans_with_device_inference(boxes8_problems):
    rb7 = W.arm7()
    prop = P.Proposal(7, rb7.lower, rb7.upper, flat(init(7, 16)))
    items, props = [], []
    for k, pb in enumerate(boxes8_problems):
        items.append((P.make_robot(pb.robot), P.make_env(pb.scene), pb.q_start, pb.q_goal, 9, k))
        props.append(prop if k % 2 == 0 else None)
    res = P.prrtc_plan_batch_learned(items, props, P.params(learned_ratio=0.5))
    orc = O.plan_batch(boxes8_problems, seed=9, problem_ids=list(range(len(boxes8_problems))), range=1.0,
                       resolution=F32(1 / 32), goal_bias=F32(0.05))
    for r in res:
        assert r["status"] == P.SOLVED
    # the re-check at 4x resolution flags segments at the oracle's own rate on these problems
    H.assert_same_revalidation_rate(
        H.revalidation_counts([(pb.robot, pb.scene, r["path"], None) for pb, r in zip(boxes8_problems, res)],
                              F32(1 / 32) / 4),
        H.revalidation_counts([(pb.robot, pb.scene, o["path"], None) for pb, o in zip(boxes8_problems, orc)
                               if o["status"] == 0], F32(1 / 32) / 4), "learned batch")


def test_learned_inference_replay_is_exact(boxes8_problems):
    """The inference chain runs eagerly, is captured on its second call with the same
    buffers and replayed afterwards: serial plans of all three calls are identical, and
    a different batch size in between does not disturb the replay."""
    rb7 = W.arm7()
    prop = P.Proposal(7, rb7.lower, rb7.upper, flat(init(7, 17)))
    items = [(P.make_robot(pb.robot), P.make_env(pb.scene), pb.q_start, pb.q_goal, 5, k)
             for k, pb in enumerate(boxes8_problems)]
    prm = P.params(learned_ratio=0.5, mode=P.MODE_SERIAL, tree_capacity=1 << 14)
    runs = [P.prrtc_plan_batch_learned(items, [prop] * len(items), prm) for _ in range(3)]
    P.prrtc_plan_batch_learned(items[:2], [prop] * 2, prm)
    runs.append(P.prrtc_plan_batch_learned(items, [prop] * len(items), prm))
    for r in runs[1:]:
        for a, b in zip(runs[0], r):
            assert a["status"] == b["status"] and a["iterations"] == b["iterations"]
            np.testing.assert_array_equal(a["path"], b["path"])


@pytest.mark.parametrize("distinct,B", [(False, 24), (True, 24), (True, 40), (False, 300)])
def test_planner_mixtures_match_oracle(distinct, B):
    """The mixtures the learned planner samples from, read back.  The occupancy part
    of the first layer is computed once per distinct environment (a GEMV for up to 32
    environments, the tensor-core GEMM beyond), the rest of the network in one fused
    launch per 128-row tile (300 rows: three tiles, the last ragged)."""
    rb = W.arm7()
    params = init(rb.dof, 18)
    prop = P.Proposal(rb.dof, rb.lower, rb.upper, flat(params))
    n_sc = B if distinct else 3
    scenes = [W.scene_shelf(1000 + k) for k in range(n_sc)]
    made = [P.make_env(sc) for sc in scenes]
    envs = [made[k % n_sc] for k in range(B)]
    st = W.Stream(19, 3)
    u = st.uniform(2 * B * rb.dof).reshape(2, B, rb.dof)
    qs, qg = ((rb.lower + u[i] * (rb.upper - rb.lower)).astype(np.float32) for i in range(2))
    got = prop.mixtures(envs, qs, qg)
    occ = np.stack([O.occupancy(scenes[k % n_sc]) for k in range(B)])
    out, _ = M.forward(params, oracle_x(rb, occ, qs, qg))
    logits, mean, raw = M.split_head(out, rb.dof)
    want = np.concatenate([logits, mean.reshape(B, -1), np.clip(raw, M.LOGSIG_MIN, M.LOGSIG_MAX).reshape(B, -1)],
                          axis=1)
    assert got.shape == want.shape
    assert rel(got, want) <= FWD_TOL, rel(got, want)
    worst = max(rel(got[b], want[b]) for b in range(B))
    assert worst <= 2 * FWD_TOL, worst
    # the second call is captured, the third replays the capture: identical output
    np.testing.assert_array_equal(prop.mixtures(envs, qs, qg), got)
    np.testing.assert_array_equal(prop.mixtures(envs, qs, qg), got)


# ------------------------------------------------------------------ element-wise, layer by layer

def bf16_params(params):
    """The device's weights: the FP32 masters rounded to BF16 (biases stay FP32)."""
    return [(H.bf16_round(Wm).astype(np.float64), b.astype(np.float32).astype(np.float64)) for Wm, b in params]


def assert_layer(got, a, Wm, b, relu, bf16_out, what):
    """One layer against the oracle fed the device's own BF16 input rows `a` and
    BF16 weights, element by element: FP32 accumulation of K products in any
    order is within 2 K 2^-24 (sum |a||w| + |b|) of the exact value, and a BF16
    output adds at most half an ulp, 2^-8 of the value."""
    from oracle import mlp_oracle as M
    ref = M.layer(Wm, b, a, relu)
    K = a.shape[1]
    acc = 2.0 * K * 2.0 ** -24 * (np.abs(a) @ np.abs(Wm).T + np.abs(b))
    bound = acc * (1 + 2.0 ** -8) + (2.0 ** -8 * np.abs(ref) if bf16_out else 0.0) + 1e-30
    err = np.abs(got.astype(np.float64) - ref)
    bad = np.argwhere(err > bound)
    assert len(bad) == 0, (what, bad[:5].tolist(), float((err / bound).max()))
    return float((err / bound).max())


@pytest.mark.parametrize("name,B", [("arm7", 37), ("dual14", 140)])
def test_training_forward_layers_elementwise(name, B):
    rb = W.ROBOTS[name]()
    params = init(rb.dof, 21)
    prop = P.Proposal(rb.dof, rb.lower, rb.upper, flat(params))
    occ, qs, qg, _ = make_batch(rb, B, 7)
    x, h1, h2, h3, out = prop.forward_layers(occ, qs, qg)
    # the features: occupancy exactly, normalised start / goal as BF16 (within one BF16 ulp
    # of the FP64 value; the device rounds its FP32 value)
    ref_x = oracle_x(rb, occ, qs, qg)
    np.testing.assert_array_equal(x[:, :4096], ref_x[:, :4096])
    assert np.all(np.abs(x - ref_x) <= 2.0 ** -7 * np.abs(ref_x) + 1e-30)
    Wb = bf16_params(params)
    ins = [x.astype(np.float64), h1.astype(np.float64), h2.astype(np.float64), h3.astype(np.float64)]
    outs = [h1, h2, h3, out]
    worst = [assert_layer(outs[l], ins[l], Wb[l][0], Wb[l][1], l < 3, l < 3, f"layer {l + 1}") for l in range(4)]
    print(f"{name}: worst error / bound per layer {['%.3f' % w for w in worst]}")


@pytest.mark.parametrize("distinct,B", [(False, 300), (True, 40)])
def test_fused_inference_layers_elementwise(distinct, B):
    """The fused inference kernel layer by layer: its hidden activations read
    back, each checked against the oracle fed the previous one; the mixture rows
    against the oracle's head from its third layer (log-sigmas clamped)."""
    from oracle import mlp_oracle as M
    rb = W.arm7()
    d = rb.dof
    params = init(d, 23)
    prop = P.Proposal(d, rb.lower, rb.upper, flat(params))
    n_sc = B if distinct else 3
    scenes = [W.scene_shelf(1100 + k) for k in range(n_sc)]
    made = [P.make_env(sc) for sc in scenes]
    envs = [made[k % n_sc] for k in range(B)]
    st = W.Stream(24, 3)
    u = st.uniform(2 * B * d).reshape(2, B, d)
    qs, qg = ((rb.lower + u[i] * (rb.upper - rb.lower)).astype(np.float32) for i in range(2))
    mix = prop.mixtures(envs, qs, qg)
    h1, h2, h3 = prop.inference_layers(B)
    occ = np.stack([P.prrtc_occupancy(e) for e in envs])
    x, _, _, _, _ = prop.forward_layers(occ, qs, qg)  # the same BF16 features
    Wb = bf16_params(params)
    assert_layer(h1, x.astype(np.float64), Wb[0][0], Wb[0][1], True, True, "layer 1")
    assert_layer(h2, h1.astype(np.float64), Wb[1][0], Wb[1][1], True, True, "layer 2")
    assert_layer(h3, h2.astype(np.float64), Wb[2][0], Wb[2][1], True, True, "layer 3")
    # head -> mixture rows (logits | means | clamped log-sigmas)
    a = h3.astype(np.float64)
    ref = M.layer(Wb[3][0], Wb[3][1], a, False)
    bound = 2.0 * a.shape[1] * 2.0 ** -24 * (np.abs(a) @ np.abs(Wb[3][0]).T + np.abs(Wb[3][1])) + 1e-30
    logits, mean, raw = M.split_head(ref, d)
    lb, mb, rbnd = M.split_head(bound, d)
    want = np.concatenate([logits, mean.reshape(B, -1), np.clip(raw, M.LOGSIG_MIN, M.LOGSIG_MAX).reshape(B, -1)], 1)
    tol = np.concatenate([lb, mb.reshape(B, -1), rbnd.reshape(B, -1)], 1)
    bad = np.argwhere(np.abs(mix - want) > tol)
    assert len(bad) == 0, (bad[:5].tolist(), float((np.abs(mix - want) / tol).max()))
