"""Pins of the learned-proposal oracle (FP64 MLP, mixture NLL, Adam, occupancy,
mixture sampler) against facts independent of it: central finite differences,
scipy's normal log-density, Adam's closed-form first step, closed-form voxel
sets, and the statistics of many draws."""
import numpy as np
import pytest

from oracle import mlp_oracle as M
from oracle import oracle as O
from paper_2503_06757_gb300 import workload as W
from tests import helpers as H


def _small_params(d, seed=0, hidden=(6, 5, 4)):
    rng = np.random.default_rng(seed)
    dims = (M.IN_DIM,) + hidden + (M.head_pad(d),)
    return [(rng.normal(size=(dims[i + 1], dims[i])) * (0.05 if i == 0 else 0.4),
             rng.normal(size=dims[i + 1]) * 0.1) for i in range(4)]


def _batch(d, B=5, seed=1):
    rng = np.random.default_rng(seed)
    occ = (rng.random((B, M.N_VOX)) < 0.1).astype(float)
    us, ug = rng.uniform(-1, 1, (B, d)), rng.uniform(-1, 1, (B, d))
    return M.features(occ, us, ug), rng.uniform(-1, 1, (B, d))


@pytest.mark.parametrize("d", [2, 7])
def test_gradients_match_central_differences(d):
    params = _small_params(d)
    x, u = _batch(d)
    loss, grads = M.loss_and_grads(params, x, u, d)
    rng = np.random.default_rng(3)
    eps = 1e-6
    for li in range(4):
        for which in (0, 1):
            arr = params[li][which]
            for _ in range(6):
                idx = tuple(rng.integers(0, s) for s in arr.shape)
                if which == 0 and li == 0 and idx[1] < M.N_VOX and x[:, idx[1]].max() == 0:
                    continue
                old = arr[idx]
                arr[idx] = old + eps
                lp, _ = M.loss_and_grads(params, x, u, d)
                arr[idx] = old - eps
                lm, _ = M.loss_and_grads(params, x, u, d)
                arr[idx] = old
                num = (lp - lm) / (2 * eps)
                ana = grads[li][which][idx]
                assert abs(num - ana) <= 1e-6 * max(1.0, abs(num)) + 1e-8, (li, which, idx, num, ana)


def test_one_component_is_a_diagonal_gaussian():
    from scipy.stats import norm
    d, B = 4, 6
    rng = np.random.default_rng(7)
    out = np.zeros((B, M.head_pad(d)))
    out[:, 0] = 0.0
    out[:, 1:M.K] = -1e4                       # all other components have zero weight
    mean = rng.uniform(-0.5, 0.5, (B, d))
    ls = rng.uniform(-2, 0.5, (B, d))
    out[:, M.K:M.K + d] = mean
    out[:, M.K + M.K * d:M.K + M.K * d + d] = ls
    u = rng.uniform(-1, 1, (B, d))
    lse, _ = M.mixture_logp(out, u, d)
    want = np.sum(norm.logpdf(u, loc=mean, scale=np.exp(ls)), axis=1)
    np.testing.assert_allclose(lse, want, rtol=1e-12, atol=1e-12)


def test_identical_components_leave_logits_without_gradient():
    d, B = 3, 4
    rng = np.random.default_rng(2)
    out = np.zeros((B, M.head_pad(d)))
    out[:, :M.K] = rng.normal(size=(B, M.K))
    mean = rng.uniform(-0.5, 0.5, (B, 1, d)).repeat(M.K, 1)
    out[:, M.K:M.K + M.K * d] = mean.reshape(B, -1)
    out[:, M.K + M.K * d:M.K + 2 * M.K * d] = -1.0
    _, dout = M.nll_and_dout(out, rng.uniform(-1, 1, (B, d)), d)
    np.testing.assert_allclose(dout[:, :M.K], 0.0, atol=1e-15)


def test_log_sigma_clamp():
    d = 1
    out = np.zeros((1, M.head_pad(d)))
    out[0, M.K + M.K * d:M.K + 2 * M.K * d] = 3.0      # above the clamp
    u = np.array([[0.3]])
    lse, _ = M.mixture_logp(out, u, d)
    ref = out.copy()
    ref[0, M.K + M.K * d:M.K + 2 * M.K * d] = 2.0
    lse2, _ = M.mixture_logp(ref, u, d)
    assert lse[0] == lse2[0]
    _, dout = M.nll_and_dout(out, u, d)
    assert np.all(dout[0, M.K + M.K * d:M.K + 2 * M.K * d] == 0.0)


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(4)
    params = [(rng.normal(size=(3, 2)), rng.normal(size=3))]
    grads = [(rng.normal(size=(3, 2)), rng.normal(size=3))]
    st = M.adam_state(params)
    new = M.adam(params, grads, st, lr=1e-2, eps=1e-8)
    for (p0, p1, g) in ((params[0][0], new[0][0], grads[0][0]), (params[0][1], new[0][1], grads[0][1])):
        np.testing.assert_allclose(p1, p0 - 1e-2 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def _centres():
    i = np.arange(M.GRID)
    c = (i + 0.5) * M.CELL
    X, Y, Z = np.meshgrid(c + M.ORIGIN[0], c + M.ORIGIN[1], c + M.ORIGIN[2], indexing="ij")
    # index i + 16 j + 256 k  ->  transpose to (k, j, i) order before flattening
    return np.stack([X.transpose(2, 1, 0).ravel(), Y.transpose(2, 1, 0).ravel(), Z.transpose(2, 1, 0).ravel()], 1)


def test_occupancy_sphere_and_box_closed_form():
    P = _centres()
    sc = H.scene(spheres=[[0.13, -0.21, 0.57, 0.22]])
    occ = O.occupancy(sc)
    want = np.linalg.norm(P - [0.13, -0.21, 0.57], axis=1) < 0.22 + M.OCC_RADIUS
    np.testing.assert_array_equal(occ.astype(bool), want)
    sc = H.scene(boxes=[H.aabb([0.2, 0.1, 0.4], [0.12, 0.3, 0.07])])
    occ = O.occupancy(sc)
    ex = np.maximum(np.abs(P - [0.2, 0.1, 0.4]) - [0.12, 0.3, 0.07], 0)
    want = np.linalg.norm(ex, axis=1) < M.OCC_RADIUS
    np.testing.assert_array_equal(occ.astype(bool), want)
    assert O.occupancy(H.empty_scene()).sum() == 0


def test_learned_sampler_statistics():
    rb = W.arm7()
    d = rb.dof
    gmm = np.zeros(M.K * (1 + 2 * d))
    pi = np.array([0.4, 0.3, 0.2, 0.1, 0, 0, 0, 0], float)
    with np.errstate(divide="ignore"):
        gmm[:M.K] = np.log(np.where(pi > 0, pi, 1e-300))
    centres = np.array([-0.6, -0.2, 0.2, 0.6, 0.0, 0.0, 0.0, 0.0])   # used components 8 sigma apart
    means = centres[:, None] * np.ones((M.K, d))
    gmm[M.K:M.K + M.K * d] = means.ravel()
    gmm[M.K + M.K * d:] = np.log(0.05)
    n = 8000
    draws, kinds = [], []
    for it in range(n):
        kind, q, _ = O.sample_learned(rb, 3, 0, it, 0.0, gmm, 1.0)
        kinds.append(kind)
        draws.append(M.normalise(q, rb.lower, rb.upper))
    assert set(kinds) == {2}
    U = np.array(draws)
    comp = np.argmin(np.abs(U[:, :1] - centres[None, :4]), axis=1)
    freq = np.bincount(comp, minlength=M.K) / n
    assert np.all(np.abs(freq - pi) < 5 * np.sqrt(pi * (1 - pi) / n) + 1e-9), freq
    for k in range(4):
        sel = U[comp == k]
        np.testing.assert_allclose(sel.mean(0), means[k], atol=5 * 0.05 / np.sqrt(len(sel)))
        np.testing.assert_allclose(sel.std(0), 0.05, rtol=0.08)
    # ratio 0 falls back to the uniform draw of the plain sampler
    for it in range(50):
        kind, q, _ = O.sample_learned(rb, 3, 0, it, 0.05, gmm, 0.0)
        g, q0 = O.sample(rb, 3, 0, it, 0.05)
        assert kind == (1 if g else 0)
        if not g:
            np.testing.assert_array_equal(q, q0)
