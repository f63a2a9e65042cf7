"""FP64 oracle of the learned sampling proposal (TEST INFRASTRUCTURE).

Only the test-suite and the benchmark's CPU-baseline leg import this module;
it shares no code with the CUDA path.  Written from the definition of the
proposal (it has no counterpart in the paper):

  input   x = [occupancy (16^3 voxels, 0/1) | u_start (dof, zero-padded to 32)
               | u_goal (dof, zero-padded to 32)],  u = 2 (q - lo)/(hi - lo) - 1
  layers  h1 = relu(W1 x + b1) (1024), h2 = relu(W2 h1 + b2) (512),
          h3 = relu(W3 h2 + b3) (512), out = W4 h3 + b4
  head    out[0:8] = mixture logits, out[8:8+8d] = means (component-major),
          out[8+8d:8+16d] = log standard deviations, clamped to [-5, 2]
  loss    mean over samples of -log sum_k pi_k prod_j N(u_j | mu_kj, sigma_kj)
  update  Adam (Kingma & Ba 2015) on FP32-style master weights

Every step is plain numpy in binary64; the backward pass is the chain rule
written out layer by layer.
"""
from __future__ import annotations

import numpy as np

GRID = 16
CELL = 0.1
ORIGIN = (-0.8, -0.8, 0.0)
OCC_RADIUS = 0.05
N_VOX = GRID ** 3
Q_PAD = 32
IN_DIM = N_VOX + 2 * Q_PAD          # 4160
HIDDEN = (1024, 512, 512)
K = 8
LOGSIG_MIN, LOGSIG_MAX = -5.0, 2.0


def head_dim(d: int) -> int:
    return K * (1 + 2 * d)


def head_pad(d: int) -> int:
    return ((head_dim(d) + 127) // 128) * 128


def normalise(q, lo, hi):
    return 2.0 * (np.asarray(q, float) - lo) / (hi - lo) - 1.0


def features(occ, u_start, u_goal):
    """Rows of x for a batch: occ [B, 4096] (0/1), u_* [B, d] normalised."""
    occ = np.asarray(occ, float).reshape(-1, N_VOX)
    B = occ.shape[0]
    d = u_start.shape[1]
    x = np.zeros((B, IN_DIM))
    x[:, :N_VOX] = occ
    x[:, N_VOX:N_VOX + d] = u_start
    x[:, N_VOX + Q_PAD:N_VOX + Q_PAD + d] = u_goal
    return x


def shapes(d: int):
    dims = (IN_DIM,) + HIDDEN + (head_pad(d),)
    return [(dims[i + 1], dims[i]) for i in range(4)]


def layer(W, b, h, relu):
    """One layer: W h + b for every row of h, then ReLU on the hidden layers."""
    z = h @ W.T + b
    return np.maximum(z, 0.0) if relu else z


def forward(params, x):
    """params: list of (W, b); returns out [B, P] and the activations."""
    acts = [x]
    h = x
    for li, (W, b) in enumerate(params):
        h = layer(W, b, h, li < 3)
        acts.append(h)
    return h, acts


def split_head(out, d):
    logits = out[:, :K]
    mean = out[:, K:K + K * d].reshape(-1, K, d)
    raw = out[:, K + K * d:K + 2 * K * d].reshape(-1, K, d)
    return logits, mean, raw


def mixture_logp(out, u, d):
    """Per-sample log density of u [B, d] and the pieces the gradient needs."""
    logits, mean, raw = split_head(out, d)
    ls = np.clip(raw, LOGSIG_MIN, LOGSIG_MAX)
    sig = np.exp(ls)
    zt = (u[:, None, :] - mean) / sig
    comp = -0.5 * np.sum(zt * zt, axis=2) - np.sum(ls, axis=2) - 0.5 * d * np.log(2.0 * np.pi)
    m = np.max(logits, axis=1, keepdims=True)
    logpi = logits - m - np.log(np.sum(np.exp(logits - m), axis=1, keepdims=True))
    a = logpi + comp
    am = np.max(a, axis=1, keepdims=True)
    lse = am[:, 0] + np.log(np.sum(np.exp(a - am), axis=1))
    return lse, dict(logpi=logpi, a=a, lse=lse, zt=zt, sig=sig, raw=raw)


def nll_and_dout(out, u, d):
    """Mean negative log-likelihood and its gradient with respect to out."""
    B = out.shape[0]
    lse, c = mixture_logp(out, u, d)
    gamma = np.exp(c["a"] - lse[:, None])           # responsibilities
    pi = np.exp(c["logpi"])
    dout = np.zeros_like(out)
    dout[:, :K] = pi - gamma
    dmean = -gamma[:, :, None] * c["zt"] / c["sig"]
    inside = (c["raw"] > LOGSIG_MIN) & (c["raw"] < LOGSIG_MAX)
    dls = -gamma[:, :, None] * (c["zt"] ** 2 - 1.0) * inside
    dout[:, K:K + K * d] = dmean.reshape(B, -1)
    dout[:, K + K * d:K + 2 * K * d] = dls.reshape(B, -1)
    return float(-np.mean(lse)), dout / B


def loss_and_grads(params, x, u, d):
    out, acts = forward(params, x)
    loss, g = nll_and_dout(out, u, d)
    grads = [None] * 4
    for li in range(3, -1, -1):
        W, b = params[li]
        h_in = acts[li]
        grads[li] = (g.T @ h_in, np.sum(g, axis=0))
        if li > 0:
            g = (g @ W) * (acts[li] > 0.0)
    return loss, grads


def adam(params, grads, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (bias-corrected moments); state = {'t', 'm', 'v'}."""
    state["t"] += 1
    t = state["t"]
    new = []
    for i, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
        out = []
        for j, (p, g) in enumerate(((W, gW), (b, gb))):
            m = state["m"][i][j] = b1 * state["m"][i][j] + (1 - b1) * g
            v = state["v"][i][j] = b2 * state["v"][i][j] + (1 - b2) * g * g
            mh = m / (1 - b1 ** t)
            vh = v / (1 - b2 ** t)
            out.append(p - lr * mh / (np.sqrt(vh) + eps))
        new.append(tuple(out))
    return new


def adam_state(params):
    return {"t": 0, "m": [[np.zeros_like(W), np.zeros_like(b)] for W, b in params],
            "v": [[np.zeros_like(W), np.zeros_like(b)] for W, b in params]}
