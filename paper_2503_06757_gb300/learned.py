"""Training data, training and evaluation of the learned sampling proposal.

The proposal is trained on solution paths of the plain planner: for each
solved problem the path is resampled at a fixed arclength spacing and every
resampled configuration becomes a target of the mixture density, conditioned
on the problem's start, goal and occupancy grid.  Everything that computes
runs in libprrtc (collision checks for start/goal selection, planning,
occupancy, training, inference); this module only orchestrates calls.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import prrtc as P
from . import workload as W

WAYPOINT_SPACING = 0.25


@dataclass
class Dataset:
    dof: int
    occ: np.ndarray                 # [n_scenes, 4096] uint8
    scene_of: np.ndarray            # [N] int32
    q_start: np.ndarray             # [N, dof]
    q_goal: np.ndarray              # [N, dof]
    target: np.ndarray              # [N, dof]
    paths: int = 0
    problems: int = 0
    seconds: float = 0.0
    info: dict = field(default_factory=dict)


def waypoints(path: np.ndarray, spacing: float = WAYPOINT_SPACING, interior: bool = True) -> np.ndarray:
    """Configurations at arclength s, 2s, ... along a piecewise-linear path.  With
    `interior` the start and goal themselves (already tree roots) are left out;
    otherwise arclength 0 and the end are included."""
    seg = np.linalg.norm(np.diff(path, axis=0), axis=1)
    cum = np.concatenate([[0.0], np.cumsum(seg)])
    total = cum[-1]
    if total <= 0.0:
        return path[:0].copy() if interior else path[:1].copy()
    s = np.arange(spacing if interior else 0.0, total - (1e-9 if interior else 0.0), spacing)
    if len(s) == 0:
        return path[:0].copy()
    idx = np.clip(np.searchsorted(cum, s, side="right") - 1, 0, len(seg) - 1)
    t = np.where(seg[idx] > 0, (s - cum[idx]) / np.maximum(seg[idx], 1e-30), 0.0)
    pts = path[idx] + t[:, None] * (path[idx + 1] - path[idx])
    return pts if interior else np.concatenate([pts, path[-1:]], axis=0)


def end_effectors(robot: W.Robot, spheres: np.ndarray) -> np.ndarray:
    """Origin of the first end-effector frame, extrapolated from the two outermost
    spheres on that link's axis (the device returns sphere centres)."""
    f = robot.ee_frames[0]
    idx = np.nonzero(robot.sphere_frame == f)[0]
    order = idx[np.argsort(robot.sphere_offset[idx, 2])]
    a, b = order[-2], order[-1]
    za, zb = robot.sphere_offset[a, 2], robot.sphere_offset[b, 2]
    ca, cb = spheres[:, a, :3].astype(np.float64), spheres[:, b, :3].astype(np.float64)
    return cb + (cb - ca) * ((0.0 - zb) / (zb - za))


def scene_pairs(robot: W.Robot, scene: W.Scene, rb: P.Robot, ev: P.Env, n_pairs: int, seed: int,
                chunk: int = 16384, max_chunks: int = 8):
    """Up to n_pairs (start, goal) pairs: starts collision-free, goals collision-free
    with the end effector inside a cubby, both from seeded candidate streams."""
    starts, goals = [], []
    for ci in range(max_chunks):
        Q = W.candidates(robot, seed, 0, chunk, offset=ci * chunk).astype(np.float32)
        valid, sph = P.prrtc_check_states(rb, ev, Q, want_spheres=True)
        free = np.nonzero(valid)[0]
        ee = end_effectors(robot, sph[free])
        cells = scene.cells
        inside = np.any(np.all((ee[:, None, :] >= cells[None, :, :3]) & (ee[:, None, :] <= cells[None, :, 3:]), axis=2),
                        axis=1)
        goals += list(Q[free[inside]])
        starts += list(Q[free[~inside]])
        if len(goals) >= n_pairs and len(starts) >= n_pairs:
            break
    m = min(n_pairs, len(starts), len(goals))
    return np.array(starts[:m]), np.array(goals[:m])


def shelf_problem_batch(robot: W.Robot, n_scenes: int, pairs_per_scene: int, seed0: int):
    """Scenes, device handles and problems (scene index, start, goal)."""
    rb = P.make_robot(robot)
    scenes, envs, probs = [], [], []
    for k in range(n_scenes):
        sc = W.scene_shelf(seed0 + k, W.shelf_facing(robot))
        ev = P.make_env(sc)
        s, g = scene_pairs(robot, sc, rb, ev, pairs_per_scene, seed0 + k)
        scenes.append(sc)
        envs.append(ev)
        for i in range(len(s)):
            probs.append((k, s[i], g[i]))
    return rb, scenes, envs, probs


def build_dataset(robot: W.Robot, n_scenes: int, pairs_per_scene: int, seed0: int, batch: int = 1024,
                  params: P.prrtc_params | None = None) -> Dataset:
    """Solve seeded shelf problems with the plain planner and turn the paths into samples."""
    t0 = time.perf_counter()
    prm = params or P.params(tree_capacity=1 << 13, path_capacity=1 << 12, max_iters=20000)
    rb, scenes, envs, probs = shelf_problem_batch(robot, n_scenes, pairs_per_scene, seed0)
    occ = np.stack([P.prrtc_occupancy(ev) for ev in envs]).astype(np.uint8)
    scene_of, qs, qg, tg = [], [], [], []
    n_paths = 0
    for b0 in range(0, len(probs), batch):
        chunk = probs[b0:b0 + batch]
        items = [(rb, envs[k], s, g, seed0, b0 + i) for i, (k, s, g) in enumerate(chunk)]
        res = P.prrtc_plan_batch(items, prm)
        for (k, s, g), r in zip(chunk, res):
            if r["status"] != P.SOLVED:
                continue
            n_paths += 1
            wp = waypoints(r["path"].astype(np.float64))
            if len(wp) == 0:
                continue
            scene_of += [k] * len(wp)
            qs += [s] * len(wp)
            qg += [g] * len(wp)
            tg += list(wp)
    return Dataset(dof=robot.dof, occ=occ, scene_of=np.asarray(scene_of, np.int32),
                   q_start=np.asarray(qs, np.float32), q_goal=np.asarray(qg, np.float32),
                   target=np.asarray(tg, np.float32), paths=n_paths, problems=len(probs),
                   seconds=time.perf_counter() - t0)


def concat_datasets(parts: list[Dataset]) -> Dataset:
    """One dataset from several built on disjoint scene ranges (scene indices renumbered)."""
    occ, scene_of, off = [], [], 0
    for d in parts:
        occ.append(d.occ)
        scene_of.append(d.scene_of + off)
        off += d.occ.shape[0]
    cat = lambda name: np.concatenate([getattr(d, name) for d in parts])
    return Dataset(dof=parts[0].dof, occ=np.concatenate(occ), scene_of=np.concatenate(scene_of).astype(np.int32),
                   q_start=cat("q_start"), q_goal=cat("q_goal"), target=cat("target"),
                   paths=sum(d.paths for d in parts), problems=sum(d.problems for d in parts),
                   seconds=sum(d.seconds for d in parts))


def train(robot: W.Robot, data: Dataset, steps: int, batch: int = 512, lr: float = 1e-3, seed: int = 1,
          init_seed: int = 7) -> tuple[P.Proposal, np.ndarray, float]:
    init = W.proposal_init(robot.dof, init_seed)
    flat = np.concatenate([np.concatenate([Wm.ravel(), b]) for Wm, b in init]).astype(np.float32)
    prop = P.Proposal(robot.dof, robot.lower, robot.upper, flat)
    t0 = time.perf_counter()
    losses = prop.train(data.occ, data.scene_of, data.q_start, data.q_goal, data.target, batch=batch, steps=steps,
                        lr=lr, seed=seed)
    return prop, losses, time.perf_counter() - t0


def held_out_nll(prop: P.Proposal, data: Dataset, limit: int = 4096) -> float:
    n = min(limit, len(data.target))
    occ = data.occ[data.scene_of[:n]]
    loss, _ = prop.loss_and_grads(occ, data.q_start[:n], data.q_goal[:n], data.target[:n])
    return loss


def evaluate(robot: W.Robot, n_scenes: int, pairs_per_scene: int, seed0: int, prop: P.Proposal,
             ratio: float = 0.5, keys=(1, 2, 3), params: P.prrtc_params | None = None):
    """Plain vs learned batched planning on the same held-out problems and keys."""
    rb, scenes, envs, probs = shelf_problem_batch(robot, n_scenes, pairs_per_scene, seed0)
    items = [(rb, envs[k], s, g, 0, i) for i, (k, s, g) in enumerate(probs)]
    out = {}
    # one untimed call per mode first: both launch sequences are then replayed
    # from CUDA graphs, as in steady use
    warm = P.params() if params is None else params
    P.prrtc_plan_batch([it[:4] + (97, it[5]) for it in items], warm)
    warm_l = P.params() if params is None else params
    warm_l.learned_ratio = ratio
    for _ in range(2):
        P.prrtc_plan_batch_learned([it[:4] + (97, it[5]) for it in items], [prop] * len(items), warm_l)
    for name in ("plain", "learned"):
        ttfs, ok, iters, cost, dev_ms, prep_ms = [], 0, [], [], 0.0, 0.0
        for key in keys:
            its = [it[:4] + (key, it[5]) for it in items]
            if name == "plain":
                prm = params or P.params()
                res = P.prrtc_plan_batch(its, prm)
            else:
                prm = params or P.params()
                prm.learned_ratio = ratio
                res = P.prrtc_plan_batch_learned(its, [prop] * len(its), prm)
            st = P.prrtc_last_launch_stats()
            dev_ms += st["kernel_ms"] + st["setup_ms"] + st["prep_ms"]
            prep_ms += st["prep_ms"]
            for r in res:
                if r["status"] == P.SOLVED:
                    ok += 1
                    # from the call's first device work: inference (learned) + upload + planning
                    ttfs.append(r["solve_time_us"] + 1e3 * (st["prep_ms"] + st["setup_ms"]))
                    iters.append(r["iterations"])
                    cost.append(r["cost"])
        n = len(items) * len(keys)
        out[name] = dict(success_rate=ok / n, ttfs_us_p50=float(np.percentile(ttfs, 50)) if ttfs else None,
                         ttfs_us_p95=float(np.percentile(ttfs, 95)) if ttfs else None,
                         iterations_mean=float(np.mean(iters)) if iters else None,
                         cost_mean=float(np.mean(cost)) if cost else None, device_ms=dev_ms / len(keys),
                         prep_ms=prep_ms / len(keys),
                         problems=len(items), keys=len(keys))
    return out


def train_on_plain_solutions(robot: W.Robot, rb: P.Robot, ev: P.Env, starts: np.ndarray, goals: np.ndarray,
                             params: P.prrtc_params, steps: int, batch: int = 256, lr: float = 1e-3,
                             init_seed: int = 7, seed: int = 1, key: int = 3):
    """A proposal for one environment trained on the plain planner's solutions of
    (starts[k], goals[k]) -- waypoints of each solution path as targets, the pair as
    input.  Returns (proposal, training samples, losses)."""
    res = P.prrtc_plan_batch([(rb, ev, starts[k], goals[k], key, k) for k in range(len(starts))], params)
    qs, qg, tg = [], [], []
    for k, r in enumerate(res):
        if r["status"] != P.SOLVED:
            continue
        wp = waypoints(r["path"].astype(np.float64), spacing=0.05)
        qs += [starts[k]] * len(wp)
        qg += [goals[k]] * len(wp)
        tg += list(wp)
    init = W.proposal_init(robot.dof, init_seed)
    prop = P.Proposal(robot.dof, robot.lower, robot.upper,
                      np.concatenate([np.concatenate([Wm.ravel(), b]) for Wm, b in init]).astype(np.float32))
    losses = prop.train(P.prrtc_occupancy(ev)[None, :], np.zeros(len(tg), np.int32), np.array(qs, np.float32),
                        np.array(qg, np.float32), np.array(tg, np.float32), batch=batch, steps=steps, lr=lr,
                        seed=seed)
    return prop, len(tg), losses


def batched_ttfs(rb: P.Robot, ev: P.Env, starts: np.ndarray, goals: np.ndarray, params: P.prrtc_params,
                 proposal: P.Proposal | None, keys=(1, 2, 3), warmup: int = 2):
    """Plan every pair in one batched call per key (plain when proposal is None,
    else with the learned proposal) and return per-problem TTFS in microseconds
    (device prep, which includes the inference, + setup + the problem's solve
    time), success rate, mean iterations, and the mean prep and inference
    times."""
    def call(key):
        items = [(rb, ev, starts[k], goals[k], key, k) for k in range(len(starts))]
        if proposal is None:
            return P.prrtc_plan_batch(items, params)
        return P.prrtc_plan_batch_learned(items, [proposal] * len(items), params)

    for _ in range(warmup):
        call(97)
    ttfs, iters, ok, prep, infer = [], [], 0, [], []
    for key in keys:
        rs = call(key)
        st = P.prrtc_last_launch_stats()
        prep.append(st["prep_ms"] * 1e3)
        infer.append(st["infer_ms"] * 1e3)
        for r in rs:
            iters.append(r["iterations"])
            if r["status"] == P.SOLVED:
                ok += 1
                ttfs.append(r["solve_time_us"] + 1e3 * (st["prep_ms"] + st["setup_ms"]))
    return dict(ttfs_us=np.array(ttfs), success_rate=ok / (len(starts) * len(keys)),
                iterations_mean=float(np.mean(iters)), prep_us_mean=float(np.mean(prep)),
                infer_us_mean=float(np.mean(infer)))
