"""Serving workload: Poisson arrivals of planning queries against resident,
dynamically updated environments, driven through the library's request loop
(prrtc_server_*).

Scenes are mixed 7/8/14-DoF arms among 40-120 random obstacles plus five
spheres (radius 0.05-0.15 m) that move at 0.5 m/s; their new positions are
published with prrtc_env_update at 30 Hz while queries are in flight.  Each
admitted query plans against a snapshot of its scene taken at admission.
"""
from __future__ import annotations

import threading
import time
from dataclasses import dataclass

import numpy as np

from . import prrtc as P
from . import workload as W

N_MOVING = 5


@dataclass
class ServeScene:
    robot: W.Robot
    rb: P.Robot
    env: P.Env
    scene: W.Scene
    moving: W.MovingSpheres
    moving_ids: list
    queries: list


def build_scenes(n_scenes: int, pairs: int, seed0: int, n_obs=(40, 120)):
    kinds = ["arm7", "arm8", "dual14"]
    out = []
    robots = {k: (W.ROBOTS[k](), None) for k in kinds}
    handles = {}
    for k in range(n_scenes):
        kind = kinds[k % 3]
        robot = robots[kind][0]
        if kind not in handles:
            handles[kind] = P.make_robot(robot)
        seed = seed0 + k
        st = W.Stream(seed, 16)
        base = W.scene_mixed(seed, st.integers(n_obs[0], n_obs[1]), bases=W.robot_bases(robot))
        mv = W.moving_spheres(seed, N_MOVING, bases=W.robot_bases(robot))
        sph = np.concatenate([base.spheres, np.concatenate([mv.centres0, mv.radii[:, None]], axis=1)])
        scene = W.Scene(boxes=base.boxes, cylinders=base.cylinders, spheres=sph)
        env = P.make_env(scene)
        n_total = scene.n_obstacles
        ids = list(range(n_total - N_MOVING, n_total))
        Q = W.candidates(robot, seed, 0, 8192).astype(np.float32)
        free = Q[P.prrtc_check_states(handles[kind], env, Q)]
        m = min(pairs, len(free) // 2)
        qs = [(free[2 * i], free[2 * i + 1]) for i in range(m)]
        out.append(ServeScene(robot, handles[kind], env, scene, mv, ids, qs))
    return out


class ObstacleMover(threading.Thread):
    """Publishes the moving spheres' positions at `rate_hz` until stopped."""

    def __init__(self, scenes, rate_hz: float = 30.0, seconds: float = 30.0):
        super().__init__(daemon=True)
        self.scenes = scenes
        self.period = 1.0 / rate_hz
        self.stop_flag = threading.Event()
        self.ticks = 0
        self.n_ticks = int(seconds * rate_hz) + 1  # pre-computed positions for `seconds` of ticks
        self.tracks = [sc.moving for sc in scenes]
        # the positions last published per scene (read by clients that record what a query saw)
        self.current = [sc.moving.centres0.copy() for sc in scenes]

    def run(self):
        k = 0
        paths = [mv.positions_track(self.n_ticks) for mv in self.tracks]
        while not self.stop_flag.is_set():
            t0 = time.perf_counter()
            k += 1
            for i, (sc, tr) in enumerate(zip(self.scenes, paths)):
                pos = tr[min(k, len(tr) - 1)]
                obs = P.obstacles_from_scene(W.Scene(boxes=np.zeros((0, 15)), cylinders=np.zeros((0, 8)),
                                                     spheres=np.concatenate([pos, sc.moving.radii[:, None]], 1)))
                sc.env.update(sc.moving_ids, obs)
                self.current[i] = np.array(pos, copy=True)
            self.ticks = k
            dt = self.period - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)


def run_rate(server: P.Server, scenes, rate: float, duration_s: float, seed: int, proposals=None, mover=None,
             record=None):
    """Submit queries with exponential inter-arrival gaps for duration_s, then drain.
    With `record` (a list) and `mover`, every query is appended as a dict of its
    scene, query, seed, problem id, the moving spheres' positions published when
    it was submitted, and (after the drain) its status."""
    rng = np.random.default_rng(seed)
    pool = [(si, qi) for si, sc in enumerate(scenes) for qi in range(len(sc.queries))]
    order = rng.permutation(len(pool))
    t0 = time.perf_counter()
    t_next = t0
    k = drawn = skipped = 0
    before = server.stats()["completed"]
    while True:
        now = time.perf_counter()
        if now - t0 >= duration_s:
            break
        if now < t_next:
            time.sleep(min(t_next - now, 0.0005))
            continue
        # like a client that re-reads its sensors, only submit endpoints that are
        # free against the obstacles as currently published
        for _ in range(len(pool)):
            si, qi = pool[order[drawn % len(pool)]]
            drawn += 1
            sc = scenes[si]
            qs, qg = sc.queries[qi]
            if P.prrtc_check_states(sc.rb, sc.env, np.stack([qs, qg])).all():
                break
            skipped += 1
        prop = proposals.get(sc.robot.name) if proposals else None
        ticket = server.submit(sc.rb, sc.env, qs, qg, seed=seed + k, problem_id=k, proposal=prop)
        if record is not None and mover is not None:
            record.append(dict(ticket=ticket, scene=si, query=qi, seed=seed + k, problem_id=k,
                               moving=np.array(mover.current[si], copy=True), learned=prop is not None))
        k += 1
        t_next += rng.exponential(1.0 / rate)
    submitted = k
    server.wait(before + submitted, timeout_s=120.0)
    wall = time.perf_counter() - t0
    res = []
    while len(res) < submitted:
        got = server.poll()
        if not got:
            break
        res += got
    if record is not None:
        by_ticket = {r["ticket"]: r for r in res}
        for q in record:
            if q["ticket"] in by_ticket and "status" not in q:
                q["status"] = by_ticket[q["ticket"]]["status"]
    lat = np.array([r["latency_ms"] for r in res])
    que = np.array([r["queue_ms"] for r in res])
    ok = [r for r in res if r["status"] == P.SOLVED]
    in_coll = sum(r["status"] in (P.START_IN_COLLISION, P.GOAL_IN_COLLISION) for r in res)
    pct = lambda a, p: float(np.percentile(a, p)) if len(a) else None
    return dict(rate_qps=rate, submitted=submitted, completed=len(res), seconds=wall,
                throughput_qps=len(res) / wall if wall > 0 else None,
                latency_ms=dict(p50=pct(lat, 50), p95=pct(lat, 95), p99=pct(lat, 99), mean=float(lat.mean()) if len(lat) else None),
                queue_ms=dict(p50=pct(que, 50), p99=pct(que, 99)),
                success_rate=len(ok) / max(len(res), 1), endpoint_in_collision=in_coll,
                skipped_blocked_endpoints=skipped)


def scene_at(sc: ServeScene, moving_positions) -> W.Scene:
    """The scene with its moving spheres at the given positions (what a query saw)."""
    sph = sc.scene.spheres.copy()
    sph[len(sph) - N_MOVING:, :3] = moving_positions
    return W.Scene(boxes=sc.scene.boxes, cylinders=sc.scene.cylinders, spheres=sph)
