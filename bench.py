#!/usr/bin/env python
"""Benchmark of the pRRTC hot path on GB300 (one JSON line on stdout).

Step = one batched planning launch (prrtc_plan_batch) over the 200-problem
cubby-shelf workload: a synthetic 7-DoF arm, 3x3 shelf of 0.3 m cells plus
clutter (30 cuboids, 10 capped cylinders, 10 spheres), goals inside cubbies,
edge resolution 1/32, range 1.0, 5% goal bias, at most 50k iterations per
problem.  All inputs are seeded and synthetic (stand-ins for the paper's
MotionBenchMaker scenes, which are not available here).

Reported:
  value      edge states checked per second over the device time of the
             setup + planner kernels (CUDA events on the launching stream).
             A state counts once its collision verdict is established: all
             states of a free edge, the first colliding state of a colliding
             one; states an early exit skipped are not counted (they are in
             edge_states_begun_per_s).
  e2e        the same metric over the wall time of the whole C-ABI call with
             host buffers (descriptor upload and result download included).
  ttfs       time to first solution per problem (device %globaltimer from
             launch start), p50/p95/p99; plus single-problem TTFS through
             prrtc_plan (host wall clock, environment resident).
  roofline   the planner kernel's executed lane-ops (the multi-stage check as
             run, counted by the kernel) against the issue-rate bound of the
             SMs (128 lane-instructions / clock / SM).
  mixed_600  the 600-problem mixed 7/8/14-DoF batch in one launch.
  oracle_agreement  serial, lockstep and async statistics against the oracle.
  cpu_baseline  the FP64 oracle on the host cores (bounded sample).

`--impl reference` times the oracle alone on the same workload and metric.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "p50/p95 time-to-first-solution & edge states checked/s; learned vs plain, 1 GB300"
# A state counts once its collision verdict is established: every state of a
# free edge, and the first colliding state of a colliding edge (the states an
# early exit skips do not count).
UNIT = "edge states checked/s"
WORKLOAD = "shelf-200: 200 cubby-shelf problems, 7-DoF arm (28 spheres), 50 obstacles each, one launch"

# Counted arithmetic per test (lane-level instructions of the test as written:
# FADD/FMUL/FFMA/FMNMX/FSETP, MUFU counted once).
OPS = dict(centre=9, aabb=13, obb=22, cyl=24, sph=9, pair=7, joint=17)


def kernel_source_hash():
    """Hash of the planner kernel's code (its sources with comments and blank lines
    removed), to tell whether the committed ncu counters still describe it."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in ["prrtc_device.cuh", "prrtc_launch.h", "prrtc_plan.cu"]:
        h.update(f.encode())
        with open(os.path.join(ROOT, "paper_2503_06757_gb300", "csrc", f), encoding="utf-8") as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        code = "\n".join(line.rstrip() for line in text.splitlines() if line.strip())
        h.update(code.encode())
    return h.hexdigest()[:16]


def profiled_traffic(problems):
    """DRAM bytes per planner launch from the committed ncu summary, scaled by
    problems, or None when the kernel source changed since the capture."""
    try:
        text = open(os.path.join(ROOT, "profiles", "plan_kernel_shelf200_full.md")).read()
        src = text.split("kernel_source:")[1].split()[0]
        per = float(text.split("dram_bytes_per_problem:")[1].split()[0])
    except Exception:
        return None
    return per * problems if src == kernel_source_hash() else None


def result_rows(out):
    """Per-problem dicts of a BatchResult's scalar columns (outside timed regions)."""
    names = [n for n in out._v.dtype.names if n != "q"]
    return [dict(zip(names, row)) for row in out._v[names].tolist()]


def percentiles(v, ps=(50, 95, 99)):
    if not len(v):
        return {f"p{p}": None for p in ps}
    return {f"p{p}": float(np.percentile(v, p)) for p in ps}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """SM clock, power and clock-event reasons read through NVML (read-only)
    every ~1 ms during the timed region; falls back to nvidia-smi."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
               0x80: "hw_power_brake_slowdown"}

    def __init__(self, index=0, period_s=0.001):
        self.index = index
        self.period = period_s
        self.samples = []
        self.running = False
        self.nvml = None
        try:
            import ctypes
            nv = ctypes.CDLL("libnvidia-ml.so.1")
            if nv.nvmlInit_v2() != 0:
                raise OSError("nvmlInit failed")
            h = ctypes.c_void_p()
            if nv.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(index), ctypes.byref(h)) != 0:
                raise OSError("no handle")
            self.nvml, self.h, self.ct = nv, h, ctypes
            mx = ctypes.c_uint()
            nv.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx))
            self.max_mhz = float(mx.value)
            self.reason_fn = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                nv.nvmlDeviceGetCurrentClocksThrottleReasons
        except Exception:
            self.nvml = None

    def _loop(self):
        ct, nv, h = self.ct, self.nvml, self.h
        clk, rs, pw = ct.c_uint(), ct.c_ulonglong(), ct.c_uint()
        while self.running:
            nv.nvmlDeviceGetClockInfo(h, 1, ct.byref(clk))
            self.reason_fn(h, ct.byref(rs))
            nv.nvmlDeviceGetPowerUsage(h, ct.byref(pw))
            self.samples.append((clk.value, rs.value, pw.value))
            time.sleep(self.period)

    def start(self):
        if self.nvml is None:
            return
        self.running = True
        self.t = threading.Thread(target=self._loop, daemon=True)
        self.t.start()

    def stop(self):
        if self.nvml is None:
            return self._smi_once()
        self.running = False
        self.t.join()
        sm = [c for c, _, _ in self.samples]
        reasons = set()
        for _, r, _ in self.samples:
            for bit, name in self.REASONS.items():
                if r & bit:
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": self.max_mhz,
                "reasons": sorted(reasons), "samples": len(sm), "source": "nvml",
                "power_w_max": max(p for _, _, p in self.samples) / 1000.0 if self.samples else None}

    def _smi_once(self):
        try:
            out = subprocess.run(["nvidia-smi", "--query-gpu=clocks.sm,clocks.max.sm", "--format=csv,noheader,nounits"],
                                 capture_output=True, text=True, timeout=20).stdout.split(",")
            return {"sm_mhz": float(out[0]), "sm_max_mhz": float(out[1]), "reasons": [], "samples": 1,
                    "source": "nvidia-smi (after the run)"}
        except Exception:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["clock query unavailable"], "samples": 0}


# ------------------------------------------------------------------ workload

def gpu_accept_factory(P):
    """Start/goal acceptance through the device collision checker."""
    from paper_2503_06757_gb300.accept import device_accept
    return device_accept()


def shelf_problems(accept, count=200, seed0=1000):
    from paper_2503_06757_gb300 import workload as W
    return W.problem_set("shelf", count, seed0, accept)


def boxes8_problem(accept):
    from paper_2503_06757_gb300 import workload as W
    return W.problem_set("boxes8", 1, 1, accept)[0]


PRIM_KINDS = ("aabb", "obb", "cyl", "sph")


def op_count(path, env_counts, dof, dpad):
    """Counted arithmetic of one problem: sphere passes over the whole obstacle set
    (fine spheres of one-stage frames and bounding spheres of two-stage frames),
    second-stage sphere-primitive tests, self pairs, FK joints, NN row distances."""
    a, o, c, s = env_counts
    per_sphere = OPS["centre"] + OPS["aabb"] * a + OPS["obb"] * o + OPS["cyl"] * c + OPS["sph"] * s
    prim = sum(n * OPS[k] for n, k in zip(path["prim_tests"], PRIM_KINDS))
    return (path["sphere_tests"] * per_sphere + prim + path["pair_tests"] * OPS["pair"] +
            path["fk_states"] * OPS["joint"] * dof + path["nn_nodes"] * (2 * dpad + 1))


def one_stage_ops_per_state(env_counts, dof, n_spheres, n_pairs):
    """Algorithmic work of one collision verdict, in counted lane-ops: FK of every
    joint, every distinct sphere against every primitive, every self pair -- the
    one-stage check, whatever the kernel skips."""
    a, o, c, s = env_counts
    per_sphere = OPS["centre"] + OPS["aabb"] * a + OPS["obb"] * o + OPS["cyl"] * c + OPS["sph"] * s
    return OPS["joint"] * dof + n_spheres * per_sphere + n_pairs * OPS["pair"]


def algorithmic_ops(path, env_counts, dof, dpad, n_spheres, n_pairs):
    """States with an established verdict x the one-stage work per state, plus the
    nearest-neighbour distances (2 dpad + 1 per row scanned)."""
    return (path["verdict_states"] * one_stage_ops_per_state(env_counts, dof, n_spheres, n_pairs) +
            path["nn_nodes"] * (2 * dpad + 1))


# ------------------------------------------------------------------ multi-GPU (weak scaling)

def rank_problem_seed(rank: int) -> int:
    """First scene seed of a rank's problem set: every rank plans its own problems
    (independent units, no data-path collective)."""
    return 1000 + 10000 * rank


def reduce_over_ranks(dist, torch, device_s, wall_s, units, device):
    """Whole-job timing and work: the slowest rank's device and wall time, the sum
    of the units all ranks processed.  Without a process group: the inputs."""
    if dist is None:
        return device_s, wall_s, units
    t = torch.tensor([device_s, wall_s], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    n = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(n)
    return float(t[0]), float(t[1]), float(n[0])


# ------------------------------------------------------------------ CPU baseline

def oracle_sample(problems, budget_s=12.0, threads=None):
    """The oracle as it stands on the host cores: whole problems, in chunks of
    `threads`, until the time budget is used."""
    from oracle import oracle as O
    threads = threads or os.cpu_count() or 1
    done, states, wall, solved, costs, per_problem, serial_states = 0, 0, 0.0, 0, [], [], 0
    while done < len(problems) and wall < budget_s:
        chunk = problems[done:done + threads]
        t = time.perf_counter()
        rs = O.plan_batch(chunk, threads=threads, seed=1, problem_ids=list(range(done, done + len(chunk))),
                          range=1.0, resolution=float(np.float32(1 / 32)), goal_bias=float(np.float32(0.05)))
        wall += time.perf_counter() - t
        done += len(chunk)
        for r in rs:
            # the oracle checks an edge's states in order and stops at the first
            # collision: states_checked counts the verdicts it established
            states += r["states_checked"]
            serial_states += r["states_checked"]
            per_problem.append(r["seconds"])
            solved += r["status"] == 0
            if r["status"] == 0:
                costs.append(r["cost"])
    pp = np.array(per_problem) if per_problem else np.zeros(1)
    return dict(value=states / wall if wall > 0 else None, unit=UNIT, cores=threads, kind="oracle",
                sample=f"first {done} of {len(problems)} shelf problems, 1 Philox key, one problem per thread",
                problems=done, seconds=wall, success_rate=solved / max(done, 1),
                mean_cost=float(np.mean(costs)) if costs else None,
                single_core=dict(value=serial_states / max(float(pp.sum()), 1e-12), unit=UNIT,
                                 seconds_per_problem=dict(percentiles(list(pp * 1e3)), unit="ms"),
                                 note="each problem's own thread time: one core per problem"))


def oracle_agreement(P, probs, items, keys=(1, 2, 3), workers=8):
    """Planner statistics against the oracle on the same problems and Philox keys.

    serial:   Alg. 1 in iteration order on one warp against the serial oracle
              (identical trees wherever no decision is ambiguous).
    lockstep: `workers` concurrent iterations per round on a fixed schedule,
              against the oracle's lockstep form (identical trees likewise).
    async:    the concurrent mode with exactly `workers` warps per problem (one
              block per problem, no other blocks joining), against the oracle's
              lockstep form at the same concurrency: the same semantics up to
              the hardware's interleaving, held to success +-1 pp, cost +-2%.
    timed:    the timed launch itself (blocks move to unsolved problems, so a
              problem's concurrency grows as others finish), for reference."""
    import dataclasses
    from oracle import oracle as O
    f32 = lambda x: float(np.float32(x))
    n = len(items)
    out = dict(problems=n, keys=list(keys), workers=workers)
    # the oracle plans from the binary32 start and goal the device receives
    probs = [dataclasses.replace(pb, q_start=pb.q_start.astype(np.float32).astype(np.float64),
                                 q_goal=pb.q_goal.astype(np.float32).astype(np.float64)) for pb in probs]

    def stats(rs):
        ok = [r for r in rs if r["status"] == 0]
        return dict(success_rate=len(ok) / max(len(rs), 1),
                    mean_cost=float(np.mean([r["cost"] for r in ok])) if ok else None)

    def oracle_runs(B):
        rs = []
        for key in keys:
            rs += O.plan_batch(probs, seed=key, problem_ids=list(range(n)), range=1.0, resolution=f32(1 / 32),
                               goal_bias=f32(0.05), workers=B)
        return rs

    def gpu_runs(prm, single=False):
        rs = []
        for key in keys:
            sub = [it[:4] + (key, k) for k, it in enumerate(items)]
            if single:
                for it in sub:
                    rs += P.prrtc_plan_batch([it], prm)
            else:
                rs += P.prrtc_plan_batch(sub, prm)
        return rs

    o_serial, o_lock = oracle_runs(0), oracle_runs(workers)
    out["oracle_serial"] = stats(o_serial)
    out["oracle_lockstep"] = stats(o_lock)
    for name, prm, single, ref in (
            ("serial", P.params(mode=P.MODE_SERIAL), False, o_serial),
            ("lockstep", P.params(mode=P.MODE_LOCKSTEP, workers=workers), False, o_lock),
            ("async", P.params(mode=P.MODE_ASYNC, blocks=1, warps_per_block=workers), True, o_lock)):
        g = gpu_runs(prm, single)
        out[name] = stats(g)
        same = sum(1 for a, b in zip(g, ref) if a["status"] == b["status"] == 0 and abs(a["cost"] - b["cost"]) <= 1e-4 * b["cost"])
        out[name]["same_cost_as_oracle"] = same / max(len(g), 1)
        if out[name]["mean_cost"] and stats(ref)["mean_cost"]:
            out[name]["cost_vs_oracle"] = out[name]["mean_cost"] / stats(ref)["mean_cost"] - 1.0
        out[name]["success_vs_oracle_pp"] = 100.0 * (out[name]["success_rate"] - stats(ref)["success_rate"])
    out["timed"] = stats(gpu_runs(P.params()))
    return out


# ------------------------------------------------------------------ learned proposal and serving

def learned_section(args, P):
    """Train the proposal on plain-planner solution paths (shelf scenes, 7-DoF) and
    compare learned (50% mixture / 50% uniform) with plain sampling on held-out scenes."""
    from paper_2503_06757_gb300 import learned as L
    from paper_2503_06757_gb300 import workload as W
    rb = W.arm7()
    ds = L.build_dataset(rb, args.learned_scenes, args.learned_pairs, 100000)
    prop, losses, tt = L.train(rb, ds, steps=args.learned_steps, batch=512)
    held = L.build_dataset(rb, 30, 10, 900000)
    untrained = L.train(rb, ds, steps=0)[0]
    train = dict(paths=ds.paths, problems=ds.problems, samples=int(len(ds.target)), data_seconds=ds.seconds,
                 steps=args.learned_steps, batch=512, train_seconds=tt,
                 loss_first=float(np.mean(losses[:10])), loss_last=float(np.mean(losses[-10:])),
                 heldout_nll=L.held_out_nll(prop, held), heldout_nll_untrained=L.held_out_nll(untrained, held))
    ev = L.evaluate(rb, args.learned_eval_scenes, 1, 9000, prop, ratio=0.5)
    ev_25 = L.evaluate(rb, args.learned_eval_scenes, 1, 9000, prop, ratio=0.25)["learned"]
    return dict(workload="cubby shelf, 7-DoF arm; held-out scenes 9000.. (one problem each), Philox keys 1..3",
                ratio=0.5, train=train, eval=ev, learned_ratio_0_25=ev_25,
                note="TTFS includes the on-device inference (occupancy grids, layer 1 per distinct scene, one "
                     "fused kernel for the rest) that precedes planning"), prop


def learned_full_section(P, dofs=(7, 14), paths=50000, steps=20000, eval_scenes=500):
    """The learned proposal at its stated size: per arm (7-DoF, and the 14-DoF dual
    arm with the shelf turned to face both arms), at least `paths` plain-planner
    solution paths on seeded shelf scenes, `steps` Adam steps of 512 samples, then
    plain vs 50% learned / 50% uniform sampling on `eval_scenes` held-out scenes
    (one problem each) with the same Philox keys."""
    from paper_2503_06757_gb300 import learned as L
    from paper_2503_06757_gb300 import workload as W
    out = dict(paths_target=paths, steps=steps, eval_scenes=eval_scenes, ratio=0.5)
    for dof in dofs:
        rb = W.arm7() if dof == 7 else W.dual14()
        t0 = time.perf_counter()
        parts, seed0, got = [], 100000, 0
        while got < paths:
            part = L.build_dataset(rb, 500, 40, seed0)
            parts.append(part)
            got += part.paths
            seed0 += 500
        ds = L.concat_datasets(parts)
        data_s = time.perf_counter() - t0
        prop, losses, tt = L.train(rb, ds, steps=steps, batch=512)
        held = L.build_dataset(rb, 30, 10, 900000)
        ev = L.evaluate(rb, eval_scenes, 1, 9000, prop, ratio=0.5)
        out[f"dof{dof}"] = dict(
            robot=rb.name, train=dict(paths=ds.paths, problems=ds.problems, samples=int(len(ds.target)),
                                      data_seconds=data_s, train_seconds=tt, loss_first=float(np.mean(losses[:20])),
                                      loss_last=float(np.mean(losses[-20:])), heldout_nll=L.held_out_nll(prop, held)),
            eval=ev)
    return out


def door_section(P, door, keys=(1, 2, 3)):
    """The learned proposal where its gain is structural: a point robot in two rooms
    joined by a door in a wall (opening `door` in y).  Train on 256 plain-planner
    solutions, then plan 200 held-out pairs in one batched launch, plain vs 50%
    learned, same keys; TTFS includes the call's device prep (for the learned form
    the on-device inference) and setup."""
    from paper_2503_06757_gb300 import learned as L
    from paper_2503_06757_gb300 import workload as W
    rb, sc = W.point2(), W.scene_two_rooms(door=door)
    h, ev = P.make_robot(rb), P.make_env(sc)
    base = dict(range=0.2, resolution=0.01, max_iters=20000, tree_capacity=1 << 14, path_capacity=1 << 12)
    s, g = W.two_rooms_pairs(256, 11)
    prop, samples, losses = L.train_on_plain_solutions(rb, h, ev, s, g, P.params(mode=P.MODE_SERIAL, **base),
                                                        steps=1500)
    s2, g2 = W.two_rooms_pairs(200, 12)
    width = door[1] - door[0]
    out = dict(workload=f"point robot (2 cm sphere), two rooms joined by a {100 * width:.0f} cm door "
                        f"({100 * (width - 0.04):.0f} cm free for the centre); 256 training, 200 held-out pairs, "
                        f"keys {keys[0]}..{keys[-1]}",
               train=dict(samples=samples, loss_first=float(losses[:10].mean()), loss_last=float(losses[-10:].mean())))
    for name in ("plain", "learned"):
        for mode_name, mode in (("async", P.MODE_ASYNC), ("serial", P.MODE_SERIAL)):
            prm = P.params(mode=mode, learned_ratio=0.5 if name == "learned" else 0.0, **base)
            m = L.batched_ttfs(h, ev, s2, g2, prm, prop if name == "learned" else None, keys=keys)
            out[f"{name}_{mode_name}"] = dict(success_rate=m["success_rate"], iterations_mean=m["iterations_mean"],
                                              ttfs_us=percentiles(m["ttfs_us"], (50, 95)) if mode == P.MODE_ASYNC
                                              else None,
                                              prep_us_mean=m["prep_us_mean"], infer_us_mean=m["infer_us_mean"])
    return out


def serving_section(args, P, proposals):
    from paper_2503_06757_gb300 import serving as S
    scenes = S.build_scenes(30, 12, 3000)
    prm = P.params(max_iters=20000, tree_capacity=1 << 13, path_capacity=1 << 12, learned_ratio=0.5)
    server = P.Server(prm, slice_us=300)
    mover = S.ObstacleMover(scenes)
    mover.start()
    out = dict(workload="30 resident scenes (7/8/14-DoF in turn, 40-120 obstacles + 5 spheres moving at "
                        "0.5 m/s, updated at 30 Hz), Poisson arrivals; learned proposal on the 7-DoF queries",
               slice_us=300, slots=server.stats()["slots"])
    try:
        for rate in (200, 1000):
            out[f"rate_{rate}"] = S.run_rate(server, scenes, rate, args.serve_seconds, seed=rate, proposals=proposals)
    finally:
        mover.stop_flag.set()
        mover.join()
        out["obstacle_updates"] = mover.ticks
        out["slices"] = server.stats()["slices"]
        server.close()
    return out


def serving_full_section(args, P, proposals, queries=10000, oracle_sample=96):
    """The serving loop at its stated size: at least `queries` Poisson arrivals per
    rate (200 and 1000 queries/s), then the oracle on a seeded sample of the same
    queries (the scene each one saw at submission, the same seed, budget and tree
    capacity; serial plain sampling): success rates side by side."""
    from oracle import oracle as O
    from paper_2503_06757_gb300 import serving as S
    scenes = S.build_scenes(30, 12, 3000)
    prm = P.params(max_iters=20000, tree_capacity=1 << 13, path_capacity=1 << 12, learned_ratio=0.5)
    server = P.Server(prm, slice_us=300)
    rates = (200, 1000)
    mover = S.ObstacleMover(scenes, seconds=sum(queries / r for r in rates) + 30.0)
    mover.start()
    out = dict(workload="30 resident scenes (7/8/14-DoF in turn, 40-120 obstacles + 5 spheres moving at "
                        "0.5 m/s, updated at 30 Hz), Poisson arrivals; learned proposal on the 7-DoF queries",
               slice_us=300, slots=server.stats()["slots"], queries_per_rate=queries)
    records = {}
    try:
        for rate in rates:
            rec = []
            out[f"rate_{rate}"] = S.run_rate(server, scenes, rate, queries / rate, seed=rate, proposals=proposals,
                                             mover=mover, record=rec)
            records[rate] = rec
    finally:
        mover.stop_flag.set()
        mover.join()
        out["obstacle_updates"] = mover.ticks
        out["slices"] = server.stats()["slices"]
        server.close()
    rng = np.random.default_rng(5)
    for rate, rec in records.items():
        done = [q for q in rec if "status" in q]
        pick = [done[i] for i in sorted(rng.choice(len(done), min(oracle_sample, len(done)), replace=False))]
        probs = []
        for q in pick:
            sc = scenes[q["scene"]]
            qs, qg = sc.queries[q["query"]]
            probs.append(dataclasses_replace_problem(sc.robot, S.scene_at(sc, q["moving"]), qs, qg, q["seed"]))
        t = time.perf_counter()
        orc = O.plan_batch(probs, seeds=[q["seed"] for q in pick], problem_ids=[q["problem_id"] for q in pick],
                           range=1.0, resolution=float(np.float32(1 / 32)), goal_bias=float(np.float32(0.05)),
                           max_iters=20000, tree_capacity=1 << 13, path_capacity=1 << 12)
        secs = time.perf_counter() - t
        rows = dict(plain_both=[], learned_on_gpu=[])
        for q, o in zip(pick, orc):
            rows["learned_on_gpu" if q["learned"] else "plain_both"].append((q["status"] == P.SOLVED, o["status"] == 0))
        out[f"rate_{rate}"]["oracle_sample"] = dict(
            queries=len(pick), oracle_seconds=secs,
            **{k: dict(queries=len(v), gpu_success=float(np.mean([a for a, _ in v])) if v else None,
                       oracle_success=float(np.mean([b for _, b in v])) if v else None) for k, v in rows.items()})
    return out


def dataclasses_replace_problem(robot, scene, qs, qg, seed):
    from paper_2503_06757_gb300 import workload as W
    return W.Problem(robot, scene, np.asarray(qs, np.float64), np.asarray(qg, np.float64), seed)


# ------------------------------------------------------------------ tensor-core GEMM

GEMM_SHAPES = [
    ("proposal layer 1 forward, training batch 512", 512, 1024, 4160),
    ("proposal layer 1 weight gradient, training batch 512", 1024, 4160, 512),
    ("proposal layer 1 inference, 200 problems", 200, 1024, 4160),
    ("proposal layer 2 forward, training batch 512", 512, 512, 1024),
    ("square 8192", 8192, 8192, 8192),
]


def gemm_section(P, torch, peak_tflops, reps=20):
    """The tcgen05 GEMM (BF16 in, FP32 accumulate, BF16 out) at the learned
    proposal's shapes and one large square; CUDA events on the launching stream
    around a CUDA-graph replay of `reps` calls (device time), and around the
    same calls issued one by one (device time plus host call cost); inputs
    resident, split-K reduction included where the library splits."""
    out = dict(peak_tflops=peak_tflops, peak="bf16_tflops (burst) of MEASURED_PEAKS.json", shapes=[])
    stream = torch.cuda.current_stream()
    for name, M, N, K in GEMM_SHAPES:
        g = torch.Generator(device="cuda").manual_seed(M + N + K)
        A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
        B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
        C16 = torch.empty(M, N, device="cuda", dtype=torch.bfloat16)
        call_on = lambda st: P.prrtc_gemm_bf16(A.data_ptr(), B.data_ptr(), M, N, K, 0, False, 0, C16.data_ptr(),
                                               st.cuda_stream)
        call = lambda: call_on(stream)
        n = reps if M * N * K < 1 << 36 else 5
        # launches replayed from a CUDA graph, so host-side call cost does not
        # hide the device time of these short kernels
        side = torch.cuda.Stream()
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            for _ in range(3):
                call_on(side)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=side):
            for _ in range(n):
                call_on(side)
        graph.replay()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        graph.replay()
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / n
        # and through the C ABI call by call (host cost included)
        for _ in range(3):
            call()
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(n):
            call()
        ev1.record(stream)
        torch.cuda.synchronize()
        ms_calls = ev0.elapsed_time(ev1) / n
        tf = 2.0 * M * N * K / (ms * 1e-3) * 1e-12
        err = P.prrtc_gemm_error()
        out["shapes"].append(dict(name=name, M=M, N=N, K=K, us=ms * 1e3, tflops=tf, frac=tf / peak_tflops,
                                  us_per_call_unbatched=ms_calls * 1e3, error=err))
        del A, B, C16, graph
    return out


# ------------------------------------------------------------------ distance-field environments

ESDF_GRID = dict(origin=(-0.8, -0.8, 0.0), voxel=0.02, dims=(80, 80, 80))


def esdf_section(P, torch, items, prm, flush, F, rb_check, steps=5):
    """The benchmark batch against distance fields instead of primitives: each
    scene voxelised (2 cm voxels over the 1.6 m workspace, 80^3) and turned into
    an ESDF environment on the device; then the same planning step and the
    collision-check microbenchmark against one of them."""
    import copy
    g = ESDF_GRID
    t = time.perf_counter()
    envs = {}
    for it in items:
        ev = it[1]
        if id(ev) not in envs:
            occ = ev.voxelize(g["origin"], g["voxel"], g["dims"])
            envs[id(ev)] = P.Env.from_occupancy(occ, g["origin"], g["voxel"])
    build_s = time.perf_counter() - t
    its = [(it[0], envs[id(it[1])]) + tuple(it[2:]) for it in items]
    p = copy.copy(prm)
    for _ in range(2):
        P.prrtc_plan_batch(its, p)
    dev_ms, states, ttfs, solved, pre = 0.0, 0, [], 0, 0
    for _ in range(steps):
        flush.zero_()
        torch.cuda.synchronize()
        res = P.prrtc_plan_batch(its, p)
        st = P.prrtc_last_launch_stats()
        dev_ms += st["kernel_ms"] + st["setup_ms"]
        for r in res:
            states += r["verdict_states"]
            pre += r["status"] in (P.START_IN_COLLISION, P.GOAL_IN_COLLISION)
            if r["status"] == P.SOLVED:
                solved += 1
                ttfs.append(r["solve_time_us"])
    n = len(items) * steps
    ev0 = envs[id(items[0][1])]
    for _ in range(3):
        P.prrtc_check_states(rb_check, ev0, F)
    ms = []
    for _ in range(5):
        flush.zero_()
        torch.cuda.synchronize()
        P.prrtc_check_states(rb_check, ev0, F)
        ms.append(P.prrtc_last_launch_stats()["kernel_ms"])
    kms = float(np.median(ms))
    return dict(grid=g, environments=len(envs), build_ms_per_env=build_s * 1e3 / len(envs),
                ms_per_step=dev_ms / steps, states_checked_per_s=states / (dev_ms * 1e-3), ttfs_us=percentiles(ttfs),
                success_rate=solved / n, endpoint_in_collision_rate=pre / n,
                check_states_microbench=dict(states=int(len(F)), kernel_ms=kms, states_per_s=len(F) / (kms * 1e-3)),
                note="start/goal pairs were chosen against the primitives; the voxelised scene can cover some")


# ------------------------------------------------------------------ mixed-DoF batch

MIXED_WORKLOAD = ("mixed-600: 200 problems each of the 7-, 8- and 14-DoF arms (28 / 32 / 56 spheres), 10-120 "
                  "obstacles per scene (cuboid : cylinder : sphere = 3 : 1 : 1), one persistent autotuned launch")


def mixed_section(args, P, flush, torch, peak_gops, steps=3):
    """The largest single-GPU configuration: 600 problems of uneven DoF, obstacle
    count and tree size in one persistent launch, launch shape from the autotuner."""
    from paper_2503_06757_gb300 import workload as W
    t0 = time.perf_counter()
    probs = W.problem_set("mixed", 600, 2000, gpu_accept_factory(P))
    gen_s = time.perf_counter() - t0
    robots, items, counts = {}, [], []
    for k, pb in enumerate(probs):
        if pb.robot.name not in robots:
            robots[pb.robot.name] = P.make_robot(pb.robot)
        rb = robots[pb.robot.name]
        ev = P.make_env(pb.scene)
        info = rb.info()
        counts.append((ev.info(), pb.robot.dof, info["dpad"], info["n_spheres"], info["n_pairs"]))
        items.append((rb, ev, pb.q_start, pb.q_goal, 1, k))
    prm, tuned_ms = P.prrtc_autotune(items, P.params(), trials=3)
    batch = P.PlanBatch(items)
    for _ in range(2):
        batch.run(prm)
    dev_ms = kms = 0.0
    states = begun = ops = alg = 0
    by = {d: dict(ttfs=[], solved=0, n=0, costs=[]) for d in (7, 8, 14)}
    for _ in range(steps):
        flush.zero_()
        torch.cuda.synchronize()
        res = result_rows(batch.run(prm))
        st = P.prrtc_last_launch_stats()
        dev_ms += st["kernel_ms"] + st["setup_ms"]
        kms += st["kernel_ms"]
        for r, (ec, dof, dpad, nsph, npair) in zip(res, counts):
            states += r["verdict_states"]
            begun += r["edge_states"]
            ops += op_count(r, ec, dof, dpad)
            alg += algorithmic_ops(r, ec, dof, dpad, nsph, npair)
            b = by[dof]
            b["n"] += 1
            if r["status"] == P.SOLVED:
                b["solved"] += 1
                b["ttfs"].append(r["solve_time_us"])
                b["costs"].append(r["cost"])
    executed = ops / (kms * 1e-3) * 1e-9
    one_stage = alg / (kms * 1e-3) * 1e-9
    all_ttfs = [t for b in by.values() for t in b["ttfs"]]
    return dict(
        workload=MIXED_WORKLOAD, problems=len(items), steps=steps, problem_set_seconds=gen_s,
        launch=dict(blocks=prm.blocks, warps_per_block=prm.warps_per_block, obstacle_tile=prm.obstacle_tile,
                    expansions=prm.expansions, autotuned_score_ms=tuned_ms, trials=3),
        ms_per_step=dev_ms / steps, states_checked_per_s=states / (dev_ms * 1e-3),
        edge_states_begun_per_s=begun / (dev_ms * 1e-3),
        ttfs_us=dict(percentiles(all_ttfs), note="solved problems, device time from launch start"),
        success_rate=sum(b["solved"] for b in by.values()) / max(1, sum(b["n"] for b in by.values())),
        by_dof={str(d): dict(success_rate=b["solved"] / max(b["n"], 1), ttfs_us=percentiles(b["ttfs"]),
                             mean_cost=float(np.mean(b["costs"])) if b["costs"] else None) for d, b in by.items()},
        roofline=dict(bound="alu", achieved=executed, peak=peak_gops, unit="Gop/s", frac=executed / peak_gops,
                      one_stage_equivalent_gops=one_stage, one_stage_equivalent_frac=one_stage / peak_gops,
                      note="planner kernel over the whole launch, counted as on the main line"))


# ------------------------------------------------------------------ sampler / check variants

DD_PARAMS = dict(dd_radius=5.0, dd_alpha=0.02, dd_min_radius=4.0)


def variants_section(args, P, items, prm, counts, flush, torch, steps=5):
    """The method's optional parts on the benchmark batch, same keys and launch
    shape: one-stage vs multi-stage check, Philox vs Halton sampling,
    dynamic-domain sampling on/off."""
    import copy
    robots = {id(it[0]): it[0] for it in items}
    variants = [("baseline", {}, True), ("one_stage", {}, False),
                ("halton", dict(sampler=P.SAMPLER_HALTON), True),
                ("dynamic_domain", dict(DD_PARAMS), True),
                ("halton_dynamic_domain", dict(DD_PARAMS, sampler=P.SAMPLER_HALTON), True)]
    out = dict(workload=WORKLOAD, steps=steps, dynamic_domain_params=DD_PARAMS,
               note="baseline = multi-stage check, Philox sampling, no dynamic domain (the main line's step)")
    for name, kw, two in variants:
        for rb in robots.values():
            rb.set_two_stage(two)
        p = copy.copy(prm)
        for k, v in kw.items():
            setattr(p, k, v)
        for _ in range(2):
            P.prrtc_plan_batch(items, p)
        dev_ms, kms, states, ops, ttfs, iters, costs, solved, rej = 0.0, 0.0, 0, 0, [], [], [], 0, 0
        begun = 0
        alg = 0
        for _ in range(steps):
            flush.zero_()
            torch.cuda.synchronize()
            res = P.prrtc_plan_batch(items, p)
            st = P.prrtc_last_launch_stats()
            dev_ms += st["kernel_ms"] + st["setup_ms"]
            kms += st["kernel_ms"]
            for r, (ec, dof, dpad, nsph, npair) in zip(res, counts):
                states += r["verdict_states"]
                begun += r["edge_states"]
                ops += op_count(r, ec, dof, dpad)
                alg += algorithmic_ops(r, ec, dof, dpad, nsph, npair)
                iters.append(r["iterations"])
                rej += r["dd_rejected"]
                if r["status"] == P.SOLVED:
                    solved += 1
                    ttfs.append(r["solve_time_us"])
                    costs.append(r["cost"])
        n = len(items) * steps
        out[name] = dict(ms_per_step=dev_ms / steps, states_checked_per_s=states / (dev_ms * 1e-3),
                         edge_states_begun_per_s=begun / (dev_ms * 1e-3),
                         ttfs_us=percentiles(ttfs), success_rate=solved / n,
                         iterations_mean=float(np.mean(iters)), cost_mean=float(np.mean(costs)) if costs else None,
                         dd_rejected_per_problem=rej / n, planner_executed_gops=ops / (kms * 1e-3) * 1e-9,
                         planner_one_stage_equivalent_gops=alg / (kms * 1e-3) * 1e-9)
    for rb in robots.values():
        rb.set_two_stage(True)
    return out


# ------------------------------------------------------------------ arms

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import oracle as O
    # the oracle builds its own start/goal acceptance
    probs = shelf_problems(O.accept, count=args.problems)
    budget = max(2.0, 60.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        oracle_sample(probs, budget_s=budget / 4)
    vals, secs = [], []
    last = None
    for _ in range(args.steps):
        r = oracle_sample(probs, budget_s=budget)
        vals.append(r["value"])
        secs.append(r["seconds"])
        last = r
    value = float(np.mean(vals))
    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=args.gpus, steps=args.steps, warmup=args.warmup,
                ms_per_step=1e3 * float(np.mean(secs)), higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f64", data="synthetic", impl="reference",
                config=dict(workload=WORKLOAD, problems=args.problems, sample="bounded per step"),
                cpu_baseline=dict(last, value=value),
                e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line))
    return 0


def run_ours(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        # the library keeps its own CUDA runtime state: give each rank one visible GPU
        os.environ["CUDA_VISIBLE_DEVICES"] = str(local)
    import torch
    from paper_2503_06757_gb300 import build as B
    B.build()
    from paper_2503_06757_gb300 import prrtc as P
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.init()
    dev_props = torch.cuda.get_device_properties(0)
    sms = dev_props.multi_processor_count

    accept = gpu_accept_factory(P)
    probs = shelf_problems(accept, count=args.problems, seed0=rank_problem_seed(rank))
    robots, envs, items, counts = {}, [], [], []
    for k, pb in enumerate(probs):
        if pb.robot.name not in robots:
            robots[pb.robot.name] = P.make_robot(pb.robot)
        rb = robots[pb.robot.name]
        ev = P.make_env(pb.scene)
        envs.append(ev)
        info = rb.info()
        counts.append((ev.info(), pb.robot.dof, info["dpad"], info["n_spheres"], info["n_pairs"]))
        items.append((rb, ev, pb.q_start, pb.q_goal, 1, rank * args.problems + k))
    prm = P.params(tree_capacity=args.tree_capacity)
    tuned = None
    if args.blocks or args.warps:
        # a fixed launch shape (e.g. to profile the shape the autotuner picked)
        prm.blocks, prm.warps_per_block = args.blocks, args.warps
    elif not args.no_autotune:
        prm, tuned_ms = P.prrtc_autotune(items, prm, trials=16)
        tuned = dict(blocks=prm.blocks, warps_per_block=prm.warps_per_block, obstacle_tile=prm.obstacle_tile,
                     expansions=prm.expansions, score_ms=tuned_ms,
                     score="mean of the batch p50 and p95 time to first solution, averaged over trials", trials=16)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    batch = P.PlanBatch(items)  # marshalled once; every run uploads its descriptors again
    for _ in range(args.warmup):
        batch.run(prm)
    torch.cuda.synchronize()

    clocks = ClockSampler(0)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("timed")
    dev_ms, wall_s, edge_states, ops, launches, h2d, d2h = 0.0, 0.0, 0, 0, 0, 0, 0
    verdict_states = 0
    alg_ops = 0
    kernel_ms = 0.0
    ttfs, solved, costs = [], 0, []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        out = batch.run(prm)
        wall_s += time.perf_counter() - t
        res = result_rows(out)
        st = P.prrtc_last_launch_stats()
        dev_ms += st["kernel_ms"] + st["setup_ms"]
        kernel_ms += st["kernel_ms"]
        launches += st["kernels"]
        h2d += st["h2d_bytes"]
        d2h += st["d2h_bytes"]
        for r, (ec, dof, dpad, nsph, npair) in zip(res, counts):
            edge_states += r["edge_states"]
            verdict_states += r["verdict_states"]
            ops += op_count(r, ec, dof, dpad)
            alg_ops += algorithmic_ops(r, ec, dof, dpad, nsph, npair)
            if r["status"] == P.SOLVED:
                solved += 1
                ttfs.append(r["solve_time_us"])
                costs.append(r["cost"])
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    plan_grid = dict(blocks=st["grid"], threads=st["block_threads"], smem=st["smem_bytes"])
    if dist:
        dist.barrier()
    clk = clocks.stop()

    device_s, wall_s, total_states = reduce_over_ranks(dist, torch, dev_ms * 1e-3, wall_s, verdict_states,
                                                       "cuda" if torch.cuda.is_available() else "cpu")
    value = total_states / device_s
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak_gops = sms * 128 * sm_max * 1e-3
    achieved_gops = alg_ops / (kernel_ms * 1e-3) * 1e-9
    executed_gops = ops / (kernel_ms * 1e-3) * 1e-9

    extra = {}
    if rank == 0 and not args.quick:
        # single-problem TTFS through prrtc_plan (host wall clock, env resident)
        boxes8 = boxes8_problem(accept)
        rb1, ev1 = P.make_robot(boxes8.robot), P.make_env(boxes8.scene)
        p1 = P.params()
        if not args.no_autotune:
            p1, _ = P.prrtc_autotune([(rb1, ev1, boxes8.q_start, boxes8.q_goal, 101, 0)], p1, trials=8)
        for key in range(1, 4):
            p1.seed = key
            P.prrtc_plan(rb1, ev1, boxes8.q_start, boxes8.q_goal, p1)
        tt, ok = [], 0
        for key in range(1, 101):
            p1.seed = key
            t = time.perf_counter()
            r = P.prrtc_plan(rb1, ev1, boxes8.q_start, boxes8.q_goal, p1)
            tt.append((time.perf_counter() - t) * 1e3)
            ok += r["status"] == P.SOLVED
        extra["ttfs_single_boxes8_ms"] = dict(percentiles(tt), success_rate=ok / 100, keys=100,
                                          launch=dict(blocks=p1.blocks, warps_per_block=p1.warps_per_block),
                                          workload="boxes8: 7-DoF arm, 8 random cuboids, one problem, keys 1..100")
        # collision-check microbenchmark: collision-free shelf states, every test runs
        pb = probs[0]
        rb, ev = robots[pb.robot.name], envs[0]
        from paper_2503_06757_gb300 import workload as W
        Q = W.candidates(pb.robot, 7, 3, 1 << 21).astype(np.float32)
        F = Q[P.prrtc_check_states(rb, ev, Q)][: 1 << 20]
        ec = ev.info()
        per_sphere = OPS["centre"] + OPS["aabb"] * ec[0] + OPS["obb"] * ec[1] + OPS["cyl"] * ec[2] + OPS["sph"] * ec[3]
        micro = {}
        for name, two in (("two_stage", True), ("one_stage", False)):
            rb.set_two_stage(two)
            for _ in range(3):
                P.prrtc_check_states(rb, ev, F)
            ms = []
            for _ in range(5):
                flush.zero_()
                torch.cuda.synchronize()
                P.prrtc_check_states(rb, ev, F)
                ms.append(P.prrtc_last_launch_stats()["kernel_ms"])
            st = P.prrtc_last_launch_stats()
            cc_ops = (st["sphere_tests"] * per_sphere + st["pair_tests"] * OPS["pair"] +
                      st["fk_states"] * OPS["joint"] * 7 +
                      sum(n * OPS[k] for n, k in zip(st["prim_tests"], PRIM_KINDS)))
            kms = float(np.median(ms))
            info = rb.info()
            alg_state = one_stage_ops_per_state(ec, pb.robot.dof, info["n_spheres"], info["n_pairs"])
            alg_gops = len(F) * alg_state / (kms * 1e-3) * 1e-9
            micro[name] = dict(
                bound="alu", achieved=alg_gops, peak=peak_gops, unit="Gop/s", frac=alg_gops / peak_gops,
                executed_gops=cc_ops / (kms * 1e-3) * 1e-9, executed_frac=cc_ops / (kms * 1e-3) * 1e-9 / peak_gops,
                states=int(len(F)), kernel_ms=kms, states_per_s=len(F) / (kms * 1e-3),
                executed_ops_per_state=cc_ops / len(F), algorithmic_ops_per_state=alg_state)
        rb.set_two_stage(True)
        extra["roofline_cc_microbench"] = dict(micro["two_stage"], one_stage=micro["one_stage"],
                                               workload="1M collision-free 7-DoF states vs one shelf scene "
                                                        "(every test runs)")
        # the roofline's denominator checked on the device: an FP32 FMA loop
        fma_rate, fma_ms = P.prrtc_alu_peak(16384)
        extra["alu_peak_microbench"] = dict(
            measured_gops=fma_rate * 1e-9, peak_gops=peak_gops, ratio=fma_rate * 1e-9 / peak_gops,
            kernel_ms=fma_ms, note="8 independent FMA chains per thread, 64 warps per SM; one FMA = one lane-op")
        if not args.no_mixed:
            extra["mixed_600"] = mixed_section(args, P, flush, torch, peak_gops)
        extra["variants"] = variants_section(args, P, items, prm, counts, flush, torch)
        extra["esdf"] = esdf_section(P, torch, items, prm, flush, F, rb)
        extra["roofline_gemm"] = gemm_section(P, torch, float(peaks.get("bf16_tflops", 1900.0)))
        extra["cpu_baseline"] = oracle_sample(probs, budget_s=args.cpu_budget)
        extra["oracle_agreement"] = oracle_agreement(P, probs, items)
        prop = None
        if not args.no_learned:
            extra["learned"], prop = learned_section(args, P)
            extra["learned"]["door_8cm"] = door_section(P, (0.85, 0.93))
            extra["learned"]["door_5cm"] = door_section(P, (0.865, 0.915))
        if not args.no_serving:
            extra["serving"] = serving_section(args, P, {"arm7": prop} if prop is not None else None)

    line = dict(
        metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
        ms_per_step=dev_ms / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f32",
        data="synthetic",
        config=dict(workload=WORKLOAD, problems=args.problems, problems_per_gpu=args.problems,
                    l2="flushed between steps (256 MiB write)", mode="async", range=1.0, resolution=1 / 32,
                    goal_bias=0.05, max_iters=50000, grid=plan_grid, autotuned=tuned, parallelism=f"problems sharded over {world} GPU(s)"),
        ttfs_us=dict(percentiles(ttfs), note="device time from launch start to each problem's solution"),
        success_rate=solved / (len(items) * args.steps), mean_cost=float(np.mean(costs)) if costs else None,
        edge_states_begun_per_s=edge_states / (dev_ms * 1e-3),
        roofline=dict(bound="alu", achieved=executed_gops, peak=peak_gops, unit="Gop/s",
                      frac=executed_gops / peak_gops, traffic=profiled_traffic(args.problems),
                      one_stage_equivalent_gops=achieved_gops, one_stage_equivalent_frac=achieved_gops / peak_gops,
                      peak_at_sampled_clock_gops=(sms * 128 * clk["sm_mhz"] * 1e-3) if clk.get("sm_mhz") else None,
                      note="planner kernel: the lane-ops the method ran (FK, the multi-stage sphere hierarchy of "
                           "Sec. III-A as executed, self pairs, NN row distances; counted by the kernel) per "
                           "kernel time, against SMs x 128 lanes x max SM clock (of measured sm_max_mhz).  "
                           "one_stage_equivalent_*: the same verdicts priced as a one-stage check (every sphere "
                           "against every primitive), which the hierarchy never runs"),
        e2e=dict(value=total_states / wall_s, unit=UNIT, h2d_bytes_per_step=h2d // args.steps,
                 d2h_bytes_per_step=d2h // args.steps),
        gpu_launches=launches, clocks=clk, learned=None, serving=None,
    )
    line.update(extra)
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--problems", type=int, default=200)
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--quick", action="store_true", help="skip the side measurements")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--blocks", type=int, default=0, help="fixed planner grid (skips the autotuner)")
    ap.add_argument("--warps", type=int, default=0, help="fixed warps per planner block (skips the autotuner)")
    ap.add_argument("--tree-capacity", type=int, default=1 << 16, help="nodes per tree per problem")
    ap.add_argument("--no-mixed", action="store_true", help="skip the 600-problem mixed-DoF section")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--learned-scenes", type=int, default=1250)
    ap.add_argument("--learned-pairs", type=int, default=40)
    ap.add_argument("--learned-steps", type=int, default=3000)
    ap.add_argument("--learned-eval-scenes", type=int, default=500)
    ap.add_argument("--serve-seconds", type=float, default=2.0)
    ap.add_argument("--serving-full", action="store_true",
                    help="only the serving loop at its stated size (10^4 queries per rate) with an oracle sample; "
                         "one JSON line")
    ap.add_argument("--learned-full", action="store_true",
                    help="only the learned proposal at its stated size (7- and 14-DoF networks, 50k paths each, "
                         "500 held-out scenes); one JSON line")
    ap.add_argument("--gemm-only", action="store_true",
                    help="only the tensor-core GEMM microbenchmark (one JSON line; for profiling the GEMM)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.serving_full:
        import torch
        from paper_2503_06757_gb300 import build as B
        B.build()
        from paper_2503_06757_gb300 import prrtc as P
        torch.cuda.init()
        _, prop = learned_section(args, P)
        print(json.dumps(dict(section="serving_full", **serving_full_section(args, P, {"arm7": prop}))))
        return 0
    if args.learned_full:
        import torch
        from paper_2503_06757_gb300 import build as B
        B.build()
        from paper_2503_06757_gb300 import prrtc as P
        torch.cuda.init()
        print(json.dumps(dict(section="learned_full", **learned_full_section(P))))
        return 0
    if args.gemm_only:
        import torch
        from paper_2503_06757_gb300 import build as B
        B.build()
        from paper_2503_06757_gb300 import prrtc as P
        torch.cuda.init()
        print(json.dumps(gemm_section(P, torch, float(measured_peaks().get("bf16_tflops", 1900.0)))))
        return 0
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
