"""ctypes front end of the FP64 CPU oracle (prrtc_oracle.c).

TEST INFRASTRUCTURE: only the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` import this module.  It builds and loads its
own shared library with gcc and never touches the CUDA path.

Functions follow pRRTC (Huang et al. 2025): Alg. 1 (top-level loop), Alg. 2
(pEXTEND), Sec. III-A (sphere-model collision checking), Sec. III-C (nearest
neighbour); sampling uses Philox4x32-10 (Salmon et al., SC'11) or the paper's Halton
sequence (Sec. IV-A); dynamic-domain sampling (Yershova et al. 2005, adaptive
radius of Jaillet et al. 2005) is the heuristic the paper adds to Alg. 1.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "prrtc_oracle.c")
HDR = os.path.join(HERE, "prrtc_oracle.h")
LIB = os.path.join(HERE, "_build", "liboracle.so")

_PD = C.POINTER(C.c_double)
_PI = C.POINTER(C.c_int32)


class OrcRobot(C.Structure):
    _fields_ = [
        ("dof", C.c_int32), ("joint_type", _PI), ("joint_parent", _PI), ("joint_base", _PD),
        ("link_length", _PD), ("lower", _PD), ("upper", _PD), ("n_spheres", C.c_int32),
        ("sphere_frame", _PI), ("sphere_offset", _PD), ("sphere_radius", _PD),
        ("n_pairs", C.c_int32), ("pairs", _PI),
    ]


class OrcEnv(C.Structure):
    _fields_ = [
        ("n_box", C.c_int32), ("box", _PD), ("n_cyl", C.c_int32), ("cyl", _PD),
        ("n_sph", C.c_int32), ("sph", _PD), ("esdf", _PD), ("esdf_origin", C.c_double * 3),
        ("esdf_voxel", C.c_double), ("esdf_dims", C.c_int32 * 3),
    ]


class OrcParams(C.Structure):
    _fields_ = [
        ("range", C.c_double), ("resolution", C.c_double), ("goal_bias", C.c_double),
        ("amb_band", C.c_double), ("amb_rel", C.c_double), ("seed", C.c_uint64),
        ("problem", C.c_uint32), ("max_iters", C.c_int32), ("tree_capacity", C.c_int32),
        ("path_capacity", C.c_int32), ("gmm", _PD), ("learned_ratio", C.c_double),
        ("sampler", C.c_int32), ("halton_offset", C.c_uint32), ("dd_radius", C.c_double),
        ("dd_alpha", C.c_double), ("dd_min_radius", C.c_double), ("workers", C.c_int32),
    ]


class OrcResult(C.Structure):
    _fields_ = [
        ("status", C.c_int32), ("iterations", C.c_int32), ("n_a", C.c_int32), ("n_b", C.c_int32),
        ("join_a", C.c_int32), ("join_b", C.c_int32), ("path_n", C.c_int32),
        ("first_amb_iter", C.c_int32), ("first_amb_kind", C.c_int32), ("pad_", C.c_int32),
        ("cost", C.c_double), ("edges_checked", C.c_int64), ("states_checked", C.c_int64),
        ("edge_states", C.c_int64), ("dd_rejected", C.c_int64), ("nodes_a", _PD), ("parent_a", _PI),
        ("nodes_b", _PD), ("parent_b", _PI), ("path", _PD), ("radius_a", _PD), ("radius_b", _PD),
    ]


class OrcProblem(C.Structure):
    _fields_ = [
        ("robot", C.POINTER(OrcRobot)), ("env", C.POINTER(OrcEnv)), ("q_start", _PD),
        ("q_goal", _PD), ("params", OrcParams), ("result", C.POINTER(OrcResult)),
        ("seconds", C.c_double),
    ]


STATUS = {0: "solved", 1: "start_in_collision", 2: "goal_in_collision", 3: "no_solution",
          4: "path_overflow", -1: "bad_input"}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (binary64, no FMA contraction)."""
    newest = max(os.path.getmtime(SRC), os.path.getmtime(HDR))
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    tmp = LIB + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11",
                           "-D_POSIX_C_SOURCE=200809L", "-o", tmp, SRC, "-lm", "-lpthread"])
    os.replace(tmp, LIB)
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        try:
            _lib = C.CDLL(LIB)
        except OSError:  # stale binary for another architecture
            build(force=True)
            _lib = C.CDLL(LIB)
        _lib.orc_sd_box.restype = C.c_double
        _lib.orc_sd_cyl.restype = C.c_double
        _lib.orc_sd_sph.restype = C.c_double
        _lib.orc_clearance.restype = C.c_double
        _lib.orc_plan.restype = C.c_int32
        _lib.orc_revalidate.restype = C.c_int32
        _lib.orc_sample.restype = C.c_int
        _lib.orc_sample_learned.restype = C.c_int
        _lib.orc_esdf_query.restype = C.c_double
        _lib.orc_esdf_at.restype = C.c_double
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_PD)


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(_PI)


class _Holder:
    """Keeps numpy buffers alive while a ctypes struct points into them."""

    def __init__(self):
        self.keep = []

    def d(self, a):
        a, p = _d(a)
        self.keep.append(a)
        return p

    def i(self, a):
        a, p = _i(a)
        self.keep.append(a)
        return p


def make_robot(robot):
    h = _Holder()
    s = OrcRobot(
        dof=robot.dof, joint_type=h.i(robot.joint_type), joint_parent=h.i(robot.joint_parent),
        joint_base=h.d(robot.joint_base.reshape(-1)), link_length=h.d(robot.link_length),
        lower=h.d(robot.lower), upper=h.d(robot.upper), n_spheres=robot.n_spheres,
        sphere_frame=h.i(robot.sphere_frame), sphere_offset=h.d(robot.sphere_offset.reshape(-1)),
        sphere_radius=h.d(robot.sphere_radius), n_pairs=int(robot.self_pairs.shape[0]),
        pairs=h.i(robot.self_pairs.reshape(-1) if robot.self_pairs.size else np.zeros(2, np.int32)),
    )
    s._holder = h
    return s


def make_env(scene, esdf=None):
    """esdf (optional): (values [nz, ny, nx] or flat, origin xyz, voxel size)."""
    h = _Holder()
    b = scene.boxes.reshape(-1) if scene.boxes.size else np.zeros(15)
    c = scene.cylinders.reshape(-1) if scene.cylinders.size else np.zeros(8)
    p = scene.spheres.reshape(-1) if scene.spheres.size else np.zeros(4)
    s = OrcEnv(n_box=int(scene.boxes.shape[0]), box=h.d(b), n_cyl=int(scene.cylinders.shape[0]),
               cyl=h.d(c), n_sph=int(scene.spheres.shape[0]), sph=h.d(p))
    if esdf is not None:
        vals, origin, voxel, dims = esdf
        s.esdf = h.d(np.asarray(vals, np.float64).reshape(-1))
        s.esdf_origin[:] = [float(x) for x in origin]
        s.esdf_voxel = float(voxel)
        s.esdf_dims[:] = [int(x) for x in dims]
    s._holder = h
    return s


def voxelize(scene, origin, voxel, dims):
    """Occupancy [nz, ny, nx] (uint8): voxel centre strictly inside some primitive."""
    e = make_env(scene)
    o = np.ascontiguousarray(origin, dtype=np.float64)
    d = (C.c_int32 * 3)(*[int(x) for x in dims])
    out = np.zeros(int(np.prod(dims)), dtype=np.uint8)
    lib().orc_voxelize(C.byref(e), o.ctypes.data_as(_PD), C.c_double(voxel), d,
                       out.ctypes.data_as(C.POINTER(C.c_uint8)))
    return out.reshape(dims[2], dims[1], dims[0])


def esdf(occ, dims, voxel):
    """Signed Euclidean distance field [nz, ny, nx] of an occupancy grid (brute force)."""
    o = np.ascontiguousarray(np.asarray(occ, np.uint8).reshape(-1))
    d = (C.c_int32 * 3)(*[int(x) for x in dims])
    out = np.zeros(o.size)
    lib().orc_esdf(o.ctypes.data_as(C.POINTER(C.c_uint8)), d, C.c_double(voxel), out.ctypes.data_as(_PD))
    return out.reshape(dims[2], dims[1], dims[0])


def esdf_at(occ, dims, voxel, i, j, k):
    o = np.ascontiguousarray(np.asarray(occ, np.uint8).reshape(-1))
    d = (C.c_int32 * 3)(*[int(x) for x in dims])
    return float(lib().orc_esdf_at(o.ctypes.data_as(C.POINTER(C.c_uint8)), d, C.c_double(voxel), C.c_int32(i),
                                   C.c_int32(j), C.c_int32(k)))


def esdf_query(values, origin, voxel, dims, p):
    v = np.ascontiguousarray(np.asarray(values, np.float64).reshape(-1))
    o = np.ascontiguousarray(origin, dtype=np.float64)
    d = (C.c_int32 * 3)(*[int(x) for x in dims])
    pp = np.ascontiguousarray(p, dtype=np.float64)
    return float(lib().orc_esdf_query(v.ctypes.data_as(_PD), o.ctypes.data_as(_PD), C.c_double(voxel), d,
                                      pp.ctypes.data_as(_PD)))


# ------------------------------------------------------------------ primitives

def philox(ctr, key):
    ctr = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    key = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    out = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(ctr, key, out)
    return [int(x) for x in out]


def philox_blocks(ctr, key64):
    """Philox4x32-10 of n counters ([n x 4] uint32) under a 64-bit key (low word first)."""
    c = np.ascontiguousarray(np.asarray(ctr, np.uint32).reshape(-1, 4))
    out = np.zeros_like(c)
    key = (C.c_uint32 * 2)(int(key64) & 0xFFFFFFFF, (int(key64) >> 32) & 0xFFFFFFFF)
    P32 = C.POINTER(C.c_uint32)
    lib().orc_philox_blocks(c.ctypes.data_as(P32), C.c_int32(c.shape[0]), key, out.ctypes.data_as(P32))
    return out


def sample(robot, seed, problem, it, goal_bias):
    r = make_robot(robot)
    q = np.zeros(robot.dof)
    g = lib().orc_sample(C.byref(r), C.c_uint64(seed), C.c_uint32(problem), C.c_uint32(it),
                         C.c_double(goal_bias), q.ctypes.data_as(_PD))
    return bool(g), q


def sample_learned(robot, seed, problem, it, goal_bias, gmm, learned_ratio, amb_rel=1e-5):
    r = make_robot(robot)
    q = np.zeros(robot.dof)
    g = np.ascontiguousarray(gmm, dtype=np.float64)
    amb = C.c_int()
    kind = lib().orc_sample_learned(C.byref(r), C.c_uint64(seed), C.c_uint32(problem), C.c_uint32(it),
                                    C.c_double(goal_bias), g.ctypes.data_as(_PD), C.c_double(learned_ratio),
                                    C.c_double(amb_rel), q.ctypes.data_as(_PD), C.byref(amb))
    return int(kind), q, bool(amb.value)


def halton(index, dim):
    u = np.zeros(dim)
    lib().orc_halton(C.c_uint32(index), C.c_int32(dim), u.ctypes.data_as(_PD))
    return u


def occupancy(scene, origin=(-0.8, -0.8, 0.0), cell=0.1, n=16, radius=0.05):
    e = make_env(scene)
    o = np.ascontiguousarray(origin, dtype=np.float64)
    out = np.zeros(n * n * n, dtype=np.uint8)
    lib().orc_occupancy(C.byref(e), o.ctypes.data_as(_PD), C.c_double(cell), C.c_int32(n), C.c_double(radius),
                        out.ctypes.data_as(C.POINTER(C.c_uint8)))
    return out


def fk(robot, q):
    r = make_robot(robot)
    q, qp = _d(q)
    cen = np.zeros((robot.n_spheres, 3))
    fr = np.zeros((robot.dof, 4, 4))
    lib().orc_fk(C.byref(r), qp, cen.ctypes.data_as(_PD), fr.ctypes.data_as(_PD))
    return cen, fr


def sd_box(box15, p):
    b, bp = _d(box15)
    p, pp = _d(p)
    return float(lib().orc_sd_box(bp, pp))


def sd_cyl(cyl8, p):
    b, bp = _d(cyl8)
    p, pp = _d(p)
    return float(lib().orc_sd_cyl(bp, pp))


def sd_sph(sph4, p):
    b, bp = _d(sph4)
    p, pp = _d(p)
    return float(lib().orc_sd_sph(bp, pp))


def clearance(robot, scene, q, esdf=None):
    r, e = make_robot(robot), make_env(scene, esdf)
    q, qp = _d(q)
    ce, cs = C.c_double(), C.c_double()
    t = lib().orc_clearance(C.byref(r), C.byref(e), qp, C.byref(ce), C.byref(cs))
    return float(t), float(ce.value), float(cs.value)


def check_states(robot, scene, Q, esdf=None):
    r, e = make_robot(robot), make_env(scene, esdf)
    Q, qp = _d(np.asarray(Q).reshape(-1, robot.dof))
    n = Q.shape[0]
    free = np.zeros(n, dtype=np.uint8)
    cl = np.zeros(n)
    lib().orc_check_states(C.byref(r), C.byref(e), qp, C.c_int32(n),
                           free.ctypes.data_as(C.POINTER(C.c_uint8)), cl.ctypes.data_as(_PD))
    return free.astype(bool), cl


def accept(robot, scene, Q):
    """Start/goal acceptance for workload.choose_problem: free mask + end-effector positions."""
    free, _ = check_states(robot, scene, Q)
    ee = np.zeros((Q.shape[0], len(robot.ee_frames), 3))
    for i in np.nonzero(free)[0]:
        _, fr = fk(robot, Q[i])
        for k, f in enumerate(robot.ee_frames):
            ee[i, k] = fr[f, :3, 3]
    return free, ee


# ------------------------------------------------------------------ planner

DEFAULT_PARAMS = dict(range=1.0, resolution=1.0 / 32.0, goal_bias=0.05, amb_band=1e-5, amb_rel=1e-5,
                      seed=1, problem=0, max_iters=50000, tree_capacity=1 << 16, path_capacity=1 << 14,
                      gmm=None, learned_ratio=0.5, sampler=0, halton_offset=0, dd_radius=0.0,
                      dd_alpha=0.0, dd_min_radius=0.0, workers=0)
SAMPLER_PHILOX, SAMPLER_HALTON = 0, 1


def _params(keep=None, **kw):
    p = dict(DEFAULT_PARAMS)
    p.update(kw)
    prm = OrcParams(range=p["range"], resolution=p["resolution"], goal_bias=p["goal_bias"],
                    amb_band=p["amb_band"], amb_rel=p["amb_rel"], seed=int(p["seed"]),
                    problem=int(p["problem"]), max_iters=int(p["max_iters"]),
                    tree_capacity=int(p["tree_capacity"]), path_capacity=int(p["path_capacity"]),
                    sampler=int(p["sampler"]), halton_offset=int(p["halton_offset"]),
                    dd_radius=float(p["dd_radius"]), dd_alpha=float(p["dd_alpha"]),
                    dd_min_radius=float(p["dd_min_radius"]), workers=int(p["workers"]))
    g = p.get("gmm")
    if g is not None:
        g = np.ascontiguousarray(g, dtype=np.float64)
        if keep is not None:
            keep.append(g)
        prm.gmm = g.ctypes.data_as(_PD)
        prm.learned_ratio = float(p.get("learned_ratio", 0.5))
    return prm


def _result_dict(res, d, trees=None, path=None):
    out = dict(status=int(res.status), status_name=STATUS.get(int(res.status), "?"),
               iterations=int(res.iterations), n_a=int(res.n_a), n_b=int(res.n_b),
               join_a=int(res.join_a), join_b=int(res.join_b), cost=float(res.cost),
               path_n=int(res.path_n), first_amb_iter=int(res.first_amb_iter),
               first_amb_kind=int(res.first_amb_kind), edges_checked=int(res.edges_checked),
               states_checked=int(res.states_checked), edge_states=int(res.edge_states),
               dd_rejected=int(res.dd_rejected))
    if path is not None:
        out["path"] = path[: min(out["path_n"], path.shape[0])].copy()
    if trees is not None:
        na, pa, nb, pb, ra, rb = trees
        out["nodes_a"] = na[: out["n_a"]].copy()
        out["parent_a"] = pa[: out["n_a"]].copy()
        out["nodes_b"] = nb[: out["n_b"]].copy()
        out["parent_b"] = pb[: out["n_b"]].copy()
        out["radius_a"] = ra[: out["n_a"]].copy()
        out["radius_b"] = rb[: out["n_b"]].copy()
    return out


def plan(robot, scene, q_start, q_goal, want_trees=False, esdf=None, **kw):
    r, e = make_robot(robot), make_env(scene, esdf)
    keep = []
    prm = _params(keep, **kw)
    d = robot.dof
    res = OrcResult()
    path = np.zeros((prm.path_capacity, d))
    res.path = path.ctypes.data_as(_PD)
    trees = None
    if want_trees:
        cap = prm.tree_capacity
        trees = (np.zeros((cap, d)), np.zeros(cap, np.int32), np.zeros((cap, d)), np.zeros(cap, np.int32),
                 np.zeros(cap), np.zeros(cap))
        res.nodes_a, res.parent_a = trees[0].ctypes.data_as(_PD), trees[1].ctypes.data_as(_PI)
        res.nodes_b, res.parent_b = trees[2].ctypes.data_as(_PD), trees[3].ctypes.data_as(_PI)
        res.radius_a, res.radius_b = trees[4].ctypes.data_as(_PD), trees[5].ctypes.data_as(_PD)
    s, sp = _d(q_start)
    g, gp = _d(q_goal)
    lib().orc_plan(C.byref(r), C.byref(e), sp, gp, C.byref(prm), C.byref(res))
    return _result_dict(res, d, trees, path)


def revalidate(robot, scene, path, res, esdf=None):
    r, e = make_robot(robot), make_env(scene, esdf)
    p, pp = _d(np.asarray(path).reshape(-1, robot.dof))
    mc = C.c_double()
    bad = lib().orc_revalidate(C.byref(r), C.byref(e), pp, C.c_int32(p.shape[0]), C.c_double(res), C.byref(mc))
    return int(bad), float(mc.value)


def plan_batch(problems, threads=None, **kw):
    """Plan each workload.Problem on its own thread.  kw: planner params shared by all
    (``seeds`` / ``problem_ids`` lists override seed / problem per entry)."""
    threads = threads or os.cpu_count() or 1
    seeds = kw.pop("seeds", None)
    pids = kw.pop("problem_ids", None)
    n = len(problems)
    keep = []
    arr = (OrcProblem * n)()
    paths = []
    results = []
    for k, pb in enumerate(problems):
        r, e = make_robot(pb.robot), make_env(pb.scene)
        s, sp = _d(pb.q_start)
        g, gp = _d(pb.q_goal)
        prm = _params(keep, **kw)
        prm.seed = int(seeds[k]) if seeds is not None else int(kw.get("seed", pb.seed))
        prm.problem = int(pids[k]) if pids is not None else int(kw.get("problem", 0))
        res = OrcResult()
        path = np.zeros((prm.path_capacity, pb.robot.dof))
        res.path = path.ctypes.data_as(_PD)
        keep += [r, e, s, g, res, path]
        paths.append(path)
        results.append(res)
        arr[k].robot = C.pointer(r)
        arr[k].env = C.pointer(e)
        arr[k].q_start = sp
        arr[k].q_goal = gp
        arr[k].params = prm
        arr[k].result = C.pointer(res)
    lib().orc_plan_batch(arr, C.c_int32(n), C.c_int32(threads))
    out = []
    for k, pb in enumerate(problems):
        dct = _result_dict(results[k], pb.robot.dof, None, paths[k])
        dct["seconds"] = float(arr[k].seconds)
        out.append(dct)
    return out
