"""Python binding of libprrtc (include/prrtc.h): argument marshalling only.

Every function here forwards to the C ABI of the same name; all planning and
collision-checking work runs in the library's CUDA kernels.  There is no CPU
fallback: if the library has not been built, or no CUDA device is present,
the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import workload as W

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libprrtc.so")

OK = 0
ERR_INVALID_ARG, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_DEVICE_INDEX, ERR_NO_DEVICE, ERR_UNSUPPORTED = -1, -2, -3, -4, -5, -6, -7
SOLVED, START_IN_COLLISION, GOAL_IN_COLLISION, NO_SOLUTION, PATH_OVERFLOW, TIME_LIMIT = 0, 1, 2, 3, 4, 5
MODE_ASYNC, MODE_SERIAL, MODE_LOCKSTEP = 0, 1, 2
OBS_BOX, OBS_CYLINDER, OBS_SPHERE = 0, 1, 2

_f = C.POINTER(C.c_float)
_i = C.POINTER(C.c_int32)


class prrtc_obstacle(C.Structure):
    _fields_ = [("type", C.c_int32), ("center", C.c_float * 3), ("half", C.c_float * 3),
                ("axis", C.c_float * 3), ("rot", C.c_float * 9)]


class prrtc_robot_desc(C.Structure):
    _fields_ = [("dof", C.c_int32), ("joint_type", _i), ("joint_parent", _i), ("joint_base", _f),
                ("link_length", _f), ("lower", _f), ("upper", _f), ("n_spheres", C.c_int32),
                ("sphere_frame", _i), ("sphere_offset", _f), ("sphere_radius", _f),
                ("n_pairs", C.c_int32), ("self_pairs", _i)]


class prrtc_params(C.Structure):
    _fields_ = [("range", C.c_float), ("resolution", C.c_float), ("goal_bias", C.c_float),
                ("max_iters", C.c_int32), ("tree_capacity", C.c_int32), ("path_capacity", C.c_int32),
                ("mode", C.c_int32), ("blocks", C.c_int32), ("warps_per_block", C.c_int32),
                ("learned_ratio", C.c_float), ("seed", C.c_uint64), ("time_limit_s", C.c_double),
                ("sampler", C.c_int32), ("halton_offset", C.c_uint32), ("dd_radius", C.c_float),
                ("dd_alpha", C.c_float), ("dd_min_radius", C.c_float), ("workers", C.c_int32),
                ("debug_wait_polls", C.c_int32), ("expansions", C.c_int32), ("obstacle_tile", C.c_int32),
                ("reserved", C.c_int32 * 2)]


SAMPLER_PHILOX, SAMPLER_HALTON = 0, 1


class prrtc_path(C.Structure):
    _fields_ = [("status", C.c_int32), ("n", C.c_int32), ("dof", C.c_int32), ("iterations", C.c_int32),
                ("q", _f), ("cost", C.c_double), ("nodes_a", C.c_int32), ("nodes_b", C.c_int32),
                ("edges_checked", C.c_int64), ("edge_states", C.c_int64), ("solve_time_us", C.c_double),
                ("sphere_tests", C.c_int64), ("pair_tests", C.c_int64), ("fk_states", C.c_int64),
                ("nn_nodes", C.c_int64), ("dd_rejected", C.c_int64), ("prim_tests", C.c_int64 * 4),
                ("verdict_states", C.c_int64)]


class prrtc_launch_stats(C.Structure):
    _fields_ = [("kernel_ms", C.c_double), ("setup_ms", C.c_double), ("edges_checked", C.c_int64),
                ("edge_states", C.c_int64), ("sphere_tests", C.c_int64), ("env_tests", C.c_int64),
                ("pair_tests", C.c_int64), ("fk_states", C.c_int64), ("nn_nodes", C.c_int64),
                ("iterations", C.c_int64), ("grid", C.c_int32), ("block_threads", C.c_int32),
                ("smem_bytes", C.c_int32), ("problems", C.c_int32), ("h2d_bytes", C.c_int64),
                ("d2h_bytes", C.c_int64), ("kernels", C.c_int32), ("lean_kernel", C.c_int32),
                ("prep_ms", C.c_double), ("prim_tests", C.c_int64 * 4), ("dd_rejected", C.c_int64),
                ("verdict_states", C.c_int64), ("infer_ms", C.c_double)]


class prrtc_server_config(C.Structure):
    _fields_ = [("max_slots", C.c_int32), ("slice_us", C.c_int32), ("memory_budget_bytes", C.c_int64),
                ("params", prrtc_params)]


class prrtc_server_stats(C.Structure):
    _fields_ = [("slots", C.c_int32), ("active", C.c_int32), ("submitted", C.c_int64), ("admitted", C.c_int64),
                ("completed", C.c_int64), ("pending", C.c_int64), ("slices", C.c_int64), ("busy_s", C.c_double),
                ("uptime_s", C.c_double)]


class prrtc_problem(C.Structure):
    _fields_ = [("robot", C.c_void_p), ("env", C.c_void_p), ("q_start", _f), ("q_goal", _f),
                ("seed", C.c_uint64), ("problem_id", C.c_uint32), ("reserved", C.c_int32), ("gmm", _f)]


EXPORTS = [
    "prrtc_params_default", "prrtc_path_free", "prrtc_paths_free", "prrtc_last_launch_stats", "prrtc_status_string",
    "prrtc_version", "prrtc_last_error", "prrtc_env_create", "prrtc_env_update", "prrtc_env_destroy",
    "prrtc_robot_create", "prrtc_robot_destroy", "prrtc_robot_info", "prrtc_env_info",
    "prrtc_robot_set_two_stage", "prrtc_robot_bounds", "prrtc_env_create_esdf", "prrtc_env_update_esdf",
    "prrtc_env_esdf_values", "prrtc_voxelize",
    "prrtc_check_states", "prrtc_check_states_device", "prrtc_philox", "prrtc_alu_peak", "prrtc_plan", "prrtc_plan_batch", "prrtc_debug_tree",
    "prrtc_plan_noalloc", "prrtc_gemm_bf16", "prrtc_gemm_bf16_splitk", "prrtc_gemm_error",
    "prrtc_proposal_create", "prrtc_proposal_destroy", "prrtc_proposal_info", "prrtc_proposal_get_params",
    "prrtc_proposal_forward", "prrtc_proposal_forward_layers", "prrtc_proposal_inference_layers",
    "prrtc_proposal_grads", "prrtc_proposal_train", "prrtc_proposal_save",
    "prrtc_proposal_load", "prrtc_occupancy", "prrtc_proposal_mixtures", "prrtc_plan_batch_learned",
    "prrtc_server_config_default", "prrtc_server_create", "prrtc_server_submit", "prrtc_server_poll",
    "prrtc_server_wait", "prrtc_server_get_stats", "prrtc_server_destroy", "prrtc_autotune",
]

_lib = None


class PrrtcError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        super().__init__(f"{what}: {status_string(code)} ({code}): {last_error()}")


def lib():
    """Load the in-tree CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libprrtc is not built ({LIB_PATH}); run __graft_entry__.build()")
    L = C.CDLL(LIB_PATH)
    L.prrtc_status_string.restype = C.c_char_p
    L.prrtc_version.restype = C.c_char_p
    L.prrtc_last_error.restype = C.c_char_p
    L.prrtc_env_create.argtypes = [C.POINTER(prrtc_obstacle), C.c_int32, C.POINTER(C.c_void_p)]
    L.prrtc_env_update.argtypes = [C.c_void_p, _i, C.POINTER(prrtc_obstacle), C.c_int32]
    L.prrtc_env_destroy.argtypes = [C.c_void_p]
    L.prrtc_robot_create.argtypes = [C.POINTER(prrtc_robot_desc), C.POINTER(C.c_void_p)]
    L.prrtc_robot_destroy.argtypes = [C.c_void_p]
    L.prrtc_robot_info.argtypes = [C.c_void_p, _i, _i, _i, _i]
    L.prrtc_env_info.argtypes = [C.c_void_p, _i]
    L.prrtc_robot_set_two_stage.argtypes = [C.c_void_p, C.c_int32]
    L.prrtc_env_create_esdf.argtypes = [C.POINTER(C.c_float), C.c_float, C.POINTER(C.c_int32), C.POINTER(C.c_uint8),
                                        C.POINTER(C.c_void_p)]
    L.prrtc_env_update_esdf.argtypes = [C.c_void_p, C.POINTER(C.c_uint8)]
    L.prrtc_env_esdf_values.argtypes = [C.c_void_p, _f]
    L.prrtc_voxelize.argtypes = [C.c_void_p, C.POINTER(C.c_float), C.c_float, C.POINTER(C.c_int32),
                                 C.POINTER(C.c_uint8)]
    L.prrtc_robot_bounds.argtypes = [C.c_void_p, _f]
    L.prrtc_check_states.argtypes = [C.c_void_p, C.c_void_p, _f, C.c_int32, C.POINTER(C.c_uint8), _f]
    L.prrtc_alu_peak.argtypes = [C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.prrtc_check_states_device.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p,
                                            C.c_void_p, C.c_void_p]
    L.prrtc_plan.argtypes = [C.c_void_p, C.c_void_p, _f, _f, C.POINTER(prrtc_params), C.POINTER(prrtc_path)]
    L.prrtc_plan_batch.argtypes = [C.POINTER(prrtc_problem), C.c_int32, C.POINTER(prrtc_params),
                                   C.POINTER(prrtc_path), _i]
    L.prrtc_path_free.argtypes = [C.POINTER(prrtc_path)]
    L.prrtc_paths_free.argtypes = [C.POINTER(prrtc_path), C.c_int32]
    L.prrtc_params_default.argtypes = [C.POINTER(prrtc_params)]
    L.prrtc_last_launch_stats.argtypes = [C.POINTER(prrtc_launch_stats)]
    L.prrtc_debug_tree.argtypes = [C.c_int32, C.c_int32, _f, _i, C.c_int32, _i]
    L.prrtc_gemm_bf16.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_void_p, C.c_int32,
                                  C.c_void_p, C.c_void_p, C.c_void_p]
    L.prrtc_gemm_bf16_splitk.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_void_p,
                                         C.c_int32, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]
    _u8 = C.POINTER(C.c_uint8)
    L.prrtc_proposal_create.argtypes = [C.c_int32, _f, _f, _f, C.POINTER(C.c_void_p)]
    L.prrtc_proposal_destroy.argtypes = [C.c_void_p]
    L.prrtc_proposal_info.argtypes = [C.c_void_p, _i, _i, C.POINTER(C.c_int64), _i]
    L.prrtc_proposal_get_params.argtypes = [C.c_void_p, _f, _f]
    L.prrtc_proposal_forward.argtypes = [C.c_void_p, _u8, _f, _f, C.c_int32, _f]
    L.prrtc_proposal_forward_layers.argtypes = [C.c_void_p, _u8, _f, _f, C.c_int32, _f, _f, _f, _f, _f]
    L.prrtc_proposal_inference_layers.argtypes = [C.c_void_p, C.c_int32, _f, _f, _f]
    L.prrtc_proposal_grads.argtypes = [C.c_void_p, _u8, _f, _f, _f, C.c_int32, _f]
    L.prrtc_proposal_train.argtypes = [C.c_void_p, _u8, C.c_int32, _i, _f, _f, _f, C.c_int32, C.c_int32, C.c_int32,
                                       C.c_float, C.c_uint64, _f]
    L.prrtc_proposal_save.argtypes = [C.c_void_p, C.c_char_p]
    L.prrtc_proposal_load.argtypes = [C.c_char_p, C.POINTER(C.c_void_p)]
    L.prrtc_occupancy.argtypes = [C.c_void_p, _u8]
    L.prrtc_proposal_mixtures.argtypes = [C.c_void_p, C.POINTER(C.c_void_p), _f, _f, C.c_int32, _f]
    L.prrtc_plan_batch_learned.argtypes = [C.POINTER(prrtc_problem), C.POINTER(C.c_void_p), C.c_int32,
                                           C.POINTER(prrtc_params), C.POINTER(prrtc_path), _i]
    L.prrtc_server_config_default.argtypes = [C.POINTER(prrtc_server_config)]
    L.prrtc_server_create.argtypes = [C.POINTER(prrtc_server_config), C.POINTER(C.c_void_p)]
    L.prrtc_server_submit.argtypes = [C.c_void_p, C.POINTER(prrtc_problem), C.c_void_p, C.POINTER(C.c_uint64)]
    L.prrtc_server_poll.argtypes = [C.c_void_p, C.c_int32, C.POINTER(prrtc_path), C.POINTER(C.c_uint64),
                                    C.POINTER(C.c_double), C.POINTER(C.c_double), _i]
    L.prrtc_server_wait.argtypes = [C.c_void_p, C.c_int64, C.c_double]
    L.prrtc_server_get_stats.argtypes = [C.c_void_p, C.POINTER(prrtc_server_stats)]
    L.prrtc_server_destroy.argtypes = [C.c_void_p]
    L.prrtc_autotune.argtypes = [C.POINTER(prrtc_problem), C.c_int32, C.POINTER(prrtc_params), C.c_int32,
                                 C.POINTER(prrtc_params), C.POINTER(C.c_double)]
    L.prrtc_plan_noalloc.argtypes = [C.c_void_p, C.c_void_p, _f, _f, C.POINTER(prrtc_params), _f, C.c_int32,
                                     C.POINTER(prrtc_path), C.c_void_p]
    _lib = L
    return L


def status_string(code: int) -> str:
    return lib().prrtc_status_string(int(code)).decode()


def last_error() -> str:
    return lib().prrtc_last_error().decode()


def version() -> str:
    return lib().prrtc_version().decode()


def _check(rc, what):
    if rc != OK:
        raise PrrtcError(rc, what)


def _fa(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a, a.ctypes.data_as(_f)


def _ia(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(_i)


# ------------------------------------------------------------------ handles

class Env:
    """Device-resident obstacle set (prrtc_env_create / _update / _destroy)."""

    def __init__(self, obstacles):
        self._lib = lib()
        arr = (prrtc_obstacle * max(1, len(obstacles)))(*obstacles)
        h = C.c_void_p()
        _check(self._lib.prrtc_env_create(arr, len(obstacles), C.byref(h)), "prrtc_env_create")
        self.handle = h
        self.n = len(obstacles)

    def update(self, ids, obstacles):
        ids_a, ids_p = _ia(ids)
        arr = (prrtc_obstacle * max(1, len(obstacles)))(*obstacles)
        _check(self._lib.prrtc_env_update(self.handle, ids_p, arr, len(obstacles)), "prrtc_env_update")

    def info(self):
        out = (C.c_int32 * 4)()
        _check(self._lib.prrtc_env_info(self.handle, out), "prrtc_env_info")
        return tuple(out)

    @classmethod
    def from_occupancy(cls, occupancy, origin, voxel: float):
        """Distance-field environment (prrtc_env_create_esdf); occupancy [nz, ny, nx]."""
        occ = np.ascontiguousarray(np.asarray(occupancy) != 0, dtype=np.uint8)
        nz, ny, nx = occ.shape
        self = cls.__new__(cls)
        self._lib = lib()
        o = (C.c_float * 3)(*[float(x) for x in origin])
        d = (C.c_int32 * 3)(nx, ny, nz)
        h = C.c_void_p()
        _check(self._lib.prrtc_env_create_esdf(o, C.c_float(voxel), d, occ.ctypes.data_as(C.POINTER(C.c_uint8)),
                                               C.byref(h)), "prrtc_env_create_esdf")
        self.handle = h
        self.n = 0
        self.grid = ((nx, ny, nz), tuple(float(x) for x in origin), float(voxel))
        return self

    def update_occupancy(self, occupancy):
        occ = np.ascontiguousarray(np.asarray(occupancy) != 0, dtype=np.uint8)
        _check(self._lib.prrtc_env_update_esdf(self.handle, occ.ctypes.data_as(C.POINTER(C.c_uint8))),
               "prrtc_env_update_esdf")

    def esdf(self) -> np.ndarray:
        (nx, ny, nz), _, _ = self.grid
        out = np.zeros((nz, ny, nx), np.float32)
        _check(self._lib.prrtc_env_esdf_values(self.handle, out.ctypes.data_as(_f)), "prrtc_env_esdf_values")
        return out

    def voxelize(self, origin, voxel: float, dims) -> np.ndarray:
        """Occupancy [nz, ny, nx] of this environment's primitives (prrtc_voxelize)."""
        nx, ny, nz = (int(x) for x in dims)
        out = np.zeros((nz, ny, nx), np.uint8)
        o = (C.c_float * 3)(*[float(x) for x in origin])
        d = (C.c_int32 * 3)(nx, ny, nz)
        _check(self._lib.prrtc_voxelize(self.handle, o, C.c_float(voxel), d, out.ctypes.data_as(C.POINTER(C.c_uint8))),
               "prrtc_voxelize")
        return out

    def close(self):
        if getattr(self, "handle", None):
            self._lib.prrtc_env_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Robot:
    """Device-resident sphere model (prrtc_robot_create / _destroy)."""

    def __init__(self, rb: W.Robot):
        self._lib = lib()
        keep = []

        def f(a):
            a, p = _fa(a)
            keep.append(a)
            return p

        def i(a):
            a, p = _ia(a)
            keep.append(a)
            return p

        desc = prrtc_robot_desc(
            dof=rb.dof, joint_type=i(rb.joint_type), joint_parent=i(rb.joint_parent),
            joint_base=f(rb.joint_base.reshape(-1)), link_length=f(rb.link_length), lower=f(rb.lower),
            upper=f(rb.upper), n_spheres=rb.n_spheres, sphere_frame=i(rb.sphere_frame),
            sphere_offset=f(rb.sphere_offset.reshape(-1)), sphere_radius=f(rb.sphere_radius),
            n_pairs=int(rb.self_pairs.shape[0]),
            self_pairs=i(rb.self_pairs.reshape(-1) if rb.self_pairs.size else np.zeros(2, np.int32)))
        h = C.c_void_p()
        _check(self._lib.prrtc_robot_create(C.byref(desc), C.byref(h)), "prrtc_robot_create")
        self.handle = h
        self.dof = rb.dof
        self.n_raw = rb.n_spheres
        self.model = rb

    def info(self):
        v = [C.c_int32() for _ in range(4)]
        _check(self._lib.prrtc_robot_info(self.handle, *[C.byref(x) for x in v]), "prrtc_robot_info")
        return dict(dof=v[0].value, n_spheres=v[1].value, n_pairs=v[2].value, dpad=v[3].value)

    def set_two_stage(self, enabled: bool):
        _check(self._lib.prrtc_robot_set_two_stage(self.handle, int(bool(enabled))), "prrtc_robot_set_two_stage")

    def bounds(self) -> np.ndarray:
        out = np.zeros((self.dof, 4), np.float32)
        _check(self._lib.prrtc_robot_bounds(self.handle, out.ctypes.data_as(_f)), "prrtc_robot_bounds")
        return out

    def close(self):
        if getattr(self, "handle", None):
            self._lib.prrtc_robot_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def obstacles_from_scene(scene: W.Scene):
    obs = []
    for b in scene.boxes:
        o = prrtc_obstacle(type=OBS_BOX)
        o.center[:] = [float(x) for x in b[0:3]]
        o.half[:] = [float(x) for x in b[3:6]]
        o.rot[:] = [float(x) for x in b[6:15]]
        obs.append(o)
    for c in scene.cylinders:
        o = prrtc_obstacle(type=OBS_CYLINDER)
        o.center[:] = [float(x) for x in c[0:3]]
        o.axis[:] = [float(x) for x in c[3:6]]
        o.half[:] = [float(c[6]), float(c[7]), 0.0]
        obs.append(o)
    for s in scene.spheres:
        o = prrtc_obstacle(type=OBS_SPHERE)
        o.center[:] = [float(x) for x in s[0:3]]
        o.half[:] = [float(s[3]), 0.0, 0.0]
        obs.append(o)
    return obs


def make_env(scene: W.Scene) -> Env:
    return Env(obstacles_from_scene(scene))


def make_robot(rb: W.Robot) -> Robot:
    return Robot(rb)


# ------------------------------------------------------------------ calls

def prrtc_params_default() -> prrtc_params:
    p = prrtc_params()
    lib().prrtc_params_default(C.byref(p))
    return p


def params(**kw) -> prrtc_params:
    p = prrtc_params_default()
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def prrtc_check_states(robot: Robot, env: Env, Q, want_spheres: bool = False):
    """Verdicts (True = collision-free) and, optionally, [n, S, 4] sphere centres+radii."""
    Q, qp = _fa(np.asarray(Q).reshape(-1, robot.dof))
    n = Q.shape[0]
    valid = np.zeros(n, dtype=np.uint8)
    sph = np.zeros((n, robot.n_raw, 4), dtype=np.float32) if want_spheres else None
    _check(lib().prrtc_check_states(robot.handle, env.handle, qp, n, valid.ctypes.data_as(C.POINTER(C.c_uint8)),
                                    sph.ctypes.data_as(_f) if want_spheres else None), "prrtc_check_states")
    return (valid.astype(bool), sph) if want_spheres else valid.astype(bool)


def prrtc_check_states_device(robot: Robot, env: Env, q_ptr: int, n: int, valid_ptr: int, spheres_ptr: int = 0,
                              stream: int = 0):
    """Device-pointer form (e.g. torch tensors' data_ptr(), stream.cuda_stream)."""
    _check(lib().prrtc_check_states_device(robot.handle, env.handle, C.c_void_p(q_ptr), n, C.c_void_p(valid_ptr),
                                           C.c_void_p(spheres_ptr or None), C.c_void_p(stream or None)),
           "prrtc_check_states_device")


def _path_dict(p: prrtc_path):
    d = dict(status=int(p.status), n=int(p.n), dof=int(p.dof), iterations=int(p.iterations), cost=float(p.cost),
             nodes_a=int(p.nodes_a), nodes_b=int(p.nodes_b), edges_checked=int(p.edges_checked),
             edge_states=int(p.edge_states), solve_time_us=float(p.solve_time_us),
             sphere_tests=int(p.sphere_tests), pair_tests=int(p.pair_tests), fk_states=int(p.fk_states),
             nn_nodes=int(p.nn_nodes), dd_rejected=int(p.dd_rejected), prim_tests=[int(x) for x in p.prim_tests],
             verdict_states=int(p.verdict_states))
    if p.q and p.n > 0:
        d["path"] = np.ctypeslib.as_array(p.q, shape=(p.n * p.dof,)).reshape(p.n, p.dof).copy()
    else:
        d["path"] = np.zeros((0, p.dof), np.float32)
    return d


def prrtc_philox(ctr, key: int):
    """Philox4x32-10 blocks on the device: ctr [n x 4] uint32 counters -> [n x 4] words."""
    c = np.ascontiguousarray(np.asarray(ctr, np.uint32).reshape(-1, 4))
    out = np.zeros_like(c)
    P32 = C.POINTER(C.c_uint32)
    _check(lib().prrtc_philox(c.ctypes.data_as(P32), c.shape[0], C.c_uint64(int(key) & (2 ** 64 - 1)),
                              out.ctypes.data_as(P32)), "prrtc_philox")
    return out


def prrtc_alu_peak(iters: int = 16384):
    """FP32 FMA issue rate of the device (lane-ops/s, one FMA = one lane-op) and
    the timed launch's milliseconds."""
    rate, ms = C.c_double(), C.c_double()
    _check(lib().prrtc_alu_peak(int(iters), C.byref(rate), C.byref(ms)), "prrtc_alu_peak")
    return rate.value, ms.value


def prrtc_plan(robot: Robot, env: Env, q_start, q_goal, prm: prrtc_params | None = None):
    prm = prm or prrtc_params_default()
    s, sp = _fa(q_start)
    g, gp = _fa(q_goal)
    out = prrtc_path()
    _check(lib().prrtc_plan(robot.handle, env.handle, sp, gp, C.byref(prm), C.byref(out)), "prrtc_plan")
    try:
        return _path_dict(out)
    finally:
        lib().prrtc_path_free(C.byref(out))


def _numpy_dtype(cls):
    """numpy structured dtype with the layout of a ctypes Structure (pointers as
    uint64), so that arrays of it can be filled and read column-wise."""
    def np_type(t):
        if issubclass(t, C.Array):
            return (np_type(t._type_), (t._length_,))
        if t in (C.c_void_p, C.c_char_p) or issubclass(t, C._Pointer):
            return np.uint64
        return np.dtype(t)
    names = [n for n, _ in cls._fields_]
    return np.dtype(dict(names=names, formats=[np_type(t) for _, t in cls._fields_],
                         offsets=[getattr(cls, n).offset for n in names], itemsize=C.sizeof(cls)))


_PROBLEM_DT = _numpy_dtype(prrtc_problem)
_PATH_DT = _numpy_dtype(prrtc_path)
_PATH_FIELDS = [n for n, _ in prrtc_path._fields_ if n != "q"]


def _handle(x):
    h = x.handle
    return h.value if isinstance(h, C.c_void_p) else int(h)


def _problem_array(problems, keep):
    """The C problem array for a sequence of (Robot, Env, q_start, q_goal, seed,
    problem_id[, gmm]), filled column-wise; `keep` holds what it points into."""
    n = len(problems)
    v = np.zeros(n, _PROBLEM_DT)
    qs = [np.ascontiguousarray(it[2], np.float32).ravel() for it in problems]
    qg = [np.ascontiguousarray(it[3], np.float32).ravel() for it in problems]
    lens = np.fromiter((len(q) for q in qs), np.int64, n)
    flat = np.concatenate(qs + qg) if n else np.zeros(0, np.float32)
    keep.append(flat)
    base = flat.ctypes.data
    off = np.concatenate([[0], np.cumsum(lens)[:-1]]) if n else np.zeros(0, np.int64)
    v["q_start"] = base + 4 * off
    v["q_goal"] = base + 4 * (off + int(lens.sum()))
    v["robot"] = np.fromiter((_handle(it[0]) for it in problems), np.uint64, n)
    v["env"] = np.fromiter((_handle(it[1]) for it in problems), np.uint64, n)
    v["seed"] = np.fromiter((int(it[4]) for it in problems), np.uint64, n)
    v["problem_id"] = np.fromiter((int(it[5]) for it in problems), np.uint32, n)
    for k, it in enumerate(problems):
        if len(it) > 6 and it[6] is not None:
            m = np.ascontiguousarray(it[6], np.float32)
            keep.append(m)
            v["gmm"][k] = m.ctypes.data
    keep.append(v)
    return v.ctypes.data_as(C.POINTER(prrtc_problem))


def _collect(paths, n):
    """Per-problem result dicts (and path arrays); frees the C paths."""
    v = np.frombuffer((C.c_char * (n * C.sizeof(prrtc_path))).from_address(C.addressof(paths)), _PATH_DT, n)
    rows = v[_PATH_FIELDS].tolist()
    out = []
    for k in range(n):
        d = dict(zip(_PATH_FIELDS, rows[k]))
        d["prim_tests"] = list(d["prim_tests"])
        p = paths[k]
        if p.q and p.n > 0:
            d["path"] = np.ctypeslib.as_array(p.q, shape=(p.n * p.dof,)).reshape(p.n, p.dof).copy()
        else:
            d["path"] = np.zeros((0, p.dof), np.float32)
        out.append(d)
    lib().prrtc_paths_free(paths, n)
    return out


class PlanBatch:
    """A batch of planning problems marshalled once and planned many times
    (prrtc_plan_batch / prrtc_plan_batch_learned).  run() returns a BatchResult
    whose per-problem scalars are numpy columns; paths are read from the C
    buffers on first access."""

    def __init__(self, problems, proposals=None):
        self._keep = []
        self.n = len(problems)
        self._arr = _problem_array(problems, self._keep)
        self._view = self._keep[-1]
        self._props = None
        if proposals is not None:
            self._props = (C.c_void_p * self.n)(*[(pp.handle.value if pp is not None else None) for pp in proposals])

    def set_seeds(self, seeds):
        self._view["seed"] = np.asarray(seeds, np.uint64)

    def run(self, prm: prrtc_params | None = None):
        prm = prm or prrtc_params_default()
        paths = (prrtc_path * self.n)()
        status = (C.c_int32 * self.n)()
        if self._props is None:
            rc = lib().prrtc_plan_batch(self._arr, self.n, C.byref(prm), paths, status)
        else:
            rc = lib().prrtc_plan_batch_learned(self._arr, self._props, self.n, C.byref(prm), paths, status)
        _check(rc, "prrtc_plan_batch")
        return BatchResult(paths, self.n)


class BatchResult:
    """Results of one PlanBatch.run: numpy columns named as prrtc_path's fields
    (result["status"], result["edge_states"], ...), paths(k) for problem k."""

    def __init__(self, paths, n):
        self._paths = paths
        self.n = n
        self._v = np.frombuffer((C.c_char * (n * C.sizeof(prrtc_path))).from_address(C.addressof(paths)), _PATH_DT,
                                n).copy()

    def __getitem__(self, name):
        return self._v[name]

    def path(self, k):
        p = self._paths[k]
        if not p.q or p.n <= 0:
            return np.zeros((0, p.dof), np.float32)
        return np.ctypeslib.as_array(p.q, shape=(p.n * p.dof,)).reshape(p.n, p.dof).copy()

    def __del__(self):
        try:
            lib().prrtc_paths_free(self._paths, self.n)
        except Exception:
            pass


def prrtc_plan_batch(problems, prm: prrtc_params | None = None):
    """problems: sequence of (Robot, Env, q_start, q_goal, seed, problem_id[, gmm])."""
    prm = prm or prrtc_params_default()
    keep = []
    n = len(problems)
    arr = _problem_array(problems, keep)
    paths = (prrtc_path * n)()
    status = (C.c_int32 * n)()
    _check(lib().prrtc_plan_batch(arr, n, C.byref(prm), paths, status), "prrtc_plan_batch")
    del keep
    return _collect(paths, n)


def prrtc_plan_batch_learned(problems, proposals, prm: prrtc_params | None = None):
    """As prrtc_plan_batch, with proposals[p] (Proposal or None) inferring each mixture on the device."""
    prm = prm or prrtc_params_default()
    keep = []
    n = len(problems)
    arr = _problem_array(problems, keep)
    props = (C.c_void_p * n)(*[(pp.handle.value if pp is not None else None) for pp in proposals])
    paths = (prrtc_path * n)()
    status = (C.c_int32 * n)()
    _check(lib().prrtc_plan_batch_learned(arr, props, n, C.byref(prm), paths, status), "prrtc_plan_batch_learned")
    return _collect(paths, n)


class Proposal:
    """Learned sampling proposal (prrtc_proposal_*)."""

    def __init__(self, dof=None, lower=None, upper=None, params=None, handle=None):
        self._lib = lib()
        if handle is None:
            lo, lp = _fa(lower)
            hi, hp = _fa(upper)
            pr, pp = _fa(params) if params is not None else (None, None)
            h = C.c_void_p()
            _check(self._lib.prrtc_proposal_create(int(dof), lp, hp, pp, C.byref(h)), "prrtc_proposal_create")
            handle = h
        self.handle = handle
        d, hd, npar, st = C.c_int32(), C.c_int32(), C.c_int64(), C.c_int32()
        _check(self._lib.prrtc_proposal_info(self.handle, C.byref(d), C.byref(hd), C.byref(npar), C.byref(st)),
               "prrtc_proposal_info")
        self.dof, self.head, self.n_params = d.value, hd.value, npar.value

    @property
    def step(self):
        st = C.c_int32()
        _check(self._lib.prrtc_proposal_info(self.handle, None, None, None, C.byref(st)), "prrtc_proposal_info")
        return st.value

    @classmethod
    def load(cls, path):
        h = C.c_void_p()
        _check(lib().prrtc_proposal_load(str(path).encode(), C.byref(h)), "prrtc_proposal_load")
        return cls(handle=h)

    def save(self, path):
        _check(self._lib.prrtc_proposal_save(self.handle, str(path).encode()), "prrtc_proposal_save")

    def params(self):
        out = np.zeros(self.n_params, np.float32)
        _check(self._lib.prrtc_proposal_get_params(self.handle, out.ctypes.data_as(_f), None), "get_params")
        return out

    def grads(self):
        out = np.zeros(self.n_params, np.float32)
        _check(self._lib.prrtc_proposal_get_params(self.handle, None, out.ctypes.data_as(_f)), "get_params")
        return out

    def forward(self, occ, q_start, q_goal):
        occ = np.ascontiguousarray(occ, np.uint8).reshape(-1, 4096)
        B = occ.shape[0]
        s, sp = _fa(np.asarray(q_start).reshape(B, self.dof))
        g, gp = _fa(np.asarray(q_goal).reshape(B, self.dof))
        out = np.zeros((B, self.head), np.float32)
        _check(self._lib.prrtc_proposal_forward(self.handle, occ.ctypes.data_as(C.POINTER(C.c_uint8)), sp, gp, B,
                                                out.ctypes.data_as(_f)), "prrtc_proposal_forward")
        return out

    def loss_and_grads(self, occ, q_start, q_goal, target):
        occ = np.ascontiguousarray(occ, np.uint8).reshape(-1, 4096)
        B = occ.shape[0]
        s, sp = _fa(np.asarray(q_start).reshape(B, self.dof))
        g, gp = _fa(np.asarray(q_goal).reshape(B, self.dof))
        t, tp = _fa(np.asarray(target).reshape(B, self.dof))
        loss = C.c_float()
        _check(self._lib.prrtc_proposal_grads(self.handle, occ.ctypes.data_as(C.POINTER(C.c_uint8)), sp, gp, tp, B,
                                              C.byref(loss)), "prrtc_proposal_grads")
        return float(loss.value), self.grads()

    def train(self, occ, scene_of, q_start, q_goal, target, batch, steps, lr=1e-3, seed=1):
        occ = np.ascontiguousarray(occ, np.uint8).reshape(-1, 4096)
        so, sop = _ia(scene_of)
        N = len(so)
        s, sp = _fa(np.asarray(q_start).reshape(N, self.dof))
        g, gp = _fa(np.asarray(q_goal).reshape(N, self.dof))
        t, tp = _fa(np.asarray(target).reshape(N, self.dof))
        losses = np.zeros(max(steps, 1), np.float32)
        _check(self._lib.prrtc_proposal_train(self.handle, occ.ctypes.data_as(C.POINTER(C.c_uint8)), occ.shape[0], sop,
                                              sp, gp, tp, N, int(batch), int(steps), float(lr), int(seed),
                                              losses.ctypes.data_as(_f)), "prrtc_proposal_train")
        return losses[:steps]

    def forward_layers(self, occ, q_start, q_goal):
        """(x, h1, h2, h3, head) of the training forward, BF16 values widened to FP32."""
        occ = np.ascontiguousarray(occ, np.uint8).reshape(-1, 4096)
        B = occ.shape[0]
        s, sp = _fa(np.asarray(q_start).reshape(B, self.dof))
        g, gp = _fa(np.asarray(q_goal).reshape(B, self.dof))
        outs = [np.zeros((B, w), np.float32) for w in (4160, 1024, 512, 512, self.head)]
        _check(self._lib.prrtc_proposal_forward_layers(self.handle, occ.ctypes.data_as(C.POINTER(C.c_uint8)), sp, gp, B,
                                                       *[o.ctypes.data_as(_f) for o in outs]),
               "prrtc_proposal_forward_layers")
        return tuple(outs)

    def inference_layers(self, B):
        """Hidden activations (h1, h2, h3) of the first B rows of the last inference batch."""
        outs = [np.zeros((B, w), np.float32) for w in (1024, 512, 512)]
        _check(self._lib.prrtc_proposal_inference_layers(self.handle, B, *[o.ctypes.data_as(_f) for o in outs]),
               "prrtc_proposal_inference_layers")
        return tuple(outs)

    def mixtures(self, envs, q_start, q_goal):
        """Mixtures the learned planner samples from, one row of 8 + 16 dof
        floats per (env, start, goal) triple (prrtc_proposal_mixtures)."""
        B = len(envs)
        s, sp = _fa(np.asarray(q_start).reshape(B, self.dof))
        g, gp = _fa(np.asarray(q_goal).reshape(B, self.dof))
        eh = (C.c_void_p * B)(*[e.handle for e in envs])
        out = np.zeros((B, 8 + 16 * self.dof), np.float32)
        _check(self._lib.prrtc_proposal_mixtures(self.handle, eh, sp, gp, B, out.ctypes.data_as(_f)),
               "prrtc_proposal_mixtures")
        return out

    def close(self):
        if getattr(self, "handle", None):
            self._lib.prrtc_proposal_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def prrtc_occupancy(env: Env):
    out = np.zeros(4096, np.uint8)
    _check(lib().prrtc_occupancy(env.handle, out.ctypes.data_as(C.POINTER(C.c_uint8))), "prrtc_occupancy")
    return out


def prrtc_last_launch_stats():
    s = prrtc_launch_stats()
    _check(lib().prrtc_last_launch_stats(C.byref(s)), "prrtc_last_launch_stats")
    return {k: (list(getattr(s, k)) if isinstance(getattr(s, k), C.Array) else getattr(s, k)) for k, _ in s._fields_}


def prrtc_debug_tree(problem: int, tree: int, dof: int):
    """Rows and parents (root: -1) of one tree of the last planning launch."""
    n = C.c_int32()
    _check(lib().prrtc_debug_tree(problem, tree, None, None, 0, C.byref(n)), "prrtc_debug_tree")
    m = n.value
    nodes = np.zeros((max(m, 1), dof), np.float32)
    par = np.zeros(max(m, 1), np.int32)
    _check(lib().prrtc_debug_tree(problem, tree, nodes.ctypes.data_as(_f), par.ctypes.data_as(_i), m, C.byref(n)),
           "prrtc_debug_tree")
    return nodes[:m], par[:m]


def prrtc_plan_noalloc(robot: Robot, env: Env, q_start, q_goal, prm: prrtc_params | None = None, path_rows: int = 4096,
                       stream: int = 0):
    """Plan one problem without any device allocation (fixed static scratch).

    The caller owns the host path buffer; returns the same dict as prrtc_plan.
    Raises PrrtcError with the C status code on failure."""
    prm = prm or prrtc_params_default()
    s, sp = _fa(q_start)
    g, gp = _fa(q_goal)
    buf = np.zeros((max(path_rows, 1), robot.dof), np.float32)
    info = prrtc_path()
    rc = lib().prrtc_plan_noalloc(robot.handle, env.handle, sp, gp, C.byref(prm), buf.ctypes.data_as(_f), path_rows,
                                  C.byref(info), C.c_void_p(stream or None))
    if rc != OK:
        raise PrrtcError(rc, "prrtc_plan_noalloc")
    d = _path_dict(info)  # copies the rows out of buf
    return d


def prrtc_gemm_bf16(a_ptr: int, b_ptr: int, M: int, N: int, K: int, bias_ptr: int = 0, relu: bool = False,
                    c32_ptr: int = 0, c16_ptr: int = 0, stream: int = 0):
    """C[M,N] = A[M,K] B[N,K]^T (+bias, ReLU) on the tensor cores; device pointers."""
    _check(lib().prrtc_gemm_bf16(C.c_void_p(a_ptr), C.c_void_p(b_ptr), M, N, K, C.c_void_p(bias_ptr or None),
                                 int(bool(relu)), C.c_void_p(c32_ptr or None), C.c_void_p(c16_ptr or None),
                                 C.c_void_p(stream or None)), "prrtc_gemm_bf16")


def prrtc_gemm_bf16_splitk(a_ptr: int, b_ptr: int, M: int, N: int, K: int, bias_ptr: int = 0, relu: bool = False,
                           c32_ptr: int = 0, c16_ptr: int = 0, splits: int = 0, stream: int = 0):
    """prrtc_gemm_bf16 with an explicit split of K (0 = the library's choice)."""
    _check(lib().prrtc_gemm_bf16_splitk(C.c_void_p(a_ptr), C.c_void_p(b_ptr), M, N, K, C.c_void_p(bias_ptr or None),
                                        int(bool(relu)), C.c_void_p(c32_ptr or None), C.c_void_p(c16_ptr or None),
                                        int(splits), C.c_void_p(stream or None)), "prrtc_gemm_bf16_splitk")


def prrtc_gemm_error() -> int:
    return int(lib().prrtc_gemm_error())


class Server:
    """Continuous-batching request loop (prrtc_server_*)."""

    def __init__(self, params: prrtc_params | None = None, slice_us: int = 500, memory_budget_bytes: int = 2 << 30,
                 max_slots: int = 0):
        self._lib = lib()
        cfg = prrtc_server_config()
        self._lib.prrtc_server_config_default(C.byref(cfg))
        if params is not None:
            cfg.params = params
        cfg.slice_us = int(slice_us)
        cfg.memory_budget_bytes = int(memory_budget_bytes)
        cfg.max_slots = int(max_slots)
        h = C.c_void_p()
        _check(self._lib.prrtc_server_create(C.byref(cfg), C.byref(h)), "prrtc_server_create")
        self.handle = h
        self._keep = {}

    def submit(self, robot: Robot, env: Env, q_start, q_goal, seed=1, problem_id=0, proposal=None, gmm=None):
        keep = []
        arr = _problem_array([(robot, env, q_start, q_goal, seed, problem_id) + ((gmm,) if gmm is not None else ())],
                             keep)
        t = C.c_uint64()
        _check(self._lib.prrtc_server_submit(self.handle, arr, proposal.handle if proposal is not None else None,
                                             C.byref(t)), "prrtc_server_submit")
        return int(t.value)

    def poll(self, max_n: int = 4096):
        paths = (prrtc_path * max_n)()
        tickets = (C.c_uint64 * max_n)()
        lat = (C.c_double * max_n)()
        que = (C.c_double * max_n)()
        n = C.c_int32()
        _check(self._lib.prrtc_server_poll(self.handle, max_n, paths, tickets, lat, que, C.byref(n)),
               "prrtc_server_poll")
        out = []
        for k in range(n.value):
            d = _path_dict(paths[k])
            d.update(ticket=int(tickets[k]), latency_ms=float(lat[k]), queue_ms=float(que[k]))
            out.append(d)
        lib().prrtc_paths_free(paths, n.value)
        return out

    def wait(self, completed: int, timeout_s: float = 60.0):
        _check(self._lib.prrtc_server_wait(self.handle, int(completed), float(timeout_s)), "prrtc_server_wait")

    def stats(self):
        st = prrtc_server_stats()
        _check(self._lib.prrtc_server_get_stats(self.handle, C.byref(st)), "prrtc_server_get_stats")
        return {k: getattr(st, k) for k, _ in st._fields_}

    def close(self):
        if getattr(self, "handle", None):
            self._lib.prrtc_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def prrtc_autotune(problems, prm: prrtc_params | None = None, trials: int = 3):
    """Launch shape, obstacle tile and expansions per claim for these problems, scored by the
    batch's median time to first solution over `trials` runs; returns (params, score in ms) and
    is remembered by the library."""
    prm = prm or prrtc_params_default()
    keep = []
    n = len(problems)
    arr = _problem_array(problems, keep)
    best = prrtc_params()
    ms = C.c_double()
    _check(lib().prrtc_autotune(arr, n, C.byref(prm), int(trials), C.byref(best), C.byref(ms)), "prrtc_autotune")
    return best, float(ms.value)
