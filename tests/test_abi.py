"""The C ABI library builds, loads and exports every entry point of
include/prrtc.h; the ctypes mirrors of its structs match the C layout; and
without a GPU every call fails with PRRTC_ERR_NO_DEVICE (no CPU fallback)."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_2503_06757_gb300 import build as B
from paper_2503_06757_gb300 import prrtc as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "prrtc.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return P.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(prrtc_\w+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(names) == set(P.EXPORTS)


STRUCTS = {
    "prrtc_obstacle": P.prrtc_obstacle,
    "prrtc_robot_desc": P.prrtc_robot_desc,
    "prrtc_params": P.prrtc_params,
    "prrtc_path": P.prrtc_path,
    "prrtc_launch_stats": P.prrtc_launch_stats,
    "prrtc_problem": P.prrtc_problem,
    "prrtc_server_config": P.prrtc_server_config,
    "prrtc_server_stats": P.prrtc_server_stats,
}


def test_struct_layouts_match_c(tmp_path):
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "prrtc.h"', "int main(void){"]
    for name, cls in STRUCTS.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{name}.{fname} %zu\\n", offsetof({name}, {fname}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = dict(l.rsplit(" ", 1) for l in subprocess.check_output([str(exe)], text=True).splitlines())
    for name, cls in STRUCTS.items():
        assert int(out[name]) == C.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert int(out[f"{name}.{fname}"]) == getattr(cls, fname).offset, f"{name}.{fname}"


def _has_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.mark.skipif(_has_gpu(), reason="checks the behaviour without a GPU")
def test_no_gpu_fails_loudly(lib):
    h = C.c_void_p()
    rc = lib.prrtc_env_create(None, 0, C.byref(h))
    assert rc == P.ERR_NO_DEVICE
    assert "device" in P.last_error()
    from paper_2503_06757_gb300 import workload as W
    with pytest.raises(P.PrrtcError) as ei:
        P.Robot(W.arm7())
    assert ei.value.code == P.ERR_NO_DEVICE
    # argument validation still happens first
    assert lib.prrtc_check_states(None, None, None, 1, None, None) == P.ERR_INVALID_ARG


def test_params_default(lib):
    p = P.prrtc_params_default()
    assert p.range == 1.0 and abs(p.resolution - 1 / 32) < 1e-9 and abs(p.goal_bias - 0.05) < 1e-7
    assert p.max_iters == 50000 and p.mode == P.MODE_ASYNC and p.seed == 1


def test_status_strings(lib):
    for code in (0, 1, 2, 3, 4, 5, -1, -2, -3, -4, -5, -6, -7):
        assert P.status_string(code) != "unknown status"


def test_numpy_views_match_the_ctypes_structs():
    """The column-wise views used to marshal batches have the C layout."""
    for cls, dt in ((P.prrtc_problem, P._PROBLEM_DT), (P.prrtc_path, P._PATH_DT)):
        assert dt.itemsize == C.sizeof(cls)
        for name, _ in cls._fields_:
            assert dt.fields[name][1] == getattr(cls, name).offset, (cls.__name__, name)


def test_problem_array_points_at_each_problems_data():
    import numpy as np

    class Handle:
        def __init__(self, v):
            self.handle = C.c_void_p(v)

    items = [(Handle(100 + k), Handle(200 + k), np.arange(d, dtype=np.float32) + k,
              -np.arange(d, dtype=np.float32) - k, 7 * k, k) for k, d in enumerate((7, 8, 14, 7))]
    items.append(items[0][:6] + (np.full(8 + 16 * 7, 0.5, np.float32),))
    keep = []
    arr = P._problem_array(items, keep)
    for k, it in enumerate(items):
        pb = arr[k]
        d = len(it[2])
        assert pb.robot == 100 + (k % 4) and pb.env == 200 + (k % 4)
        assert pb.seed == it[4] and pb.problem_id == it[5]
        np.testing.assert_array_equal(np.ctypeslib.as_array(pb.q_start, shape=(d,)), it[2])
        np.testing.assert_array_equal(np.ctypeslib.as_array(pb.q_goal, shape=(d,)), it[3])
        assert bool(pb.gmm) == (len(it) > 6)


def test_paths_free_releases_a_batch_in_one_call(lib):
    """prrtc_paths_free frees library-allocated rows of every path and clears
    them; a null array or n = 0 does nothing (host-only: no GPU needed)."""
    n = 3
    paths = (P.prrtc_path * n)()
    libc = C.CDLL(None)
    libc.malloc.restype = C.c_void_p
    for k in range(n):
        paths[k].n, paths[k].dof = 2, 7
        paths[k].q = C.cast(libc.malloc(2 * 7 * 4), C.POINTER(C.c_float))
    lib.prrtc_paths_free(paths, n)
    assert all(not paths[k].q and paths[k].n == 0 for k in range(n))
    lib.prrtc_paths_free(None, 5)
    lib.prrtc_paths_free(paths, 0)
