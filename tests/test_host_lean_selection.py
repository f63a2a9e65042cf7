"""Host logic of the planner-instance choice, on the CPU: `problem_is_lean`
(csrc/prrtc_launch.h) decides whether a problem may run on the lean kernel
instance, the one compiled without the learned mixture draw, Halton sampling,
dynamic domain, distance fields, oriented boxes, one-stage links and the
wide-range sine/cosine.  A small host program built with nvcc (device code is
cross-compiled, nothing runs on a GPU) evaluates it on synthetic descriptors:
the plain case is lean, and each feature the lean instance leaves out makes the
problem full."""
import os
import subprocess

import pytest

from paper_2503_06757_gb300 import build as B

PROGRAM = r'''
#include <cstdio>
#include <cstring>
#include "prrtc_launch.h"
using namespace prrtc;

static void plain(RobotHeader& H, ProblemDesc& D, float4* env) {
  std::memset(&H, 0, sizeof(H));
  std::memset(&D, 0, sizeof(D));
  H.dof = 3;
  H.two_stage = 1;
  const int types[3] = {kRevZ, kRevY, kPrismZ};
  for (int f = 0; f < 3; ++f) {
    H.jtype[f] = types[f];
    H.lo[f] = f == 2 ? 0.f : -2.8f;
    H.span[f] = f == 2 ? 5.f : 5.6f;   // the prismatic joint may exceed +-3.2
    H.sph_begin[f] = 2 * f;
    H.coarse[f] = make_float4(0.f, 0.f, 0.f, 0.1f);
  }
  H.sph_begin[3] = 6;
  D.env.data = env;
  D.env.n_aabb = 2;
  for (int f = 0; f < 3; ++f) D.q_start[f] = D.q_goal[f] = 0.5f;
}

int main() {
  RobotHeader H;
  ProblemDesc D;
  float4 env[8];
  float grid[1];
  plain(H, D, env);
  printf("plain %d\n", problem_is_lean(H, D));
  plain(H, D, env); D.gmm = grid;                        printf("mixture %d\n", problem_is_lean(H, D));
  plain(H, D, env); D.env.esdf.v = grid;                 printf("esdf %d\n", problem_is_lean(H, D));
  plain(H, D, env); D.env.n_obb = 1;                     printf("obb %d\n", problem_is_lean(H, D));
  plain(H, D, env); D.env.n_aabb = 0;                    printf("empty %d\n", problem_is_lean(H, D));
  plain(H, D, env); H.two_stage = 0;                     printf("one_stage_robot %d\n", problem_is_lean(H, D));
  plain(H, D, env); H.coarse[1].w = 0.f;                 printf("link_without_bound %d\n", problem_is_lean(H, D));
  plain(H, D, env); H.sph_begin[2] = 2; H.coarse[1].w = 0.f;
  printf("empty_link_without_bound %d\n", problem_is_lean(H, D));
  plain(H, D, env); H.span[0] = 6.1f;                    printf("wide_limit %d\n", problem_is_lean(H, D));
  plain(H, D, env); D.q_start[1] = 3.25f;                printf("wide_start %d\n", problem_is_lean(H, D));
  plain(H, D, env); D.q_goal[1] = -3.25f;                printf("wide_goal %d\n", problem_is_lean(H, D));
  plain(H, D, env); D.q_goal[2] = 4.5f;                  printf("prismatic_far %d\n", problem_is_lean(H, D));
  return 0;
}
'''


@pytest.fixture(scope="module")
def verdicts(tmp_path_factory):
    d = tmp_path_factory.mktemp("lean")
    src, exe = os.path.join(d, "lean.cu"), os.path.join(d, "lean")
    with open(src, "w") as f:
        f.write(PROGRAM)
    try:
        nvcc = B.nvcc()
    except Exception as e:  # pragma: no cover - the image always has nvcc
        pytest.skip(f"nvcc not available: {e}")
    cmd = [nvcc] + B.ARCH + ["-std=c++17", "--expt-relaxed-constexpr", "-I", B.CSRC, "-I", B.INCLUDE, src, "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    return {line.split()[0]: int(line.split()[1]) for line in out.splitlines()}


def test_plain_problem_is_lean(verdicts):
    assert verdicts["plain"] == 1


@pytest.mark.parametrize("case", ["mixture", "esdf", "obb", "empty", "one_stage_robot", "link_without_bound",
                                  "wide_limit", "wide_start", "wide_goal"])
def test_each_left_out_feature_needs_the_full_instance(verdicts, case):
    assert verdicts[case] == 0


def test_cases_the_lean_instance_still_serves(verdicts):
    # a link without spheres needs no bound; prismatic joints may go beyond +-3.2
    assert verdicts["empty_link_without_bound"] == 1
    assert verdicts["prismatic_far"] == 1
