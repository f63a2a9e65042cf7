"""GPU parity of the distance-field (ESDF) collision path with the FP64 oracle.

* Voxelisation: bit-exact wherever the voxel centre is farther than 1e-5 m
  from every primitive surface.
* Signed distance transform: integer squared distances are exact on both
  sides, so the fields agree to FP32 rounding of sqrt and the voxel scale;
  at full size, spot checks against the oracle's single-voxel definition.
* Collision verdicts and serial-mode plans against an ESDF environment
  equal the oracle's outside the 1e-5 m clearance band.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_06757_gb300 import prrtc as P
from paper_2503_06757_gb300 import workload as W
from tests import helpers as H

pytestmark = pytest.mark.gpu

F32 = lambda x: float(np.float32(x))
BAND = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2503_06757_gb300 import build
    build.build()


def f32v(v):
    return [F32(x) for x in v]


def grid_for(voxel, dims, origin):
    return f32v(origin), F32(voxel), tuple(dims)


@pytest.mark.parametrize("kind,seed", [("shelf", 1000), ("mixed", 2003), ("mixed", 2004)])
def test_voxelize_matches_oracle(kind, seed):
    sc = W.scene_shelf(seed) if kind == "shelf" else W.scene_mixed(seed, 80)
    origin, voxel, dims = grid_for(0.07, (23, 24, 25), (-0.8, -0.8, 0.0))
    got = P.make_env(sc).voxelize(origin, voxel, dims)
    want = O.voxelize(sc, np.array(origin, np.float64), voxel, dims)
    bad = np.argwhere(got != want)
    for k, j, i in bad:
        p = np.array(origin) + (np.array([i, j, k]) + 0.5) * voxel
        sd = min([O.sd_box(b, p) for b in sc.boxes] + [O.sd_cyl(c, p) for c in sc.cylinders] +
                 [O.sd_sph(s, p) for s in sc.spheres])
        assert abs(sd) <= BAND, (i, j, k, sd)
    assert 0 < want.sum() < want.size


@pytest.mark.parametrize("dims,frac,seed", [((20, 18, 16), 0.1, 0), ((7, 31, 9), 0.3, 1), ((2, 2, 2), 0.5, 2),
                                            ((33, 5, 4), 0.02, 3)])
def test_distance_transform_matches_oracle(dims, frac, seed):
    rng = np.random.default_rng(seed)
    occ = (rng.random((dims[2], dims[1], dims[0])) < frac).astype(np.uint8)
    voxel = F32(0.03)
    env = P.Env.from_occupancy(occ, (0.0, 0.0, 0.0), voxel)
    got = env.esdf().astype(np.float64)
    want = O.esdf(occ, dims, voxel)
    np.testing.assert_allclose(got, want, rtol=2e-7, atol=1e-9)


@pytest.mark.parametrize("fill", [0, 1])
def test_distance_transform_empty_and_full(fill):
    dims = (6, 5, 4)
    occ = np.full((4, 5, 6), fill, np.uint8)
    env = P.Env.from_occupancy(occ, (0.0, 0.0, 0.0), 0.1)
    np.testing.assert_allclose(env.esdf(), O.esdf(occ, dims, F32(0.1)), rtol=2e-7)


def test_distance_transform_full_size_spot_checks():
    """A 128^3 grid voxelised from a shelf scene (1.25 cm voxels, 2M voxels):
    the oracle's single-voxel definition at 120 sampled voxels."""
    sc = W.scene_shelf(1005)
    dims = (128, 128, 128)
    origin, voxel = f32v((-0.8, -0.8, 0.0)), F32(1.6 / 128)
    occ = P.make_env(sc).voxelize(origin, voxel, dims)
    env = P.Env.from_occupancy(occ, origin, voxel)
    field = env.esdf()
    rng = np.random.default_rng(7)
    # half of the samples next to the surfaces, where the field changes sign
    near = np.argwhere(np.abs(field) < 2.5 * voxel)
    pick = list(near[rng.choice(len(near), 60, replace=False)]) + \
        [rng.integers(0, 128, 3) for _ in range(60)]
    for k, j, i in pick:
        want = O.esdf_at(occ, dims, voxel, int(i), int(j), int(k))
        assert abs(field[k, j, i] - want) <= 2e-7 * abs(want) + 1e-9, (i, j, k, field[k, j, i], want)


def _esdf_setup(seed=1000, dims=(22, 22, 22), extent=1.6):
    sc = W.scene_shelf(seed)
    origin, voxel = f32v((-0.8, -0.8, 0.0)), F32(extent / dims[0])
    occ = O.voxelize(sc, np.array(origin, np.float64), voxel, dims)  # the oracle's occupancy is the input
    field = O.esdf(occ, dims, voxel)
    return sc, occ, origin, voxel, dims, field


def test_check_states_against_esdf_env_matches_oracle():
    sc, occ, origin, voxel, dims, field = _esdf_setup()
    env = P.Env.from_occupancy(occ, origin, voxel)
    for name in ("arm7", "arm8"):
        rb = W.ROBOTS[name]()
        h = P.make_robot(rb)
        Q = W.candidates(rb, 23, 5, 2000).astype(np.float32)
        got = P.prrtc_check_states(h, env, Q)
        free, cl = O.check_states(rb, H.empty_scene(), Q.astype(np.float64),
                                  esdf=(field, np.array(origin, np.float64), voxel, dims))
        clear = np.abs(cl) > BAND
        np.testing.assert_array_equal(got[clear], free[clear])
        assert 0.05 < free.mean() < 0.95


def test_esdf_update_changes_verdicts():
    rb = H.robot([W.JOINT_PRISM_X], [0.0], bases=[[0.0, 0.0, 0.5]], lower=[-0.7], upper=[0.7],
                 spheres=[(0, (0.0, 0.0, 0.0), 0.05)], name="slider")
    h = P.make_robot(rb)
    dims = (32, 32, 32)
    origin, voxel = (-0.8, -0.8, 0.0), 0.05
    occ = np.zeros((32, 32, 32), np.uint8)
    env = P.Env.from_occupancy(occ, origin, voxel)
    Q = np.array([[-0.5], [0.0], [0.5]], np.float32)
    assert P.prrtc_check_states(h, env, Q).tolist() == [True, True, True]
    occ[:, :, 18:] = 1  # x >= 0.1 occupied
    env.update_occupancy(occ)
    assert P.prrtc_check_states(h, env, Q).tolist() == [True, True, False]


@pytest.fixture(scope="module")
def esdf_problems():
    sc, occ, origin, voxel, dims, field = _esdf_setup(seed=1002)
    rb = W.arm7()
    env = P.Env.from_occupancy(occ, origin, voxel)
    Q = W.candidates(rb, 31, 7, 4000)
    free, cl = O.check_states(rb, H.empty_scene(), Q, esdf=(field, np.array(origin, np.float64), voxel, dims))
    ok = np.nonzero(free & (cl > 1e-3))[0]
    return rb, env, (field, np.array(origin, np.float64), voxel, dims), [(Q[ok[2 * m]], Q[ok[2 * m + 1]])
                                                                        for m in range(4)]


@pytest.mark.parametrize("k", range(4))
def test_serial_plan_against_esdf_matches_oracle(esdf_problems, k):
    rb, env, esdf, pairs = esdf_problems
    s, g = (x.astype(np.float32) for x in pairs[k])
    h = P.make_robot(rb)
    r = P.prrtc_plan(h, env, s, g, P.params(seed=4, mode=P.MODE_SERIAL, tree_capacity=1 << 14, max_iters=3000))
    o = O.plan(rb, H.empty_scene(), s.astype(np.float64), g.astype(np.float64), seed=4, want_trees=True,
               tree_capacity=1 << 14, max_iters=3000, range=1.0, resolution=F32(1 / 32), goal_bias=F32(0.05),
               esdf=esdf)
    amb = o["first_amb_iter"]
    if amb != -1 and amb < o["iterations"]:
        pytest.skip(f"oracle met an ambiguous decision at iteration {amb} (kind {o['first_amb_kind']})")
    assert r["status"] == o["status"]
    assert r["iterations"] == o["iterations"]
    assert (r["nodes_a"], r["nodes_b"]) == (o["n_a"], o["n_b"])
    for t, (nodes, par) in enumerate(((o["nodes_a"], o["parent_a"]), (o["nodes_b"], o["parent_b"]))):
        gn, gp = P.prrtc_debug_tree(0, t, rb.dof)
        np.testing.assert_array_equal(gp, par)
        np.testing.assert_allclose(gn, nodes, atol=1e-4)
    if o["status"] == 0:
        np.testing.assert_allclose(r["path"], o["path"], atol=1e-4)


def test_async_plans_against_esdf_revalidate(esdf_problems):
    rb, env, esdf, pairs = esdf_problems
    h = P.make_robot(rb)
    items = [(h, env, s.astype(np.float32), g.astype(np.float32), 3, k) for k, (s, g) in enumerate(pairs)]
    res = P.prrtc_plan_batch(items, P.params())
    g_items, o_items = [], []
    for k, ((s, g), r) in enumerate(zip(pairs, res)):
        assert r["status"] == P.SOLVED
        g_items.append((rb, H.empty_scene(), r["path"], esdf))
        o = O.plan(rb, H.empty_scene(), s.astype(np.float32).astype(np.float64), g.astype(np.float32).astype(np.float64),
                   seed=3, problem=k, range=1.0, resolution=F32(1 / 32), goal_bias=F32(0.05), esdf=esdf)
        assert o["status"] == 0
        o_items.append((rb, H.empty_scene(), o["path"], esdf))
    # re-checked at 4x resolution against the field, GPU and oracle paths are flagged alike
    H.assert_same_revalidation_rate(H.revalidation_counts(g_items, F32(1 / 32) / 4),
                                    H.revalidation_counts(o_items, F32(1 / 32) / 4), "distance field")


def test_esdf_grid_validation():
    occ = np.zeros((4, 4, 4), np.uint8)
    for origin, voxel, shape in (((0, 0, 0), 0.0, (4, 4, 4)), ((0, 0, float("nan")), 0.1, (4, 4, 4)),
                                 ((0, 0, 0), 0.1, (1, 4, 4))):
        with pytest.raises(P.PrrtcError) as e:
            P.Env.from_occupancy(np.zeros(shape, np.uint8), origin, voxel)
        assert e.value.code == P.ERR_INVALID_ARG
    env = P.make_env(H.empty_scene())
    with pytest.raises(P.PrrtcError):
        env.update_occupancy(occ)
