"""Host logic of the workloads and training data, on CPU: the two-room scene's
door, the start/goal rooms, and the waypoints taken from solution paths."""
import numpy as np
import pytest

from paper_2503_06757_gb300 import learned as L
from paper_2503_06757_gb300 import workload as W


@pytest.mark.parametrize("door", [(0.85, 0.93), (0.865, 0.915)])
def test_two_rooms_wall_leaves_exactly_the_door_open(door):
    sc = W.scene_two_rooms(door=door)
    assert sc.boxes.shape[0] == 2 and sc.cylinders.shape[0] == 0 and sc.spheres.shape[0] == 0
    # every box is axis-aligned, 4 cm thick, centred on x = 0.6
    for b in sc.boxes:
        np.testing.assert_allclose(b[6:], np.eye(3).reshape(9))
        assert abs(b[0] - 0.6) < 1e-6 and abs(b[3] - 0.02) < 1e-6
    # the wall covers y in [0, 1.2] except the door
    spans = sorted((b[1] - b[4], b[1] + b[4]) for b in sc.boxes)
    assert abs(spans[0][0]) < 1e-6 and abs(spans[1][1] - 1.2) < 1e-6
    assert abs(spans[0][1] - door[0]) < 1e-6 and abs(spans[1][0] - door[1]) < 1e-6


def test_two_rooms_pairs_lie_in_opposite_rooms():
    s, g = W.two_rooms_pairs(500, 3)
    assert s.shape == g.shape == (500, 2)
    # values are binary32 numbers, so both sides of the parity tests see the same inputs
    np.testing.assert_array_equal(s, s.astype(np.float32).astype(s.dtype))
    assert np.all((s[:, 0] >= 0.05) & (s[:, 0] <= 0.5)) and np.all((g[:, 0] >= 0.7) & (g[:, 0] <= 1.15))
    assert np.all((s[:, 1] >= 0.05) & (s[:, 1] <= 1.15)) and np.all((g[:, 1] >= 0.05) & (g[:, 1] <= 1.15))
    s2, _ = W.two_rooms_pairs(500, 3)
    np.testing.assert_array_equal(s, s2)  # seeded


def test_waypoints_are_evenly_spaced_on_the_path():
    path = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0]])
    wp = L.waypoints(path, spacing=0.25)
    # arclength 0.25, 0.5, ..., 1.75 (interior only: not 0, not 2)
    assert len(wp) == 7
    cum = np.minimum(np.arange(1, 8) * 0.25, 1.0)
    np.testing.assert_allclose(wp[:4, 0], cum[:4])
    np.testing.assert_allclose(wp[4:], [[1.0, 0.25], [1.0, 0.5], [1.0, 0.75]])
    full = L.waypoints(path, spacing=0.25, interior=False)
    np.testing.assert_allclose(full[0], path[0])
    np.testing.assert_allclose(full[-1], path[-1])
    assert len(L.waypoints(path[:1], spacing=0.25)) == 0


def test_shelf_facing_both_arms():
    """The dual arm's shelf is the single arm's scene turned 90 degrees about z:
    four turns give the scene back, the cells sit behind the plane y = 0.45, and
    the dual arm has collision-free configurations in it (the oracle's check)."""
    import numpy as np
    from oracle import oracle as O
    sc = W.scene_shelf(1234)
    r = sc
    for _ in range(4):
        r = W.rotate_scene_z90(r)
    np.testing.assert_allclose(r.boxes, sc.boxes, atol=1e-6)
    np.testing.assert_allclose(r.cylinders, sc.cylinders, atol=1e-6)
    np.testing.assert_allclose(r.spheres, sc.spheres, atol=1e-6)
    y = W.scene_shelf(1234, W.shelf_facing(W.dual14()))
    assert W.shelf_facing(W.arm7()) == "x" and W.shelf_facing(W.dual14()) == "y"
    assert np.all(y.cells[:, 1] >= 0.45 - 1e-6)
    rb = W.dual14()
    free, _ = O.check_states(rb, y, W.candidates(rb, 1234, 0, 256))
    assert free.mean() > 0.3


def test_concat_datasets_renumbers_scenes():
    import numpy as np
    from paper_2503_06757_gb300 import learned as L
    a = L.Dataset(dof=2, occ=np.zeros((2, 4096), np.uint8), scene_of=np.array([0, 1, 1], np.int32),
                  q_start=np.zeros((3, 2), np.float32), q_goal=np.zeros((3, 2), np.float32),
                  target=np.zeros((3, 2), np.float32), paths=2, problems=2)
    b = L.Dataset(dof=2, occ=np.ones((3, 4096), np.uint8), scene_of=np.array([2, 0], np.int32),
                  q_start=np.ones((2, 2), np.float32), q_goal=np.ones((2, 2), np.float32),
                  target=np.ones((2, 2), np.float32), paths=1, problems=3)
    c = L.concat_datasets([a, b])
    assert c.occ.shape == (5, 4096) and c.paths == 3 and c.problems == 5
    np.testing.assert_array_equal(c.scene_of, [0, 1, 1, 4, 2])
    assert np.all(c.occ[c.scene_of[3:]] == 1)


def test_scene_at_places_the_moving_spheres():
    """The scene a served query saw: the static obstacles as built, the moving
    spheres at the positions recorded when it was submitted."""
    import numpy as np
    from paper_2503_06757_gb300 import serving as S
    mv = W.moving_spheres(3000, S.N_MOVING)
    base = W.scene_mixed(3000, 40)
    sph = np.concatenate([base.spheres, np.concatenate([mv.centres0, mv.radii[:, None]], 1)])
    sc = S.ServeScene(W.arm7(), None, None, W.Scene(base.boxes, base.cylinders, sph), mv, [], [])
    pos = mv.positions_track(10)[7]
    at = S.scene_at(sc, pos)
    np.testing.assert_array_equal(at.boxes, base.boxes)
    np.testing.assert_array_equal(at.spheres[:len(base.spheres)], base.spheres)
    np.testing.assert_array_equal(at.spheres[len(base.spheres):, :3], pos)
    np.testing.assert_array_equal(at.spheres[len(base.spheres):, 3], mv.radii)
    assert not np.array_equal(pos, mv.centres0)
