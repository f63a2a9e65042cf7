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
