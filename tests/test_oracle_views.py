"""Synthetic camera poses: look_at_view is a rigid world-to-camera map that
sends the eye to the origin and the target onto the +z axis, with image y
pointing against the world up vector."""
import numpy as np

from paper_2606_05650_gb300 import synthetic as syn


def test_look_at_view_is_rigid_and_aims_at_target():
    eye, tgt = np.array([2.0, -1.0, 0.7]), np.array([0.5, 0.4, 0.3])
    V = syn.look_at_view(eye, tgt)
    R, t = V[:, :3], V[:, 3]
    assert np.allclose(R @ R.T, np.eye(3)) and np.isclose(np.linalg.det(R), 1.0)
    assert np.allclose(R @ eye + t, 0)
    c = R @ tgt + t
    assert np.allclose(c[:2], 0) and c[2] > 0
    up = R @ np.array([0, 0, 1.0])
    assert up[1] < 0  # world up is image up (negative y)


def test_orbit_views_surround_centre():
    vs = syn.orbit_views(6, radius=2.0)
    for V in vs:
        eye = -V[:, :3].T @ V[:, 3]
        assert np.isclose(np.linalg.norm(eye - 0.5), 2.0)
        c = V[:, :3] @ np.full(3, 0.5) + V[:, 3]
        assert np.allclose(c[:2], 0)
