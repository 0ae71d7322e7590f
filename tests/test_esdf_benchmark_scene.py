"""Pins of the simulated ESDF benchmark scene (Sec. VI-B): its analytic signed distance at
points with closed-form answers, noiseless returns lying on that surface, and the pose rule."""
import numpy as np
import pytest

from paper_1611_03631_gb300 import scenes


@pytest.mark.parametrize(
    "x,expected",
    [
        ((6.5, 4.0, 2.0), -1.5),  # sphere centre: minus the radius
        ((3.0, 6.5, 1.0), -1.0),  # cube centre: minus the half-size
        ((5.0, 5.0, 5.0), 2.0),  # nearest: the sphere, |(-1.5, 1, 3)| - 1.5 = 3.5 - 1.5
        ((8.0, 1.0, 0.5), 0.5),  # above the ground
        ((0.25, 1.0, 4.0), 0.25),  # next to the wall x = 0
        ((8.0, 9.0, 6.0), 1.0),  # next to the wall y = 10
        ((3.0, 6.5, 2.75), 0.75),  # above the cube's top face
        ((4.0 + 0.6, 7.5 + 0.8, 2.0), 1.0),  # off the cube's top edge corner (0.6, 0.8, 0)
    ],
)
def test_analytic_distance_closed_forms(x, expected):
    assert scenes.esdf_benchmark_sdf(np.array([x]))[0] == pytest.approx(expected, abs=1e-12)


def test_noiseless_returns_lie_on_the_surface_and_poses_keep_clearance():
    s = scenes.esdf_benchmark(poses=6, width=80, height=60, fx=65.625)
    assert len(s) == 6
    n_valid = 0
    for p, T in zip(s.points, s.poses):
        T = T.astype(np.float64)
        assert scenes.esdf_benchmark_sdf(T[None, :3, 3])[0] >= 1.0
        ok = ~np.isnan(p[:, 0])
        n_valid += ok.sum()
        if not ok.any():  # a pose may see nothing within 5 m
            continue
        pw = p[ok].astype(np.float64) @ T[:3, :3].T + T[:3, 3]
        assert np.max(np.abs(scenes.esdf_benchmark_sdf(pw))) < 1e-5
        depth = p[ok, 2]
        assert (depth > 0).all() and (depth <= 5.0 + 1e-5).all()
    assert n_valid > 1000
