"""Pins of oracle/travel.py (Eq. e1 and the Euclidean alternative) against closed forms
and an independent formula (no GPU needed)."""
import math

import numpy as np
import pytest

from oracle import travel
from paper_2002_11710_gb300 import gen

R = travel.EARTH_RADIUS_KM


def test_euclidean_closed_forms():
    d = travel.euclidean_km([[0.0, 0.0], [3.0, 4.0], [3.0, 0.0]])
    assert d[0, 1] == 5.0 and d[1, 0] == 5.0 and d[0, 2] == 3.0 and d[1, 2] == 4.0
    assert (np.diag(d) == 0).all()


def test_minutes_round_half_to_even():
    # 60 km/h: one kilometre is one minute
    xy = [[0.0, 0.0], [2.5, 0.0], [3.5, 0.0], [0.5, 0.0], [1.25, 0.0]]
    m = travel.travel_minutes(xy, [60.0, 120.0], travel.EUCLIDEAN)
    assert m.dtype == np.int32 and m.shape == (2, 5, 5)
    assert m[0, 0, 1] == 2 and m[0, 0, 2] == 4 and m[0, 0, 3] == 0 and m[0, 0, 4] == 1
    assert m[1, 0, 2] == 2 and m[1, 0, 1] == 1  # 1.75 -> 2, 1.25 -> 1


@pytest.mark.parametrize("pts,want", [
    ([[0.0, 0.0], [0.0, 90.0]], R * math.pi / 2),      # a quarter of the equator
    ([[0.0, 0.0], [45.0, 0.0]], R * math.pi / 4),      # along a meridian
    ([[0.0, 0.0], [0.0, 180.0]], R * math.pi),         # antipodes (the clip keeps it finite)
    ([[90.0, 0.0], [-90.0, 0.0]], R * math.pi),        # pole to pole
    ([[52.0, 13.0], [52.0, 13.0]], 0.0),
])
def test_haversine_closed_forms(pts, want):
    d = travel.haversine_km(pts)
    assert d[0, 1] == pytest.approx(want, rel=1e-12, abs=1e-9)
    assert d[0, 1] == d[1, 0]


def test_haversine_against_chord_formula():
    """Independent: the chord between unit vectors c gives the arc 2 asin(c / 2)."""
    rng = np.random.default_rng(3)
    ll = np.stack([rng.uniform(-80, 80, 60), rng.uniform(-180, 180, 60)], axis=1)
    d = travel.haversine_km(ll)
    lat, lon = np.radians(ll[:, 0]), np.radians(ll[:, 1])
    u = np.stack([np.cos(lat) * np.cos(lon), np.cos(lat) * np.sin(lon), np.sin(lat)], axis=1)
    chord = np.linalg.norm(u[:, None, :] - u[None, :, :], axis=2)
    want = 2 * R * np.arcsin(np.minimum(chord / 2, 1.0))
    np.testing.assert_allclose(d, want, rtol=1e-9, atol=1e-6)
    assert np.all(d <= d[:, :1] + d[:1, :] + 1e-6)  # triangle inequality through point 0


def test_generator_matrices_follow_the_definition():
    """gen's matrices (np.hypot) equal the oracle's Euclidean minutes on the workloads."""
    for inst, speeds in [(gen.paper_shaped(0), [250.0]), (gen.paper_fleet(3, 30), [300.0, 500.0]),
                         (gen.tiny(0), [250.0])]:
        m = travel.travel_minutes(inst.coords, speeds, travel.EUCLIDEAN)
        np.testing.assert_array_equal(m, inst.travel)
