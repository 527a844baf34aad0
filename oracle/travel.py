"""Travel-time matrices from coordinates, the plain way (test infrastructure only).

Eq. e1 (Section 3): the time between locations i and j for a vehicle of type l is the
Haversine distance between them divided by the vehicle's speed K_s,

    d_ijl = 2 r asin( sqrt( sin^2((phi_i - phi_j) / 2)
                            + cos(phi_i) cos(phi_j) sin^2((psi_i - psi_j) / 2) ) ) / K_s,

phi latitude and psi longitude in radians, r the Earth's radius. The synthetic workloads
place points in a square kilometre box instead, where the distance is Euclidean. Times
are integer minutes: rint(distance_km / speed_kmh * 60), half to even, in float64 (the
paper's own code is Python, float64).

Readings: the radius is 6371 km unless given; sqrt(a) is clipped to 1 before the
arcsine (rounding can push it a hair above 1 for antipodal points). Every step below is
a single numpy float64 operation, in the order written, so a device implementation
that rounds each step the same way gets the same integers for the Euclidean metric.
Only the callers allowed to use the oracle import this module.
"""
from __future__ import annotations

import math

import numpy as np

EUCLIDEAN, HAVERSINE = 0, 1
EARTH_RADIUS_KM = 6371.0


def euclidean_km(xy):
    """[L][L] distances between points (x, y) in kilometres."""
    xy = np.asarray(xy, dtype=np.float64)
    dx = xy[:, None, 0] - xy[None, :, 0]
    dy = xy[:, None, 1] - xy[None, :, 1]
    return np.sqrt(dx * dx + dy * dy)


def haversine_km(latlon_deg, radius_km: float = EARTH_RADIUS_KM):
    """[L][L] great-circle distances (Eq. e1's numerator) between (latitude, longitude)
    points given in degrees."""
    ll = np.asarray(latlon_deg, dtype=np.float64)
    k = math.pi / 180.0
    phi = ll[:, 0] * k
    psi = ll[:, 1] * k
    s1 = np.sin((phi[:, None] - phi[None, :]) * 0.5)
    s2 = np.sin((psi[:, None] - psi[None, :]) * 0.5)
    c = np.cos(phi)
    a = s1 * s1 + (c[:, None] * c[None, :]) * (s2 * s2)
    return (2.0 * radius_km) * np.arcsin(np.minimum(np.sqrt(a), 1.0))


def distance_km(coords, metric: int, radius_km: float = EARTH_RADIUS_KM):
    if metric == EUCLIDEAN:
        return euclidean_km(coords)
    if metric == HAVERSINE:
        return haversine_km(coords, radius_km)
    raise ValueError(metric)


def minutes_unrounded(coords, speeds_kmh, metric: int, radius_km: float = EARTH_RADIUS_KM):
    """[n_types][L][L] times in minutes before rounding."""
    d = distance_km(coords, metric, radius_km)
    return np.stack([d / float(s) * 60.0 for s in speeds_kmh])


def travel_minutes(coords, speeds_kmh, metric: int, radius_km: float = EARTH_RADIUS_KM):
    """[n_types][L][L] int32 travel minutes (Eq. e1 with the readings above)."""
    return np.rint(minutes_unrounded(coords, speeds_kmh, metric, radius_km)).astype(np.int32)
