"""Seeded synthetic instances for the air-ambulance scheduling problem.

This module only draws inputs. It holds none of the scheduling arithmetic (no
route cost, no move, no feasibility rule), so both the CPU oracle and the CUDA
path can take their inputs from it.

The paper's own eight datasets (real coordinates of air bases and health
facilities, Section 5) are not available, so seeded instances with the same
structure stand in for them:

* locations ``0 .. B-1`` are bases, ``B .. B+F-1`` are health facilities;
* a mission is a (pickup facility, delivery facility) pair with pickup !=
  delivery (the 6-tuple of Section 3 without coordinates, which live in the
  travel-time matrix);
* the travel-time matrix ``T[type][i][j]`` holds integer minutes,
  ``rint(dist_km / speed_kmh * 60)`` (Eq. e1 divides a distance by the vehicle
  speed; the configurations here use Euclidean kilometres in a square box);
* vehicles sit on bases round-robin (``veh_base[v] = v mod B``); bases and
  vehicles are interchangeable in the paper's model (Section 3).

Draw order for a given ``numpy.random.default_rng(seed)`` is fixed:
base coordinates, facility coordinates (cluster centres, memberships, Gaussian
offsets, outlier mask, outlier coordinates, then clipping), missions (pickups,
then deliveries), then optional heli-only flags and deadlines.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

HARD = 0
PENALTY = 1


@dataclasses.dataclass
class Instance:
    """One scheduling problem, all arrays int32 and C-contiguous.

    travel     [n_types, L, L] minutes, type 0 = helicopter, 1 = plane
    veh_base   [V] base location of each vehicle
    veh_type   [V] 0 (helicopter) or 1 (plane)
    pickup     [M], delivery [M] facility locations, pickup != delivery
    heli_only  [M] 1 if only a helicopter may fly the mission, or None
    deadline   [M] arrive-by minute at the delivery, or None (no deadlines)
    duty_cap   maximum flight minutes per vehicle (the constant p)
    horizon    latest return-to-base minute when deadlines are on (24 h)
    coords     [L, 2] float64 location coordinates the matrix was built from (x, y km),
               or None
    """

    travel: np.ndarray
    veh_base: np.ndarray
    veh_type: np.ndarray
    pickup: np.ndarray
    delivery: np.ndarray
    heli_only: Optional[np.ndarray]
    deadline: Optional[np.ndarray]
    duty_cap: int
    horizon: int = 1440
    name: str = ""
    coords: Optional[np.ndarray] = None

    @property
    def n_loc(self) -> int:
        return int(self.travel.shape[1])

    @property
    def n_types(self) -> int:
        return int(self.travel.shape[0])

    @property
    def n_vehicles(self) -> int:
        return int(self.veh_base.shape[0])

    @property
    def n_missions(self) -> int:
        return int(self.pickup.shape[0])

    def subinstance(self, missions) -> "Instance":
        """The same fleet and matrix with only the listed missions."""
        idx = np.asarray(list(missions), dtype=np.int64)
        return dataclasses.replace(
            self,
            pickup=np.ascontiguousarray(self.pickup[idx]),
            delivery=np.ascontiguousarray(self.delivery[idx]),
            heli_only=None if self.heli_only is None else np.ascontiguousarray(self.heli_only[idx]),
            deadline=None if self.deadline is None else np.ascontiguousarray(self.deadline[idx]),
            name=self.name + f"[{len(idx)} missions]",
        )


@dataclasses.dataclass
class Params:
    """Tabu search parameters.

    tenure      iterations a (mission, vehicle it left) pair stays tabu
    iterations  fixed iteration budget
    cap_mode    HARD (duty cap is a constraint) or PENALTY (lambda per minute over)
    lam         penalty weight in PENALTY mode
    """

    tenure: int
    iterations: int
    cap_mode: int = HARD
    lam: int = 1000


def minutes_matrix(xy: np.ndarray, speed_kmh: float) -> np.ndarray:
    """Integer-minute travel times between all point pairs (float64, half-to-even)."""
    d = np.hypot(xy[:, None, 0] - xy[None, :, 0], xy[:, None, 1] - xy[None, :, 1])
    return np.rint(d / speed_kmh * 60.0).astype(np.int32)


def _uniform_points(rng, n, box):
    return rng.uniform(0.0, box, size=(n, 2))


def _clustered_points(rng, n, box, n_clusters=4, sigma=80.0, outlier_frac=0.2):
    centres = rng.uniform(0.0, box, size=(n_clusters, 2))
    member = rng.integers(0, n_clusters, size=n)
    offs = rng.normal(0.0, sigma, size=(n, 2))
    outlier = rng.random(n) < outlier_frac
    out_xy = rng.uniform(0.0, box, size=(n, 2))
    xy = centres[member] + offs
    xy[outlier] = out_xy[outlier]
    return np.clip(xy, 0.0, box)


def _uniform_pairs(rng, n_fac, m):
    p = rng.integers(0, n_fac, size=m)
    d = (p + 1 + rng.integers(0, n_fac - 1, size=m)) % n_fac
    return p, d


def _zipf_pairs(rng, n_fac, m, s):
    perm = rng.permutation(n_fac)
    w = 1.0 / np.arange(1, n_fac + 1, dtype=np.float64) ** s
    w /= w.sum()
    p = perm[rng.choice(n_fac, size=m, p=w)]
    d = perm[rng.choice(n_fac, size=m, p=w)]
    clash = p == d
    while clash.any():
        d[clash] = perm[rng.choice(n_fac, size=int(clash.sum()), p=w)]
        clash = p == d
    return p, d


def make_instance(seed: int, *, n_bases: int, n_vehicles: int, n_facilities: int,
                  n_missions: int, box_km: float, geography: str = "uniform",
                  pairs: str = "uniform", zipf_s: float = 1.1, speed_kmh: float = 250.0,
                  duty_cap: int = 720, horizon: int = 1440, plane_speed_kmh: Optional[float] = None,
                  n_planes: int = 0, heli_only_frac: float = 0.0, deadlines: bool = False,
                  deadline_lo: int = 0, deadline_window: bool = False, name: str = "") -> Instance:
    """Draw one instance; see the module docstring for the fixed draw order.

    With ``plane_speed_kmh`` set there are two travel layers (type 0 helicopter at
    ``speed_kmh``, type 1 plane at ``plane_speed_kmh``) and the first ``n_planes``
    bases hold planes, as in the paper's 4 plane + 8 helicopter fleet (Section 5).

    ``deadline_window``: instead of uniform in [deadline_lo, horizon], each mission's
    arrive-by time is drawn inside a window that some vehicle allowed to fly it can meet
    on its own (leave base at 0, arrive by w, be home by the horizon): one compatible
    vehicle with a non-empty window is drawn uniformly, then w uniformly in it. Every
    mission is then feasible alone (the paper only kept valid scenarios, Section 5);
    together they may still not be.
    """
    rng = np.random.default_rng(seed)
    base_xy = _uniform_points(rng, n_bases, box_km)
    if geography == "uniform":
        fac_xy = _uniform_points(rng, n_facilities, box_km)
    elif geography == "clustered":
        fac_xy = _clustered_points(rng, n_facilities, box_km)
    else:
        raise ValueError(geography)
    if pairs == "uniform":
        p, d = _uniform_pairs(rng, n_facilities, n_missions)
    elif pairs == "zipf":
        p, d = _zipf_pairs(rng, n_facilities, n_missions, zipf_s)
    else:
        raise ValueError(pairs)
    xy = np.concatenate([base_xy, fac_xy], axis=0)
    layers = [minutes_matrix(xy, speed_kmh)]
    if plane_speed_kmh is not None:
        layers.append(minutes_matrix(xy, plane_speed_kmh))
    travel = np.ascontiguousarray(np.stack(layers).astype(np.int32))
    veh_base = (np.arange(n_vehicles) % n_bases).astype(np.int32)
    if plane_speed_kmh is not None:
        veh_type = (veh_base < n_planes).astype(np.int32)
    else:
        veh_type = np.zeros(n_vehicles, dtype=np.int32)
    heli = None
    if heli_only_frac > 0.0:
        heli = (rng.random(n_missions) < heli_only_frac).astype(np.int32)
    dl = None
    if deadlines and not deadline_window:
        dl = rng.integers(deadline_lo, horizon + 1, size=n_missions).astype(np.int32)
    elif deadlines:
        # windows [lo, hi] per (mission, vehicle): leave base at 0, arrive by w, home by the horizon
        pk, dv = p + n_bases, d + n_bases
        T = travel[veh_type]  # [V][L][L], each vehicle's own layer
        vi = np.arange(n_vehicles)[None, :]
        lo = np.maximum(deadline_lo, T[vi, veh_base[None, :], pk[:, None]] + T[vi, pk[:, None], dv[:, None]])
        hi = horizon - T[vi, dv[:, None], veh_base[None, :]]
        ok = lo <= hi
        if heli is not None:
            ok &= ~((heli[:, None] != 0) & (veh_type[None, :] != 0))
        n_ok = ok.sum(axis=1)
        if (n_ok == 0).any():
            raise ValueError(f"mission {int(np.argmin(n_ok))} fits no vehicle within the horizon")
        # one vehicle window per mission (uniform over the valid ones), then w uniform in it
        pick = np.minimum((rng.random(n_missions) * n_ok).astype(np.int64), n_ok - 1)
        col = np.argmax(np.cumsum(ok, axis=1) > pick[:, None], axis=1)
        rows = np.arange(n_missions)
        lo_j, hi_j = lo[rows, col], hi[rows, col]
        dl = (lo_j + np.minimum((rng.random(n_missions) * (hi_j - lo_j + 1)).astype(np.int64),
                                hi_j - lo_j)).astype(np.int32)
    return Instance(
        travel=travel,
        veh_base=veh_base,
        veh_type=veh_type,
        pickup=(p + n_bases).astype(np.int32),
        delivery=(d + n_bases).astype(np.int32),
        heli_only=heli,
        deadline=dl,
        duty_cap=int(duty_cap),
        horizon=int(horizon),
        name=name,
        coords=np.ascontiguousarray(xy, dtype=np.float64),
    )


# --- the named workloads -------------------------------------------------------------

def tiny(seed: int = 0) -> Instance:
    """3 bases with one vehicle each, 6 facilities, 10 missions, uniform 1000 km box, 12 h cap."""
    return make_instance(seed, n_bases=3, n_vehicles=3, n_facilities=6, n_missions=10,
                         box_km=1000.0, duty_cap=720, name=f"tiny-s{seed}")


TINY_PARAMS = Params(tenure=7, iterations=200, cap_mode=HARD)


def paper_shaped(seed: int = 0) -> Instance:
    """12 bases, 20 vehicles, 60 clustered facilities in a 1500 km box, 100 uniform missions."""
    return make_instance(seed, n_bases=12, n_vehicles=20, n_facilities=60, n_missions=100,
                         box_km=1500.0, geography="clustered", duty_cap=720,
                         name=f"paper-shaped-s{seed}")


PAPER_SHAPED_PARAMS = Params(tenure=10, iterations=5000, cap_mode=PENALTY, lam=1000)


def large(seed: int = 0) -> Instance:
    """40 bases, 50 vehicles, 200 clustered facilities in a 3000 km box, 400 Zipf missions."""
    return make_instance(seed, n_bases=40, n_vehicles=50, n_facilities=200, n_missions=400,
                         box_km=3000.0, geography="clustered", pairs="zipf", duty_cap=960,
                         name=f"large-s{seed}")


LARGE_PARAMS = Params(tenure=15, iterations=10000, cap_mode=PENALTY, lam=1000)


def batched_member(i: int) -> Instance:
    """Instance i of the 1,024-instance batch: V ~ U[3,30], M ~ U[10,200], paper-shaped geography."""
    seed = 1000 + i
    rng = np.random.default_rng(seed)
    v = int(rng.integers(3, 31))
    m = int(rng.integers(10, 201))
    return make_instance(seed, n_bases=12, n_vehicles=v, n_facilities=60, n_missions=m,
                         box_km=1500.0, geography="clustered", duty_cap=720,
                         name=f"batched-{i}")


BATCHED_PARAMS = Params(tenure=10, iterations=2000, cap_mode=PENALTY, lam=1000)


def serving_size(rng) -> tuple[int, int]:
    """Request size: M = clip(round(lognormal(ln 60, 0.5)), 10, 400), V = ceil(M / 5)."""
    m = int(np.clip(np.rint(rng.lognormal(math.log(60.0), 0.5)), 10, 400))
    return m, int(math.ceil(m / 5))


def paper_model(seed: int, n_missions: int, *, heli_only_frac: float = 0.3,
                deadlines: bool = True) -> Instance:
    """The paper's fleet (Section 5): 4 plane bases (500 km/h) + 8 helicopter bases (300 km/h),
    one vehicle each, heli-only missions, random arrive-by times within 24 h, 10 h cap."""
    return make_instance(seed, n_bases=12, n_vehicles=12, n_facilities=40,
                         n_missions=n_missions, box_km=1000.0, geography="clustered",
                         speed_kmh=300.0, plane_speed_kmh=500.0, n_planes=4,
                         heli_only_frac=heli_only_frac, deadlines=deadlines,
                         deadline_lo=240, duty_cap=600, name=f"paper-model-s{seed}-m{n_missions}")



def paper_fleet(seed: int, n_missions: int, *, heli_only_frac: float = 0.3) -> Instance:
    """The paper's fleet as paper_model, with arrive-by times drawn inside windows a
    compatible vehicle can meet (``deadline_window``), so that no mission is infeasible
    on its own. The workload of the paper's own sweeps (Algorithms 2 and 3)."""
    return make_instance(seed, n_bases=12, n_vehicles=12, n_facilities=40,
                         n_missions=n_missions, box_km=1000.0, geography="clustered",
                         speed_kmh=300.0, plane_speed_kmh=500.0, n_planes=4,
                         heli_only_frac=heli_only_frac, deadlines=True, deadline_lo=240,
                         deadline_window=True, duty_cap=600,
                         name=f"paper-fleet-s{seed}-m{n_missions}")


def sweep_orders(seed: int, n_vehicles: int, n_missions: int):
    """The random loop orders of one run of the paper's sweeps (its permutation vectors
    for the loops over bases and over a base's missions): a permutation of the vehicles
    and a rank for every mission, both uniform, from their own seed."""
    rng = np.random.default_rng(seed)
    vorder = rng.permutation(n_vehicles).astype(np.int32)
    mrank = rng.permutation(n_missions).astype(np.int32)
    return vorder, mrank


def random_instance(seed: int, *, n_loc: int, n_vehicles: int, n_missions: int,
                    n_types: int = 1, max_minutes: int = 300, heli_only_frac: float = 0.0,
                    deadlines: bool = False, deadline_lo: int = 0, horizon: int = 1440,
                    duty_cap: int = 720, n_bases: Optional[int] = None,
                    name: str = "") -> Instance:
    """A test instance with an arbitrary (asymmetric, non-metric) integer matrix.

    The method never assumes symmetry or the triangle inequality, and a matrix
    that has neither shows transposed operands and dropped legs that a Euclidean
    matrix hides. Diagonal entries are 0. Draw order: matrix, bases, vehicle
    types, missions (pickups, then deliveries), heli-only flags, deadlines.
    """
    rng = np.random.default_rng(seed)
    travel = rng.integers(1, max_minutes + 1, size=(n_types, n_loc, n_loc)).astype(np.int32)
    for t in range(n_types):
        np.fill_diagonal(travel[t], 0)
    nb = n_bases if n_bases is not None else max(1, min(n_vehicles, n_loc // 2))
    veh_base = rng.integers(0, nb, size=n_vehicles).astype(np.int32)
    veh_type = rng.integers(0, n_types, size=n_vehicles).astype(np.int32)
    p = rng.integers(0, n_loc, size=n_missions)
    d = (p + 1 + rng.integers(0, n_loc - 1, size=n_missions)) % n_loc
    heli = None
    if heli_only_frac > 0.0:
        heli = (rng.random(n_missions) < heli_only_frac).astype(np.int32)
    dl = None
    if deadlines:
        dl = rng.integers(deadline_lo, horizon + 1, size=n_missions).astype(np.int32)
    return Instance(travel=np.ascontiguousarray(travel), veh_base=veh_base, veh_type=veh_type,
                    pickup=p.astype(np.int32), delivery=d.astype(np.int32), heli_only=heli,
                    deadline=dl, duty_cap=int(duty_cap), horizon=int(horizon),
                    name=name or f"random-s{seed}")


SERVING_PARAMS = Params(tenure=10, iterations=1000, cap_mode=PENALTY, lam=1000)


def serving_request(seed: int) -> Instance:
    """One re-planning request: M = clip(round(lognormal(ln 60, 0.5)), 10, 400) missions,
    V = ceil(M / 5) vehicles, paper-shaped geography (12 bases, 60 clustered facilities
    in a 1500 km box), 12 h cap. Drawn from its own seed."""
    rng = np.random.default_rng(seed)
    m, v = serving_size(rng)
    return make_instance(seed, n_bases=12, n_vehicles=v, n_facilities=60, n_missions=m,
                         box_km=1500.0, geography="clustered", duty_cap=720,
                         name=f"request-{seed}")


def poisson_arrivals(seed: int, rate_per_s: float, duration_s: float) -> np.ndarray:
    """Arrival times (seconds) of a Poisson stream: exponential gaps of mean 1 / rate."""
    rng = np.random.default_rng(seed)
    n = int(rate_per_s * duration_s * 1.2) + 16
    t = np.cumsum(rng.exponential(1.0 / rate_per_s, size=n))
    return t[t < duration_s]
