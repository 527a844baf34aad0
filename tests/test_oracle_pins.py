"""Pins of the CPU oracle against things other than itself (no GPU needed).

* closed forms: the neighbourhood size, one-mission and empty routes;
* the ILP's arc form of obj_s and con1-con11 (Section 3), written independently in
  tests/ilp.py, on every schedule of tiny instances (brute force);
* an independent characterisation of the neighbourhood (relocation = equal after
  deleting the mission, swap = two exchanged places), compared as a set with the
  oracle's canonical move list, deltas and flags;
* a brute-force re-derivation of each Tabu iteration (readings R5-R7);
* the hand-worked instance under tests/golden/line3.json.

Instances use asymmetric, non-metric matrices so that transposed operands and
dropped legs cannot hide.
"""
import json
import math
import os

import numpy as np
import pytest

import ilp
import oracle
from paper_2002_11710_gb300 import gen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_instance(g):
    gi = g["instance"]
    inst = gen.Instance(travel=np.array(gi["travel"], dtype=np.int32),
                        veh_base=np.array(gi["veh_base"], dtype=np.int32),
                        veh_type=np.array(gi["veh_type"], dtype=np.int32),
                        pickup=np.array(gi["pickup"], dtype=np.int32),
                        delivery=np.array(gi["delivery"], dtype=np.int32),
                        heli_only=None, deadline=None, duty_cap=gi["duty_cap"],
                        horizon=gi["horizon"], name="line3")
    return inst, gi["cap_mode"], gi["lambda"]


@pytest.fixture(scope="module")
def line3():
    with open(os.path.join(GOLDEN, "line3.json")) as f:
        return json.load(f)


def test_num_moves_closed_form():
    for M in range(0, 12):
        for V in range(1, 6):
            assert oracle.num_moves(M, V) == M * (M + V - 2) + M * (M - 1) // 2
    assert oracle.num_moves(10, 3) == 155
    assert oracle.num_moves(100, 20) == 16750
    assert oracle.num_moves(400, 50) == 259000


def test_golden_greedy(line3):
    inst, mode, lam = _golden_instance(line3)
    pb = oracle.Problem(inst, mode, lam)
    rc, off, route = oracle.greedy_init(pb)
    assert rc == 0
    assert off.tolist() == line3["greedy"]["route_off"]
    assert route.tolist() == line3["greedy"]["route"]
    z, fl, ov = oracle.cost(pb, off, route)
    assert z == line3["greedy"]["z"]
    assert fl.tolist() == line3["greedy"]["flight"]


def test_golden_neighbourhood(line3):
    inst, mode, lam = _golden_instance(line3)
    pb = oracle.Problem(inst, mode, lam)
    g = line3["greedy"]
    tabu = -np.ones((3, 2), dtype=np.int32)
    ids, delta, flags, chosen = oracle.eval_neighbourhood(pb, g["route_off"], g["route"], tabu, 0, 140)
    want = {mv["id"]: mv["delta"] for mv in line3["neighbourhood_of_greedy"]["moves"]}
    got = {int(i): int(d) for i, d in zip(ids, delta)}
    assert got == want
    assert list(ids) == sorted(ids)
    assert int(ids[chosen]) == 3


def test_golden_tabu_trajectory(line3):
    inst, mode, lam = _golden_instance(line3)
    pb = oracle.Problem(inst, mode, lam)
    t = line3["tabu_tenure_2"]
    r = oracle.tabu_search(pb, 2, 3)
    assert r["status"] == 0
    assert [int(x) for x in r["traj_move"]] == t["traj_move"]
    assert [int(x) for x in r["traj_z"]] == t["traj_z"]
    assert r["z_best"] == t["z_best"] and r["best_it"] == t["best_it"]


def test_golden_optimum_by_brute_force(line3):
    inst, mode, lam = _golden_instance(line3)
    zs = [ilp.objective(inst, s, mode, lam) for s in ilp.all_schedules(3, 2)
          if ilp.feasible(inst, s, mode)]
    assert min(zs) == line3["optimum"]["z"]


def test_closed_form_single_mission_routes():
    inst = gen.random_instance(11, n_loc=7, n_vehicles=3, n_missions=1, n_types=2)
    for mode in (ilp.HARD, ilp.PENALTY):
        pb = oracle.Problem(inst, mode, 7)
        for v in range(3):
            routes = tuple((0,) if k == v else () for k in range(3))
            off, route = ilp.routes_to_csr(routes)
            z, fl, _ = oracle.cost(pb, off, route)
            T = inst.travel[inst.veh_type[v]]
            b, p, d = inst.veh_base[v], inst.pickup[0], inst.delivery[0]
            f = int(T[b, p] + T[p, d] + T[d, b])
            assert fl.tolist() == [f if k == v else 0 for k in range(3)]
            want = f + (7 * max(0, f - inst.duty_cap) if mode == ilp.PENALTY else 0)
            assert z == want


TINY_CASES = [
    # seed, L, V, M, types, heli, deadlines, cap
    (1, 6, 3, 5, 1, 0.0, False, 400),
    (2, 5, 2, 6, 2, 0.4, False, 500),
    (3, 7, 3, 5, 2, 0.3, True, 700),
    (4, 6, 2, 5, 1, 0.0, True, 900),
]


def _tiny(case):
    seed, L, V, M, nt, heli, dl, cap = case
    return gen.random_instance(seed, n_loc=L, n_vehicles=V, n_missions=M, n_types=nt,
                               heli_only_frac=heli, deadlines=dl, deadline_lo=200,
                               duty_cap=cap, max_minutes=200)


@pytest.mark.parametrize("case", TINY_CASES)
@pytest.mark.parametrize("mode", [ilp.HARD, ilp.PENALTY])
def test_cost_and_feasibility_on_every_schedule(case, mode):
    inst = _tiny(case)
    pb = oracle.Problem(inst, mode, 1000)
    M, V = inst.n_missions, inst.n_vehicles
    n = 0
    for s in ilp.all_schedules(M, V):
        off, route = ilp.routes_to_csr(s)
        z, fl, ov = oracle.cost(pb, off, route)
        assert z == ilp.objective(inst, s, mode, 1000)
        assert fl.tolist() == ilp.flights(inst, s)
        assert oracle.feasible(pb, off, route) == ilp.feasible(inst, s, mode)
        n += 1
    assert n == math.factorial(M) * math.comb(M + V - 1, V - 1)


def _universe(inst):
    return list(ilp.all_schedules(inst.n_missions, inst.n_vehicles))


@pytest.mark.parametrize("case", TINY_CASES[:3])
def test_neighbourhood_matches_characterisation(case):
    inst = _tiny(case)
    uni = _universe(inst)
    rng = np.random.default_rng(case[0])
    for mode in (ilp.HARD, ilp.PENALTY):
        pb = oracle.Problem(inst, mode, 1000)
        for trial in range(4):
            s = uni[int(rng.integers(len(uni)))]
            off, route = ilp.routes_to_csr(s)
            M, V = inst.n_missions, inst.n_vehicles
            tabu = rng.integers(-1, 3, size=(M, V)).astype(np.int32)
            it = 1
            z0 = ilp.objective(inst, s, mode, 1000)
            z_best = z0 - int(rng.integers(0, 50))
            ids, delta, flags, chosen = oracle.eval_neighbourhood(pb, off, route, tabu, it, z_best)
            assert len(ids) == oracle.num_moves(M, V)
            want = {}
            for mid, s2, moved in ilp.neighbours(s, uni):
                z1 = ilp.objective(inst, s2, mode, 1000)
                fe = ilp.feasible(inst, s2, mode)
                tb = any(tabu[x, to] >= it for (x, _, to) in moved)
                asp = z1 < z_best
                fl = (1 if fe else 0) | (2 if tb else 0) | (4 if asp else 0)
                fl |= 8 if fe and (not tb or asp) else 0
                want[mid] = (z1 - z0, fl)
            got = {int(i): (int(d), int(f)) for i, d, f in zip(ids, delta, flags)}
            assert got == want
            adm = [(d, i) for i, (d, f) in want.items() if f & 8]
            if adm:
                assert int(ids[chosen]) == min(adm)[1]
            else:
                assert chosen == -1


@pytest.mark.parametrize("case", TINY_CASES)
def test_tabu_trajectory_rederived_by_brute_force(case):
    inst = _tiny(case)
    uni = _universe(inst)
    tenure, iters = 3, 12
    for mode in (ilp.HARD, ilp.PENALTY):
        pb = oracle.Problem(inst, mode, 1000)
        rc, off, route = oracle.greedy_init(pb)
        if rc != 0:
            continue
        r = oracle.tabu_search(pb, tenure, iters)
        assert r["status"] == 0
        s = ilp.csr_to_routes(off, route, inst.n_vehicles)
        z = ilp.objective(inst, s, mode, 1000)
        z_best, best_it = z, -1
        tabu = {}
        for it in range(iters):
            mid, s2, moved = ilp.tabu_step(inst, s, uni, tabu, it, z_best, mode, 1000)
            got = int(r["traj_move"][it])
            assert got == (0xFFFFFFFF if mid is None else mid), (mode, it)
            for (x, frm, _) in moved:
                tabu[(x, frm)] = it + tenure
            s = s2
            z = ilp.objective(inst, s, mode, 1000)
            assert int(r["traj_z"][it]) == z
            if z < z_best:
                z_best, best_it = z, it
        assert r["z_best"] == z_best and r["best_it"] == best_it


@pytest.mark.parametrize("case", TINY_CASES)
def test_greedy_rederived(case):
    """Algorithm 1 (reading R8): each mission in (heli-only, deadline, id) order goes to
    the feasible vehicle with the least objective increase, lowest index on ties."""
    inst = _tiny(case)
    M, V = inst.n_missions, inst.n_vehicles
    for mode in (ilp.HARD, ilp.PENALTY):
        pb = oracle.Problem(inst, mode, 1000)
        rc, off, route = oracle.greedy_init(pb)
        heli = inst.heli_only if inst.heli_only is not None else np.zeros(M, int)
        dl = inst.deadline if inst.deadline is not None else np.zeros(M, int)
        order = sorted(range(M), key=lambda m: (0 if heli[m] else 1, int(dl[m]), m))
        routes = [[] for _ in range(V)]
        status = 0
        for m in order:
            z0 = ilp.objective(inst, tuple(map(tuple, routes)), mode, 1000)
            best = None
            for v in range(V):
                trial = [list(r) for r in routes]
                trial[v].append(m)
                # feasibility of the partial schedule: check the placed missions only
                placed = [x for r in trial for x in r]
                sub = inst.subinstance(sorted(placed))
                remap = {x: i for i, x in enumerate(sorted(placed))}
                st = tuple(tuple(remap[x] for x in r) for r in trial)
                if not ilp.feasible(sub, st, mode):
                    continue
                dz = ilp.objective(inst, tuple(map(tuple, trial)), mode, 1000) - z0
                if best is None or dz < best[0]:
                    best = (dz, v)
            if best is None:
                status = -4
                break
            routes[best[1]].append(m)
        assert rc == status
        if rc == 0:
            assert ilp.csr_to_routes(off, route, V) == tuple(map(tuple, routes))


@pytest.mark.parametrize("seed", range(8))
def test_tabu_reaches_brute_force_optimum_or_reports_gap(seed):
    """Brute force over all schedules (M=5, V=2) gives the optimum; the oracle's Tabu
    best is never below it, and on these tiny instances it reaches it."""
    inst = gen.random_instance(100 + seed, n_loc=6, n_vehicles=2, n_missions=5,
                               max_minutes=120, duty_cap=2000)
    pb = oracle.Problem(inst, ilp.HARD, 1000)
    opt = min(ilp.objective(inst, s, ilp.HARD, 1000) for s in ilp.all_schedules(5, 2)
              if ilp.feasible(inst, s, ilp.HARD))
    r = oracle.tabu_search(pb, 3, 60)
    assert r["status"] == 0
    assert r["z_best"] >= opt
    assert r["z_best"] == opt, f"gap {r['z_best'] - opt}"
    best = ilp.csr_to_routes(r["route_off"], r["route"], 2)
    assert ilp.objective(inst, best, ilp.HARD, 1000) == r["z_best"]
    assert ilp.feasible(inst, best, ilp.HARD)


def test_oracle_outputs_satisfy_ilp_constraints():
    for inst, mode in [(gen.tiny(0), ilp.PENALTY), (gen.paper_model(3, 14), ilp.HARD),
                       (gen.paper_model(5, 20), ilp.PENALTY)]:
        pb = oracle.Problem(inst, mode, 1000)
        rc, off, route = oracle.greedy_init(pb)
        if rc != 0:
            continue
        r = oracle.tabu_search(pb, 5, 40)
        assert r["status"] == 0
        s = ilp.csr_to_routes(r["route_off"], r["route"], inst.n_vehicles)
        assert ilp.feasible(inst, s, mode)
        assert ilp.objective(inst, s, mode, 1000) == r["z_best"]
        z0 = oracle.cost(pb, off, route)[0]
        assert r["z_best"] == min([z0] + [int(z) for z in r["traj_z"]])


def test_infeasible_init_reported():
    inst = gen.random_instance(7, n_loc=5, n_vehicles=2, n_missions=6, duty_cap=10)
    pb = oracle.Problem(inst, ilp.HARD, 1000)
    rc, _, _ = oracle.greedy_init(pb)
    assert rc == oracle.E_INFEASIBLE_INIT


def test_thread_count_does_not_change_results():
    """The loop over moves runs on OpenMP threads; the chosen move is picked afterwards in
    canonical order, so per-move deltas, flags and whole trajectories are the same on one
    thread and on every core."""
    import oracle

    inst = gen.random_instance(49, n_loc=12, n_vehicles=6, n_missions=23, n_types=2, heli_only_frac=0.25,
                               deadlines=True, deadline_lo=1000, duty_cap=2500, max_minutes=60)
    pb = oracle.Problem(inst, gen.PENALTY, 1000)
    runs = []
    before = oracle.set_threads(0)
    try:
        for threads in (1, 3, 0):
            oracle.set_threads(threads if threads else before)
            r = oracle.tabu_search(pb, 4, 40)
            rc, off, route = oracle.greedy_init(pb)
            tabu = np.random.default_rng(1).integers(-1, 5, size=(pb.M, pb.V)).astype(np.int32)
            ev = oracle.eval_neighbourhood(pb, off, route, tabu, 2, oracle.cost(pb, off, route)[0] - 5)
            runs.append((r, ev))
    finally:
        oracle.set_threads(before)
    (r0, e0) = runs[0]
    assert r0["status"] == 0
    for r, e in runs[1:]:
        np.testing.assert_array_equal(r["traj_move"], r0["traj_move"])
        np.testing.assert_array_equal(r["traj_z"], r0["traj_z"])
        for a, b in zip(e[:3], e0[:3]):
            np.testing.assert_array_equal(a, b)
        assert e[3] == e0[3]
