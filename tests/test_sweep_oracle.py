"""Pins of the oracle's Algorithm 2 / Algorithm 3 sweeps (readings S1-S5) against things
other than the oracle itself (no GPU needed).

* the hand-worked instance tests/golden/line_sweep.json;
* every trace replayed on plain Python routes, its objectives recomputed with the
  ILP's arc form (tests/ilp.py) and every schedule on the way checked against
  con1-con11;
* every step re-derived by brute force: the mission tried, its candidates built as
  explicit schedules, the break rule, the least (delta, k, q), the tabu pairs;
* closed properties: Neighbourhood Search ends in a local optimum of its own
  candidate set and descends strictly; tenure 0 reduces Algorithm 3 to Algorithm 2;
  a single vehicle has no candidate.
"""
import json
import os

import numpy as np
import pytest

import ilp
import oracle
from paper_2002_11710_gb300 import gen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
NULL = 0xFFFFFFFF


def _line_sweep():
    with open(os.path.join(GOLDEN, "line_sweep.json")) as f:
        g = json.load(f)
    gi = g["instance"]
    x = gi["coordinates_minutes"]
    n = len(x)
    T = np.array([[abs(x[str(i)] - x[str(j)]) for j in range(n)] for i in range(n)], dtype=np.int32)
    inst = gen.Instance(travel=T[None], veh_base=np.array(gi["veh_base"], dtype=np.int32),
                        veh_type=np.array(gi["veh_type"], dtype=np.int32),
                        pickup=np.array(gi["pickup"], dtype=np.int32),
                        delivery=np.array(gi["delivery"], dtype=np.int32), heli_only=None,
                        deadline=None, duty_cap=gi["duty_cap"], horizon=gi["horizon"],
                        name="line_sweep")
    return g, inst


def test_golden_line_sweep():
    g, inst = _line_sweep()
    pb = oracle.Problem(inst, g["instance"]["cap_mode"], g["instance"]["lambda"])
    rc, off, route = oracle.greedy_init(pb)
    assert rc == 0
    assert off.tolist() == g["greedy"]["route_off"] and route.tolist() == g["greedy"]["route"]
    ns = oracle.neighbourhood_search(pb, 50)
    e = g["neighbourhood_search"]
    assert ns["status"] == 0 and ns["z_init"] == g["greedy"]["z"]
    assert ns["trace_move"].tolist() == e["trace_move"]
    assert ns["trace_z"].tolist() == e["trace_z"]
    assert ns["route_off"].tolist() == e["route_off"] and ns["route"].tolist() == e["route"]
    assert (ns["z_best"], ns["best_step"], ns["sweeps"], ns["n_moves"], ns["steps"]) == \
        (e["z_best"], e["best_step"], e["sweeps"], e["moves"], e["steps"])
    ts = oracle.tabu_sweep(pb, 2, 50)
    assert ts["trace_move"].tolist() == g["tabu_sweep_tenure_2"]["trace_move"]
    assert ts["z_best"] == g["tabu_sweep_tenure_2"]["z_best"]


# (seed, n_loc, V, M, n_types, heli-only fraction, deadlines, duty cap)
# Seeds chosen so that Algorithm 1 finds a feasible start in both cap modes (a case
# without one would test nothing but the error).
CASES = [
    (17, 6, 2, 4, 1, 0.0, False, 400),
    (12, 7, 3, 5, 2, 0.4, False, 500),
    (13, 8, 3, 6, 2, 0.3, True, 900),
    (20, 9, 4, 7, 2, 0.3, False, 350),
    (15, 10, 4, 9, 2, 0.25, True, 1200),
    (16, 12, 5, 11, 2, 0.2, False, 600),
]


def _inst(case):
    seed, L, V, M, nt, heli, dl, cap = case
    return gen.random_instance(seed, n_loc=L, n_vehicles=V, n_missions=M, n_types=nt,
                               heli_only_frac=heli, deadlines=dl, deadline_lo=300,
                               duty_cap=cap, max_minutes=200)


def _variants():
    # (name, runner, is_tabu, tenure, accept_worse)
    return [("ns", lambda pb: oracle.neighbourhood_search(pb, 40), False, 0, False),
            ("ts3", lambda pb: oracle.tabu_sweep(pb, 3, 40), True, 3, False),
            ("ts3w", lambda pb: oracle.tabu_sweep(pb, 3, 12, accept_worse=True), True, 3, True),
            ("ts9w", lambda pb: oracle.tabu_sweep(pb, 9, 12, accept_worse=True), True, 9, True)]


def _routes_of(pb, off, route):
    return [list(r) for r in ilp.csr_to_routes(off, route, pb.V)]


def _where(routes, m):
    for v, r in enumerate(routes):
        if m in r:
            return v, r.index(m)
    raise AssertionError(m)


def _compatible(inst, m, k):
    return inst.heli_only is None or not int(inst.heli_only[m]) or int(inst.veh_type[k]) == 0


def _partial_ok(inst, routes, mode):
    """con1-con11 on the missions placed so far (the sub-instance of those missions)."""
    placed = sorted(m for r in routes for m in r)
    remap = {m: i for i, m in enumerate(placed)}
    return ilp.feasible(inst.subinstance(placed), tuple(tuple(remap[m] for m in r) for r in routes), mode)


def _pass(inst, mode, lam, routes, st, is_tabu, tenure, accept_worse, vorder=None, mrank=None):
    """One sweep (S1, S2, S3 / S4 / S4b) on explicit, possibly partial, schedules;
    st holds z, z_best, best, tabu and the trace. Returns whether a move was applied."""
    M, V = inst.n_missions, inst.n_vehicles
    applied = False
    for i in (range(V) if vorder is None else [int(x) for x in vorder]):
        turn = list(routes[i])
        if mrank is not None:
            turn.sort(key=lambda m: int(mrank[m]))
        for j in turn:
            rec = NULL
            if j in routes[i]:
                kj = routes[i].index(j)
                cands = []
                for k in range(V):
                    if k == i or not _compatible(inst, j, k):
                        continue
                    if is_tabu and st["tabu"].get((j, k), -1) >= len(st["trace"]):
                        continue
                    for q in range(len(routes[k]) + 1):
                        t = [list(r) for r in routes]
                        del t[i][kj]
                        t[k].insert(q, j)
                        if not _partial_ok(inst, t, mode):
                            break
                        cands.append((ilp.objective(inst, tuple(map(tuple, t)), mode, lam) - st["z"], k, q))
                if cands:
                    d, k, q = min(cands)
                    if d < 0 or accept_worse:
                        y = routes[k][q] if q < len(routes[k]) else M + k
                        del routes[i][kj]
                        routes[k].insert(q, j)
                        st["z"] += d
                        if is_tabu:
                            st["tabu"][(j, i)] = len(st["trace"]) + tenure
                        rec = (j << 13) | y
                        applied = True
                        if st["z"] < st["z_best"]:
                            st["z_best"], st["best"] = st["z"], [list(r) for r in routes]
            st["trace"].append((rec, st["z"]))
    return applied


def _state(inst, routes, mode, lam):
    z = ilp.objective(inst, tuple(map(tuple, routes)), mode, lam)
    return {"z": z, "z_best": z, "best": [list(r) for r in routes], "tabu": {}, "trace": []}


def _rederive(inst, mode, lam, routes, is_tabu, tenure, accept_worse, max_sweeps, vorder=None, mrank=None):
    """Algorithm 2/3 re-derived step by step on explicit schedules (readings S1-S5)."""
    st = _state(inst, routes, mode, lam)
    sweeps = 0
    go_on = True
    while go_on and sweeps < max_sweeps:
        zb0 = st["z_best"]
        applied = _pass(inst, mode, lam, routes, st, is_tabu, tenure, accept_worse, vorder, mrank)
        sweeps += 1
        go_on = (st["z_best"] < zb0) if accept_worse else applied
    return st["trace"], st["z_best"], st["best"], sweeps


def _greedy(inst, mode, lam, repair):
    """Algorithm 1 (R8, and the repair of R12) re-derived on explicit partial schedules."""
    M, V = inst.n_missions, inst.n_vehicles
    heli = inst.heli_only
    dl = inst.deadline
    order = sorted(range(M), key=lambda m: (0 if heli is not None and heli[m] else 1,
                                            int(dl[m]) if dl is not None else 0, m))
    routes = [[] for _ in range(V)]

    def pick(m):
        z0 = ilp.objective(inst, tuple(map(tuple, routes)), mode, lam)
        best = None
        for v in range(V):
            t = [list(r) for r in routes]
            t[v].append(m)
            if not _partial_ok(inst, t, mode):
                continue
            sc = ilp.objective(inst, tuple(map(tuple, t)), mode, lam) - z0
            if best is None or sc < best[0]:
                best = (sc, v)
        return best

    for n, m in enumerate(order):
        b = pick(m)
        if b is None and repair and n > 0:
            if _pass(inst, mode, lam, routes, _state(inst, routes, mode, lam), False, 0, False):
                b = pick(m)
        if b is None:
            return None
        routes[b[1]].append(m)
    return routes


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("mode", [ilp.HARD, ilp.PENALTY])
def test_sweeps_rederived_by_brute_force(case, mode):
    inst = _inst(case)
    pb = oracle.Problem(inst, mode, 1000)
    rc, off, route = oracle.greedy_init(pb)
    assert rc == 0, "every case has a feasible greedy start"
    for name, run, is_tabu, tenure, aw in _variants():
        r = run(pb)
        assert r["status"] == 0, name
        max_sweeps = 40 if not aw else 12
        trace, zb, best, sweeps = _rederive(inst, mode, 1000, _routes_of(pb, off, route), is_tabu,
                                            tenure, aw, max_sweeps)
        assert r["trace_move"].tolist() == [t[0] for t in trace], name
        assert r["trace_z"].tolist() == [t[1] for t in trace], name
        assert r["z_best"] == zb and r["sweeps"] == sweeps, name
        assert _routes_of(pb, r["route_off"], r["route"]) == best, name


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("mode", [ilp.HARD, ilp.PENALTY])
def test_trace_replays_on_feasible_schedules(case, mode):
    """Each applied move relocates one mission to another, compatible vehicle; each
    schedule on the way satisfies con1-con11 and has the traced objective."""
    inst = _inst(case)
    pb = oracle.Problem(inst, mode, 1000)
    rc, off, route = oracle.greedy_init(pb)
    assert rc == 0, "every case has a feasible greedy start"
    M = inst.n_missions
    for name, run, is_tabu, tenure, aw in _variants():
        r = run(pb)
        routes = _routes_of(pb, off, route)
        z = ilp.objective(inst, tuple(map(tuple, routes)), mode, 1000)
        assert r["z_init"] == z
        zs = [z]
        left = {}
        for s, (mv, zt) in enumerate(zip(r["trace_move"].tolist(), r["trace_z"].tolist())):
            if mv != NULL:
                j, y = mv >> 13, mv & 0x1FFF
                vi, ki = _where(routes, j)
                del routes[vi][ki]
                if y < M:
                    k, q = _where(routes, y)
                else:
                    k, q = y - M, len(routes[y - M])
                assert k != vi and _compatible(inst, j, k)
                if is_tabu:
                    assert left.get((j, k), -1) < s, "move onto a tabu base"
                    left[(j, vi)] = s + tenure
                routes[k].insert(q, j)
                tt = tuple(map(tuple, routes))
                assert ilp.feasible(inst, tt, mode)
                znew = ilp.objective(inst, tt, mode, 1000)
                if not aw:
                    assert znew < zs[-1], "Algorithm 2 / 3 apply improving moves only"
                zs.append(znew)
            assert zt == zs[-1]
        assert r["z_final"] == zs[-1]
        assert r["z_best"] == min(zs)
        assert ilp.objective(inst, ilp.csr_to_routes(r["route_off"], r["route"], pb.V), mode,
                             1000) == r["z_best"]


@pytest.mark.parametrize("case", CASES)
def test_neighbourhood_search_ends_in_a_local_optimum(case):
    inst = _inst(case)
    pb = oracle.Problem(inst, ilp.PENALTY, 1000)
    r = oracle.neighbourhood_search(pb, 1000)
    assert r["status"] == 0 and r["sweeps"] < 1000
    routes = _routes_of(pb, r["route_off"], r["route"])
    z = ilp.objective(inst, tuple(map(tuple, routes)), ilp.PENALTY, 1000)
    for i, ri in enumerate(routes):
        for kj, j in enumerate(ri):
            for k in range(inst.n_vehicles):
                if k == i or not _compatible(inst, j, k):
                    continue
                for q in range(len(routes[k]) + 1):
                    t = [list(x) for x in routes]
                    del t[i][kj]
                    t[k].insert(q, j)
                    tt = tuple(map(tuple, t))
                    if not ilp.feasible(inst, tt, ilp.PENALTY):
                        break
                    assert ilp.objective(inst, tt, ilp.PENALTY, 1000) >= z


def test_tenure_zero_is_neighbourhood_search():
    for seed, m in [(0, 20), (2, 24), (8, 33)]:
        pb = oracle.Problem(gen.paper_model(seed, m), ilp.PENALTY, 1000)
        a = oracle.neighbourhood_search(pb, 100)
        b = oracle.tabu_sweep(pb, 0, 100)
        assert a["trace_move"].tolist() == b["trace_move"].tolist()
        assert a["z_best"] == b["z_best"]


def test_single_vehicle_has_no_candidate():
    inst = gen.random_instance(21, n_loc=8, n_vehicles=1, n_missions=6, n_types=1, duty_cap=10000)
    pb = oracle.Problem(inst, ilp.PENALTY, 1000)
    for r in (oracle.neighbourhood_search(pb, 10), oracle.tabu_sweep(pb, 3, 10, accept_worse=True)):
        assert r["n_moves"] == 0 and r["steps"] == 6
        assert (r["trace_move"] == NULL).all()
        assert r["z_best"] == r["z_init"] == r["z_final"]


def test_sweep_reports_infeasible_start():
    bad = gen.random_instance(401, n_loc=8, n_vehicles=2, n_missions=12, duty_cap=10)
    pb = oracle.Problem(bad, ilp.HARD, 1000)
    assert oracle.neighbourhood_search(pb, 5)["status"] == oracle.E_INFEASIBLE_INIT
    assert oracle.tabu_sweep(pb, 3, 5)["status"] == oracle.E_INFEASIBLE_INIT


REPAIR_CASES = [(235, 18, ilp.HARD), (23, 22, ilp.HARD), (162, 22, ilp.HARD), (3, 26, ilp.HARD),
                (13, 30, ilp.HARD), (75, 30, ilp.PENALTY), (110, 30, ilp.PENALTY)]


@pytest.mark.parametrize("case", REPAIR_CASES)
def test_greedy_repair_rederived(case):
    """Paper-fleet instances where Algorithm 1 gets stuck and the repair sweep (R12)
    frees a place: the oracle's start equals the re-derived one."""
    seed, m, mode = case
    inst = gen.paper_fleet(seed, m)
    pb = oracle.Problem(inst, mode, 1000)
    assert oracle.greedy_init(pb)[0] == oracle.E_INFEASIBLE_INIT
    assert _greedy(inst, mode, 1000, repair=False) is None
    rc, off, route = oracle.greedy_init(pb, repair=True)
    assert rc == 0
    want = _greedy(inst, mode, 1000, repair=True)
    assert _routes_of(pb, off, route) == want
    assert ilp.feasible(inst, tuple(map(tuple, want)), mode)


@pytest.mark.parametrize("mode", [ilp.HARD, ilp.PENALTY])
def test_repair_changes_nothing_when_algorithm_1_succeeds(mode):
    for seed in range(40):
        inst = gen.paper_fleet(seed, 12 + seed % 20)
        pb = oracle.Problem(inst, mode, 1000)
        a = oracle.greedy_init(pb)
        b = oracle.greedy_init(pb, repair=True)
        if a[0] == 0:
            assert b[0] == 0 and a[1].tolist() == b[1].tolist() and a[2].tolist() == b[2].tolist()
        else:
            assert a[0] == oracle.E_INFEASIBLE_INIT


@pytest.mark.parametrize("seed", [0, 3, 7])
def test_plain_greedy_rederived_on_paper_fleet(seed):
    inst = gen.paper_fleet(seed, 16)
    for mode in (ilp.HARD, ilp.PENALTY):
        pb = oracle.Problem(inst, mode, 1000)
        rc, off, route = oracle.greedy_init(pb)
        want = _greedy(inst, mode, 1000, repair=False)
        assert (rc == 0) == (want is not None)
        if want is not None:
            assert _routes_of(pb, off, route) == want


def test_paper_fleet_deadlines_sit_in_a_vehicle_window():
    """gen.paper_fleet: every mission can be flown alone by a vehicle allowed to fly it."""
    for seed in range(10):
        inst = gen.paper_fleet(seed, 33)
        for j in range(inst.n_missions):
            ok = False
            for v in range(inst.n_vehicles):
                if not _compatible(inst, j, v):
                    continue
                T = inst.travel[inst.veh_type[v]]
                b, p, d = inst.veh_base[v], inst.pickup[j], inst.delivery[j]
                w = int(inst.deadline[j])
                ok |= T[b, p] + T[p, d] <= w and w + T[d, b] <= inst.horizon and w >= 240
            assert ok


@pytest.mark.parametrize("case", CASES[1:5])
@pytest.mark.parametrize("mode", [ilp.HARD, ilp.PENALTY])
def test_sweeps_with_random_orders_rederived(case, mode):
    """The paper's permutation vectors (S1): vehicle turns in a given order, each turn's
    missions by a given rank; re-derived step by step."""
    inst = _inst(case)
    pb = oracle.Problem(inst, mode, 1000)
    rc, off, route = oracle.greedy_init(pb)
    assert rc == 0, "every case has a feasible greedy start"
    for seed in range(3):
        vo, mr = gen.sweep_orders(seed, inst.n_vehicles, inst.n_missions)
        for is_tabu, tenure, aw in ((False, 0, False), (True, 3, False), (True, 3, True)):
            if is_tabu:
                r = oracle.tabu_sweep(pb, tenure, 12, accept_worse=aw, vorder=vo, mrank=mr)
            else:
                r = oracle.neighbourhood_search(pb, 12, vorder=vo, mrank=mr)
            trace, zb, best, sweeps = _rederive(inst, mode, 1000, _routes_of(pb, off, route), is_tabu,
                                                tenure, aw, 12, vo, mr)
            assert r["trace_move"].tolist() == [t[0] for t in trace]
            assert r["trace_z"].tolist() == [t[1] for t in trace]
            assert r["z_best"] == zb and r["sweeps"] == sweeps
            assert _routes_of(pb, r["route_off"], r["route"]) == best


def test_identity_orders_equal_the_default_and_bad_orders_are_rejected():
    inst = gen.paper_fleet(5, 24)
    pb = oracle.Problem(inst, ilp.HARD, 1000)
    a = oracle.tabu_sweep(pb, 7, 20, repair=True)
    b = oracle.tabu_sweep(pb, 7, 20, repair=True, vorder=np.arange(inst.n_vehicles),
                          mrank=np.arange(inst.n_missions))
    assert a["trace_move"].tolist() == b["trace_move"].tolist() and a["z_best"] == b["z_best"]
    bad = np.arange(inst.n_vehicles)
    bad[0] = 1
    assert oracle.neighbourhood_search(pb, 5, vorder=bad)["status"] == oracle.E_INVALID
    assert oracle.neighbourhood_search(pb, 5, mrank=np.full(inst.n_missions, 3))["status"] == oracle.E_INVALID


def test_random_orders_give_different_runs():
    """Different permutation vectors are different runs of the same method (the paper
    reports the best, worst and mean of 10 runs): on paper-fleet instances the runs do
    not all end at the same objective, and each run's result is feasible."""
    differ = 0
    for seed in range(6):
        inst = gen.paper_fleet(100 + seed, 26)
        pb = oracle.Problem(inst, ilp.HARD, 1000)
        zs = set()
        for run in range(10):
            vo, mr = gen.sweep_orders(1000 * seed + run, inst.n_vehicles, inst.n_missions)
            r = oracle.neighbourhood_search(pb, 100, repair=True, vorder=vo, mrank=mr)
            if r["status"] != 0:
                continue
            assert ilp.feasible(inst, ilp.csr_to_routes(r["route_off"], r["route"], pb.V), ilp.HARD)
            zs.add(r["z_best"])
        differ += len(zs) > 1
    assert differ >= 3
