"""asched_sweep_batch (Algorithm 2 and the per-mission sweep of Algorithm 3) against the
oracle: the per-step trace, the counters and the best schedule of every instance are
identical (integer arithmetic, so bit-exact). Needs a GB300."""
import numpy as np
import pytest
import torch

import oracle
from paper_2002_11710_gb300 import api, gen

pytestmark = pytest.mark.gpu

PENALTY, HARD = gen.PENALTY, gen.HARD
NULL = 0xFFFFFFFF

# (name, algorithm, tenure, accept_worse, max_sweeps)
VARIANTS = [("alg2", api.SWEEP_NEIGHBOURHOOD, 0, False, 50),
            ("alg3", api.SWEEP_TABU, 7, False, 50),
            ("alg3w", api.SWEEP_TABU, 5, True, 20)]


def _oracle(inst, mode, algorithm, tenure, aw, max_sweeps):
    pb = oracle.Problem(inst, mode, 1000)
    if algorithm == api.SWEEP_NEIGHBOURHOOD:
        return oracle.neighbourhood_search(pb, max_sweeps)
    return oracle.tabu_sweep(pb, tenure, max_sweeps, accept_worse=aw)


def _check(bp, out, trace, b, r):
    got = bp.unpack(out, b)
    info = got["info"]
    assert info[api.INFO_STATUS] == r["status"]
    if r["status"] != 0:
        return
    assert info[api.INFO_Z_BEST] == r["z_best"]
    assert info[api.INFO_Z_INIT] == r["z_init"]
    assert info[api.INFO_Z_FINAL] == r["z_final"]
    assert info[api.INFO_BEST_IT] == r["best_step"]
    assert info[api.INFO_ITERS] == r["sweeps"]
    assert info[api.INFO_MOVES] == r["n_moves"]
    assert info[api.INFO_STEPS] == r["steps"]
    np.testing.assert_array_equal(got["route_off"], r["route_off"])
    np.testing.assert_array_equal(got["route"], r["route"])
    if trace is not None:
        cap = trace.capacity
        n = min(r["steps"], cap)
        mv = trace.move[b * cap: b * cap + n].cpu().numpy().view(np.uint32)
        zz = trace.z[b * cap: b * cap + n].cpu().numpy()
        np.testing.assert_array_equal(mv, r["trace_move"][:n])
        np.testing.assert_array_equal(zz, r["trace_z"][:n])


def _flight_pin(bp, out, b, inst, mode):
    got = bp.unpack(out, b)
    pb = oracle.Problem(inst, mode, 1000)
    z, fl, ov = oracle.cost(pb, got["route_off"], got["route"])
    np.testing.assert_array_equal(got["flight"], fl)
    np.testing.assert_array_equal(got["overflow"], ov)
    assert z == got["info"][api.INFO_Z_BEST]


def _paper_instances():
    out = []
    for s, m in [(0, 20), (2, 24), (8, 33), (3, 16), (6, 12), (9, 28)]:
        out.append(gen.paper_model(s, m))
    return out


@pytest.mark.parametrize("variant", VARIANTS, ids=[v[0] for v in VARIANTS])
@pytest.mark.parametrize("mode", [HARD, PENALTY], ids=["hard", "penalty"])
def test_paper_model_batch_matches_oracle(variant, mode):
    name, alg, tenure, aw, ms = variant
    insts = _paper_instances()
    bp = api.BatchProblem(insts)
    out, trace = api.sweep_batch(bp, alg, api.sweep_params(ms, mode, 1000, tenure, aw), trace_capacity=4096)
    torch.cuda.synchronize()
    for b, inst in enumerate(insts):
        r = _oracle(inst, mode, alg, tenure, aw, ms)
        _check(bp, out, trace, b, r)
        if r["status"] == 0:
            _flight_pin(bp, out, b, inst, mode)


def _random_instances(deadlines):
    """Without deadlines: up to 120 missions on 9 vehicles. With deadlines: about three
    missions per vehicle, arrive-by times clipped to leave room for the flight home, so
    that Algorithm 1 finds a start (a long route rarely meets random deadlines)."""
    if deadlines:
        sizes = [(8, 4, 10), (12, 12, 37), (6, 1, 0), (9, 2, 1), (15, 22, 65), (10, 11, 33),
                 (20, 40, 120), (7, 3, 2), (11, 3, 9), (9, 6, 3)]
    else:
        sizes = [(8, 3, 10), (12, 5, 37), (6, 1, 0), (9, 2, 1), (15, 7, 65), (10, 4, 33),
                 (20, 9, 120), (7, 3, 2), (11, 1, 9), (9, 6, 3)]
    out = []
    for s, (L, V, M) in enumerate(sizes):
        mm = 60 if deadlines else 120
        inst = gen.random_instance(700 + s, n_loc=L, n_vehicles=V, n_missions=M, n_types=2,
                                   heli_only_frac=0.2, deadlines=deadlines, deadline_lo=200,
                                   duty_cap=1500, max_minutes=mm)
        if deadlines:
            inst.deadline = np.minimum(inst.deadline, inst.horizon - 2 * mm).astype(np.int32)
        out.append(inst)
    return out


@pytest.mark.parametrize("variant", VARIANTS, ids=[v[0] for v in VARIANTS])
@pytest.mark.parametrize("mode", [HARD, PENALTY], ids=["hard", "penalty"])
@pytest.mark.parametrize("deadlines", [False, True], ids=["nodl", "dl"])
def test_random_batch_matches_oracle(variant, mode, deadlines):
    """Asymmetric, non-metric matrices; sizes from empty (M = 0) and single-vehicle
    instances to 120 missions (several candidates per thread)."""
    name, alg, tenure, aw, ms = variant
    insts = _random_instances(deadlines)
    bp = api.BatchProblem(insts)
    out, trace = api.sweep_batch(bp, alg, api.sweep_params(ms, mode, 1000, tenure, aw), trace_capacity=8192)
    torch.cuda.synchronize()
    for b, inst in enumerate(insts):
        _check(bp, out, trace, b, _oracle(inst, mode, alg, tenure, aw, ms))


def test_more_vehicles_than_threads_matches_oracle():
    """Every thread covers several vehicles in Algorithm 1 and several candidates in the
    sweep (one warp for 70 vehicles and 150 missions)."""
    insts = [gen.random_instance(900 + s, n_loc=25, n_vehicles=70, n_missions=150, n_types=2,
                                 heli_only_frac=0.2, duty_cap=900, max_minutes=100) for s in range(3)]
    bp = api.BatchProblem(insts)
    for alg, tenure, aw in ((api.SWEEP_NEIGHBOURHOOD, 0, False), (api.SWEEP_TABU, 4, True)):
        out, trace = api.sweep_batch(bp, alg, api.sweep_params(6, PENALTY, 1000, tenure, aw, block_threads=32),
                                     trace_capacity=2048)
        torch.cuda.synchronize()
        for b, inst in enumerate(insts):
            _check(bp, out, trace, b, _oracle(inst, PENALTY, alg, tenure, aw, 6))


@pytest.mark.parametrize("threads", [32, 64, 96, 256, 512])
def test_block_size_does_not_change_results(threads):
    insts = _random_instances(True)
    bp = api.BatchProblem(insts)
    p0 = api.sweep_params(20, PENALTY, 1000, 5, True)
    ref, tr0 = api.sweep_batch(bp, api.SWEEP_TABU, p0, trace_capacity=2048)
    p1 = api.sweep_params(20, PENALTY, 1000, 5, True, block_threads=threads)
    got, tr1 = api.sweep_batch(bp, api.SWEEP_TABU, p1, trace_capacity=2048)
    torch.cuda.synchronize()
    assert torch.equal(ref.info, got.info) and torch.equal(ref.route, got.route)
    assert torch.equal(ref.route_off, got.route_off) and torch.equal(tr0.move, tr1.move)


def test_result_independent_of_the_mix():
    insts = _paper_instances() + _random_instances(True)
    insts = [i for i in insts if i.travel.shape[0] == 2]
    p = api.sweep_params(50, PENALTY, 1000, 7)
    bp1 = api.BatchProblem(insts)
    o1, _ = api.sweep_batch(bp1, api.SWEEP_TABU, p)
    perm = list(reversed(range(len(insts))))
    bp2 = api.BatchProblem([insts[i] for i in perm])
    o2, _ = api.sweep_batch(bp2, api.SWEEP_TABU, p)
    torch.cuda.synchronize()
    for j, i in enumerate(perm):
        a, c = bp1.unpack(o1, i), bp2.unpack(o2, j)
        for k in ("route_off", "route", "flight", "info"):
            np.testing.assert_array_equal(a[k], c[k])


def test_large_batch_sample_matches_oracle():
    """4,096 paper-model instances (12-33 missions) in one launch; a sample against the
    oracle, and every instance's objective against the oracle's cost of its schedule."""
    rng = np.random.default_rng(5)
    sizes = rng.integers(12, 34, size=4096)
    insts = [gen.paper_model(10_000 + i, int(m)) for i, m in enumerate(sizes)]
    p = api.sweep_params(100, PENALTY, 1000, 7)
    bp = api.BatchProblem(insts)
    out, trace = api.sweep_batch(bp, api.SWEEP_TABU, p, trace_capacity=512)
    torch.cuda.synchronize()
    info = out.info.view(-1, api.INFO_LEN).cpu().numpy()
    for b in list(range(0, 4096, 97)) + [4095]:
        _check(bp, out, trace, b, _oracle(insts[b], PENALTY, api.SWEEP_TABU, 7, False, 100))
    ok = info[:, api.INFO_STATUS] == 0
    assert ok.mean() > 0.5
    for b in np.nonzero(ok)[0][::53]:
        _flight_pin(bp, out, int(b), insts[int(b)], PENALTY)


def test_device_status_codes():
    good = gen.random_instance(400, n_loc=8, n_vehicles=3, n_missions=12, duty_cap=5000)
    infeasible = gen.random_instance(401, n_loc=8, n_vehicles=2, n_missions=12, duty_cap=10)
    bad = gen.random_instance(402, n_loc=8, n_vehicles=2, n_missions=5, duty_cap=500)
    bad.pickup = bad.pickup.copy()
    bad.pickup[2] = 8  # location out of range
    huge = gen.random_instance(403, n_loc=8, n_vehicles=2, n_missions=5, duty_cap=500, max_minutes=300)
    huge.travel = huge.travel.copy()
    huge.travel[0, 1, 2] = 100_000_000  # the int32 objective guard trips
    bp = api.BatchProblem([good, infeasible, bad, huge])
    out, _ = api.sweep_batch(bp, api.SWEEP_NEIGHBOURHOOD, api.sweep_params(10, HARD, 1000))
    torch.cuda.synchronize()
    st = [int(bp.unpack(out, b)["info"][api.INFO_STATUS]) for b in range(4)]
    assert st == [0, api.E_INFEASIBLE_INIT, api.E_INVALID, api.E_OVERFLOW_GUARD]


def test_host_errors():
    insts = _random_instances(False)[:3]
    bp = api.BatchProblem(insts)
    cases = [(9, api.sweep_params(5)),
             (api.SWEEP_NEIGHBOURHOOD, api.sweep_params(5, accept_worse=True)),
             (api.SWEEP_TABU, api.sweep_params(5, block_threads=48)),
             (api.SWEEP_TABU, api.sweep_params(-1))]
    for alg, p in cases:
        with pytest.raises(api.AschedError) as e:
            api.sweep_batch(bp, alg, p)
        assert e.value.status == api.E_INVALID
    big = gen.random_instance(9, n_loc=30, n_vehicles=1000, n_missions=3000, n_types=1, duty_cap=100)
    with pytest.raises(api.AschedError) as e:
        api.sweep_batch(api.BatchProblem([big]), api.SWEEP_TABU, api.sweep_params(1))
    assert e.value.status == api.E_TOO_LARGE


@pytest.mark.parametrize("mode", [HARD, PENALTY], ids=["hard", "penalty"])
@pytest.mark.parametrize("repair", [False, True], ids=["plain", "repair"])
def test_paper_fleet_batch_with_repair_matches_oracle(mode, repair):
    """512 paper-fleet instances (12-33 missions, arrive-by times inside vehicle windows);
    with repair, Algorithm 1's stuck placements go through one Neighbourhood Search
    sweep first. Every instance against the oracle."""
    rng = np.random.default_rng(11)
    sizes = rng.integers(12, 34, size=512)
    insts = [gen.paper_fleet(s, int(m)) for s, m in enumerate(sizes)]
    bp = api.BatchProblem(insts)
    for alg, tenure in ((api.SWEEP_NEIGHBOURHOOD, 0), (api.SWEEP_TABU, 7)):
        p = api.sweep_params(60, mode, 1000, tenure, repair=repair)
        out, trace = api.sweep_batch(bp, alg, p, trace_capacity=2048)
        torch.cuda.synchronize()
        for b, inst in enumerate(insts):
            pb = oracle.Problem(inst, mode, 1000)
            if alg == api.SWEEP_NEIGHBOURHOOD:
                r = oracle.neighbourhood_search(pb, 60, repair=repair)
            else:
                r = oracle.tabu_sweep(pb, tenure, 60, repair=repair)
            _check(bp, out, trace, b, r)


@pytest.mark.parametrize("mode", [HARD, PENALTY], ids=["hard", "penalty"])
def test_random_loop_orders_match_oracle(mode):
    """The paper's permutation vectors: every instance with its own vehicle order and
    mission ranks (Algorithm 1's repair sweep uses them too)."""
    rng = np.random.default_rng(21)
    sizes = rng.integers(12, 34, size=256)
    insts = [gen.paper_fleet(500 + s, int(m)) for s, m in enumerate(sizes)]
    orders = [gen.sweep_orders(9000 + s, i.n_vehicles, i.n_missions) for s, i in enumerate(insts)]
    bp = api.BatchProblem(insts)
    for alg, tenure, aw in ((api.SWEEP_NEIGHBOURHOOD, 0, False), (api.SWEEP_TABU, 5, False),
                            (api.SWEEP_TABU, 5, True)):
        ms = 20 if aw else 60
        p = api.sweep_params(ms, mode, 1000, tenure, aw, repair=True)
        out, trace = api.sweep_batch(bp, alg, p, trace_capacity=2048, orders=orders)
        torch.cuda.synchronize()
        for b, inst in enumerate(insts):
            pb = oracle.Problem(inst, mode, 1000)
            vo, mr = orders[b]
            if alg == api.SWEEP_NEIGHBOURHOOD:
                r = oracle.neighbourhood_search(pb, ms, repair=True, vorder=vo, mrank=mr)
            else:
                r = oracle.tabu_sweep(pb, tenure, ms, accept_worse=aw, repair=True, vorder=vo, mrank=mr)
            _check(bp, out, trace, b, r)


def test_multi_start_runs_of_one_instance():
    """Ten runs of one instance with ten order pairs in one launch (the paper's 10 runs):
    each equals its own oracle run; best, worst and mean follow."""
    inst = gen.paper_fleet(77, 30)
    runs = [gen.sweep_orders(k, inst.n_vehicles, inst.n_missions) for k in range(10)]
    bp = api.BatchProblem([inst] * 10)
    out, trace = api.sweep_batch(bp, api.SWEEP_TABU, api.sweep_params(100, HARD, 1000, 7, repair=True),
                                 trace_capacity=4096, orders=runs)
    torch.cuda.synchronize()
    zs = []
    for b, (vo, mr) in enumerate(runs):
        r = oracle.tabu_sweep(oracle.Problem(inst, HARD, 1000), 7, 100, repair=True, vorder=vo, mrank=mr)
        _check(bp, out, trace, b, r)
        if r["status"] == 0:
            zs.append(r["z_best"])
    assert zs


def test_orders_that_are_not_permutations_are_rejected():
    insts = [gen.paper_fleet(1, 20), gen.paper_fleet(2, 20)]
    bp = api.BatchProblem(insts)
    good = gen.sweep_orders(0, 12, 20)
    bad_v = (np.zeros(12, np.int32), None)
    out, _ = api.sweep_batch(bp, api.SWEEP_NEIGHBOURHOOD, api.sweep_params(5), orders=[good, bad_v])
    bad_m = (None, np.full(20, 25, np.int32))
    out2, _ = api.sweep_batch(bp, api.SWEEP_NEIGHBOURHOOD, api.sweep_params(5), orders=[bad_m, good])
    torch.cuda.synchronize()
    st = out.info.view(-1, api.INFO_LEN)[:, api.INFO_STATUS].cpu().tolist()
    st2 = out2.info.view(-1, api.INFO_LEN)[:, api.INFO_STATUS].cpu().tolist()
    assert st[1] == api.E_INVALID and st2[0] == api.E_INVALID
    assert st[0] != api.E_INVALID and st2[1] != api.E_INVALID
