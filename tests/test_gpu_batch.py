"""asched_solve_batch: every instance of a batch gets exactly the result it gets alone
(and that the oracle gets), whatever else is in the batch (needs a GB300)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2002_11710_gb300 import api, gen

pytestmark = pytest.mark.gpu

PENALTY, HARD = gen.PENALTY, gen.HARD


def _single(inst, params):
    dp = api.DeviceProblem(inst)
    out = api.solve(dp, params)
    torch.cuda.synchronize()
    return {"route_off": out.route_off.cpu().numpy()[: dp.V + 1],
            "route": out.route.cpu().numpy()[: dp.M],
            "flight": out.flight.cpu().numpy()[: dp.V],
            "overflow": out.overflow.cpu().numpy()[: dp.V],
            "info": out.info.cpu().numpy()}


def _same(a, b):
    assert a["info"][api.INFO_STATUS] == b["info"][api.INFO_STATUS]
    if a["info"][api.INFO_STATUS] != 0:
        return
    for k in (api.INFO_Z_BEST, api.INFO_BEST_IT, api.INFO_Z_INIT, api.INFO_Z_FINAL, api.INFO_ITERS):
        assert a["info"][k] == b["info"][k], k
    for k in ("route_off", "route", "flight", "overflow"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


def _mixed_instances():
    out = []
    for s, (L, V, M) in enumerate([(8, 3, 10), (12, 5, 37), (6, 1, 0), (9, 2, 1), (15, 7, 65),
                                   (10, 4, 33), (20, 9, 120), (7, 3, 2)]):
        out.append(gen.random_instance(300 + s, n_loc=L, n_vehicles=V, n_missions=M, n_types=2,
                                       heli_only_frac=0.2, duty_cap=1500, max_minutes=120))
    return out


@pytest.mark.parametrize("compact", [False, True], ids=["tables", "compact"])
def test_batch_members_equal_single_solves_and_oracle(compact):
    insts = _mixed_instances()
    params = api.make_params(5, 60, PENALTY, 1000, compact=compact)
    bp = api.BatchProblem(insts)
    out = api.solve_batch(bp, params)
    torch.cuda.synchronize()
    for b, inst in enumerate(insts):
        got = bp.unpack(out, b)
        _same(got, _single(inst, params))
        if inst.n_missions <= 40:
            r = oracle.tabu_search(oracle.Problem(inst, PENALTY, 1000), 5, 60)
            assert got["info"][api.INFO_Z_BEST] == r["z_best"]
            np.testing.assert_array_equal(got["route"], r["route"])
            np.testing.assert_array_equal(got["route_off"], r["route_off"])


def _route_flight(inst, v, r):
    T = inst.travel[inst.veh_type[v]]
    e, f = inst.veh_base[v], 0
    for m in r:
        f += T[e][inst.pickup[m]] + T[inst.pickup[m]][inst.delivery[m]]
        e = inst.delivery[m]
    return f + T[e][inst.veh_base[v]] if r else 0


@pytest.mark.parametrize("compact", [False, True], ids=["tables", "compact"])
def test_batch_hard_cap_where_a_removal_lengthens_its_route(compact):
    """HARD mode with caps just above the greedy schedule's longest route, on non-metric
    matrices where taking a mission out of its route can lengthen that route past the cap:
    such relocations are infeasible, which the batch kernel reads from its per-mission
    source-route records. Every member equals its single solve and the oracle."""
    insts = []
    for seed, cap in ((500, 1790), (501, 2929), (503, 1444), (507, 1452), (510, 1958), (515, 1999)):
        base = gen.random_instance(seed, n_loc=10, n_vehicles=3, n_missions=14, max_minutes=300,
                                   duty_cap=100000)
        inst = gen.Instance(**{**base.__dict__, "duty_cap": cap})
        pb = oracle.Problem(inst, HARD, 1000)
        status, off, route = oracle.greedy_init(pb)
        assert status == 0
        over = [m for v in range(inst.n_vehicles) for m in route[off[v]:off[v + 1]]
                if _route_flight(inst, v, [x for x in route[off[v]:off[v + 1]] if x != m]) > cap]
        assert over, seed  # the case this test is about occurs in the start schedule
        insts.append(inst)
    params = api.make_params(3, 60, HARD, 1000, compact=compact)
    bp = api.BatchProblem(insts)
    out = api.solve_batch(bp, params)
    torch.cuda.synchronize()
    for b, inst in enumerate(insts):
        got = bp.unpack(out, b)
        _same(got, _single(inst, params))
        r = oracle.tabu_search(oracle.Problem(inst, HARD, 1000), 3, 60)
        assert got["info"][api.INFO_STATUS] == 0
        assert got["info"][api.INFO_Z_BEST] == r["z_best"]
        np.testing.assert_array_equal(got["route"], r["route"])
        np.testing.assert_array_equal(got["route_off"], r["route_off"])


@pytest.mark.parametrize("compact", [False, True], ids=["tables", "compact"])
def test_batch_relocation_items_of_four_missions_at_every_remainder(compact):
    """The batch kernel evaluates relocations four missions per item: instances with every
    mission count mod 4, with one and two vehicles (where the last item's missions run past
    the route ends into the location arrays' padding) and with several vehicles, in both
    layouts, HARD and PENALTY: every member equals its single solve and the oracle."""
    insts = []
    for s, (V, M) in enumerate([(1, 1), (1, 2), (1, 3), (1, 5), (2, 1), (2, 2), (2, 3), (2, 4),
                                (2, 6), (2, 7), (3, 9), (5, 11), (4, 14), (6, 17)]):
        insts.append(gen.random_instance(600 + s, n_loc=7 + V, n_vehicles=V, n_missions=M,
                                         n_types=2, heli_only_frac=0.2 if s % 3 == 0 else 0.0,
                                         duty_cap=100000, max_minutes=150))
    bp = api.BatchProblem(insts)
    for mode in (PENALTY, HARD):
        params = api.make_params(3, 40, mode, 1000, compact=compact)
        out = api.solve_batch(bp, params)
        torch.cuda.synchronize()
        for b, inst in enumerate(insts):
            got = bp.unpack(out, b)
            _same(got, _single(inst, params))
            r = oracle.tabu_search(oracle.Problem(inst, mode, 1000), 3, 40)
            assert got["info"][api.INFO_STATUS] == r["status"]
            if r["status"] == 0:
                assert got["info"][api.INFO_Z_BEST] == r["z_best"]
                np.testing.assert_array_equal(got["route"], r["route"])
                np.testing.assert_array_equal(got["route_off"], r["route_off"])


def test_batch_result_independent_of_the_mix():
    insts = _mixed_instances()
    params = api.make_params(4, 40, PENALTY, 1000)
    bp1 = api.BatchProblem(insts)
    o1 = api.solve_batch(bp1, params)
    perm = [5, 0, 7, 2, 6, 1, 4, 3]
    extra = gen.random_instance(399, n_loc=9, n_vehicles=4, n_missions=21, n_types=2, duty_cap=900)
    bp2 = api.BatchProblem([insts[i] for i in perm] + [extra])
    o2 = api.solve_batch(bp2, params)
    torch.cuda.synchronize()
    for j, i in enumerate(perm):
        _same(bp1.unpack(o1, i), bp2.unpack(o2, j))


def test_batch_hard_mode_reports_per_instance_status():
    good = gen.random_instance(400, n_loc=8, n_vehicles=3, n_missions=12, duty_cap=5000)
    bad = gen.random_instance(401, n_loc=8, n_vehicles=2, n_missions=12, duty_cap=10)
    params = api.make_params(3, 30, HARD, 1000)
    bp = api.BatchProblem([good, bad, good])
    out = api.solve_batch(bp, params)
    torch.cuda.synchronize()
    assert bp.unpack(out, 0)["info"][api.INFO_STATUS] == 0
    assert bp.unpack(out, 1)["info"][api.INFO_STATUS] == api.E_INFEASIBLE_INIT
    _same(bp.unpack(out, 2), _single(good, params))


def test_batch_with_deadlines_matches_single():
    insts = [gen.random_instance(s, n_loc=12, n_vehicles=6, n_missions=23, n_types=2,
                                 heli_only_frac=0.25, deadlines=True, deadline_lo=800,
                                 duty_cap=2500, max_minutes=60) for s in (43, 49, 50, 57)]
    params = api.make_params(4, 50, HARD, 1000)
    bp = api.BatchProblem(insts)
    out = api.solve_batch(bp, params)
    torch.cuda.synchronize()
    for b, inst in enumerate(insts):
        _same(bp.unpack(out, b), _single(inst, params))


def test_batched_workload_sample_matches_single_solves():
    """The 1,024-instance batched workload (shortened to 40 iterations): every member
    equals its own single solve."""
    insts = [gen.batched_member(i) for i in range(1024)]
    params = api.params_from(gen.BATCHED_PARAMS, iterations=40)
    bp = api.BatchProblem(insts)
    out = api.solve_batch(bp, params)
    torch.cuda.synchronize()
    info = out.info.view(-1, api.INFO_LEN).cpu().numpy()
    assert (info[:, api.INFO_STATUS] == 0).all()
    assert (info[:, api.INFO_ITERS] == 40).all()
    for b in list(range(0, 1024, 37)) + [1023]:
        _same(bp.unpack(out, b), _single(insts[b], params))


def test_batch_host_errors():
    insts = _mixed_instances()[:3]
    bp = api.BatchProblem(insts)
    with pytest.raises(api.AschedError) as e:
        api.solve_batch(bp, api.make_params(3, 5, PENALTY, 1000, cluster_size=3))
    assert e.value.status == api.E_INVALID
    huge = gen.random_instance(9, n_loc=300, n_vehicles=60, n_missions=900, n_types=2,
                               duty_cap=100000)
    with pytest.raises(api.AschedError) as e:
        api.solve_batch(api.BatchProblem([insts[0], huge]), api.make_params(3, 5, PENALTY, 1))
    assert e.value.status == api.E_TOO_LARGE


def test_batch_independent_of_block_size_and_autotuner_picks_a_candidate():
    insts = _mixed_instances()
    params = api.make_params(4, 30, PENALTY, 1000)
    bp = api.BatchProblem(insts)
    outs = []
    for thr in (512, 256, 128, 64):
        params.block_threads = thr
        outs.append(api.solve_batch(bp, params))
    torch.cuda.synchronize()
    for o in outs[1:]:
        for b in range(len(insts)):
            _same(bp.unpack(outs[0], b), bp.unpack(o, b))
    cands = ((256, False), (128, True), (256, False, 2))
    best, times = api.autotune_batch(bp, api.make_params(4, 30, PENALTY, 1000), candidates=cands,
                                     probe_iterations=10, repeats=1)
    assert best in times and set(times) == {(256, False, 1), (128, True, 1), (256, False, 2)}
    assert api.batch_moves_per_warp(bp, (256, False, 2)) * 2 == pytest.approx(
        api.batch_moves_per_warp(bp, (256, False, 1)))
    tuned = api.tuned_params(api.make_params(4, 30, PENALTY, 1000), best)
    got = api.solve_batch(bp, tuned)
    torch.cuda.synchronize()
    for b in range(len(insts)):
        _same(bp.unpack(outs[0], b), bp.unpack(got, b))


def test_batch_replayed_from_a_cuda_graph_matches_direct_calls():
    insts = _mixed_instances()
    params = api.make_params(5, 50, PENALTY, 1000)
    bp = api.BatchProblem(insts)
    direct = api.solve_batch(bp, params)
    torch.cuda.synchronize()
    g, out = api.capture_batch(bp, params)
    for _ in range(3):
        out.info.zero_()
        out.route.zero_()
        g.replay()
        torch.cuda.synchronize()
        for b in range(len(insts)):
            _same(bp.unpack(out, b), bp.unpack(direct, b))


@pytest.mark.parametrize("cluster", [2, 4, 16])
def test_batch_solved_by_clusters_equals_one_cta_per_instance(cluster):
    """CTAs per instance (a thread-block cluster solving each instance) changes nothing in
    the results: every member equals the one-CTA batch, which equals single solves."""
    insts = _mixed_instances()
    params = api.make_params(5, 40, PENALTY, 1000)
    bp = api.BatchProblem(insts)
    ref = api.solve_batch(bp, params)
    got = api.solve_batch(bp, api.make_params(5, 40, PENALTY, 1000, cluster_size=cluster, block_threads=128))
    torch.cuda.synchronize()
    for b in range(len(insts)):
        _same(bp.unpack(ref, b), bp.unpack(got, b))
    _same(bp.unpack(got, 0), _single(insts[0], params))
