"""CUDA path vs the CPU oracle, through the C ABI (needs a GB300).

All travel times are integers, so every comparison is exact: per-move delta and
flags, chosen move ids, whole trajectories of (move, objective), best schedules.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2002_11710_gb300 import api, gen

pytestmark = pytest.mark.gpu

HARD, PENALTY = gen.HARD, gen.PENALTY


def _replay_states(pb, tenure, traj_moves, init):
    """Yield (it, off, route, tabu, z, z_best) before each iteration, replaying the
    given moves with the oracle's own apply."""
    off, route = (np.array(init[0], np.int32), np.array(init[1], np.int32))
    tabu = -np.ones((pb.M, pb.V), dtype=np.int32)
    z = oracle.cost(pb, off, route)[0]
    z_best = z
    for it, mv in enumerate(traj_moves):
        yield it, off, route, tabu, z, z_best
        oracle.apply_tabu_move(pb, tenure, it, off, route, tabu, int(mv))
        z = oracle.cost(pb, off, route)[0]
        z_best = min(z_best, z)


def _dev(a, dtype=torch.int32):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype=dtype)


def _gpu_eval(dp, params, off, route, tabu, it, z_best):
    delta, flags, ids, key, info = api.eval_neighbourhood(dp, params, _dev(off), _dev(route),
                                                          _dev(tabu), it, z_best)
    torch.cuda.synchronize()
    assert int(info[api.INFO_STATUS]) == 0, int(info[api.INFO_STATUS])
    return (delta.cpu().numpy().astype(np.int64), flags.cpu().numpy(),
            ids.cpu().numpy().view(np.uint32), int(key.cpu().numpy().view(np.uint64)[0]))


def _oracle_key(ids, delta, chosen):
    if chosen < 0:
        return 0xFFFFFFFFFFFFFFFF
    d = int(delta[chosen]) & 0xFFFFFFFF
    return ((d ^ 0x80000000) << 32) | int(ids[chosen])


EVAL_CASES = [
    ("tiny-penalty", lambda: gen.tiny(0), PENALTY, 7),
    ("random-hard", lambda: gen.random_instance(21, n_loc=9, n_vehicles=4, n_missions=13,
                                                duty_cap=900, max_minutes=150), HARD, 4),
    ("random-2types-heli", lambda: gen.random_instance(22, n_loc=11, n_vehicles=5, n_missions=37,
                                                       n_types=2, heli_only_frac=0.3,
                                                       duty_cap=1500, max_minutes=120), PENALTY, 5),
    ("random-deadlines", lambda: gen.random_instance(23, n_loc=10, n_vehicles=6, n_missions=19,
                                                     deadlines=True, deadline_lo=700,
                                                     duty_cap=2000, max_minutes=100), HARD, 3),
    ("paper-model-14", lambda: gen.paper_model(3, 14), PENALTY, 4),
    ("paper-shaped", lambda: gen.paper_shaped(0), PENALTY, 10),
]


@pytest.mark.parametrize("compact", [False, True], ids=["tables", "compact"])
@pytest.mark.parametrize("name,mk,mode,tenure", EVAL_CASES, ids=[c[0] for c in EVAL_CASES])
def test_eval_neighbourhood_matches_oracle(name, mk, mode, tenure, compact):
    inst = mk()
    pb = oracle.Problem(inst, mode, 1000)
    rc, off0, route0 = oracle.greedy_init(pb)
    assert rc == 0
    iters = 30 if inst.n_missions < 50 else 6
    r = oracle.tabu_search(pb, tenure, iters)
    dp = api.DeviceProblem(inst)
    params = api.make_params(tenure, 0, mode, 1000, compact=compact)
    checked = 0
    for it, off, route, tabu, z, z_best in _replay_states(pb, tenure, r["traj_move"], (off0, route0)):
        if it % 3 and it != iters - 1:
            continue
        ids, delta, flags, chosen = oracle.eval_neighbourhood(pb, off, route, tabu, it, z_best)
        gd, gf, gi, gkey = _gpu_eval(dp, params, off, route, tabu, it, z_best)
        np.testing.assert_array_equal(gi, ids)
        np.testing.assert_array_equal(gd, delta)
        np.testing.assert_array_equal(gf, flags)
        assert gkey == _oracle_key(ids, delta, chosen)
        checked += 1
    assert checked > 0


@pytest.mark.parametrize("cluster,threads", [(1, 64), (1, 512), (2, 96), (4, 256), (8, 512),
                                             (16, 512), (16, 64)])
def test_eval_independent_of_launch_shape(cluster, threads):
    inst = gen.random_instance(31, n_loc=12, n_vehicles=7, n_missions=45, n_types=2,
                               heli_only_frac=0.2, duty_cap=1200, max_minutes=140)
    pb = oracle.Problem(inst, PENALTY, 1000)
    rc, off, route = oracle.greedy_init(pb)
    tabu = np.random.default_rng(0).integers(-1, 6, size=(pb.M, pb.V)).astype(np.int32)
    z = oracle.cost(pb, off, route)[0]
    ids, delta, flags, chosen = oracle.eval_neighbourhood(pb, off, route, tabu, 3, z - 10)
    dp = api.DeviceProblem(inst)
    params = api.make_params(5, 0, PENALTY, 1000, cluster_size=cluster, block_threads=threads)
    gd, gf, gi, gkey = _gpu_eval(dp, params, off, route, tabu, 3, z - 10)
    np.testing.assert_array_equal(gd, delta)
    np.testing.assert_array_equal(gf, flags)
    assert gkey == _oracle_key(ids, delta, chosen)


TRAJ_CASES = [
    ("tiny-200", lambda: gen.tiny(0), PENALTY, 7, 200),
    ("random-hard", lambda: gen.random_instance(41, n_loc=9, n_vehicles=4, n_missions=15,
                                                duty_cap=1000, max_minutes=150), HARD, 5, 150),
    ("random-deadlines-2types", lambda: gen.random_instance(49, n_loc=12, n_vehicles=6,
                                                            n_missions=23, n_types=2,
                                                            heli_only_frac=0.25, deadlines=True,
                                                            deadline_lo=1000, duty_cap=2500,
                                                            max_minutes=60), HARD, 4, 120),
    ("paper-model-24", lambda: gen.paper_model(5, 24), PENALTY, 5, 150),
    ("paper-model-20-hard", lambda: gen.paper_model(2, 20), HARD, 5, 150),
    ("ragged-33", lambda: gen.random_instance(43, n_loc=15, n_vehicles=3, n_missions=33,
                                              duty_cap=3000, max_minutes=100), PENALTY, 6, 100),
    ("paper-shaped-150", lambda: gen.paper_shaped(0), PENALTY, 10, 150),
]


def _check_solve_vs_oracle(inst, mode, tenure, iters, **launch):
    pb = oracle.Problem(inst, mode, 1000)
    r = oracle.tabu_search(pb, tenure, iters)
    assert r["status"] == 0, "pick an instance with a feasible greedy start"
    dp = api.DeviceProblem(inst)
    params = api.make_params(tenure, iters, mode, 1000, **launch)
    out = api.solve(dp, params, trajectory=True)
    torch.cuda.synchronize()
    info = out.info.cpu().numpy()
    assert info[api.INFO_STATUS] == 0, info
    gm = out.traj_move.cpu().numpy().view(np.uint32)[:iters]
    gz = out.traj_z.cpu().numpy()[:iters]
    first_bad = np.nonzero(gm != r["traj_move"])[0]
    assert first_bad.size == 0, f"first differing iteration {first_bad[:1]}"
    np.testing.assert_array_equal(gz, r["traj_z"])
    assert info[api.INFO_Z_BEST] == r["z_best"] and info[api.INFO_BEST_IT] == r["best_it"]
    np.testing.assert_array_equal(out.route_off.cpu().numpy()[: pb.V + 1], r["route_off"])
    np.testing.assert_array_equal(out.route.cpu().numpy()[: pb.M], r["route"])
    z, fl, ov = oracle.cost(pb, r["route_off"], r["route"])
    np.testing.assert_array_equal(out.flight.cpu().numpy()[: pb.V], fl)
    np.testing.assert_array_equal(out.overflow.cpu().numpy()[: pb.V], ov)
    return gm, gz


@pytest.mark.parametrize("compact", [False, True], ids=["tables", "compact"])
@pytest.mark.parametrize("name,mk,mode,tenure,iters", TRAJ_CASES, ids=[c[0] for c in TRAJ_CASES])
def test_solve_trajectory_matches_oracle(name, mk, mode, tenure, iters, compact):
    _check_solve_vs_oracle(mk(), mode, tenure, iters, compact=compact)


@pytest.mark.parametrize("cluster,threads,grid", [(1, 512, 1), (2, 512, 1), (4, 128, 1), (8, 448, 1), (16, 256, 1),
                                                  (1, 128, 5), (2, 96, 3), (4, 64, 7), (8, 256, 2), (16, 512, 2),
                                                  (16, 128, 4), (1, 64, 37)])
def test_trajectory_independent_of_launch_shape(cluster, threads, grid):
    """Any launch shape, also spanning several clusters that exchange keys through the
    workspace, gives the oracle's trajectory."""
    inst = gen.random_instance(51, n_loc=14, n_vehicles=8, n_missions=40, n_types=2,
                               heli_only_frac=0.2, duty_cap=900, max_minutes=120)
    _check_solve_vs_oracle(inst, PENALTY, 6, 80, cluster_size=cluster, block_threads=threads, grid_clusters=grid)


@pytest.mark.parametrize("grid", [2, 5])
def test_grid_launch_compact_layout_with_deadlines_and_two_types(grid):
    inst = gen.random_instance(49, n_loc=12, n_vehicles=6, n_missions=23, n_types=2, heli_only_frac=0.25,
                               deadlines=True, deadline_lo=1000, duty_cap=2500, max_minutes=60)
    _check_solve_vs_oracle(inst, HARD, 4, 120, cluster_size=4, grid_clusters=grid, compact=True)


GREEDY_CASES = [
    (lambda: gen.tiny(0), PENALTY),
    (lambda: gen.paper_model(7, 24), HARD),
    (lambda: gen.random_instance(61, n_loc=10, n_vehicles=5, n_missions=30, n_types=2,
                                 heli_only_frac=0.3, deadlines=True, deadline_lo=900,
                                 duty_cap=3000), HARD),
    (lambda: gen.random_instance(57, n_loc=12, n_vehicles=6, n_missions=23, n_types=2,
                                 heli_only_frac=0.25, deadlines=True, deadline_lo=800,
                                 duty_cap=2500, max_minutes=60), HARD),
    (lambda: gen.large(0), PENALTY),
]


@pytest.mark.parametrize("mk,mode", GREEDY_CASES)
def test_greedy_init_matches_oracle(mk, mode):
    inst = mk()
    pb = oracle.Problem(inst, mode, 1000)
    rc, off, route = oracle.greedy_init(pb)
    dp = api.DeviceProblem(inst)
    params = api.make_params(5, 0, mode, 1000)
    out = api.solve(dp, params)  # every case fits one of the two on-chip layouts
    torch.cuda.synchronize()
    info = out.info.cpu().numpy()
    if rc != 0:
        assert info[api.INFO_STATUS] == api.E_INFEASIBLE_INIT
        return
    assert info[api.INFO_STATUS] == 0
    np.testing.assert_array_equal(out.route_off.cpu().numpy()[: pb.V + 1], off)
    np.testing.assert_array_equal(out.route.cpu().numpy()[: pb.M], route)
    assert info[api.INFO_Z_BEST] == oracle.cost(pb, off, route)[0]


@pytest.mark.parametrize("mk,mode", GREEDY_CASES)
def test_greedy_init_entry_point_matches_oracle(mk, mode):
    """asched_greedy_init: Algorithm 1 alone, as its own entry point."""
    inst = mk()
    pb = oracle.Problem(inst, mode, 1000)
    rc, off, route = oracle.greedy_init(pb)
    dp = api.DeviceProblem(inst)
    g_off, g_route, info = api.greedy_init(dp, api.make_params(5, 50, mode, 1000))
    torch.cuda.synchronize()
    info = info.cpu().numpy()
    if rc != 0:
        assert info[api.INFO_STATUS] == api.E_INFEASIBLE_INIT
        return
    assert info[api.INFO_STATUS] == 0 and info[api.INFO_ITERS] == 0
    np.testing.assert_array_equal(g_off.cpu().numpy()[: pb.V + 1], off)
    np.testing.assert_array_equal(g_route.cpu().numpy()[: pb.M], route)
    assert info[api.INFO_Z_BEST] == info[api.INFO_Z_INIT] == oracle.cost(pb, off, route)[0]


@pytest.mark.parametrize("grid", [1, 3])
def test_tabu_solve_entry_point_equals_solve(grid):
    """asched_tabu_solve (through ctypes, with a workspace when the launch spans several
    clusters) gives what asched_solve gives on one cluster, bit for bit."""
    import ctypes

    inst = gen.random_instance(72, n_loc=9, n_vehicles=4, n_missions=17, duty_cap=2000, n_types=2,
                               heli_only_frac=0.2)
    dp = api.DeviceProblem(inst)
    params = api.make_params(5, 80, PENALTY, 1000)
    a = api.solve_one_cluster(dp, params, trajectory=True)
    gp = api.make_params(5, 80, PENALTY, 1000, cluster_size=2, grid_clusters=grid)
    nb = api.workspace_bytes(dp, gp)
    assert (nb > 0) == (grid > 1)
    ws = torch.zeros(max(nb, 8) // 8, dtype=torch.int64, device="cuda")
    b = api.alloc_output(dp, params.iterations, trajectory=True)
    res = b.struct()
    rc = api._lib.load().asched_tabu_solve(ctypes.byref(dp.struct), ctypes.byref(gp), None, None,
                                           ctypes.byref(res), ctypes.c_void_p(ws.data_ptr()), ctypes.c_size_t(nb),
                                           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == api.OK
    torch.cuda.synchronize()
    for k in ("route_off", "route", "info", "traj_move", "traj_z"):
        assert torch.equal(getattr(a, k), getattr(b, k)), k
    if grid > 1:  # a workspace that is too small is refused before anything is queued
        rc = api._lib.load().asched_tabu_solve(ctypes.byref(dp.struct), ctypes.byref(gp), None, None,
                                               ctypes.byref(res), ctypes.c_void_p(ws.data_ptr()),
                                               ctypes.c_size_t(nb - 8),
                                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == api.E_INVALID


def test_solve_from_given_schedule():
    inst = gen.random_instance(71, n_loc=9, n_vehicles=4, n_missions=17, duty_cap=2000)
    pb = oracle.Problem(inst, PENALTY, 1000)
    # an arbitrary feasible start: missions dealt round-robin
    V, M = pb.V, pb.M
    routes = [[m for m in range(M) if m % V == v] for v in range(V)]
    off = np.array([0] + list(np.cumsum([len(r) for r in routes])), np.int32)
    route = np.array([m for r in routes for m in r], np.int32)
    r = oracle.tabu_search(pb, 4, 60, init=(off, route))
    dp = api.DeviceProblem(inst)
    out = api.solve(dp, api.make_params(4, 60, PENALTY, 1000), init=(_dev(off), _dev(route)),
                    trajectory=True)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.traj_move.cpu().numpy().view(np.uint32), r["traj_move"])
    np.testing.assert_array_equal(out.traj_z.cpu().numpy(), r["traj_z"])


def test_paper_shaped_full_run_sampled_against_oracle():
    """The full 5,000-iteration run on the paper-shaped instance (the benchmark's
    workload and launch shape): every objective on the trajectory is recomputed by
    the oracle from the replayed schedule, and at sampled iterations the oracle's own
    neighbourhood evaluation must choose the same move."""
    inst, p = gen.paper_shaped(0), gen.PAPER_SHAPED_PARAMS
    dp = api.DeviceProblem(inst)
    out = api.solve(dp, api.params_from(p), trajectory=True)
    torch.cuda.synchronize()
    info = out.info.cpu().numpy()
    assert info[api.INFO_STATUS] == 0 and info[api.INFO_ITERS] == p.iterations
    gm = out.traj_move.cpu().numpy().view(np.uint32)
    gz = out.traj_z.cpu().numpy()
    pb = oracle.Problem(inst, p.cap_mode, p.lam)
    rc, off0, route0 = oracle.greedy_init(pb)
    assert info[api.INFO_Z_INIT] == oracle.cost(pb, off0, route0)[0]
    sample = set(range(0, 12)) | set(range(0, p.iterations, 401)) | {p.iterations - 1}
    z_best, best_it = None, -1
    for it, off, route, tabu, z, zb in _replay_states(pb, p.tenure, gm, (off0, route0)):
        if it in sample:
            ids, delta, flags, chosen = oracle.eval_neighbourhood(pb, off, route, tabu, it, zb)
            want = 0xFFFFFFFF if chosen < 0 else int(ids[chosen])
            assert int(gm[it]) == want, f"iteration {it}"
        if it > 0:
            assert int(gz[it - 1]) == z, f"objective after iteration {it - 1}"
    z_end = oracle.cost(pb, off, route)[0]
    assert int(gz[-1]) == z_end
    zs = np.concatenate([[info[api.INFO_Z_INIT]], gz])
    assert info[api.INFO_Z_BEST] == zs.min()
    assert info[api.INFO_BEST_IT] == int(np.argmin(zs)) - 1


@pytest.mark.parametrize("compact", [False, True], ids=["tables", "compact"])
def test_edge_sizes(compact):
    for M, V in [(0, 3), (1, 1), (2, 1), (1, 5), (3, 2), (64, 1), (65, 2)]:
        inst = gen.random_instance(80 + M + V, n_loc=8, n_vehicles=V, n_missions=M,
                                   duty_cap=100000, max_minutes=50)
        _check_solve_vs_oracle(inst, PENALTY, 3, 25, compact=compact)


def test_plan_launch_shapes():
    """The default launch shape: one thread per item on few CTAs for small neighbourhoods;
    from 1,024 moves up, 16 CTAs with the fewest warps (4, 8, 12 or 16) that keep the
    largest per-warp share of 32-item chunks at its least."""
    two_types = gen.random_instance(8, n_loc=40, n_vehicles=25, n_missions=120, n_types=2,
                                    duty_cap=3000, max_minutes=120)  # 495 chunks: 12 warps leave 3 to some
    cases = [(gen.tiny(0), 1, 192), (gen.batched_member(10), 16, 128), (gen.paper_shaped(0), 16, 384),
             (two_types, 16, 512)]
    for inst, C, T in cases:
        dp = api.DeviceProblem(inst)
        pl = api.plan(dp, api.make_params(5, 10, PENALTY, 1000))
        assert (pl.cluster_size, pl.block_threads, pl.grid_clusters) == (C, T, 1), inst.name
        assert pl.workspace_bytes == 0
    # the large neighbourhood (5,307 chunks) spreads over every cluster the device holds
    dp = api.DeviceProblem(gen.large(0))
    pl = api.plan(dp, api.make_params(15, 10, PENALTY, 1000))
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert pl.grid_clusters >= 2 and pl.grid_clusters * pl.cluster_size <= sms
    assert pl.grid_clusters * pl.cluster_size >= sms // 2
    assert pl.workspace_bytes >= 16 * pl.grid_clusters


def test_large_instance_sampled_against_oracle():
    """The large configuration (400 missions, 50 vehicles, 240 locations) only fits in
    the compact layout. Its first 120 iterations: every objective is recomputed by the
    oracle from the replayed schedule and sampled iterations must choose the oracle's
    move."""
    inst, p = gen.large(0), gen.LARGE_PARAMS
    iters = 120
    dp = api.DeviceProblem(inst)
    params = api.params_from(p, iterations=iters)
    # the gather tables alone (2 x L x M rounded up to 32, int32) exceed a CTA's shared
    # memory, so the plan that launches is the int16 matrix layout
    assert 2 * inst.n_loc * ((inst.n_missions + 31) // 32 * 32) * 4 > 232448
    assert api.plan(dp, params).smem_bytes <= 232448
    out = api.solve(dp, params, trajectory=True)
    torch.cuda.synchronize()
    info = out.info.cpu().numpy()
    assert info[api.INFO_STATUS] == 0 and info[api.INFO_ITERS] == iters
    gm = out.traj_move.cpu().numpy().view(np.uint32)
    gz = out.traj_z.cpu().numpy()
    pb = oracle.Problem(inst, p.cap_mode, p.lam)
    rc, off0, route0 = oracle.greedy_init(pb)
    assert rc == 0 and info[api.INFO_Z_INIT] == oracle.cost(pb, off0, route0)[0]
    sample = {0, 1, 59, iters - 1}
    for it, off, route, tabu, z, zb in _replay_states(pb, p.tenure, gm, (off0, route0)):
        if it in sample:
            ids, delta, flags, chosen = oracle.eval_neighbourhood(pb, off, route, tabu, it, zb)
            assert int(gm[it]) == (0xFFFFFFFF if chosen < 0 else int(ids[chosen])), f"iteration {it}"
        if it > 0:
            assert int(gz[it - 1]) == z, f"objective after iteration {it - 1}"


def test_large_full_run_sampled_against_oracle():
    """The benchmark's workload at full length: the large instance, all 10,000 iterations,
    on the default launch shape (several clusters). Every objective on the trajectory is
    recomputed by the oracle from the replayed schedule, the best objective and its
    iteration follow, and at sampled iterations the oracle's own neighbourhood evaluation
    must choose the same move."""
    inst, p = gen.large(0), gen.LARGE_PARAMS
    dp = api.DeviceProblem(inst)
    params = api.params_from(p)
    assert api.plan(dp, params).grid_clusters >= 2
    out = api.solve(dp, params, trajectory=True)
    torch.cuda.synchronize()
    info = out.info.cpu().numpy()
    assert info[api.INFO_STATUS] == 0 and info[api.INFO_ITERS] == p.iterations
    gm = out.traj_move.cpu().numpy().view(np.uint32)
    gz = out.traj_z.cpu().numpy()
    pb = oracle.Problem(inst, p.cap_mode, p.lam)
    rc, off0, route0 = oracle.greedy_init(pb)
    assert rc == 0 and info[api.INFO_Z_INIT] == oracle.cost(pb, off0, route0)[0]
    sample = {0, 1, 2, 997, 4001, p.iterations - 1}
    for it, off, route, tabu, z, zb in _replay_states(pb, p.tenure, gm, (off0, route0)):
        if it in sample:
            ids, delta, flags, chosen = oracle.eval_neighbourhood(pb, off, route, tabu, it, zb)
            assert int(gm[it]) == (0xFFFFFFFF if chosen < 0 else int(ids[chosen])), f"iteration {it}"
        if it > 0:
            assert int(gz[it - 1]) == z, f"objective after iteration {it - 1}"
    assert int(gz[-1]) == oracle.cost(pb, off, route)[0]
    zs = np.concatenate([[info[api.INFO_Z_INIT]], gz])
    assert info[api.INFO_Z_BEST] == zs.min()
    assert info[api.INFO_BEST_IT] == int(np.argmin(zs)) - 1
    z, fl, ov = oracle.cost(pb, out.route_off.cpu().numpy()[: pb.V + 1], out.route.cpu().numpy()[: pb.M])
    assert z == info[api.INFO_Z_BEST]
    np.testing.assert_array_equal(out.flight.cpu().numpy()[: pb.V], fl)
    np.testing.assert_array_equal(out.overflow.cpu().numpy()[: pb.V], ov)


def test_plain_launch_gives_the_same_trajectory():
    """ASCHED_PLAIN_LAUNCH (no cooperative attribute) changes nothing in the results."""
    inst = gen.random_instance(51, n_loc=14, n_vehicles=8, n_missions=40, n_types=2,
                               heli_only_frac=0.2, duty_cap=900, max_minutes=120)
    _check_solve_vs_oracle(inst, PENALTY, 6, 80, cluster_size=4, block_threads=128, grid_clusters=5,
                           plain_launch=True)


def test_large_grid_equals_one_cluster():
    """The large instance on every cluster of the device (asched_tabu_solve) and on one
    cluster (asched_solve): identical trajectories and outputs."""
    inst, p = gen.large(0), gen.LARGE_PARAMS
    dp = api.DeviceProblem(inst)
    params = api.params_from(p, iterations=400)
    a = api.solve(dp, params, trajectory=True)
    b = api.solve_one_cluster(dp, params, trajectory=True)
    torch.cuda.synchronize()
    assert int(a.info[api.INFO_STATUS]) == 0
    for k in ("route_off", "route", "flight", "overflow", "info", "traj_move", "traj_z"):
        assert torch.equal(getattr(a, k), getattr(b, k)), k


def test_device_status_codes():
    base = gen.random_instance(90, n_loc=8, n_vehicles=3, n_missions=10, duty_cap=2000)
    params = api.make_params(3, 5, HARD, 1000)
    # pickup out of range -> invalid
    bad = gen.Instance(**{**base.__dict__, "pickup": base.pickup.copy()})
    bad.pickup[3] = 99
    out = api.solve(api.DeviceProblem(bad), params)
    torch.cuda.synchronize()
    assert int(out.info[api.INFO_STATUS]) == api.E_INVALID
    # tiny duty cap in HARD mode -> no feasible greedy start
    tight = gen.Instance(**{**base.__dict__, "duty_cap": 5})
    out = api.solve(api.DeviceProblem(tight), params)
    torch.cuda.synchronize()
    assert int(out.info[api.INFO_STATUS]) == api.E_INFEASIBLE_INIT
    # huge minutes -> overflow guard
    big = gen.Instance(**{**base.__dict__, "travel": base.travel * 200000})
    out = api.solve(api.DeviceProblem(big), api.make_params(3, 5, PENALTY, 1000))
    torch.cuda.synchronize()
    assert int(out.info[api.INFO_STATUS]) == api.E_OVERFLOW_GUARD
    # a start schedule that lists a mission twice -> invalid
    dp = api.DeviceProblem(base)
    off = _dev(np.array([0, 4, 7, 10], np.int32))
    route = _dev(np.array([0, 1, 2, 3, 3, 5, 6, 7, 8, 9], np.int32))
    out = api.solve(dp, params, init=(off, route))
    torch.cuda.synchronize()
    assert int(out.info[api.INFO_STATUS]) == api.E_INVALID


def test_host_side_errors():
    base = gen.random_instance(91, n_loc=8, n_vehicles=3, n_missions=10)
    dp = api.DeviceProblem(base)
    with pytest.raises(api.AschedError) as e:
        api.solve(dp, api.make_params(3, 5, 7, 1000))
    assert e.value.status == api.E_INVALID
    with pytest.raises(api.AschedError) as e:
        api.solve(dp, api.make_params(3, 5, HARD, 1000, cluster_size=3))
    assert e.value.status == api.E_INVALID
    huge = gen.random_instance(92, n_loc=300, n_vehicles=60, n_missions=900, duty_cap=100000)
    with pytest.raises(api.AschedError) as e:
        api.solve(api.DeviceProblem(huge), api.make_params(3, 5, PENALTY, 1))
    assert e.value.status == api.E_TOO_LARGE
    # the compact layout's int16 stamps cap iterations + tenure
    with pytest.raises(api.AschedError) as e:
        api.solve(dp, api.make_params(3, 40000, PENALTY, 1000, compact=True))
    assert e.value.status == api.E_TOO_LARGE
    # travel times above int16 cannot use the compact layout
    wide = gen.Instance(**{**base.__dict__, "travel": base.travel * 200})
    out = api.solve(api.DeviceProblem(wide), api.make_params(3, 5, PENALTY, 1, compact=True))
    torch.cuda.synchronize()
    assert int(out.info[api.INFO_STATUS]) == api.E_TOO_LARGE


@pytest.mark.parametrize("cluster,grid", [(2, 1), (16, 1), (2, 3), (1, 4), (16, 2)])
def test_bounded_wait_reports_timeout_and_context_stays_usable(cluster, grid):
    """A CTA (one cluster) or a cluster (several) that never publishes its key (test hook)
    makes every other bounded wait run out: the call ends with ASCHED_E_TIMEOUT, and the
    next solve in the same context is correct."""
    inst = gen.random_instance(95, n_loc=10, n_vehicles=4, n_missions=30, duty_cap=2000)
    dp = api.DeviceProblem(inst)
    params = api.make_params(4, 50, PENALTY, 1000, cluster_size=cluster, timeout_ns=50_000_000,
                             grid_clusters=grid)
    params.flags |= api._lib.TEST_WITHHOLD_KEY
    out = api.solve(dp, params)
    torch.cuda.synchronize()
    assert int(out.info[api.INFO_STATUS]) == api.E_TIMEOUT
    assert int(out.info[api.INFO_ITERS]) == 0
    _check_solve_vs_oracle(inst, PENALTY, 4, 50, cluster_size=cluster, grid_clusters=grid)
