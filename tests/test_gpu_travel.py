"""asched_travel_matrix (Eq. e1 on the device) against the oracle's definition, and the
whole path coordinates -> matrices -> search (needs a GB300)."""
import numpy as np
import pytest
import torch

from oracle import travel
from paper_2002_11710_gb300 import api, gen

pytestmark = pytest.mark.gpu


def _coords_tensor(insts):
    return torch.from_numpy(np.concatenate([i.coords for i in insts])).to("cuda", torch.float64)


def test_euclidean_bit_exact_on_the_workloads():
    """Every batched-workload member's matrix rebuilt on the device from its coordinates
    equals the oracle's (and so the generator's) integers exactly."""
    insts = [gen.batched_member(i) for i in range(1024)]
    bp = api.BatchProblem(insts)
    want = bp.travel.clone()
    bp.travel.zero_()
    status = api.travel_into_batch(bp, _coords_tensor(insts), [250.0])
    torch.cuda.synchronize()
    assert int(status.item()) == api.OK
    assert torch.equal(bp.travel, want)
    for b in (0, 17, 1023):
        o = travel.travel_minutes(insts[b].coords, [250.0], travel.EUCLIDEAN)
        t0 = int(bp.h_travel_off[b])
        L = insts[b].n_loc
        np.testing.assert_array_equal(bp.travel[t0:t0 + L * L].cpu().numpy().reshape(1, L, L), o)


def _batch_of(coords, nt):
    """A batch whose instance b has the locations coords[b] (matrices zeroed)."""
    insts = []
    for c in coords:
        L = len(c)
        inst = gen.random_instance(1, n_loc=max(L, 2), n_vehicles=1, n_missions=0, n_types=nt)
        inst.travel = np.zeros((nt, L, L), np.int32)
        inst.veh_base = np.zeros(1, np.int32)
        inst.coords = c
        insts.append(inst)
    return api.BatchProblem(insts), insts


def _check_batch(coords, speeds, metric, exact=True):
    """Build the batch's matrices on the device and compare them with the oracle's
    (metric: the oracle's travel.EUCLIDEAN or travel.HAVERSINE)."""
    bp, insts = _batch_of(coords, len(speeds))
    bp.travel.fill_(-7)  # every entry must be written
    api_metric = api.METRIC_HAVERSINE if metric == travel.HAVERSINE else api.METRIC_EUCLIDEAN
    status = api.travel_into_batch(bp, _coords_tensor(insts), speeds, api_metric)
    torch.cuda.synchronize()
    assert int(status.item()) == api.OK
    nt = len(speeds)
    for b, c in enumerate(coords):
        L = len(c)
        t0 = int(bp.h_travel_off[b])
        got = bp.travel[t0:t0 + nt * L * L].cpu().numpy().reshape(nt, L, L)
        want = travel.travel_minutes(c, speeds, metric)
        if exact:
            np.testing.assert_array_equal(got, want)
        else:  # Haversine: exact away from half minutes, else within 1
            raw = travel.minutes_unrounded(c, speeds, metric)
            near_half = np.abs(np.abs(raw - np.floor(raw)) - 0.5) < 1e-6
            assert np.array_equal(got[~near_half], want[~near_half])
            assert np.abs(got.astype(np.int64) - want).max() <= 1
    return bp


def test_euclidean_two_layers_and_ragged_sizes():
    rng = np.random.default_rng(2)
    sizes = [1, 2, 31, 32, 33, 64, 95, 300]
    _check_batch([rng.uniform(-500.0, 2500.0, size=(L, 2)) for L in sizes], [300.0, 500.0], travel.EUCLIDEAN)


@pytest.mark.parametrize("speeds", [[300.0, 500.0], [250.0]])
def test_euclidean_every_small_size_and_alignment(speeds):
    """Sizes around the limit of the shared-memory build (L <= 55 for two types, 78 for
    one) and every 16-byte phase of an instance's block in the output."""
    rng = np.random.default_rng(11)
    lim = 55 if len(speeds) == 2 else 78
    sizes = list(range(1, 20)) + [lim - 2, lim - 1, lim, lim + 1, lim + 2] + [int(x) for x in rng.integers(1, lim + 3, 40)]
    coords = [rng.uniform(-800.0, 1800.0, size=(L, 2)) for L in sizes]
    bp = _check_batch(coords, speeds, travel.EUCLIDEAN)
    # blocks of 2 L^2 words start at even words; odd L^2 blocks reach every phase
    phases = {0, 2} if len(speeds) == 2 else {0, 1, 2, 3}
    assert {int(o) % 4 for o in bp.h_travel_off[:len(sizes)]} == phases


def test_haversine_small_instances():
    rng = np.random.default_rng(12)
    coords = []
    for L in [1, 2, 5, 17, 40, 52, 55, 56, 64, 70]:
        coords.append(np.stack([rng.uniform(42.0, 56.0, L), rng.uniform(-95.0, -74.0, L)], axis=1))
    coords.append(np.stack([rng.uniform(-89.0, 89.0, 50), rng.uniform(-180.0, 180.0, 50)], axis=1))
    _check_batch(coords, [300.0, 500.0], travel.HAVERSINE, exact=False)


def test_half_minute_ties_overflow_the_float64_queue():
    """Points 0.5 km apart on a line at 60 and 120 km/h: a quarter to a half of all times
    are exact ties, far more than the float64 queue of a small instance holds (and a
    large instance beside them); half to even, as the float64 definition."""
    coords = [np.stack([0.5 * np.arange(L) + 1000.0, np.zeros(L)], axis=1) for L in (55, 50, 7, 63)]
    bp = _check_batch(coords, [60.0, 120.0], travel.EUCLIDEAN)
    L = 55
    got = bp.travel[:L * L].cpu().numpy().reshape(L, L)
    assert got[0, 1] == 0 and got[0, 3] == 2 and got[0, 5] == 2 and got[0, 7] == 4  # 0.5, 1.5, 2.5, 3.5 -> even


@pytest.mark.parametrize("region", ["ontario", "globe"])
def test_haversine_matches_the_oracle(region):
    """Exact wherever the oracle's unrounded time is not within 1e-6 minutes of a half
    minute (device and host trigonometry may differ in the last bits), else within 1."""
    rng = np.random.default_rng(4)
    if region == "ontario":  # the paper's setting: bases and hospitals in one province
        ll = np.stack([rng.uniform(42.0, 56.0, 400), rng.uniform(-95.0, -74.0, 400)], axis=1)
    else:
        ll = np.stack([rng.uniform(-89.0, 89.0, 400), rng.uniform(-180.0, 180.0, 400)], axis=1)
    got = api.travel_matrix(ll, [300.0, 500.0], api.METRIC_HAVERSINE).cpu().numpy()
    want = travel.travel_minutes(ll, [300.0, 500.0], travel.HAVERSINE)
    raw = travel.minutes_unrounded(ll, [300.0, 500.0], travel.HAVERSINE)
    near_half = np.abs(np.abs(raw - np.floor(raw)) - 0.5) < 1e-6
    assert np.array_equal(got[~near_half], want[~near_half])
    assert np.abs(got.astype(np.int64) - want).max() <= 1
    assert (got == np.transpose(got, (0, 2, 1))).all()
    assert (np.diagonal(got, axis1=1, axis2=2) == 0).all()


def test_invalid_and_far_points_in_small_instances():
    """A NaN at location 0 of a 55-location instance (every entry uncertain, far more than
    the float64 queue holds): its entries read 0, the rest are exact, status E_INVALID.
    Coordinates of 10^7 km (times may pass 2^22 minutes, so every entry goes through
    float64) stay exact; other instances of the batch are untouched."""
    rng = np.random.default_rng(13)
    good = rng.uniform(0.0, 1000.0, (40, 2))
    nan0 = rng.uniform(0.0, 1000.0, (55, 2))
    nan0[0, 0] = np.nan
    far = rng.uniform(-1e7, 1e7, (30, 2))
    coords = [good, nan0, far]
    bp, insts = _batch_of(coords, 2)
    bp.travel.fill_(-7)
    status = api.travel_into_batch(bp, _coords_tensor(insts), [300.0, 500.0], api.METRIC_EUCLIDEAN)
    torch.cuda.synchronize()
    assert int(status.item()) == api.E_INVALID
    got = []
    for b, c in enumerate(coords):
        L = len(c)
        t0 = int(bp.h_travel_off[b])
        got.append(bp.travel[t0:t0 + 2 * L * L].cpu().numpy().reshape(2, L, L))
    np.testing.assert_array_equal(got[0], travel.travel_minutes(good, [300.0, 500.0], travel.EUCLIDEAN))
    np.testing.assert_array_equal(got[2], travel.travel_minutes(far, [300.0, 500.0], travel.EUCLIDEAN))
    assert (got[1][:, 0, :] == 0).all() and (got[1][:, :, 0] == 0).all()
    np.testing.assert_array_equal(got[1][:, 1:, 1:], travel.travel_minutes(nan0[1:], [300.0, 500.0], travel.EUCLIDEAN))


def test_status_and_host_errors():
    ll = np.array([[0.0, 0.0], [np.nan, 1.0], [1.0, 1.0]])
    with pytest.raises(api.AschedError) as e:
        api.travel_matrix(ll, [300.0], api.METRIC_HAVERSINE)
    assert e.value.status == api.E_INVALID
    big = np.array([[0.0, 0.0], [1e12, 0.0]])  # 6e10 minutes at 1 km/h does not fit int32
    with pytest.raises(api.AschedError):
        api.travel_matrix(big, [1.0], api.METRIC_EUCLIDEAN)
    for speeds, metric in (([0.0], api.METRIC_EUCLIDEAN), ([300.0], 7), ([1.0, 2.0, 3.0], 0)):
        with pytest.raises((api.AschedError, ValueError)):
            api.travel_matrix([[0.0, 0.0], [1.0, 1.0]], speeds, metric)


def test_coordinates_to_schedules_end_to_end():
    """Matrices built on the device feed the batched search and the sweeps directly; the
    results equal those from the host-built matrices."""
    insts = [gen.paper_fleet(s, 12 + s % 22) for s in range(64)]
    bp_host = api.BatchProblem(insts)
    bp_dev = api.BatchProblem(insts)
    bp_dev.travel.zero_()
    status = api.travel_into_batch(bp_dev, _coords_tensor(insts), [300.0, 500.0])
    params = api.make_params(7, 200, api.PENALTY, 1000)
    a = api.solve_batch(bp_host, params)
    b = api.solve_batch(bp_dev, params)
    sp = api.sweep_params(50, api.HARD, 1000, 7, repair=True)
    c, _ = api.sweep_batch(bp_host, api.SWEEP_TABU, sp)
    d, _ = api.sweep_batch(bp_dev, api.SWEEP_TABU, sp)
    torch.cuda.synchronize()
    assert int(status.item()) == api.OK
    assert torch.equal(bp_host.travel, bp_dev.travel)
    for x, y in ((a, b), (c, d)):
        assert torch.equal(x.info, y.info) and torch.equal(x.route, y.route)


def test_half_minute_boundaries_go_through_float64():
    """Points whose times sit exactly on, or a hair off, half minutes: the float32 screen
    must hand them to float64, and the integers equal the oracle's exactly."""
    xs = [0.0]
    for k in range(1, 60):
        for eps in (0.0, 1e-12, -1e-12, 1e-9, -1e-9, 1e-6, -1e-6, 3e-5, -3e-5):
            for speed in (60.0, 300.0, 500.0):
                xs.append((k + 0.5) * speed / 60.0 + eps)
    xy = np.stack([np.array(xs), np.zeros(len(xs))], axis=1)
    for speeds in ([60.0, 300.0], [500.0]):
        got = api.travel_matrix(xy, speeds, api.METRIC_EUCLIDEAN).cpu().numpy()
        np.testing.assert_array_equal(got, travel.travel_minutes(xy, speeds, travel.EUCLIDEAN))


def test_haversine_near_antipodes_and_tiny_distances():
    rng = np.random.default_rng(9)
    lat = rng.uniform(-60, 60, 100)
    lon = rng.uniform(-180, 180, 100)
    anti = np.stack([-lat + rng.normal(0, 0.5, 100), lon + 180.0 + rng.normal(0, 0.5, 100)], axis=1)
    near = np.stack([lat + rng.normal(0, 1e-4, 100), lon + rng.normal(0, 1e-4, 100)], axis=1)
    ll = np.concatenate([np.stack([lat, lon], axis=1), anti, near])
    got = api.travel_matrix(ll, [300.0, 500.0], api.METRIC_HAVERSINE).cpu().numpy()
    want = travel.travel_minutes(ll, [300.0, 500.0], travel.HAVERSINE)
    raw = travel.minutes_unrounded(ll, [300.0, 500.0], travel.HAVERSINE)
    near_half = np.abs(np.abs(raw - np.floor(raw)) - 0.5) < 1e-6
    assert np.array_equal(got[~near_half], want[~near_half])
    assert np.abs(got.astype(np.int64) - want).max() <= 1
