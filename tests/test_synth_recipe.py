"""The input recipe: the seeded generators give the networks and trip tables
that the benchmark and the parity tests are quoted on, with the properties
stated for them (sizes, class mix, length law, signals, departure law,
route structure)."""
import numpy as np
import pytest

from paper_2007_03614_b300 import synth

KMH = 1.0 / 3.6


@pytest.fixture(scope="module")
def metro():
    return synth.metro_network()


def test_metro_network_recipe(metro):
    net = metro
    assert net.edge_src.size == 548_776 and net.node_type.size == 218_905
    # local 1 lane 40 km/h, arterial (every 8th line) 2 lanes 70 km/h, freeway (every 32nd) 4 lanes 105 km/h
    for c, lanes, kmh in ((0, 1, 40.0), (1, 2, 70.0), (2, 4, 105.0)):
        m = net.edge_class == c
        assert m.any()
        assert np.all(net.edge_lanes[m] == lanes)
        assert np.allclose(net.edge_speed_limit_mps[m], kmh * KMH, rtol=1e-4)
    # lengths: lognormal, median 120 m, sigma 0.8, clamped to [20, 2000] m per
    # segment; an overpass (a local street over a freeway) joins two segments
    L = net.edge_length_m.astype(np.float64)
    assert L.min() >= 20.0 and L.max() <= 4000.0
    assert (L <= 2000.0).mean() > 0.99
    main = L[net.edge_class > 0]                 # arterial and freeway segments are never overpasses
    assert abs(np.median(main) / 120.0 - 1.0) < 0.05
    assert abs(np.log(main).std() - 0.8) < 0.05
    # fixed-time signals at arterial crossings only; no stop signs
    assert np.sum(net.node_type == 2) == 2025    # signal
    assert np.sum(net.node_type == 1) == 0       # stop sign
    # every street is two directed edges
    pairs = set(zip(net.edge_src.tolist(), net.edge_dst.tolist()))
    assert all((d, s) in pairs for s, d in pairs)


def test_metro_trips_recipe(metro):
    net = metro
    tr = synth.metro_trips(net, n_trips=20_000)
    dep = tr.depart_time_s.astype(np.float64)
    # departures N(08:00, 75 min) truncated to [05:00, 12:00)
    assert dep.min() >= 5 * 3600.0 and dep.max() < 12 * 3600.0
    assert abs(dep.mean() - 8 * 3600.0) < 300.0
    assert abs(dep.std() / (75 * 60.0) - 1.0) < 0.1
    off = tr.route_off
    edges = tr.route_edges
    first = edges[off[:-1]]
    last = edges[off[1:] - 1]
    assert np.all(off[1:] > off[:-1])
    # routes are contiguous
    same_trip = np.ones(edges.size - 1, bool)
    same_trip[off[1:-1] - 1] = False
    assert np.all(net.edge_dst[edges[:-1]][same_trip] == net.edge_src[edges[1:]][same_trip])
    # no trip starts or ends on a freeway
    assert np.all(net.edge_class[first] != 2) and np.all(net.edge_class[last] != 2)
    # gravity model with decay length 5.4 km: mean route about 11.8 km (the paper reports 11.3 km)
    lengths = np.add.reduceat(net.edge_length_m[edges].astype(np.float64), off[:-1])
    assert 10_500.0 < lengths.mean() < 13_000.0


def test_dense_state_recipe(metro):
    """The dense starting state (synth.dense_state): every placement lies on
    its own trip's route, within its edge and lane; fronts in one lane are at
    least L = 5 cells apart; the requested share sits in the last slot of its
    edge; and the CPU oracle accepts the state and keeps its invariants
    (conservation, map bytes = speed codes, fronts >= L apart) over 20 steps."""
    from oracle import oracle as O
    net = metro
    tr = synth.metro_trips(net, n_trips=20_000)
    lo = 7.5 * 3600.0
    pl = synth.dense_state(net, tr, lo - 3600.0, lo, head_frac=0.2, seed=3)
    assert pl.n > 2000
    ro = tr.route_off
    rlen = ro[pl.trip + 1] - ro[pl.trip]
    assert np.all((pl.route_pos >= 0) & (pl.route_pos < rlen))
    e = tr.route_edges[ro[pl.trip] + pl.route_pos].astype(np.int64)
    assert np.all(pl.lane < net.edge_lanes[e])
    cells = np.maximum(8, np.floor(net.edge_length_m.astype(np.float64) + 0.5).astype(np.int64))[e]
    assert np.all((pl.x >= 0.0) & (pl.x < cells)) and np.all(pl.v >= 0.0)
    assert np.all(pl.v <= net.edge_speed_limit_mps[e])
    key = e * 16 + pl.lane
    order = np.lexsort((np.floor(pl.x), key))
    same = key[order][1:] == key[order][:-1]
    assert np.all(np.diff(np.floor(pl.x[order]))[same] >= 5)
    near_end = cells - np.floor(pl.x) <= 11
    assert near_end.mean() > 0.15
    o = O.OracleSim(net, t0_step=int(lo / 0.5), n_stats_windows=2)
    o.load_trips(tr.route_off, tr.route_edges, tr.depart_time_s)
    o.place_many(pl.trip, pl.route_pos, pl.lane, pl.x, pl.v)
    o.check()
    st = o.stats()
    assert st["on_network"] == pl.n and st["departed"] == pl.n
    for _ in range(4):
        o.step(5)
        o.check()
