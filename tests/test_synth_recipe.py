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
