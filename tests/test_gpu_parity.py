"""GPU parity: the CUDA library against the CPU oracle, through the C ABI.

Bar: bit-exact (validation = product build, -fmad=false): trajectories
(x, v as binary32 bit patterns, edge, lane, dwell, route position, id),
scalar counters, per-edge entry/exit counts, per-edge speed sums and the lane
map itself.
"""
import os

import numpy as np
import pytest

import nets
from oracle import oracle as O
from paper_2007_03614_b300 import manta, synth
from paper_2007_03614_b300.build import build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build()
    manta.load_library()


def _compare(o, g, where=""):
    a, b = o.snapshot(), g.snapshot()
    assert len(a["id"]) == len(b["id"]), (where, len(a["id"]), len(b["id"]))
    for key in ("id", "edge", "lane", "dwell", "route_pos"):
        if not np.array_equal(a[key], b[key]):
            i = int(np.nonzero(a[key] != b[key])[0][0])
            raise AssertionError(f"{where}: {key} differs first at vehicle {a['id'][i]}: {a[key][i]} vs {b[key][i]}")
    for key in ("x", "v"):
        ua, ub = a[key].view(np.uint32), b[key].view(np.uint32)
        if not np.array_equal(ua, ub):
            i = int(np.nonzero(ua != ub)[0][0])
            raise AssertionError(f"{where}: {key} differs first at vehicle {a['id'][i]}: {a[key][i]!r} vs {b[key][i]!r}")


def _compare_all(o, g, windows=(0,), where=""):
    _compare(o, g, where)
    so, sg = o.stats(), g.stats()
    for key in so:
        assert so[key] == sg[key], (where, key, so[key], sg[key])
    assert np.array_equal(o.lane_map(), g.lane_map()), where
    for w in windows:
        eo, eg = o.edge_counters(w), g.edge_counters(w)
        for key in eo:
            assert np.array_equal(eo[key], eg[key]), (where, w, key)


def _pair(net, tr, closures=(), **cfg):
    o = O.OracleSim(net, **cfg)
    g = manta.Sim(net, **cfg)
    for (e, l, k0, k1) in closures:
        o.set_lane_closure(e, l, k0, k1)
        g.set_lane_closure(e, l, k0, k1)
    nets.load(o, tr)
    nets.load(g, tr)
    return o, g


def test_tiny_workload_bit_exact():
    """10x10 grid, 2 lanes, fixed-time signals, 1,000 trips over 10 min, 30 min simulated."""
    net = synth.tiny_network()
    tr = synth.tiny_trips(net)
    o, g = _pair(net, tr)
    for k in range(0, 3600, 25):
        o.step(25)
        g.step(25)
        _compare(o, g, f"step {k + 25}")
        if (k + 25) % 600 == 0:
            _compare_all(o, g, windows=range(6), where=f"step {k + 25}")
    st = g.stats()
    assert st["arrived"] == 1000 and st["on_network"] == 0


def test_per_driver_speed_limits_bit_exact():
    """Section IV-B per-driver speed limits (speed_sigma_frac = 0.1) on the tiny
    workload: bit for bit equal to the oracle, and a different run from the one
    with every driver at the edge's limit."""
    net = synth.tiny_network()
    tr = synth.tiny_trips(net)
    o, g = _pair(net, tr, speed_sigma_frac=0.1)
    g0 = manta.Sim(net)
    nets.load(g0, tr)
    for k in range(0, 1800, 50):
        o.step(50)
        g.step(50)
        _compare(o, g, f"step {k + 50}")
        if k + 50 == 600:         # mid-run, with the network busy
            g0.step(600)
            a, b = g0.snapshot(), g.snapshot()
            assert len(a["id"]) > 100
            assert not (np.array_equal(a["id"], b["id"]) and np.array_equal(a["x"], b["x"]))
    _compare_all(o, g, windows=range(3))
    g0.close()


def test_tiny_all_stop_signs_bit_exact():
    """Red-light case of Section IV-C: every node a flashing red (stop + permit)."""
    net = synth.lattice(10, 10, arterial_every=1, len_median_m=100.0, len_sigma=0.0, len_min_m=100.0,
                        len_max_m=100.0, speed_mps=(13.889,) * 3, lanes=(2, 2, 2), all_stop=True)
    tr = synth.tiny_trips(net)
    o, g = _pair(net, tr)
    for k in range(0, 2400, 50):
        o.step(50)
        g.step(50)
        _compare(o, g, f"step {k + 50}")
    _compare_all(o, g, windows=range(4))
    assert g.stats()["arrived"] > 0


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
@pytest.mark.parametrize("ci", [0, 1, 2, 3])
def test_small_mixed_networks_every_step(seed, ci):
    """Random-walk routes on a 3x3 lattice with stop, signal and green nodes:
    every step compared (merges, queues, permits, lane changes)."""
    from test_oracle_bruteforce import CFGS, _scenario, closures_for
    net, tr = _scenario(seed, n_trips=40)
    cfg = dict(CFGS[ci])
    cfg["seed"] = 100 + seed
    o, g = _pair(net, tr, closures=closures_for(net, seed) if ci == 1 else (), **cfg)
    for k in range(600):
        o.step(1)
        g.step(1)
        _compare(o, g, f"seed {seed} cfg {ci} step {k}")
    _compare_all(o, g)


def test_edge_cases():
    # no trips at all
    net = nets.line(3)
    o, g = _pair(net, nets.trips([], []))
    o.step(10)
    g.step(10)
    _compare_all(o, g)
    # single-edge routes, departures beyond the run, a trip due before t0, many trips on one edge
    net = nets.line(2, length=60.0, lanes=2)
    routes = [[0]] * 30 + [[0, 1]] * 30 + [[1]] * 5
    times = list(np.linspace(-50.0, 40.0, 30)) + list(np.linspace(0.0, 20.0, 30)) + [1e6] * 5
    tr = nets.trips(routes, times)
    o, g = _pair(net, tr, t0_step=10)
    for k in range(300):
        o.step(1)
        g.step(1)
        _compare(o, g, f"step {k}")
    _compare_all(o, g)
    # zero steps is a no-op
    g.step(0)
    _compare_all(o, g)


def test_error_statuses():
    net = nets.line(2)
    g = manta.Sim(net)
    with pytest.raises(manta.MantaError) as ei:
        g.step(1)                                   # no trips yet
    assert ei.value.status == manta.E_STATE
    with pytest.raises(manta.MantaError) as ei:
        g.load_trips(np.array([0, 2], np.int64), np.array([1, 0], np.int32), np.array([0.0], np.float32))
    assert ei.value.status == manta.E_ROUTE       # 1 -> 0 is not contiguous
    with pytest.raises(manta.MantaError) as ei:
        g.load_trips(np.array([0, 0], np.int64), np.zeros(0, np.int32), np.array([0.0], np.float32))
    assert ei.value.status == manta.E_ROUTE       # empty route
    with pytest.raises(manta.MantaError) as ei:     # second trip: an edge out of range after its first
        g.load_trips(np.array([0, 2, 4], np.int64), np.array([0, 1, 0, 7], np.int32),
                     np.array([0.0, 0.0], np.float32))
    assert ei.value.status == manta.E_ROUTE and "trip 1" in str(ei.value)
    with pytest.raises(manta.MantaError) as ei:     # third trip: not contiguous in its middle
        g.load_trips(np.array([0, 2, 3, 6], np.int64), np.array([0, 1, 1, 0, 1, 0], np.int32),
                     np.array([0.0, 0.0, 0.0], np.float32))
    assert ei.value.status == manta.E_ROUTE and "trip 2" in str(ei.value)
    g.load_trips(np.array([0, 2], np.int64), np.array([0, 1], np.int32), np.array([0.0], np.float32))
    with pytest.raises(manta.MantaError) as ei:
        g.load_trips(np.array([0, 2], np.int64), np.array([0, 1], np.int32), np.array([0.0], np.float32))
    assert ei.value.status == manta.E_STATE
    g.step(100)
    assert g.stats()["arrived"] == 1


def test_barrier_wait_runs_out_and_context_survives():
    """A grid barrier whose last block never arrives: every waiter gives up
    after ~0.1 s and returns MANTA_E_TIMEOUT; the context keeps working."""
    assert manta.selftest_barrier_timeout(100) == manta.E_TIMEOUT
    net = nets.line(2)
    tr = nets.trips([[0, 1]], [0.0])
    o, g = _pair(net, tr)
    o.step(50)
    g.step(50)
    _compare_all(o, g)


# ------------------------------------------------------------------ metro --
def _subset(tr, lo_s, hi_s):
    sel = np.nonzero((tr.depart_time_s >= lo_s) & (tr.depart_time_s < hi_s))[0]
    routes = [tr.route_edges[tr.route_off[i]:tr.route_off[i + 1]] for i in sel]
    off = np.zeros(len(sel) + 1, np.int64)
    off[1:] = np.cumsum([len(r) for r in routes])
    return synth.Trips(route_off=off, route_edges=np.concatenate(routes).astype(np.int32),
                       depart_time_s=tr.depart_time_s[sel])


def test_metro_network_window_bit_exact(metro):
    """Full metro-shaped network (~550k edges), the trips departing 07:30-07:35,
    600 steps from an empty network at 07:30: bit-exact at checkpoints."""
    net, tr = metro
    sub = _subset(tr, 7.5 * 3600, 7.5 * 3600 + 300)
    assert sub.n_trips > 20000
    t0 = int(7.5 * 3600 / 0.5)
    o, g = _pair(net, sub, t0_step=t0, n_stats_windows=4)
    for k in range(0, 600, 100):
        o.step(100)
        g.step(100)
        _compare(o, g, f"metro step {k + 100}")
    _compare_all(o, g, windows=(0,))
    assert g.stats()["on_network"] > 10000


def test_metro_incident_closures_bit_exact(metro):
    """Stress-style incident: lane 0 closed on 200 random freeway edges from
    07:30 for 5 minutes, on the full metro network with the 07:30-07:35 trips."""
    net, tr = metro
    rng = np.random.default_rng(4)
    fw = np.nonzero(net.edge_class == synth.CLASS_FREEWAY)[0]
    t0 = int(7.5 * 3600 / 0.5)
    clo = [(int(e), 0, t0, t0 + 600) for e in rng.choice(fw, 200, replace=False)]
    sub = _subset(tr, 7.5 * 3600, 7.5 * 3600 + 300)
    o, g = _pair(net, sub, closures=clo, t0_step=t0, n_stats_windows=4)
    for k in range(0, 600, 150):
        o.step(150)
        g.step(150)
        _compare(o, g, f"closures step {k + 150}")
    _compare_all(o, g, windows=(0,))
    with pytest.raises(manta.MantaError) as ei:
        g.set_lane_closure(0, 0, 0, 1)
    assert ei.value.status == manta.E_STATE


def test_metro_dense_state_bit_exact(metro):
    """A dense mid-morning state on the full metro network, at the size the
    benchmark runs: ~500k vehicles put on the network at 07:30 by the seeded
    dense-state generator (the same placements on both sides), 600 steps in
    one 150-step launch, three 50-step launches and one of 300, bit for bit.  The state is
    built to reach the kernel's full-size paths: in the first step far more
    merge-phase items than half the warps (the record pass then shares warps
    with merge items), more arrivals than a quarter of the active list within
    150 steps (compaction), and a list long enough for guided chunk tails."""
    net, tr = metro
    lo = 7.5 * 3600
    sub = _subset(tr, lo - 2700, lo + 300)
    pl = synth.dense_state(net, sub, lo - 2700, lo, head_frac=0.15, last_edge_frac=0.3, seed=5)
    assert pl.n > 450_000
    t0 = int(lo / 0.5)
    o, g = _pair(net, sub, t0_step=t0, n_stats_windows=4)
    o.place_many(pl.trip, pl.route_pos, pl.lane, pl.x, pl.v)
    g.place(pl.trip, pl.route_pos, pl.lane, pl.x, pl.v)
    _compare_all(o, g, where="placed")
    # merge-phase items of the first step, from the oracle's own event tape:
    # crossing requests (crossed or held), arrivals
    tape = o.record_tape(1)
    o.step(1)
    out = (tape["flags"][0] >> 6) & 7
    present = (tape["flags"][0] & 1) != 0
    items = int(np.sum(present & (out >= 1)))
    assert items > 40_000, items
    o.stop_tape()
    o.step(149)
    g.step(150)
    _compare_all(o, g, where="dense step 150")
    st = o.stats()
    assert st["arrived"] > 0.25 * st["departed"]
    for k in range(150, 300, 50):
        o.step(50)
        g.step(50)
        _compare(o, g, f"dense step {k + 50}")
    _compare_all(o, g, windows=(0,), where="dense step 300")
    assert g.stats()["on_network"] > 300_000
    o.step(300)
    g.step(300)
    _compare_all(o, g, windows=(0, 1), where="dense step 600")


def test_metro_first_trips_window_bit_exact(metro):
    """05:00, the start of the morning: the trips departing 05:00-05:10 on the
    empty metro network, 600 steps in launches of 200, bit for bit."""
    net, tr = metro
    sub = _subset(tr, 5 * 3600, 5 * 3600 + 600)
    assert sub.n_trips > 1000
    o, g = _pair(net, sub, t0_step=36000, n_stats_windows=2)
    for k in range(0, 600, 200):
        o.step(200)
        g.step(200)
        _compare(o, g, f"05:00 window step {k + 200}")
    _compare_all(o, g, windows=(0,))
    assert g.stats()["on_network"] > 500


def test_metro_late_morning_dense_state_bit_exact(metro):
    """11:00: the trips departing 09:30-11:00 put along their routes (the
    dense-state generator, ~280k vehicles), 600 steps in launches of 300,
    bit for bit."""
    net, tr = metro
    lo = 11 * 3600
    sub = _subset(tr, lo - 5400, lo + 300)
    pl = synth.dense_state(net, sub, lo - 5400, lo, head_frac=0.1, seed=11)
    assert pl.n > 200_000
    o, g = _pair(net, sub, t0_step=int(lo / 0.5), n_stats_windows=2)
    o.place_many(pl.trip, pl.route_pos, pl.lane, pl.x, pl.v)
    g.place(pl.trip, pl.route_pos, pl.lane, pl.x, pl.v)
    for k in range(0, 600, 300):
        o.step(300)
        g.step(300)
        _compare(o, g, f"11:00 dense step {k + 300}")
    _compare_all(o, g, windows=(0, 1), where="11:00 dense step 600")


def test_stress_dense_state_with_incidents_bit_exact():
    """The stress configuration (~1.6M edges) at 08:00 with its incident lane
    closures active: the trips departing 07:45-08:00 put along their routes,
    none in a closed lane, 200 steps, bit for bit."""
    net = synth.stress_network()
    tr = synth.stress_trips(net)
    clo = synth.incident_closures(net)
    lo = 8 * 3600
    sub = _subset(tr, lo - 900, lo + 300)
    pl = synth.dense_state(net, sub, lo - 900, lo, head_frac=0.15, seed=13)
    closed = {(e, l) for (e, l, _, _) in clo}
    e = sub.route_edges[sub.route_off[pl.trip] + pl.route_pos]
    keep = np.array([(int(a), int(b)) not in closed for a, b in zip(e, pl.lane)])
    assert keep.sum() > 200_000
    o, g = _pair(net, sub, closures=clo, t0_step=int(lo / 0.5), n_stats_windows=2)
    args = [a[keep] for a in (pl.trip, pl.route_pos, pl.lane, pl.x, pl.v)]
    o.place_many(*args)
    g.place(*args)
    for k in range(0, 200, 100):
        o.step(100)
        g.step(100)
        _compare(o, g, f"stress dense step {k + 100}")
    _compare_all(o, g, windows=(0,), where="stress dense step 200")


def test_place_rejects_bad_placements():
    """manta_place validates what the host can see (trip, route position,
    speed) before touching the device, and is refused after the first step."""
    net = nets.line(3, length=100.0, lanes=2)
    tr = nets.trips([[0, 1, 2], [1, 2], [0, 1]], [0.0, 0.0, 50.0])
    g = manta.Sim(net)
    nets.load(g, tr)
    for bad in (dict(trip=[5]), dict(trip=[0, 0]), dict(route_pos=[3]), dict(v=[-1.0])):
        args = dict(trip=[0], route_pos=[1], lane=[0], x=[10.0], v=[5.0])
        args.update(bad)
        n = len(args["trip"])
        for k in ("route_pos", "lane", "x", "v"):
            args[k] = (args[k] * n)[:n]
        with pytest.raises(manta.MantaError) as ei:
            g.place(**args)
        assert ei.value.status == manta.E_INVALID
    o = O.OracleSim(net)
    nets.load(o, tr)
    g.place([0, 1], [1, 0], [1, 0], [10.5, 40.25], [5.0, 0.0])
    o.place_many([0, 1], [1, 0], [1, 0], [10.5, 40.25], [5.0, 0.0])
    _compare_all(o, g)
    for _ in range(40):
        o.step(1)
        g.step(1)
        _compare(o, g)
    _compare_all(o, g)
    with pytest.raises(manta.MantaError) as ei:
        g.place([2], [0], [0], [1.0], [0.0])
    assert ei.value.status == manta.E_STATE
    # what only the device sees: a lane the edge lacks, a position past its
    # end, two placements on one cell; each leaves that simulation unusable
    for bad in (([0], [1], [2], [10.0], [5.0]), ([0], [1], [0], [100.0], [5.0]),
                ([0, 1], [1, 0], [0, 0], [10.5, 10.25], [5.0, 0.0])):
        g2 = manta.Sim(net)
        nets.load(g2, tr)
        with pytest.raises(manta.MantaError) as ei:
            g2.place(*bad)
        assert ei.value.status == manta.E_INVALID
        with pytest.raises(manta.MantaError) as ei:
            g2.step(1)
        assert ei.value.status == manta.E_STATE
        g2.close()


def test_metro_full_morning_properties(metro):
    """The full 3.2M-trip table at the size the benchmark runs: conservation,
    lane-map occupancy equal to the on-network count, and fronts at least L
    apart in every lane, after 3 simulated hours from 05:00."""
    net, tr = metro
    g = manta.Sim(net, t0_step=36000)
    nets.load(g, tr)
    g.step(21600)
    st = g.stats()
    assert st["departed"] == st["arrived"] + st["on_network"]
    assert st["loaded"] == st["departed"] + st["waiting"]
    m = g.lane_map()
    occ = np.nonzero(m != 0xFF)[0]
    assert len(occ) == st["on_network"]
    ec = g.edge_counters(0)
    assert int(ec["entries"].sum()) - int(ec["exits"].sum()) == st["on_network"]
    # lane rows in canonical order: consecutive fronts within a row differ by >= L
    cells = np.maximum(np.floor(net.edge_length_m.astype(np.float64) + 0.5).astype(np.int64), 5 + 2 + 1)
    row_len = np.repeat(cells, net.edge_lanes.astype(np.int64))
    row_start = np.concatenate([[0], np.cumsum(row_len)[:-1]])
    row_of = np.searchsorted(row_start, occ, side="right") - 1
    same = row_of[1:] == row_of[:-1]
    assert np.all(np.diff(occ)[same] >= 5)
    assert st["on_network"] > 100000


def test_ensemble_union_bit_exact():
    """Batched what-if scenarios: the disjoint union of uneven scenarios runs as
    one simulation; it matches the oracle on the same union."""
    sc = synth.ensemble_scenarios(n=5, seed=7, edges_range=(800, 6000), trips_range=(300, 3000))
    ens = synth.union(sc)
    t0 = int(7 * 3600 / 0.5)
    o, g = _pair(ens.net, ens.trips, t0_step=t0, n_stats_windows=4)
    for k in range(0, 900, 150):
        o.step(150)
        g.step(150)
        _compare(o, g, f"ensemble step {k + 150}")
    _compare_all(o, g, windows=(0, 1))
    # every scenario made progress
    ec = g.edge_counters(0)
    for s in range(len(sc)):
        assert int(ec["entries"][ens.edge_off[s]:ens.edge_off[s + 1]].sum()) > 0


def test_stress_day_properties():
    """The stress configuration at full size (~1.6M edges, 10M trips, lane 0
    closed on 200 freeway edges 07:30-09:00), run from 04:00 to 08:30 in the
    launch size the benchmark uses: conservation, lane-map occupancy equal to
    the on-network count, fronts at least L apart in every lane, and no
    vehicle beyond the mid-edge obstacle of a closed lane."""
    net = synth.stress_network()
    tr = synth.stress_trips(net)
    clo = synth.incident_closures(net)
    g = manta.Sim(net, t0_step=int(4 * 7200))
    for (e, l, k0, k1) in clo:
        g.set_lane_closure(e, l, k0, k1)
    nets.load(g, tr)
    n = int(8.5 * 7200) - int(4 * 7200)
    while n > 0:
        g.step(min(1800, n))
        n -= 1800
    st = g.stats()
    assert st["departed"] == st["arrived"] + st["on_network"]
    assert st["loaded"] == st["departed"] + st["waiting"]
    assert st["on_network"] > 500_000
    m = g.lane_map()
    occ = np.nonzero(m != 0xFF)[0]
    assert len(occ) == st["on_network"]
    cells = np.maximum(np.floor(net.edge_length_m.astype(np.float64) + 0.5).astype(np.int64), 5 + 2 + 1)
    row_len = np.repeat(cells, net.edge_lanes.astype(np.int64))
    row_start = np.concatenate([[0], np.cumsum(row_len)[:-1]])
    row_of = np.searchsorted(row_start, occ, side="right") - 1
    same = row_of[1:] == row_of[:-1]
    assert np.all(np.diff(occ)[same] >= 5)
    lane0 = np.concatenate([[0], np.cumsum(net.edge_lanes.astype(np.int64))[:-1]])
    for (e, l, k0, k1) in clo:
        r = int(lane0[e]) + l
        C = int(row_len[r])
        assert np.all(m[row_start[r] + C // 2: row_start[r] + C] == 0xFF), e
